// Host-side physical parameters of a domain: Peng-Robinson coefficients
// (Eq. PREoS with the alpha function of Sec. 2.3), the viscosity interpolation,
// the interface band, and the densities where P(rho) - rho cs^2 changes sign.
#pragma once

#include <cmath>
#include <limits>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

struct EosCoeffs { double RT, b, aalpha, Tc; };

inline EosCoeffs eos_coeffs(const lbm_params& p) {
  EosCoeffs e;
  e.Tc = 0.0778 * p.a / (0.45724 * p.b * p.R);
  const double T = p.T_over_Tc * e.Tc;
  const double m = 0.37464 + 1.54226 * p.acentric - 0.26992 * p.acentric * p.acentric;
  const double s = 1.0 + m * (1.0 - std::sqrt(p.T_over_Tc));
  e.RT = p.R * T;
  e.b = p.b;
  e.aalpha = p.a * s * s;
  return e;
}

inline double pr_p(const EosCoeffs& e, double rho) {
  return rho * e.RT / (1.0 - e.b * rho) - e.aalpha * rho * rho / (1.0 + 2.0 * e.b * rho - e.b * e.b * rho * rho);
}

// True where P(rho) > rho cs^2 (s = +1), evaluated as the float64 path does.
inline bool psi_positive(const EosCoeffs& e, double rho) { return pr_p(e, rho) - rho * (1.0 / 3.0) > 0.0; }

// Sign changes of P(rho) - rho cs^2 on (0, 1/b).  Multiplied by the positive
// (1 - b rho)(1 + 2 b rho - b^2 rho^2) it is a cubic in rho, so there are at most
// three.  They are bracketed on a grid that is logarithmic towards rho = 0 and
// uniform above, and bisected down to adjacent doubles; t[k] is the upper double
// of the k-th bracket (the first density with the new sign), +inf where unused.
// *s0 is the sign below every t[k].
inline void psi_sign_changes(const EosCoeffs& e, double t[3], double* s0) {
  const double inf = std::numeric_limits<double>::infinity();
  t[0] = t[1] = t[2] = inf;
  const double top = (1.0 / e.b) * (1.0 - 1e-9);
  const int n_log = 4096, n_lin = 1 << 16;
  auto grid = [&](int j) {  // increasing in j, j in [0, n_log + n_lin]
    if (j <= n_log) return top * 1e-3 * std::pow(10.0, -12.0 * (double)(n_log - j) / n_log);
    return top * 1e-3 + (top - top * 1e-3) * (double)(j - n_log) / n_lin;
  };
  double lo = grid(0);
  bool slo = psi_positive(e, lo);
  *s0 = slo ? 1.0 : -1.0;
  int nt = 0;
  for (int j = 1; j <= n_log + n_lin && nt < 3; ++j) {
    const double hi = grid(j);
    const bool shi = psi_positive(e, hi);
    if (shi != slo) {
      double a = lo, b = hi;  // psi_positive(a) == slo, psi_positive(b) == shi
      for (int it = 0; it < 2000; ++it) {
        const double mid = a + 0.5 * (b - a);
        if (mid <= a || mid >= b) break;
        if (psi_positive(e, mid) == slo) a = mid; else b = mid;
      }
      t[nt++] = b;
    }
    lo = hi;
    slo = shi;
  }
}

// Smallest float at or above a double: a float rho satisfies rho >= this exactly
// when (double)rho >= x.
inline float float_at_or_above(double x) {
  if (std::isinf(x)) return (float)x;
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}

// Fill the physical parameters of d (both arithmetic types) from p.
inline void fill_phys(DevDomain& d, const lbm_params& p, int D) {
  Phys<double>& pd = d.pd;
  pd.kappa = p.kappa;
  for (int a = 0; a < 3; ++a) pd.g[a] = a < D ? p.body_force[a] : 0.0;
  pd.nu_v = p.nu_vapour;
  pd.dnu = p.nu_liquid - p.nu_vapour;
  pd.rho_v = p.rho_vapour;
  pd.inv_drho = 1.0 / (p.rho_liquid - p.rho_vapour);
  const EosCoeffs e = eos_coeffs(p);
  pd.RT = e.RT; pd.b = e.b; pd.aalpha = e.aalpha;
  pd.gamma_value = p.gamma_value;
  // interface band: densities between the phases, 1% of the density jump inside each bulk value
  const double span = p.rho_liquid - p.rho_vapour;
  pd.band_lo = p.rho_vapour + 0.01 * span;
  pd.band_hi = p.rho_liquid - 0.01 * span;
  psi_sign_changes(e, pd.sgn_t, &pd.sgn0);
  Phys<float>& pf = d.pf;
  pf.kappa = (float)pd.kappa;
  for (int a = 0; a < 3; ++a) pf.g[a] = (float)pd.g[a];
  pf.nu_v = (float)pd.nu_v; pf.dnu = (float)pd.dnu; pf.rho_v = (float)pd.rho_v; pf.inv_drho = (float)pd.inv_drho;
  pf.RT = (float)pd.RT; pf.b = (float)pd.b; pf.aalpha = (float)pd.aalpha;
  pf.gamma_value = (float)pd.gamma_value;
  pf.band_lo = (float)pd.band_lo; pf.band_hi = (float)pd.band_hi;
  for (int k = 0; k < 3; ++k) pf.sgn_t[k] = float_at_or_above(pd.sgn_t[k]);
  pf.sgn0 = (float)pd.sgn0;
  d.gamma_mode = p.gamma_mode;
  d.eos_fp64 = p.eos_fp64;
}

}  // namespace lbm
