/*
 * FP64 CPU oracle for the entropic multi-relaxation-time two-phase lattice
 * Boltzmann step of Hosseini, Dorschner & Karlin (arXiv:2201.12404).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it;
 * the library never calls it and shares no code, header or table with it.
 *
 * Everything is IEEE double, scalar loops, no blocking or fusion.  Build with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Layout of a population array: f[i * N + node], node = x + nx*(y + ny*z),
 * velocity index i = (cx+1) + 3(cy+1) + 9(cz+1), so the opposite direction of i
 * is Q-1-i.  The array always holds the post-streaming, pre-collision state.
 *
 * Readings of the paper used here (each is a choice where the paper is silent
 * or garbled; the CUDA library makes the same ones):
 *  - force sign: the printed stencil sum approximates grad(P-P0) - kappa rho
 *    grad lap rho, the bracket of Eq. (1); the force is its negative.
 *  - extended equilibrium: zeta* = P0/rho + xi*^2 + Phi/rho (the form whose
 *    central moments are the appendix vector a*).
 *  - Phi: second-order central difference, local omega, and q formed with the
 *    velocity of the exact-difference method, u + F dt/(2 rho), so that Phi
 *    vanishes for a fluid at rest.
 *  - nu(rho): linear in rho between the coexistence densities, clamped.
 *  - walls: half-way bounce-back; auxiliary ghosts mirrored, q negated.
 *  - gamma guards: any f*_i <= 0 -> gamma = 2 at that node; <dh|dh> <= 1e-300
 *    -> ratio 0.  No clipping.
 *  - initial state: equilibrium at the bare velocity u0 - F dt/(2 rho0), so that
 *    the reported (exact-difference-method) velocity starts at u0.
 *  - D3Q27 moment set: the 27 tensor products H_p(x)H_q(y)H_r(z), p,q,r<=2,
 *    with the three diagonal second-order moments recombined into two
 *    differences and the trace (the printed list repeats a_{x^2y^2} where
 *    a_{xyz} belongs).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXQ 27

typedef struct {
  int D, nx, ny, nz;
  double a, b, R, T_over_Tc, acentric;
  double kappa;
  double nu_liquid, nu_vapour, rho_liquid, rho_vapour;
  double g[3];
  int bc[6];          /* faces -x,+x,-y,+y,-z,+z: 0 periodic, 1 bounce-back */
  int gamma_mode;     /* 0 entropic, 1 fixed */
  double gamma_value;
} orc_params;

static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared, P0/rho */

/* ---- Lattice: velocities, one-dimensional triplet, product form (Sec. 2.1) ---- */

int orc_Q(int D) { return D == 2 ? 9 : 27; }

void orc_velocities(int D, int* c /* Q*3 */) {
  int Q = orc_Q(D);
  for (int i = 0; i < Q; ++i) {
    c[3 * i + 0] = i % 3 - 1;
    c[3 * i + 1] = (i / 3) % 3 - 1;
    c[3 * i + 2] = D == 3 ? (i / 9) - 1 : 0;
  }
}

/* Triplet Psi_{c}(xi, zeta), Eqs. (phi0)-(phis). */
double orc_psi1(int c, double xi, double zeta) {
  if (c == 0) return 1.0 - zeta;
  if (c == 1) return (xi + zeta) / 2.0;
  return (-xi + zeta) / 2.0;
}

/* Product form Eq. (prod) scaled by rho: out_i = rho * prod_alpha Psi_{c_ia}(xi_a, zeta_a). */
void orc_product_form(int D, double rho, const double* xi, const double* zeta, double* out) {
  int Q = orc_Q(D), c[3 * MAXQ];
  orc_velocities(D, c);
  for (int i = 0; i < Q; ++i) {
    double p = rho;
    for (int al = 0; al < D; ++al) p = p * orc_psi1(c[3 * i + al], xi[al], zeta[al]);
    out[i] = p;
  }
}

/* Weights, Eq. (wi): product form at xi = 0, zeta = cs^2. */
void orc_weights(int D, double* w) {
  double xi[3] = {0, 0, 0}, zeta[3] = {CS2, CS2, CS2};
  orc_product_form(D, 1.0, xi, zeta, w);
}

/* Equilibrium, Eq. (LBMeq): xi = u, zeta = P0/rho + u^2 with P0/rho = cs^2. */
void orc_feq(int D, double rho, const double* u, double* feq) {
  double xi[3] = {0, 0, 0}, zeta[3] = {CS2, CS2, CS2};
  for (int al = 0; al < D; ++al) { xi[al] = u[al]; zeta[al] = CS2 + u[al] * u[al]; }
  orc_product_form(D, rho, xi, zeta, feq);
}

/* Extended equilibrium, Eqs. (xistar), (LBMstar): xi* = u + F dt/rho,
 * zeta* = P0/rho + xi*^2 + Phi/rho (shifted reading, matches the appendix a*). */
void orc_fstar(int D, double rho, const double* u, const double* F, const double* Phi, double* fs) {
  double xi[3] = {0, 0, 0}, zeta[3] = {CS2, CS2, CS2};
  for (int al = 0; al < D; ++al) {
    xi[al] = u[al] + F[al] / rho;
    zeta[al] = CS2 + xi[al] * xi[al] + Phi[al] / rho;
  }
  orc_product_form(D, rho, xi, zeta, fs);
}

/* ---- Equation of state, Eq. (PREoS), and pseudo-potential (Sec. 2.3) ---- */

double orc_Tc(const orc_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }

double orc_pressure(const orc_params* p, double rho) {
  double T = p->T_over_Tc * orc_Tc(p);
  double m = 0.37464 + 1.54226 * p->acentric - 0.26992 * p->acentric * p->acentric;
  double sq = 1.0 + m * (1.0 - sqrt(p->T_over_Tc));
  double alpha = sq * sq;
  double b = p->b;
  return rho * p->R * T / (1.0 - b * rho) - p->a * alpha * rho * rho / (1.0 + 2.0 * rho * b - b * b * rho * rho);
}

/* Signed pseudo-potential: returns psi = sqrt(|P - P0|) and sets *sign to +1 when
 * P > P0, -1 otherwise (the "<=" branch takes the tie). */
double orc_psi(const orc_params* p, double rho, double* sign) {
  double d = orc_pressure(p, rho) - rho * CS2;
  if (d > 0.0) { *sign = 1.0; return sqrt(d); }
  *sign = -1.0;
  return sqrt(-d);
}

/* Viscosity rule across the interface, and omega = dt/(rho nu/P0 + dt/2). */
double orc_omega(const orc_params* p, double rho) {
  double phi = 0.0;
  if (p->rho_liquid > p->rho_vapour) phi = (rho - p->rho_vapour) / (p->rho_liquid - p->rho_vapour);
  if (phi < 0.0) phi = 0.0;
  if (phi > 1.0) phi = 1.0;
  double nu = p->nu_vapour + phi * (p->nu_liquid - p->nu_vapour);
  return 1.0 / (nu / CS2 + 0.5);
}

/* ---- Modified central Hermite moment basis (Appendix A) ---- */

/* One-dimensional central Hermite polynomials H_0 = 1, H_1 = x, H_2 = x^2 - cs^2. */
static double herm1(int p, double x) {
  if (p == 0) return 1.0;
  if (p == 1) return x;
  return x * x - CS2;
}

/* Row descriptors of the moment basis.  kind 0: tensor product H_p H_q H_r with
 * exponents e; kind 1: a_xx - a_yy; kind 2: a_xx - a_zz; kind 3: trace.
 * part: 0 = K (conserved), 1 = S (deviatoric second order), 2 = H (rest). */
typedef struct { int kind; int e[3]; int part; } orc_row;

static int basis_rows(int D, orc_row* rows) {
  int n = 0;
#define ROW(k, p, q, r, part_) do { rows[n].kind = (k); rows[n].e[0] = (p); rows[n].e[1] = (q); rows[n].e[2] = (r); rows[n].part = (part_); ++n; } while (0)
  if (D == 2) {
    ROW(0, 0, 0, 0, 0); ROW(0, 1, 0, 0, 0); ROW(0, 0, 1, 0, 0);
    ROW(0, 1, 1, 0, 1); ROW(1, 0, 0, 0, 1); ROW(3, 0, 0, 0, 2);
    ROW(0, 2, 1, 0, 2); ROW(0, 1, 2, 0, 2); ROW(0, 2, 2, 0, 2);
  } else {
    ROW(0, 0, 0, 0, 0); ROW(0, 1, 0, 0, 0); ROW(0, 0, 1, 0, 0); ROW(0, 0, 0, 1, 0);
    ROW(0, 1, 1, 0, 1); ROW(0, 1, 0, 1, 1); ROW(0, 0, 1, 1, 1);
    ROW(1, 0, 0, 0, 1); ROW(2, 0, 0, 0, 1); ROW(3, 0, 0, 0, 2);
    ROW(0, 2, 1, 0, 2); ROW(0, 2, 0, 1, 2); ROW(0, 1, 2, 0, 2); ROW(0, 0, 2, 1, 2);
    ROW(0, 1, 0, 2, 2); ROW(0, 0, 1, 2, 2); ROW(0, 1, 1, 1, 2);
    ROW(0, 2, 2, 0, 2); ROW(0, 2, 0, 2, 2); ROW(0, 0, 2, 2, 2);
    ROW(0, 2, 1, 1, 2); ROW(0, 1, 2, 1, 2); ROW(0, 1, 1, 2, 2);
    ROW(0, 2, 2, 1, 2); ROW(0, 2, 1, 2, 2); ROW(0, 1, 2, 2, 2);
    ROW(0, 2, 2, 2, 2);
  }
#undef ROW
  return n;
}

/* Matrix M(u) (Q x Q, row-major): a_m = sum_i M[m][i] f_i. */
static void moment_matrix(int D, const double* u, double* M) {
  int Q = orc_Q(D), c[3 * MAXQ];
  orc_row rows[MAXQ];
  orc_velocities(D, c);
  basis_rows(D, rows);
  for (int m = 0; m < Q; ++m) {
    for (int i = 0; i < Q; ++i) {
      double v[3];
      for (int al = 0; al < 3; ++al) v[al] = (al < D) ? (double)c[3 * i + al] - u[al] : 0.0;
      double val;
      if (rows[m].kind == 0) {
        val = 1.0;
        for (int al = 0; al < D; ++al) val = val * herm1(rows[m].e[al], v[al]);
      } else {
        double hxx = herm1(2, v[0]), hyy = herm1(2, v[1]), hzz = D == 3 ? herm1(2, v[2]) : 0.0;
        /* the diagonal Hermite polynomial along one axis is H_2 of that axis times H_0 of the others */
        if (rows[m].kind == 1) val = hxx - hyy;
        else if (rows[m].kind == 2) val = hxx - hzz;
        else val = hxx + hyy + hzz;
      }
      M[m * Q + i] = val;
    }
  }
}

/* Gaussian elimination with partial pivoting: solve A x = bvec (A is n x n, copied). */
static int lu_solve(int n, const double* A_in, const double* bvec, double* x) {
  double A[MAXQ * MAXQ], bb[MAXQ];
  memcpy(A, A_in, sizeof(double) * n * n);
  memcpy(bb, bvec, sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r) if (fabs(A[r * n + k]) > fabs(A[piv * n + k])) piv = r;
    if (A[piv * n + k] == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      double t = bb[k]; bb[k] = bb[piv]; bb[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double l = A[r * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[r * n + j] -= l * A[k * n + j];
      bb[r] -= l * bb[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = bb[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
    x[k] = s / A[k * n + k];
  }
  return 0;
}

/* Central moments of f in the modified basis, in the row order above. */
void orc_central_moments(int D, const double* u, const double* f, double* a) {
  int Q = orc_Q(D);
  double M[MAXQ * MAXQ];
  moment_matrix(D, u, M);
  for (int m = 0; m < Q; ++m) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) s += M[m * Q + i] * f[i];
    a[m] = s;
  }
}

/* Exponent triple and kind of each basis row (for tests that match moments by name). */
void orc_basis_rows(int D, int* kind, int* e /* Q*3 */, int* part) {
  orc_row rows[MAXQ];
  int n = basis_rows(D, rows);
  for (int m = 0; m < n; ++m) {
    kind[m] = rows[m].kind; part[m] = rows[m].part;
    for (int al = 0; al < 3; ++al) e[3 * m + al] = rows[m].e[al];
  }
}

/* k/s/h decomposition, Sec. 2.4: each part is M^{-1} applied to the moments of
 * that part with the others set to zero. */
int orc_kbc_split(int D, const double* u, const double* f, double* k, double* s, double* h) {
  int Q = orc_Q(D);
  double M[MAXQ * MAXQ], a[MAXQ], masked[MAXQ] = {0};
  orc_row rows[MAXQ];
  basis_rows(D, rows);
  moment_matrix(D, u, M);
  for (int m = 0; m < Q; ++m) {
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) acc += M[m * Q + i] * f[i];
    a[m] = acc;
  }
  double* outs[3] = {k, s, h};
  for (int part = 0; part < 3; ++part) {
    for (int m = 0; m < Q; ++m) masked[m] = rows[m].part == part ? a[m] : 0.0;
    if (lu_solve(Q, M, masked, outs[part]) != 0) return -1;
  }
  return 0;
}

/* ---- Collision of one node, Eq. (LBGK) with the entropic mirror state (Sec. 2.4) ----
 * Inputs: pre-collision f, force F (already times dt), correction Phi, omega.
 * Outputs: post-collision fp, and optionally gamma, feq, fstar, k, s, h.
 * Returns 1 when the f*_i <= 0 guard fired, 0 otherwise, -1 on a singular basis. */
int orc_collide_node(int D, const double* f, const double* F, const double* Phi, double omega,
                     int gamma_mode, double gamma_value, double* fp, double* gamma_out,
                     double* feq_out, double* fstar_out, double* k_out, double* s_out, double* h_out) {
  int Q = orc_Q(D), c[3 * MAXQ];
  orc_velocities(D, c);
  double rho = 0.0, j[3] = {0, 0, 0}, u[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) rho += f[i];
  for (int al = 0; al < D; ++al) {
    for (int i = 0; i < Q; ++i) j[al] += c[3 * i + al] * f[i];
    u[al] = j[al] / rho;
  }
  double feq[MAXQ], fs[MAXQ], k[MAXQ], s[MAXQ], h[MAXQ];
  orc_feq(D, rho, u, feq);
  orc_fstar(D, rho, u, F, Phi, fs);
  if (orc_kbc_split(D, u, f, k, s, h) != 0) return -1;

  /* equilibrium parts: k^eq = f^eq, s^eq = h^eq = 0 (central moments of f^eq are rho, 0, ...) */
  double seq[MAXQ], heq[MAXQ];
  for (int i = 0; i < Q; ++i) { seq[i] = 0.0; heq[i] = 0.0; }

  int guard = 0;
  double gamma;
  if (gamma_mode == 1) {
    gamma = gamma_value;
  } else {
    for (int i = 0; i < Q; ++i) if (!(fs[i] > 0.0)) guard = 1;
    if (guard) {
      gamma = 2.0;
    } else {
      /* entropic scalar product <X|Y> = sum_i X_i Y_i / f*_i */
      double ds_dh = 0.0, dh_dh = 0.0;
      for (int i = 0; i < Q; ++i) {
        double ds = seq[i] - s[i], dh = heq[i] - h[i];
        ds_dh += ds * dh / fs[i];
        dh_dh += dh * dh / fs[i];
      }
      double ratio = dh_dh > 1e-300 ? ds_dh / dh_dh : 0.0;
      /* gamma/2 = 1/omega - (1 - 1/omega) <ds|dh>/<dh|dh> */
      gamma = 2.0 * (1.0 / omega - (1.0 - 1.0 / omega) * ratio);
    }
  }
  for (int i = 0; i < Q; ++i) {
    double mirr = k[i] + (2.0 * seq[i] - s[i]) + (1.0 - gamma) * h[i] + gamma * heq[i];
    fp[i] = (1.0 - omega / 2.0) * f[i] + (omega / 2.0) * mirr + (fs[i] - feq[i]);
  }
  if (gamma_out) *gamma_out = gamma;
  for (int i = 0; i < Q; ++i) {
    if (feq_out) feq_out[i] = feq[i];
    if (fstar_out) fstar_out[i] = fs[i];
    if (k_out) k_out[i] = k[i];
    if (s_out) s_out[i] = s[i];
    if (h_out) h_out[i] = h[i];
  }
  return guard;
}

/* ---- Grid helpers ---- */

static long node_index(const orc_params* p, int x, int y, int z) {
  return (long)x + (long)p->nx * ((long)y + (long)p->ny * (long)z);
}

/* Map a possibly out-of-range coordinate to an interior one for the auxiliary
 * fields: periodic wrap, or mirror about the half-way wall.  *flipped counts the
 * mirrored axes. */
static int ghost_coord(int x, int n, int bc_lo, int bc_hi, int* flipped) {
  while (x < 0 || x >= n) {
    if (x < 0) {
      if (bc_lo == 0) x += n;
      else { x = -1 - x; ++*flipped; }
    } else {
      if (bc_hi == 0) x -= n;
      else { x = 2 * n - 1 - x; ++*flipped; }
    }
  }
  return x;
}

static long aux_lookup(const orc_params* p, int x, int y, int z, int* flipped) {
  *flipped = 0;
  x = ghost_coord(x, p->nx, p->bc[0], p->bc[1], flipped);
  y = ghost_coord(y, p->ny, p->bc[2], p->bc[3], flipped);
  if (p->D == 3) z = ghost_coord(z, p->nz, p->bc[4], p->bc[5], flipped);
  else z = 0;
  return node_index(p, x, y, z);
}

static long n_nodes(const orc_params* p) { return (long)p->nx * p->ny * (p->D == 3 ? p->nz : 1); }

/* ---- Macroscopic fields and auxiliary fields of a state ---- */

/* rho, bare u = sum_i c_i f_i / rho (Sec. 2.2) and the signed pseudo-potential s*psi. */
void orc_aux_fields(const orc_params* p, const double* f, double* rho, double* u /* D*N */, double* spsi) {
  int D = p->D, Q = orc_Q(D), c[3 * MAXQ];
  long N = n_nodes(p);
  orc_velocities(D, c);
  for (long n = 0; n < N; ++n) {
    double r = 0.0;
    for (int i = 0; i < Q; ++i) r += f[i * N + n];
    rho[n] = r;
    for (int al = 0; al < D; ++al) {
      double jj = 0.0;
      for (int i = 0; i < Q; ++i) jj += c[3 * i + al] * f[i * N + n];
      u[al * N + n] = jj / r;
    }
    double sg;
    double ps = orc_psi(p, r, &sg);
    spsi[n] = sg * ps;
  }
}

/* The flux whose divergence Eq. (correction) takes:
 *   q_a = rho v_a (v_a^2 + 3 P0/rho - 3 cs^2) = rho v_a^3 (P0/rho = cs^2),
 * with v = u + F dt/(2 rho), the fluid velocity of the exact-difference forcing
 * (the velocity a node reports).  The equation writes the velocity as u, and
 * Sec. 2.2 defines u as the first moment of f over rho; under a force that
 * first moment is the fluid velocity shifted by -F dt/(2 rho).  Phi corrects a
 * Galilean defect, so it has to vanish for a fluid at rest: with the shifted
 * velocity it does not, at every interface, and the vapour density of a flat
 * interface then settles well above the Maxwell value (+36% at T/Tc = 0.6,
 * W = 6.3; under 5% with v). */
void orc_qflux(const orc_params* p, const double* rho, const double* u, const double* F, double* q /* D*N */) {
  int D = p->D;
  long N = n_nodes(p);
  for (int al = 0; al < D; ++al)
    for (long n = 0; n < N; ++n) {
      double v = u[al * N + n] + F[al * N + n] / (2.0 * rho[n]);
      q[al * N + n] = rho[n] * v * (v * v + 3.0 * CS2 - 3.0 * CS2);
    }
}

/* Force of Eq. (Kforce_final), with the physical sign (negated), plus rho*g:
 * dt F = -( 2 s psi(r) G4[psi] + kappa rho(r) G3[rho] ) + rho g,
 * G4[psi] = sum_i (w_i/cs^2) c_i (4/3 psi(r+c_i) - 1/6 psi(r+2c_i)),
 * G3[rho] = sum_i (w_i/cs^2) c_i (2 rho(r+c_i) - rho(r+2c_i)). */
void orc_force(const orc_params* p, const double* rho, const double* spsi, double* F /* D*N */) {
  int D = p->D, Q = orc_Q(D), c[3 * MAXQ];
  double w[MAXQ];
  long N = n_nodes(p);
  orc_velocities(D, c);
  orc_weights(D, w);
  int nz = D == 3 ? p->nz : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long n = node_index(p, x, y, z);
        double g4[3] = {0, 0, 0}, g3[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          int fl;
          long n1 = aux_lookup(p, x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2], &fl);
          long n2 = aux_lookup(p, x + 2 * c[3 * i], y + 2 * c[3 * i + 1], z + 2 * c[3 * i + 2], &fl);
          double psi1 = fabs(spsi[n1]), psi2 = fabs(spsi[n2]);
          for (int al = 0; al < D; ++al) {
            g4[al] += (w[i] / CS2) * c[3 * i + al] * (4.0 / 3.0 * psi1 - 1.0 / 6.0 * psi2);
            g3[al] += (w[i] / CS2) * c[3 * i + al] * (2.0 * rho[n1] - rho[n2]);
          }
        }
        for (int al = 0; al < D; ++al)
          F[al * N + n] = -(2.0 * spsi[n] * g4[al] + p->kappa * rho[n] * g3[al]) + rho[n] * p->g[al];
      }
}

/* Diagonal correction of Eq. (correction), central difference:
 *   Phi_aa = -(1 - omega/2) d_a q_a,  q from orc_qflux.
 * Sec. 2.2 gives Phi the job of correcting the diagonal of the non-equilibrium
 * momentum flux.  The lattice's third moment is sum_i f^eq_i c_ia^3 = rho u_a where
 * the continuum has rho u_a^3 + 3 P0 u_a, a defect of -q_a; the Chapman-Enskog
 * balance of the second moment then needs the source -(1 - omega/2) d_a q_a.  The
 * equation as printed has a plus sign, which doubles the defect instead of
 * cancelling it (a sound wave carried at speed 0.1 damps 9% slower, against 4.5%
 * with no correction and under 0.1% with this sign); this reading takes the sign
 * that does what the text says Phi is for. */
void orc_phi(const orc_params* p, const double* rho, const double* q, double* Phi /* D*N */) {
  int D = p->D;
  long N = n_nodes(p);
  int nz = D == 3 ? p->nz : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long n = node_index(p, x, y, z);
        double om = orc_omega(p, rho[n]);
        for (int al = 0; al < D; ++al) {
          int e[3] = {0, 0, 0};
          e[al] = 1;
          int flp, flm;
          long np_ = aux_lookup(p, x + e[0], y + e[1], z + e[2], &flp);
          long nm_ = aux_lookup(p, x - e[0], y - e[1], z - e[2], &flm);
          double qp = q[al * N + np_] * (flp ? -1.0 : 1.0);
          double qm = q[al * N + nm_] * (flm ? -1.0 : 1.0);
          Phi[al * N + n] = -(1.0 - om / 2.0) * (qp - qm) / 2.0;
        }
      }
}

/* ---- Initialisation: f = f^eq(rho0, u0) ---- */
void orc_init_equilibrium(const orc_params* p, const double* rho0, const double* u0 /* D*N */, double* f) {
  int D = p->D, Q = orc_Q(D);
  long N = n_nodes(p);
  double feq[MAXQ], u[3];
  for (long n = 0; n < N; ++n) {
    for (int al = 0; al < D; ++al) u[al] = u0[al * N + n];
    orc_feq(D, rho0[n], u, feq);
    for (int i = 0; i < Q; ++i) f[i * N + n] = feq[i];
  }
}

/* Start at rest in the reported sense: f = f^eq(rho0, u0 - F(rho0) dt/(2 rho0)), F the
 * force of the initial density field (pseudo-potential and capillary terms plus rho g),
 * so that the reported velocity u + F dt/(2 rho) of the initial state is u0. */
void orc_init_physical(const orc_params* p, const double* rho0, const double* u0 /* D*N */, double* f) {
  int D = p->D;
  long N = n_nodes(p);
  double* spsi = malloc(sizeof(double) * N);
  double* F = malloc(sizeof(double) * D * N);
  double* ub = malloc(sizeof(double) * D * N);
  for (long n = 0; n < N; ++n) {
    double sg;
    double ps = orc_psi(p, rho0[n], &sg);
    spsi[n] = sg * ps;
  }
  orc_force(p, rho0, spsi, F);
  for (int al = 0; al < D; ++al)
    for (long n = 0; n < N; ++n) ub[al * N + n] = u0[al * N + n] - F[al * N + n] / (2.0 * rho0[n]);
  orc_init_equilibrium(p, rho0, ub, f);
  free(spsi); free(F); free(ub);
}

/* Reported velocity: u + F dt / (2 rho) (exact-difference-method convention). */
void orc_macroscopic(const orc_params* p, const double* f, double* rho, double* u_phys /* D*N */) {
  int D = p->D;
  long N = n_nodes(p);
  double* ub = malloc(sizeof(double) * D * N);
  double* spsi = malloc(sizeof(double) * N);
  double* F = malloc(sizeof(double) * D * N);
  orc_aux_fields(p, f, rho, ub, spsi);
  orc_force(p, rho, spsi, F);
  for (int al = 0; al < D; ++al)
    for (long n = 0; n < N; ++n) u_phys[al * N + n] = ub[al * N + n] + F[al * N + n] / (2.0 * rho[n]);
  free(ub); free(spsi); free(F);
}

/* ---- One time step: collide every node, then stream (push) into f_out ----
 * gamma_field (nullable) receives gamma per node; returns the number of nodes
 * where the f*_i <= 0 guard fired, or -1 on failure. */
long orc_step(const orc_params* p, const double* f_in, double* f_out, double* gamma_field) {
  int D = p->D, Q = orc_Q(D), c[3 * MAXQ];
  long N = n_nodes(p);
  orc_velocities(D, c);
  double* rho = malloc(sizeof(double) * N);
  double* u = malloc(sizeof(double) * D * N);
  double* spsi = malloc(sizeof(double) * N);
  double* q = malloc(sizeof(double) * D * N);
  double* F = malloc(sizeof(double) * D * N);
  double* Phi = malloc(sizeof(double) * D * N);
  if (!rho || !u || !spsi || !q || !F || !Phi) return -1;
  orc_aux_fields(p, f_in, rho, u, spsi);
  orc_force(p, rho, spsi, F);
  orc_qflux(p, rho, u, F, q);
  orc_phi(p, rho, q, Phi);

  long guards = 0;
  int failed = 0;
  int nz = D == 3 ? p->nz : 1;
#pragma omp parallel for collapse(2) reduction(+ : guards) reduction(| : failed) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long n = node_index(p, x, y, z);
        double f[MAXQ], fp[MAXQ], Fn[3] = {0, 0, 0}, Pn[3] = {0, 0, 0}, gam;
        for (int i = 0; i < Q; ++i) f[i] = f_in[i * N + n];
        for (int al = 0; al < D; ++al) { Fn[al] = F[al * N + n]; Pn[al] = Phi[al * N + n]; }
        double om = orc_omega(p, rho[n]);
        int gr = orc_collide_node(D, f, Fn, Pn, om, p->gamma_mode, p->gamma_value, fp, &gam,
                                  NULL, NULL, NULL, NULL, NULL);
        if (gr < 0) failed = 1;
        if (gr > 0) guards += 1;
        if (gamma_field) gamma_field[n] = gam;
        /* streaming: f_i(r + c_i, t + 1) = f'_i(r, t); half-way bounce-back at walls */
        for (int i = 0; i < Q; ++i) {
          int t[3] = {x + c[3 * i], y + c[3 * i + 1], z + c[3 * i + 2]};
          int n_ax[3] = {p->nx, p->ny, nz};
          int wall = 0;
          for (int al = 0; al < D; ++al) {
            if (t[al] < 0) { if (p->bc[2 * al] == 1) wall = 1; else t[al] += n_ax[al]; }
            else if (t[al] >= n_ax[al]) { if (p->bc[2 * al + 1] == 1) wall = 1; else t[al] -= n_ax[al]; }
          }
          if (wall) f_out[(Q - 1 - i) * N + n] = fp[i];
          else f_out[i * N + node_index(p, t[0], t[1], D == 3 ? t[2] : 0)] = fp[i];
        }
      }
  free(rho); free(u); free(spsi); free(q); free(F); free(Phi);
  return failed ? -1 : guards;
}

/* Run nsteps, ping-ponging between f (in/out) and a scratch buffer. */
long orc_run(const orc_params* p, double* f, long nsteps) {
  int Q = orc_Q(p->D);
  long N = n_nodes(p);
  double* tmp = malloc(sizeof(double) * Q * N);
  if (!tmp) return -1;
  long guards = 0;
  for (long s = 0; s < nsteps; ++s) {
    long g = orc_step(p, f, tmp, NULL);
    if (g < 0) { free(tmp); return -1; }
    guards += g;
    memcpy(f, tmp, sizeof(double) * Q * N);
  }
  free(tmp);
  return guards;
}

/* Sums over the domain of rho and of the momentum sum_i c_i f_i. */
void orc_totals(const orc_params* p, const double* f, double* mass, double* mom /* 3 */) {
  int D = p->D, Q = orc_Q(D), c[3 * MAXQ];
  long N = n_nodes(p);
  orc_velocities(D, c);
  double m = 0.0, j[3] = {0, 0, 0};
  for (long n = 0; n < N; ++n)
    for (int i = 0; i < Q; ++i) {
      m += f[i * N + n];
      for (int al = 0; al < 3; ++al) j[al] += c[3 * i + al] * f[i * N + n];
    }
  *mass = m;
  for (int al = 0; al < 3; ++al) mom[al] = j[al];
}

/* Threads the OpenMP loops of orc_step use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
