// Pass 2 of a time step: force + collide + stream, one thread per interior node.
//
// A block owns a tile of Blocks<D> nodes.  It first stages the density and the
// signed pseudo-potential of the tile plus a 2-node halo in shared memory
// (coalesced rows), then each thread
//   - gathers its Q pre-collision populations (A-A parity aware),
//   - forms rho, j, Pi,
//   - evaluates the force of Eq. (Kforce_final) with the physical sign from the
//     staged tile, and Phi of Eq. (correction) from q = rho u^3,
//   - builds the one-dimensional factors of f^eq (Eq. LBMeq), f* (Eq. LBMstar)
//     and of the dual basis of the central Hermite moments (Appendix A),
//   - pass A over the populations: h = f - f^eq - s and the entropic sums
//     <ds|dh> = sum s h / f*, <dh|dh> = sum h^2 / f*,
//   - gamma from Sec. 2.4, ratio refined to float64 accuracy,
//   - pass B: recomputes f^eq, f*, s, h per population and writes
//     f' = f - omega s - (omega gamma/2) h + f* - f^eq straight to its A-A slot.
// Recomputing the cheap per-population terms in pass B instead of holding h in
// registers keeps the register count low enough for several blocks per SM.
#pragma once

#include "lbm_device.cuh"

// Minimum resident blocks per SM requested from the register allocator: two
// 256-thread blocks (128 registers) in the float32 path.
#ifndef LBM_K2_MINBLOCKS_F32
#define LBM_K2_MINBLOCKS_F32 2
#endif
#define LBM_K2_MINBLOCKS(R) (sizeof(R) == 4 ? LBM_K2_MINBLOCKS_F32 : 1)

namespace lbm {

// Reciprocal for the entropic weights 1/f*_i: one MUFU approximation in float32
// (relative error ~1 ulp, enough for sums that only set gamma), exact in float64.
template <typename R> __device__ __forceinline__ R rcp_fast(R x);
template <> __device__ __forceinline__ float rcp_fast<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <> __device__ __forceinline__ double rcp_fast<double>(double x) { return 1.0 / x; }

// gamma/2 = 1/omega - (1 - 1/omega) <ds|dh>/<dh|dh> with ds = -s, dh = -h.
template <typename R>
__device__ __forceinline__ R entropic_gamma(R sA, R sB, R om) {
  if (sizeof(R) == 8) {
    const double ratio = (double)sB > 1e-300 ? (double)sA / (double)sB : 0.0;
    const double iom = 1.0 / (double)om;
    return (R)(2.0 * iom - (2.0 - 2.0 * iom) * ratio);
  }
  const float A = (float)sA, B = (float)sB;
  double ratio = 0.0;
  if (B > 1e-37f) {
    // float quotient refined once in float64: r = q + (A - q B)/B, the residual
    // A - q B being exact in a float64 fma of float operands
    const float q = A / B;
    const double r0 = (double)q;
    const double res = fma(-r0, (double)B, (double)A);
    ratio = r0 + res * (double)__frcp_rn(B);
  }
  const double tw = 2.0 * (double)__frcp_rn((float)om);
  return (R)(tw - (2.0 - tw) * ratio);
}

template <int D, int P, typename S, typename R, typename A>
__global__ void __launch_bounds__(Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz, LBM_K2_MINBLOCKS(R))
collide_stream_kernel(DevDomain d) {
  constexpr int Q = Lattice<D>::Q;
  constexpr int BX = Blocks<D>::bx, BY = Blocks<D>::by, BZ = Blocks<D>::bz;
  constexpr int HX = BX + 4, HY = BY + 4, HZ = D == 3 ? BZ + 4 : 1;
  constexpr int HN = HX * HY * HZ;
  constexpr R cs2 = (R)(1.0 / 3.0);
  __shared__ A s_rho[HN];
  __shared__ A s_psi[HN];

  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = D == 3 ? blockIdx.z * BZ : 0;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);

  // ---- stage rho and s*psi of the tile plus halo (padded coordinates start at the tile origin)
  {
    const A* a_rho = (const A*)d.aux;
    const A* a_psi = a_rho + d.PN;
    for (int k = tid; k < HN; k += BX * BY * BZ) {
      const int hx = k % HX, hy = (k / HX) % HY, hz = k / (HX * HY);
      const int xp = x0 + hx, yp = y0 + hy, zp = z0 + hz;
      if (xp < d.px && yp < d.py && zp < d.pz) {
        const long long pn = (long long)xp + (long long)d.px * ((long long)yp + (long long)d.py * zp);
        s_rho[k] = a_rho[pn];
        s_psi[k] = a_psi[pn];
      } else {
        s_rho[k] = (A)1;
        s_psi[k] = (A)0;
      }
    }
  }
  __syncthreads();

  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + (D == 3 ? threadIdx.z : 0);
  if (x >= d.nx || y >= d.ny || z >= d.nz) return;

  const Phys<R>& ph = phys<R>(d);
  R f[Q];
  gather<D, P, S, R>(d, x, y, z, f);
  R rho, j[3], Pi[6];
  moments<D, R>(f, rho, j, Pi);
  const R inv_rho = (R)1 / rho;
  R u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = j[a] * inv_rho;

  // ---- force: dt F = -(2 s psi G4[psi] + kappa rho G3[rho]) + rho g
  const int sc = (threadIdx.x + 2) + HX * ((threadIdx.y + 2) + HY * (D == 3 ? threadIdx.z + 2 : 0));
  R g4[3] = {0, 0, 0}, g3[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i == Lattice<D>::REST) continue;
    const int o = cxi(i) + HX * (cyi(i) + HY * (D == 3 ? czi(i) : 0));
    const R psi1 = fabs((R)s_psi[sc + o]), psi2 = fabs((R)s_psi[sc + 2 * o]);
    const R r1 = (R)s_rho[sc + o], r2 = (R)s_rho[sc + 2 * o];
    const R t4 = (R)(4.0 / 3.0) * psi1 - (R)(1.0 / 6.0) * psi2;
    const R t3 = (R)2 * r1 - r2;
    const R W = (R)(3.0 * wq<D>(i));  // w_i / cs^2
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int c = cq<D>(i, a);
      if (c > 0) { g4[a] += W * t4; g3[a] += W * t3; }
      else if (c < 0) { g4[a] -= W * t4; g3[a] -= W * t3; }
    }
  }
  const R spsi_c = (R)s_psi[sc];
  R F[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a)
    F[a] = -((R)2 * spsi_c * g4[a] + ph.kappa * rho * g3[a]) + rho * ph.g[a];

  // ---- Phi_aa = (1 - omega/2) d_a q_a, central difference
  const R om = omega_of<R>(ph, rho);
  R Phi[3] = {0, 0, 0};
  {
    const A* a_q = (const A*)d.aux + 2 * d.PN;
    const long long pc = pnode_of<D>(d, x, y, z);
    const long long sy = d.px, sz = (long long)d.px * d.py;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const A* qa = a_q + a * d.PN;
      const long long e = a == 0 ? 1 : (a == 1 ? sy : sz);
      Phi[a] = ((R)1 - (R)0.5 * om) * ((R)qa[pc + e] - (R)qa[pc - e]) * (R)0.5;
    }
  }

  // ---- one-dimensional factors, index c+1: equilibrium X, extended equilibrium Xs,
  //      first-order dual d1 of the central Hermite basis
  R X[3][3], Xs[3][3], d1[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      const R ua = u[a], u2 = ua * ua;
      X[a][1] = (R)1 - cs2 - u2;
      X[a][2] = (R)0.5 * (cs2 + u2 + ua);
      X[a][0] = (R)0.5 * (cs2 + u2 - ua);
      const R xi = ua + F[a] * inv_rho;
      const R ze = cs2 + xi * xi + Phi[a] * inv_rho;
      Xs[a][1] = (R)1 - ze;
      Xs[a][2] = (R)0.5 * (ze + xi);
      Xs[a][0] = (R)0.5 * (ze - xi);
      d1[a][1] = (R)-2 * ua;
      d1[a][2] = ua + (R)0.5;
      d1[a][0] = ua - (R)0.5;
    } else {
      X[a][0] = X[a][2] = Xs[a][0] = Xs[a][2] = d1[a][0] = d1[a][1] = d1[a][2] = 0;
      X[a][1] = Xs[a][1] = 1;
    }
  }
  // second-order central Hermite moments; the shear part keeps the off-diagonals
  // and the deviatoric diagonal a_aa - trace/D
  const R axy = Pi[3] - rho * u[0] * u[1];
  const R axz = D == 3 ? Pi[4] - rho * u[0] * u[2] : (R)0;
  const R ayz = D == 3 ? Pi[5] - rho * u[1] * u[2] : (R)0;
  R adiag[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) adiag[a] = a < D ? Pi[a] - rho * u[a] * u[a] - rho * cs2 : (R)0;
  const R tr = (adiag[0] + adiag[1] + adiag[2]) * (R)(1.0 / D);
  R dev[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) dev[a] = a < D ? adiag[a] - tr : (R)0;

  // Row coefficients for the populations sharing (cy, cz): f^eq = ryz X_x, f* = rsyz Xs_x,
  // s = d0_x C0 + d1_x C1 + d2_x C2 with d2 = {-1 at c = 0, 1/2 at c = +-1}.
  struct Row { R ryz, rsyz, C0, C1, C2; };
  auto row = [&](int iy, int iz) {
    const R Z0 = D == 3 ? X[2][iz] : (R)1, Zs = D == 3 ? Xs[2][iz] : (R)1;
    const R Z1 = D == 3 ? d1[2][iz] : (R)0;
    const R Z2 = D == 3 ? (iz == 1 ? (R)-1 : (R)0.5) : (R)0;
    const R Y0 = X[1][iy], Y1 = d1[1][iy], Y2 = iy == 1 ? (R)-1 : (R)0.5;
    Row r;
    r.ryz = rho * Y0 * Z0;
    r.rsyz = rho * Xs[1][iy] * Zs;
    r.C0 = ayz * Y1 * Z1 + dev[1] * Y2 * Z0 + (D == 3 ? dev[2] * Y0 * Z2 : (R)0);
    r.C1 = axy * Y1 * Z0 + (D == 3 ? axz * Y0 * Z1 : (R)0);
    r.C2 = dev[0] * Y0 * Z0;
    return r;
  };

  // ---- pass A: entropic sums
  R sA = 0, sB = 0;
  bool neg = false;
#pragma unroll
  for (int iz = 0; iz < (D == 3 ? 3 : 1); ++iz) {
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      const Row r = row(iy, iz);
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        const int i = ix + 3 * iy + 9 * iz;
        const R feq = r.ryz * X[0][ix];
        const R fst = r.rsyz * Xs[0][ix];
        const R s = X[0][ix] * r.C0 + d1[0][ix] * r.C1 + (ix == 1 ? -r.C2 : (R)0.5 * r.C2);
        const R hh = f[i] - feq - s;
        neg |= !(fst > (R)0);
        const R hr = hh * rcp_fast<R>(fst);
        sA += s * hr;
        sB += hh * hr;
      }
    }
  }

  R gamma;
  if (d.gamma_mode == 1) {
    gamma = ph.gamma_value;
  } else if (neg) {
    gamma = (R)2;
    atomicAdd(d.guards, 1ull);
  } else {
    gamma = entropic_gamma<R>(sA, sB, om);
  }
  const long long n = node_of(d, x, y, z);
  const bool inner = interior<D>(d, x, y, z);
  S* Fo = (S*)d.f;
  if (d.gamma_out) d.gamma_out[n] = (float)gamma;

  // ---- pass B: relax and stream, f' = f - omega s - (omega gamma/2) h + f* - f^eq
  const R ch = (R)0.5 * om * gamma;
#pragma unroll
  for (int iz = 0; iz < (D == 3 ? 3 : 1); ++iz) {
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      const Row r = row(iy, iz);
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        const int i = ix + 3 * iy + 9 * iz;
        const R feq = r.ryz * X[0][ix];
        const R fst = r.rsyz * Xs[0][ix];
        const R s = X[0][ix] * r.C0 + d1[0][ix] * r.C1 + (ix == 1 ? -r.C2 : (R)0.5 * r.C2);
        const R hh = f[i] - feq - s;
        st_pop<S, R>(Fo + dst_slot<D, P>(d, inner, x, y, z, n, i), f[i] - om * s - ch * hh + (fst - feq));
      }
    }
  }
}

}  // namespace lbm
