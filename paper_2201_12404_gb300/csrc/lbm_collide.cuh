// Pass 2 of a time step: force + collide + stream, one thread per interior node.
//
// A block owns a tile of Blocks<D> nodes.  One thread starts a TMA bulk-tensor
// copy of the density and the signed pseudo-potential of the tile plus a 2-node
// halo into shared memory; while it is in flight every thread gathers its
// populations, then waits on the copy's mbarrier (bounded).  Each thread
//   - gathers its Q pre-collision populations (A-A parity aware) into registers,
//   - forms rho, j, Pi from row sums (the three populations sharing (cy, cz)),
//   - evaluates the force of Eq. (Kforce_final) with the physical sign from the
//     staged tile, and Phi of Eq. (correction) from q = rho u^3,
//   - builds the one-dimensional factors of f^eq (Eq. LBMeq), f* (Eq. LBMstar)
//     and of the dual basis of the central Hermite moments (Appendix A),
//   - pass A: h = f - f^eq - s per population, the entropic sums
//     <ds|dh> = sum s h / f*, <dh|dh> = sum h^2 / f*, and the gamma-free part
//     g = f - omega s + f* - f^eq in place of f; h goes to shared memory,
//   - gamma from Sec. 2.4, ratio refined to float64 accuracy,
//   - pass B: f' = g - (omega gamma/2) h, written to the A-A slots.
// Nodes whose links all stay inside the domain take a branch with plain
// offsets for the gather and the write; the others resolve wrap and walls.
#pragma once

#include <cuda.h>

#include "lbm_device.cuh"

// Minimum resident 256-thread blocks per SM requested from the register
// allocator in the float32 path.
#ifndef LBM_K2_MINBLOCKS_F32
#define LBM_K2_MINBLOCKS_F32 3
#endif
#define LBM_K2_MINBLOCKS(R) (sizeof(R) == 4 ? LBM_K2_MINBLOCKS_F32 : 1)

namespace lbm {

// ---- TMA and mbarrier helpers (inline PTX) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}

// Wait for phase `parity` of the barrier, at most `limit` polls; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Tile copy of a D-dimensional halo box of the two staged fields (rank D + 1).
template <int D>
__device__ __forceinline__ void tma_load_tile(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z) {
  if (D == 3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
        : "memory");
  } else {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
  }
}

// Polls of the tile barrier before a block reports a timeout (bit 1 of the
// error word) and stops; far above any real copy latency.
constexpr uint32_t kTileWaitPolls = 1u << 24;

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

// Dynamic shared memory of the kernel: h_i of every node of the tile.
template <int D, typename R, int NT = Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz>
constexpr size_t collide_dyn_smem() {
  return (size_t)Lattice<D>::Q * NT * sizeof(R);
}

// Halo-tile extents of a BX x BY x BZ tile.
template <int D, int BX, int BY, int BZ> struct Halo {
  static constexpr int HX = BX + 4, HY = BY + 4, HZ = D == 3 ? BZ + 4 : 1;
  static constexpr int HN = HX * HY * HZ;
};

// One tile of pass 2 whose origin is (x0, y0, z0), run by the BX*BY*BZ threads of
// the block.  kTma: the halo tile comes from a TMA copy of the tensor map `map`,
// completed on `bar` (phase `phase`); otherwise each warp loads halo rows.
// s_aux holds 2*HN values, s_h Q*BX*BY*BZ.
template <int D, int BX, int BY, int BZ, int P, typename S, typename R, typename A, bool kTma>
__device__ __forceinline__ void collide_tile(const DevDomain& d, const CUtensorMap* map, int x0, int y0, int z0,
                                             A* s_aux, R* s_h, unsigned long long* bar, uint32_t phase) {
  constexpr int Q = Lattice<D>::Q;
  constexpr int NT = BX * BY * BZ;
  constexpr int HX = Halo<D, BX, BY, BZ>::HX, HY = Halo<D, BX, BY, BZ>::HY, HZ = Halo<D, BX, BY, BZ>::HZ;
  constexpr int HN = HX * HY * HZ;
  constexpr R cs2 = (R)(1.0 / 3.0);
  const A* s_rho = s_aux;
  const A* s_psi = s_aux + HN;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const Phys<R>& ph = phys<R>(d);

  // ---- stage rho and s*psi of the tile plus halo; padded coordinates of the halo
  //      origin are the tile origin itself
  if (kTma) {
    // x0 is a multiple of BX (>= 32), so the box starts 16-byte aligned
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, (uint32_t)(2 * HN * sizeof(A)));
      tma_load_tile<D>(s_aux, map, bar, x0, y0, z0);
    }
  } else {
    const A* a_rho = (const A*)d.aux;
    const A* a_psi = a_rho + d.PN;
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < HY * HZ; r += NT / 32) {
      const int yp = y0 + r % HY, zp = z0 + r / HY;
      const bool row_ok = yp < d.py && zp < d.pz;
      const long long base = (long long)d.px * ((long long)yp + (long long)d.py * zp) + x0;
      for (int hx = lane; hx < HX; hx += 32) {
        const bool ok = row_ok && x0 + hx < d.px;
        s_aux[r * HX + hx] = ok ? a_rho[base + hx] : (A)1;
        s_aux[HN + r * HX + hx] = ok ? a_psi[base + hx] : (A)0;
      }
    }
    __syncthreads();
  }

  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + (D == 3 ? threadIdx.z : 0);
  const bool active = x < d.nx && y < d.ny && z < d.nz;
  const long long n = node_of(d, x, y, z);
  const bool inner = interior<D>(d, x, y, z);

  R f[Q];
  if (active) gather<D, P, S, R>(d, x, y, z, f);
  if (kTma) {
    // every thread waits, so that the block cannot retire while the copy is in flight
    if (!mbar_wait_bounded(bar, phase, kTileWaitPolls)) {
      if (tid == 0) atomicOr(d.flags, 2u);
      mbar_wait_bounded(bar, phase, kTileWaitPolls);
      return;
    }
  }
  if (!active) return;

  // ---- rho, j, Pi from row sums: r0 = f- + f0 + f+, r1 = f+ - f-, r2 = f+ + f-
  R rho = 0, jx = 0, jy = 0, jz = 0, Pxx = 0, Pyy = 0, Pzz = 0, Pxy = 0, Pxz = 0, Pyz = 0;
#pragma unroll
  for (int row = 0; row < Q / 3; ++row) {
    const int cy = row % 3 - 1, cz = D == 3 ? row / 3 - 1 : 0;
    const R fm = f[3 * row], f0 = f[3 * row + 1], fp = f[3 * row + 2];
    const R r2 = fm + fp, r0 = r2 + f0, r1 = fp - fm;
    rho += r0; jx += r1; Pxx += r2;
    if (cy != 0) { jy += cy > 0 ? r0 : -r0; Pxy += cy > 0 ? r1 : -r1; Pyy += r0; }
    if (cz != 0) { jz += cz > 0 ? r0 : -r0; Pxz += cz > 0 ? r1 : -r1; Pzz += r0; }
    if (cy * cz != 0) Pyz += cy * cz > 0 ? r0 : -r0;
  }
  const R inv_rho = (R)1 / rho;
  const R u[3] = {jx * inv_rho, jy * inv_rho, jz * inv_rho};

  // ---- force: dt F = -(2 s psi G4[psi] + kappa rho G3[rho]) + rho g, sums over the
  //      lattice links row by row with weights w_i/cs^2 = 3 w(cx) w(cy) w(cz)
  const int sc = (threadIdx.x + 2) + HX * ((threadIdx.y + 2) + HY * (D == 3 ? threadIdx.z + 2 : 0));
  R g4x = 0, g4y = 0, g4z = 0, g3x = 0, g3y = 0, g3z = 0;
#pragma unroll
  for (int row = 0; row < Q / 3; ++row) {
    const int cy = row % 3 - 1, cz = D == 3 ? row / 3 - 1 : 0;
    const R wyz = (cy == 0 ? (R)2 : (R)0.5) * (D == 3 ? (cz == 0 ? (R)(2.0 / 3.0) : (R)(1.0 / 6.0)) : (R)1);
    const int orow = HX * (cy + HY * cz);
    const A* pp = s_psi + sc + orow;
    const A* pr = s_rho + sc + orow;
    const A* pp2 = s_psi + sc + 2 * orow;
    const A* pr2 = s_rho + sc + 2 * orow;
    // t4 and t3 summed over the row with the x weights 1/6, 2/3, 1/6 and signs -1, 0, +1
    R rowm4, row04, rowp4, rowm3, row03, rowp3;
    {
      const R pm = fabs((R)pp[-1]), p0 = fabs((R)pp[0]), pq = fabs((R)pp[1]);
      const R pm2 = fabs((R)pp2[-2]), p02 = fabs((R)pp2[0]), pq2 = fabs((R)pp2[2]);
      rowm4 = (R)(4.0 / 3.0) * pm - (R)(1.0 / 6.0) * pm2;
      row04 = (row == (Q / 3) / 2) ? (R)0 : (R)(4.0 / 3.0) * p0 - (R)(1.0 / 6.0) * p02;
      rowp4 = (R)(4.0 / 3.0) * pq - (R)(1.0 / 6.0) * pq2;
      rowm3 = (R)2 * (R)pr[-1] - (R)pr2[-2];
      row03 = (row == (Q / 3) / 2) ? (R)0 : (R)2 * (R)pr[0] - (R)pr2[0];
      rowp3 = (R)2 * (R)pr[1] - (R)pr2[2];
    }
    // x-component: (+1) - (-1) with weight 1/6; y, z: weighted row sum 1/6, 2/3, 1/6
    g4x += wyz * (R)(1.0 / 6.0) * (rowp4 - rowm4);
    g3x += wyz * (R)(1.0 / 6.0) * (rowp3 - rowm3);
    const R s4 = wyz * ((R)(1.0 / 6.0) * (rowp4 + rowm4) + (R)(2.0 / 3.0) * row04);
    const R s3 = wyz * ((R)(1.0 / 6.0) * (rowp3 + rowm3) + (R)(2.0 / 3.0) * row03);
    if (cy != 0) { g4y += cy > 0 ? s4 : -s4; g3y += cy > 0 ? s3 : -s3; }
    if (D == 3 && cz != 0) { g4z += cz > 0 ? s4 : -s4; g3z += cz > 0 ? s3 : -s3; }
  }
  const R spsi_c = (R)s_psi[sc];
  R F[3];
  F[0] = -((R)2 * spsi_c * g4x + ph.kappa * rho * g3x) + rho * ph.g[0];
  F[1] = -((R)2 * spsi_c * g4y + ph.kappa * rho * g3y) + rho * ph.g[1];
  F[2] = D == 3 ? -((R)2 * spsi_c * g4z + ph.kappa * rho * g3z) + rho * ph.g[2] : (R)0;

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
  // per-axis velocity, its square, and the extended-equilibrium variables xi*, zeta*
  R uu[3], ua2[3], xs[3], zs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    uu[a] = a < D ? u[a] : (R)0;
    ua2[a] = uu[a] * uu[a];
    xs[a] = a < D ? uu[a] + F[a] * inv_rho : (R)0;
    zs[a] = a < D ? cs2 + xs[a] * xs[a] + Phi[a] * inv_rho : cs2;
  }
  // factor of index k = c+1 along one axis: equilibrium, extended equilibrium, first-order dual
  auto eqf = [&](int k, int a) { return k == 1 ? (R)1 - cs2 - ua2[a] : (R)0.5 * (cs2 + ua2[a] + (k == 2 ? uu[a] : -uu[a])); };
  auto stf = [&](int k, int a) { return k == 1 ? (R)1 - zs[a] : (R)0.5 * (zs[a] + (k == 2 ? xs[a] : -xs[a])); };
  auto d1f = [&](int k, int a) { return k == 1 ? (R)-2 * uu[a] : uu[a] + (k == 2 ? (R)0.5 : (R)-0.5); };
  // x-axis factors, used for every population
  R X[3], Xs[3], d1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    X[k] = eqf(k, 0);
    Xs[k] = stf(k, 0);
    d1[k] = d1f(k, 0);
  }
  // second-order central Hermite moments; the shear part keeps the off-diagonals
  // and the deviatoric diagonal a_aa - trace/D
  const R axy = Pxy - rho * u[0] * u[1];
  const R axz = D == 3 ? Pxz - rho * u[0] * u[2] : (R)0;
  const R ayz = D == 3 ? Pyz - rho * u[1] * u[2] : (R)0;
  const R adx = Pxx - rho * u[0] * u[0] - rho * cs2;
  const R ady = Pyy - rho * u[1] * u[1] - rho * cs2;
  const R adz = D == 3 ? Pzz - rho * u[2] * u[2] - rho * cs2 : (R)0;
  const R tr = (adx + ady + adz) * (R)(1.0 / D);
  const R devx = adx - tr, devy = ady - tr, devz = D == 3 ? adz - tr : (R)0;

  // Row coefficients for the populations sharing (cy, cz): f^eq = ryz X_x, f* = rsyz Xs_x,
  // s = d0_x C0 + d1_x C1 + d2_x C2 with d2 = {-1 at c = 0, 1/2 at c = +-1}.
  struct Row { R ryz, rsyz, C0, C1, C2; };
  auto row_coef = [&](int iy, int iz) {
    const R Z0 = D == 3 ? eqf(iz, 2) : (R)1, Zs = D == 3 ? stf(iz, 2) : (R)1;
    const R Z1 = D == 3 ? d1f(iz, 2) : (R)0;
    const R Z2 = D == 3 ? (iz == 1 ? (R)-1 : (R)0.5) : (R)0;
    const R Y0 = eqf(iy, 1), Y1 = d1f(iy, 1), Y2 = iy == 1 ? (R)-1 : (R)0.5;
    Row r;
    r.ryz = rho * Y0 * Z0;
    r.rsyz = rho * stf(iy, 1) * Zs;
    r.C0 = ayz * Y1 * Z1 + devy * Y2 * Z0 + (D == 3 ? devz * Y0 * Z2 : (R)0);
    r.C1 = axy * Y1 * Z0 + (D == 3 ? axz * Y0 * Z1 : (R)0);
    r.C2 = devx * Y0 * Z0;
    return r;
  };

  // ---- pass A: entropic sums, h to shared memory, g = f - omega s + f* - f^eq
  //      = h + (1 - omega) s + f* in place of f.  Every f*_i is positive exactly when
  //      rho and the nine one-dimensional factors Xs are (each axis's three factors
  //      sum to one, so they cannot all be negative).  The weight 1/f*_i factors as
  //      1/(rho Ys Zs) times 1/Xs, so a row's three terms are summed with the x
  //      reciprocals and scaled once by the row's; partial sums per iy keep the
  //      dependency chains short.
  R fmin = rho;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) fmin = fmin < stf(k, a) ? fmin : stf(k, a);
  const R one_m_om = (R)1 - om;
  R sAy[3] = {0, 0, 0}, sBy[3] = {0, 0, 0};
  R iXs[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) iXs[k] = rcp_fast<R>(Xs[k]);
#pragma unroll
  for (int iz = 0; iz < (D == 3 ? 3 : 1); ++iz) {
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      const Row r = row_coef(iy, iz);
      R tA = 0, tB = 0;
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        const int i = ix + 3 * iy + 9 * iz;
        const R feq = r.ryz * X[ix];
        const R fst = r.rsyz * Xs[ix];
        const R s = X[ix] * r.C0 + d1[ix] * r.C1 + (ix == 1 ? -r.C2 : (R)0.5 * r.C2);
        const R hh = f[i] - feq - s;
        const R hr = hh * iXs[ix];
        tA += s * hr;
        tB += hh * hr;
        s_h[i * NT + tid] = hh;
        f[i] = hh + one_m_om * s + fst;
      }
      const R irs = rcp_fast<R>(r.rsyz);
      sAy[iy] += irs * tA;
      sBy[iy] += irs * tB;
    }
  }
  const R sA = (sAy[0] + sAy[1]) + sAy[2], sB = (sBy[0] + sBy[1]) + sBy[2];

  R gamma;
  if (d.gamma_mode == 1) {
    gamma = ph.gamma_value;
  } else if (!(fmin > (R)0)) {
    gamma = (R)2;
    atomicAdd(d.guards, 1ull);
  } else {
    gamma = entropic_gamma<R>(sA, sB, om);
  }
  if (d.gamma_out) d.gamma_out[n] = (float)gamma;

  // ---- pass B: f' = g - (omega gamma/2) h
  const R ch = (R)0.5 * om * gamma;
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] -= ch * s_h[i * NT + tid];

  // ---- float16-deviation storage: encode against this node's density, which the
  //      next step reads back as the writer density of every slot written here
  if constexpr (DevStorage<S>::value) {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = f[i] * (inv_rho * (R)(1.0 / wq<D>(i))) - (R)1;
    d.rho_w[1 - P][n] = (float)rho;
  }

  // ---- stream: A-A write
  S* Fo = (S*)d.f;
  if (inner) {
#pragma unroll
    for (int i = 0; i < Q; ++i) st_pop<S, R>(Fo + dst_slot<D, P>(d, true, x, y, z, n, i), f[i]);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) st_pop<S, R>(Fo + dst_slot<D, P>(d, false, x, y, z, n, i), f[i]);
  }
}

template <int D, int P, typename S, typename R, typename A>
__global__ void __launch_bounds__(Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz, LBM_K2_MINBLOCKS(R))
collide_stream_kernel(DevDomain d, const __grid_constant__ CUtensorMap aux_map) {
  constexpr int BX = Blocks<D>::bx, BY = Blocks<D>::by, BZ = Blocks<D>::bz;
  __shared__ __align__(128) A s_aux[2 * Halo<D, BX, BY, BZ>::HN];  // [field][z][y][x]: rho, then s*psi
  __shared__ __align__(8) unsigned long long tile_bar;
  // higher-order part h_i of every node of the tile, [i][thread] (dynamic: above 48 KB in float64)
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  if (tid == 0) mbar_init(&tile_bar, 1);
  __syncthreads();
  collide_tile<D, BX, BY, BZ, P, S, R, A, true>(d, &aux_map, blockIdx.x * BX, blockIdx.y * BY,
                                                 D == 3 ? blockIdx.z * BZ : 0, s_aux, (R*)smem_dyn, &tile_bar, 0);
}

}  // namespace lbm
