// Pass 2 of a time step: force + collide + stream, one thread per interior node.
//
// A block owns a tile of Blocks<D> nodes.  One thread starts TMA bulk-tensor
// copies of the q planes of the tile plus a 1-node halo (2 along x) into shared
// memory; while they are in flight every thread loads its node's force (Eq.
// Kforce_final, physical sign, written by pass 1b) and gathers its populations,
// then waits on the copies' mbarrier (bounded).  Each thread
//   - gathers its Q pre-collision populations (A-A parity aware) into registers,
//   - forms rho, j, Pi from row sums (the three populations sharing (cy, cz)),
//   - evaluates Phi of Eq. (correction) from the staged q = rho v^3 (with the
//     sign that cancels the lattice's third-moment defect),
//   - builds the one-dimensional factors of f^eq (Eq. LBMeq), f* (Eq. LBMstar)
//     and of the dual basis of the central Hermite moments (Appendix A),
//   - pass A: h = f - f^eq - s per population, the entropic sums
//     <ds|dh> = sum s h / f*, <dh|dh> = sum h^2 / f*, and the gamma-free part
//     g = f - omega s + f* - f^eq in place of f; h goes to shared memory,
//   - gamma from Sec. 2.4, the float32 quotient and its residual summed in float64,
//   - pass B: f' = g - (omega gamma/2) h, written to the A-A slots.
// Nodes whose links all stay inside the domain take a branch with plain
// offsets for the gather and the write; the others resolve wrap and walls.
#pragma once

#include <cuda.h>

#include "lbm_device.cuh"

// Minimum resident blocks per SM requested from the register allocator in the
// float32 path.  D3Q27: ten 64-thread blocks, i.e. up to 96 registers and no
// spills, 20 warps per SM (512x512x256 impact, pass 2 per launch: 2.72 ms, against
// 3.03 at twelve blocks and 80 registers with ~90 bytes spilled, 2.99 at eight and
// ~112 registers).  D2Q9: five 256-thread blocks, whose nine populations a node
// fit in 48 registers (2048x1024 impact: pass 2 57.6 us per launch at three
// blocks, 49.5 at four, 46.9 at five).
#ifndef LBM_K2_MINBLOCKS_F32
#define LBM_K2_MINBLOCKS_F32 10
#endif
#ifndef LBM_K2_MINBLOCKS_F32_2D
#define LBM_K2_MINBLOCKS_F32_2D 5
#endif
#define LBM_K2_MINBLOCKS(R, D) (sizeof(R) == 4 ? ((D) == 2 ? LBM_K2_MINBLOCKS_F32_2D : LBM_K2_MINBLOCKS_F32) : 1)

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

// Tile copy of a D-dimensional halo box of (rho, psi) pairs: float32 pairs are
// 8-byte elements of a rank-D map, float64 pairs the innermost dimension (2) of a
// rank-(D + 1) map.
template <int D, typename A>
__device__ __forceinline__ void tma_load_tile(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z) {
  if (sizeof(A) == 4 && D == 3) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
  } else if (sizeof(A) == 4) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
  } else if (D == 3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(0), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
  } else {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(0), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
  }
}

// Tile copy of the q_a box of axis a (rank-(D + 1) map over the q planes).
template <int D>
__device__ __forceinline__ void tma_load_q(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z, int a) {
  if (D == 3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(a), "r"(smem_u32(bar))
        : "memory");
  } else {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(a), "r"(smem_u32(bar))
        : "memory");
  }
}

// Asynchronous 4- or 8-byte copy global -> shared (cp.async; a population is
// one 4- or 8-byte word), completion tracked per thread by commit/wait groups.
template <int kBytes>
__device__ __forceinline__ void cp_async_word(void* smem, const void* gmem) {
  static_assert(kBytes == 4 || kBytes == 8, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(smem)), "l"(gmem), "n"(kBytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Orders this thread's earlier shared-memory accesses (made visible to it by a
// barrier) before its later TMA writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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
  float ratio = 0.0f;
  if (B > 1e-37f) {
    // the float32 quotient q and its correction e = (A - q B)/B, the residual being
    // exact in one float32 fma; q + e is formed in float64 and rounded once, which
    // gives the ratio to within the rounding of its float32 result
    const float q = A / B;
    const float e = fmaf(-q, B, A) * __frcp_rn(B);
    ratio = (float)((double)q + (double)e);
  }
  // gamma/2 = 1/omega + (1/omega - 1) ratio
  const float iom = __frcp_rn((float)om);
  return (R)(2.0f * fmaf(iom - 1.0f, ratio, iom));
}

// Dynamic shared memory of the persistent kernel: h_i and the staged
// populations of every node of the tile.
template <int D, typename S, typename R, int NT = Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz>
constexpr size_t persistent_dyn_smem() {
  return (size_t)Lattice<D>::Q * NT * (sizeof(R) + sizeof(S));
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
  // q_a box: the tile with one node around it in y and z, two in x (alignment)
  static constexpr int QX = BX + 4, QY = BY + 2, QZ = D == 3 ? BZ + 2 : 1;
  static constexpr int QB = QX * QY * QZ;
  // elements of type T between consecutive q boxes in shared memory (128-byte steps)
  template <typename T> static __host__ __device__ constexpr int qstride() { return (int)((QB * sizeof(T) + 127) / 128 * 128 / sizeof(T)); }
};

// Issue the TMA copies of the D q_a boxes of one tile into s_q, all completing on
// `bar`.  Called by one thread.
template <int D, int BX, int BY, int BZ, typename A>
__device__ __forceinline__ void tma_load_q_boxes(const TileMaps* maps, A* s_q, unsigned long long* bar, int x0, int y0,
                                                 int z0) {
  using H = Halo<D, BX, BY, BZ>;
  mbar_arrive_expect_tx(bar, (uint32_t)(D * H::QB * sizeof(A)));
#pragma unroll
  for (int a = 0; a < D; ++a)
    tma_load_q<D>(s_q + a * H::template qstride<A>(), &maps->q, bar, x0, y0 + 1, D == 3 ? z0 + 1 : 0, a);
}

// Rows of populations sharing (cy, cz), paired for two-lane arithmetic.  Pair
// k < kYPairs holds the rows cy = -1 (lane x) and cy = +1 (lane y) at cz = k - 1
// (2-D: cz = 0); in 3-D pair 3 holds the rows cz = -1 and cz = +1 at cy = 0.  The
// row cy = cz = 0 stays single.  Both lanes of a pair have the same weight w_i.
template <int D> struct RowPairs {
  static constexpr int kYPairs = D == 3 ? 3 : 1;
  static constexpr int kPairs = D == 3 ? 4 : 1;
  // population index of lane `lane` (0: x, 1: y) of pair k at x index ix = cx + 1
  static __host__ __device__ constexpr int pop(int k, int lane, int ix) {
    return D == 2 ? ix + 6 * lane : (k < 3 ? ix + 6 * lane + 9 * k : ix + 3 + 18 * lane);
  }
  static __host__ __device__ constexpr int single(int ix) { return D == 3 ? ix + 12 : ix + 3; }
};

struct NoHooks {
  __device__ void prefetch() const {}
  __device__ void aux() const {}
};

// Moments of one node: rho, j and the second moments Pi.
template <typename R> struct NodeMoments {
  R rho, jx, jy, jz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
};

// Pairs the rows of the node's populations f (fp: pairs, fs: the single row,
// indexed by ix = cx + 1) and forms rho, j, Pi from row sums:
// r0 = f- + f0 + f+, r1 = f+ - f-, r2 = f+ + f-.
template <int D, typename R>
__device__ __forceinline__ void row_moments(const R (&f)[Lattice<D>::Q], Two<R> (&fp)[RowPairs<D>::kPairs][3],
                                            R (&fs)[3], NodeMoments<R>& m) {
  constexpr int NY = RowPairs<D>::kYPairs, NP = RowPairs<D>::kPairs;
  using RP = RowPairs<D>;
  using R2 = Two<R>;
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) {
#pragma unroll
    for (int k = 0; k < NP; ++k) fp[k][ix] = two<R>(f[RP::pop(k, 0, ix)], f[RP::pop(k, 1, ix)]);
    fs[ix] = f[RP::single(ix)];
  }
  const R2 zero2 = both<R>((R)0), sgn = two<R>((R)-1, (R)1);
  R2 RHO = zero2, JX = zero2, PXX = zero2, JY = zero2, PXY = zero2, PYY = zero2;
  R2 JZ = zero2, PXZ = zero2, PZZ = zero2, PYZ = zero2;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const R2 r2 = add2(fp[k][0], fp[k][2]), r0 = add2(r2, fp[k][1]), r1 = sub2(fp[k][2], fp[k][0]);
    RHO = add2(RHO, r0); JX = add2(JX, r1); PXX = add2(PXX, r2);
    if (k < NY) {  // lanes cy = -1, +1 at cz = k - 1
      JY = fma2(sgn, r0, JY); PXY = fma2(sgn, r1, PXY); PYY = add2(PYY, r0);
      if (D == 3 && k != 1) {
        if (k == 0) { JZ = sub2(JZ, r0); PXZ = sub2(PXZ, r1); PYZ = fma2(two<R>((R)1, (R)-1), r0, PYZ); }
        else { JZ = add2(JZ, r0); PXZ = add2(PXZ, r1); PYZ = fma2(sgn, r0, PYZ); }
        PZZ = add2(PZZ, r0);
      }
    } else {       // lanes cz = -1, +1 at cy = 0
      JZ = fma2(sgn, r0, JZ); PXZ = fma2(sgn, r1, PXZ); PZZ = add2(PZZ, r0);
    }
  }
  const R s2 = fs[0] + fs[2], s0 = s2 + fs[1], s1 = fs[2] - fs[0];
  m.rho = (RHO.x + RHO.y) + s0;
  m.jx = (JX.x + JX.y) + s1;
  m.Pxx = (PXX.x + PXX.y) + s2;
  m.jy = JY.x + JY.y; m.Pxy = PXY.x + PXY.y; m.Pyy = PYY.x + PYY.y;
  m.jz = D == 3 ? JZ.x + JZ.y : (R)0;
  m.Pxz = D == 3 ? PXZ.x + PXZ.y : (R)0;
  m.Pzz = D == 3 ? PZZ.x + PZZ.y : (R)0;
  m.Pyz = D == 3 ? PYZ.x + PYZ.y : (R)0;
}

// The force from the node's gradient sums G = (G3[rho], G4[psi]) per axis (the
// class-weighted link sums of stencil_force, before the common (2, 4/3)) and the
// node's own (rho, psi) pair c: F = rho g - (2 kappa rho, (8/3) s psi) . G.
template <int D, typename R, typename A>
__device__ __forceinline__ void force_from_gradients(const Phys<R>& ph, R rho, const Two<A>& c, const Two<R>& GX,
                                                     const Two<R>& GY, const Two<R>& GZ, R (&F)[3]) {
  // s psi at the node: psi from the stencil, s from the node's density there
  const R spsi_c = psi_sign<R>(ph, (R)c.x) * (R)c.y;
  const Two<R> wf = two<R>((R)2 * ph.kappa * rho, (R)(8.0 / 3.0) * spsi_c);  // (kappa rho, 2 s psi) * (2, 4/3)
  const Two<R> tx = mul2(wf, GX), ty = mul2(wf, GY), tz = mul2(wf, GZ);
  F[0] = rho * ph.g[0] - (tx.x + tx.y);
  F[1] = rho * ph.g[1] - (ty.x + ty.y);
  F[2] = D == 3 ? rho * ph.g[2] - (tz.x + tz.y) : (R)0;
}

// Force of Eq. (Kforce_final) with the physical sign, plus rho g:
// dt F = -(2 s psi G4[psi] + kappa rho G3[rho]) + rho g, from the (rho, psi) pairs
// at(dx, dy, dz) of the node's radius-2 stencil (at(0, 0, 0) the node itself).
// The lattice links are summed row by row with weights w_i/cs^2 = 3 w(cx) w(cy) w(cz).
// The two lanes carry G3[rho] (x) and G4[psi] (y): a link term 2 rho(r+c) - rho(r+2c)
// and (4/3) psi(r+c) - (1/6) psi(r+2c) is (2, 4/3) times v(r+c) + (-1/2, -1/8) v(r+2c),
// the common (2, 4/3) applied once at the end.  Rows are summed by weight class
// (w_y w_z: centre 2 (2/3), edge 1/2 (2/3) or 2 (1/6), corner 1/2 (1/6); 2-D: 2,
// 1/2) and the weights applied once: GX = (1/6) sum w_yz (t(+1) - t(-1)), and the
// y/z components use u = t(-1) + t(+1) + 4 t(0) = 6 x (the row's weighted sum over cx).
template <int D, typename R, typename A, typename AuxAt>
__device__ __forceinline__ void stencil_force(const Phys<R>& ph, R rho, const AuxAt& at, R (&F)[3]) {
  constexpr int Q = Lattice<D>::Q;
  using R2 = Two<R>;
  const R2 zero2 = both<R>((R)0);
  const R2 cb = two<R>((R)-0.5, (R)-0.125), four = both<R>((R)4);
  auto v = [](const Two<A>& a) { return two<R>((R)a.x, (R)a.y); };
  R2 DXc = zero2, DXe = zero2, DXk = zero2, YE = zero2, YK = zero2, ZE = zero2, ZK = zero2;
#pragma unroll
  for (int row = 0; row < Q / 3; ++row) {
    const int cy = row % 3 - 1, cz = D == 3 ? row / 3 - 1 : 0;
    const R2 tm = fma2(cb, v(at(-2, 2 * cy, 2 * cz)), v(at(-1, cy, cz)));
    const R2 tp = fma2(cb, v(at(2, 2 * cy, 2 * cz)), v(at(1, cy, cz)));
    const R2 dx = sub2(tp, tm);
    if (cy == 0 && cz == 0) {
      DXc = add2(DXc, dx);  // the centre row adds nothing to the y and z components
      continue;
    }
    if (cy != 0 && cz != 0) DXk = add2(DXk, dx);
    else DXe = add2(DXe, dx);
    const R2 u = fma2(four, fma2(cb, v(at(0, 2 * cy, 2 * cz)), v(at(0, cy, cz))), add2(tp, tm));
    if (cy != 0) {
      R2& acc = cz == 0 ? YE : YK;
      acc = cy > 0 ? add2(acc, u) : sub2(acc, u);
    }
    if (D == 3 && cz != 0) {
      R2& acc = cy == 0 ? ZE : ZK;
      acc = cz > 0 ? add2(acc, u) : sub2(acc, u);
    }
  }
  // class weights w_yz / 6 (3-D: 4/3, 1/3, 1/12; 2-D: 2, 1/2)
  constexpr R wc = D == 3 ? (R)(4.0 / 18.0) : (R)(2.0 / 6.0);
  constexpr R we = D == 3 ? (R)(1.0 / 18.0) : (R)(0.5 / 6.0);
  constexpr R wk = (R)(1.0 / 72.0);
  const R2 GX = fma2(both<R>(wc), DXc, fma2(both<R>(we), DXe, mul2(both<R>(wk), DXk)));
  const R2 GY = fma2(both<R>(we), YE, mul2(both<R>(wk), YK));
  const R2 GZ = fma2(both<R>(we), ZE, mul2(both<R>(wk), ZK));
  force_from_gradients<D, R, A>(ph, rho, at(0, 0, 0), GX, GY, GZ, F);
}

// Equilibria, k/s/h split, gamma and relaxation of one node (Eq. LBGK with the
// entropic mirror state of Sec. 2.4): fp/fs hold the node's pre-collision
// populations in row pairs on entry and its post-collision populations on exit.
// m: the node's moments, u = j/rho, F the force (times dt), Phi the diagonal
// correction, om the local omega; s_h holds h_i of the NT threads of the block
// ([i][thread]), n is the node (for the guard count and the gamma record).
template <int D, typename R, int NT>
__device__ __forceinline__ void collide_relax(const DevDomain& d, const Phys<R>& ph, long long n,
                                              const NodeMoments<R>& m, R inv_rho, const R (&u)[3], const R (&F)[3],
                                              const R (&Phi)[3], R om, Two<R> (&fp)[RowPairs<D>::kPairs][3],
                                              R (&fs)[3], R* s_h, int tid) {
  constexpr int NY = RowPairs<D>::kYPairs, NP = RowPairs<D>::kPairs;
  using R2 = Two<R>;
  constexpr R cs2 = (R)(1.0 / 3.0);
  const R rho = m.rho;
  const R2 zero2 = both<R>((R)0);
  R2* s_h2 = (R2*)s_h;                  // [NP * 3][NT]
  R* s_h1 = s_h + 2 * (NP * 3) * NT;    // [3][NT]
  // ---- one-dimensional factors per axis, index k = c+1: equilibrium E, extended
  //      equilibrium St, first-order dual d1 of the central Hermite basis (the
  //      second-order dual is d2 = {1/2, -1, 1/2})
  //      Each axis keeps u_a, he = (cs^2 + u_a^2)/2, xi*_a and hs = zeta*_a/2; the
  //      factors are formed where they are used (fewer live registers).
  R ua[3], he[3], xs[3], hs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ua[a] = a < D ? u[a] : (R)0;
    he[a] = (R)0.5 * (cs2 + ua[a] * ua[a]);
    xs[a] = a < D ? ua[a] + F[a] * inv_rho : (R)0;
    hs[a] = (R)0.5 * (a < D ? cs2 + xs[a] * xs[a] + Phi[a] * inv_rho : cs2);
  }
  auto Ef = [&](int a, int k) { return k == 1 ? (R)1 - (R)2 * he[a] : (k == 0 ? he[a] - (R)0.5 * ua[a] : he[a] + (R)0.5 * ua[a]); };
  auto Sf = [&](int a, int k) { return k == 1 ? (R)1 - (R)2 * hs[a] : (k == 0 ? hs[a] - (R)0.5 * xs[a] : hs[a] + (R)0.5 * xs[a]); };
  auto Df = [&](int a, int k) { return k == 1 ? (R)-2 * ua[a] : (k == 0 ? ua[a] - (R)0.5 : ua[a] + (R)0.5); };
  // x-axis factors, used by every population
  R E[3], St[3], D1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) { E[k] = Ef(0, k); St[k] = Sf(0, k); D1[k] = Df(0, k); }
  // second-order central Hermite moments; the shear part keeps the off-diagonals
  // and the deviatoric diagonal a_aa - trace/D
  const R axy = m.Pxy - rho * u[0] * u[1];
  const R axz = D == 3 ? m.Pxz - rho * u[0] * u[2] : (R)0;
  const R ayz = D == 3 ? m.Pyz - rho * u[1] * u[2] : (R)0;
  const R adx = m.Pxx - rho * u[0] * u[0] - rho * cs2;
  const R ady = m.Pyy - rho * u[1] * u[1] - rho * cs2;
  const R adz = D == 3 ? m.Pzz - rho * u[2] * u[2] - rho * cs2 : (R)0;
  const R tr = (adx + ady + adz) * (R)(1.0 / D);
  const R devx = adx - tr, devy = ady - tr, devz = D == 3 ? adz - tr : (R)0;

  // Every f*_i is positive exactly when rho and the one-dimensional factors St are
  // (each axis's three factors sum to one, so they cannot all be negative).
  R fmin = rho;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) fmin = fmin < Sf(a, k) ? fmin : Sf(a, k);

  // ---- pass A: entropic sums, h to shared memory, g = f - omega s + f* - f^eq
  //      = h + (1 - omega) s + f* in place of f.  A row (cy, cz) has f^eq = ryz E_x,
  //      f* = rsyz St_x and s = E_x C0 + d1_x C1 + d2_x C2.  The weight 1/f*_i factors
  //      as 1/rsyz times 1/St_x, so a row's three terms are summed with the x
  //      reciprocals and scaled once by the row's.
  const R one_m_om = (R)1 - om;
  R iSt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) iSt[k] = rcp_fast<R>(St[k]);
  R2 SA = zero2, SB = zero2;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    // row coefficients of the two lanes
    R2 ryz, rsyz, C0, C1, C2;
    if (k < NY) {
      // lanes vary in y (cy = -1, +1); z fixed at cz = k - 1 (2-D: factors 1, 0, 0)
      const R Z0 = D == 3 ? Ef(2, k) : (R)1, Zs = D == 3 ? Sf(2, k) : (R)1;
      const R Z1 = D == 3 ? Df(2, k) : (R)0, Z2 = D == 3 ? (k == 1 ? (R)-1 : (R)0.5) : (R)0;
      const R2 Y0 = two<R>(Ef(1, 0), Ef(1, 2)), Ys = two<R>(Sf(1, 0), Sf(1, 2)), Y1 = two<R>(Df(1, 0), Df(1, 2));
      ryz = mul2(Y0, both<R>(rho * Z0));
      rsyz = mul2(Ys, both<R>(rho * Zs));
      C0 = fma2(Y1, both<R>(ayz * Z1), fma2(Y0, both<R>(devz * Z2), both<R>((R)0.5 * devy * Z0)));
      C1 = fma2(Y1, both<R>(axy * Z0), mul2(Y0, both<R>(axz * Z1)));
      C2 = mul2(Y0, both<R>(devx * Z0));
    } else {
      // lanes vary in z (cz = -1, +1); y fixed at cy = 0
      const R Y0 = Ef(1, 1), Ys = Sf(1, 1), Y1 = Df(1, 1);
      const R2 Z0 = two<R>(Ef(2, 0), Ef(2, 2)), Zs = two<R>(Sf(2, 0), Sf(2, 2)), Z1 = two<R>(Df(2, 0), Df(2, 2));
      ryz = mul2(Z0, both<R>(rho * Y0));
      rsyz = mul2(Zs, both<R>(rho * Ys));
      C0 = fma2(Z1, both<R>(ayz * Y1), fma2(Z0, both<R>(-devy), both<R>((R)0.5 * devz * Y0)));
      C1 = fma2(Z0, both<R>(axy * Y1), mul2(Z1, both<R>(axz * Y0)));
      C2 = mul2(Z0, both<R>(devx * Y0));
    }
    const R2 E0 = add2(ryz, C0);             // f^eq + (the X C0 part of s) = E_x (ryz + C0)
    const R2 C2h = mul2(both<R>((R)0.5), C2);
    R2 TA = zero2, TB = zero2;
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
      const R2 Xb = both<R>(E[ix]);
      const R2 t = ix == 1 ? sub2(mul2(both<R>(D1[1]), C1), C2) : fma2(both<R>(D1[ix]), C1, C2h);
      const R2 sv = fma2(Xb, C0, t);
      const R2 hh = sub2(fp[k][ix], fma2(Xb, E0, t));
      const R2 fst = mul2(rsyz, both<R>(St[ix]));
      const R2 hr = mul2(hh, both<R>(iSt[ix]));
      TA = fma2(sv, hr, TA);
      TB = fma2(hh, hr, TB);
      s_h2[(3 * k + ix) * NT + tid] = hh;
      fp[k][ix] = fma2(both<R>(one_m_om), sv, add2(hh, fst));
    }
    const R2 irs = two<R>(rcp_fast<R>(rsyz.x), rcp_fast<R>(rsyz.y));
    SA = fma2(irs, TA, SA);
    SB = fma2(irs, TB, SB);
  }
  R sA, sB;
  {
    // the single row cy = cz = 0
    const R Y0 = Ef(1, 1), Ys = Sf(1, 1), Y1 = Df(1, 1);
    const R Z0 = D == 3 ? Ef(2, 1) : (R)1, Zs = D == 3 ? Sf(2, 1) : (R)1;
    const R Z1 = D == 3 ? Df(2, 1) : (R)0, Z2 = D == 3 ? (R)-1 : (R)0;
    const R ryz = rho * Y0 * Z0, rsyz = rho * Ys * Zs;
    const R C0 = ayz * Y1 * Z1 - devy * Z0 + (D == 3 ? devz * Y0 * Z2 : (R)0);
    const R C1 = axy * Y1 * Z0 + (D == 3 ? axz * Y0 * Z1 : (R)0);
    const R C2 = devx * Y0 * Z0;
    R tA = 0, tB = 0;
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
      const R sv = E[ix] * C0 + D1[ix] * C1 + (ix == 1 ? -C2 : (R)0.5 * C2);
      const R hh = fs[ix] - ryz * E[ix] - sv;
      const R hr = hh * iSt[ix];
      tA += sv * hr;
      tB += hh * hr;
      s_h1[ix * NT + tid] = hh;
      fs[ix] = hh + one_m_om * sv + rsyz * St[ix];
    }
    const R irs = rcp_fast<R>(rsyz);
    sA = (SA.x + SA.y) + irs * tA;
    sB = (SB.x + SB.y) + irs * tB;
  }

  R gamma;
  if (d.gamma_mode == 1) {
    gamma = ph.gamma_value;
  } else if (!(fmin > (R)0)) {
    gamma = (R)2;
    atomicAdd(d.guards, 1ull);
  } else {
    gamma = entropic_gamma<R>(sA, sB, om);
  }
  if (d.gamma_out) ((float2*)d.gamma_out)[n] = make_float2((float)gamma, (float)om);

  // ---- pass B: f' = g - (omega gamma/2) h
  const R ch = (R)0.5 * om * gamma;
  const R2 mch = both<R>(-ch);
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) fp[k][ix] = fma2(mch, s_h2[(3 * k + ix) * NT + tid], fp[k][ix]);
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) fs[ix] -= ch * s_h1[ix * NT + tid];

}

// One tile of pass 2 whose origin is (x0, y0, z0), run by the BX*BY*BZ threads of
// the block.  kTma: the q boxes (s_q) come from TMA copies of the tensor map
// maps->q, completed on `bar` (phase `phase`); otherwise q comes from global memory.
// The force F of each node is the one pass 1b wrote over its momentum planes.
// kStaged (with kTma): the caller has already issued this tile's q copies and
// staged its populations in s_f ([i][thread], cp.async completed); once every
// thread has read its populations the tile calls hooks.prefetch() (the next
// tile's populations into s_f), and once the block is done with the q boxes it
// calls hooks.aux() (the next tile's q copies into s_q) after a block barrier that
// every thread of the block reaches.
// s_h holds Q*BX*BY*BZ values of h: the pair rows first (Two<R> [pair*3 +
// ix][thread]), then the single row.
// Returns false when the q copy did not arrive within the poll limit.
template <int D, int BX, int BY, int BZ, int P, typename S, typename R, typename A, bool kTma,
          bool kStaged = false, typename Hooks = NoHooks>
__device__ __forceinline__ bool collide_tile(const DevDomain& d, const TileMaps* maps, int x0, int y0, int z0,
                                             A* s_q, R* s_h, unsigned long long* bar, uint32_t phase,
                                             const S* s_f = nullptr, const Hooks& hooks = Hooks()) {
  constexpr int Q = Lattice<D>::Q;
  constexpr int NT = BX * BY * BZ;
  constexpr int NP = RowPairs<D>::kPairs;
  using RP = RowPairs<D>;
  using R2 = Two<R>;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  const Phys<R>& ph = phys<R>(d);

  // x0 is a multiple of BX (>= 32), so the q boxes start 16-byte aligned
  if (kTma && !kStaged && tid == 0) tma_load_q_boxes<D, BX, BY, BZ, A>(maps, s_q, bar, x0, y0, z0);

  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + (D == 3 ? threadIdx.z : 0);
  const bool active = x < d.nx && y < d.ny && z < d.nz;
  const long long n = node_of(d, x, y, z);
  const bool fast = P == 0 || fast_links<D>(d, x, y, z);
  const long long pc = active ? bc_pnode(d, pnode_of<D>(d, x, y, z)) : 0;

  // the node's force (Eq. Kforce_final), from pass 1b
  A Fa[3] = {0, 0, 0};
  if (active) {
    const A* aF = (const A*)d.aux + (2 + D) * d.PN + pc;
#pragma unroll
    for (int a = 0; a < D; ++a) Fa[a] = aF[a * d.PN];
  }
  R f[Q];
  if (kStaged) {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = active ? ld_pop<S, R>(s_f + i * NT + tid) : (R)wq<D>(i);
  } else if (active) {
    gather<D, P, S, R>(d, x, y, z, f);
  }
  bool tile_ok = true;
  if (kTma) {
    // every thread waits, so that the block cannot retire while the copy is in flight
    tile_ok = mbar_wait_bounded(bar, phase, kTileWaitPolls);
    if (!kStaged && !tile_ok) {
      if (tid == 0) atomicOr(d.flags, 2u);
      mbar_wait_bounded(bar, phase, kTileWaitPolls);
      return false;
    }
  }
  if (!kStaged && !active) return true;

  R2 fp[NP][3];
  R fs[3];
  NodeMoments<R> m;
  row_moments<D, R>(f, fp, fs, m);
  const R rho = m.rho;
  const R inv_rho = (R)1 / rho;
  const R u[3] = {m.jx * inv_rho, m.jy * inv_rho, m.jz * inv_rho};
  // every staged population has been consumed: s_f may take the next tile's
  if (kStaged) hooks.prefetch();

  const R F[3] = {(R)Fa[0], (R)Fa[1], (R)Fa[2]};

  // ---- Phi_aa = -(1 - omega/2) d_a q_a, central difference.  The sign is the one
  // that cancels the lattice's third-moment defect (sum f^eq c_a^3 = rho u_a where
  // rho u_a^3 + 3 P0 u_a is due) in the diagonal momentum flux, the purpose Sec. 2.2
  // gives Phi; Eq. (correction) prints the opposite sign, which doubles the defect.
  const R om = omega_of<R>(ph, rho);
  R Phi[3] = {0, 0, 0};
  if (kTma) {
    using H = Halo<D, BX, BY, BZ>;
    const int qc = (threadIdx.x + 2) + H::QX * ((threadIdx.y + 1) + H::QY * (D == 3 ? threadIdx.z + 1 : 0));
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const A* qa = s_q + a * H::template qstride<A>() + qc;
      const int e = a == 0 ? 1 : (a == 1 ? H::QX : H::QX * H::QY);
      Phi[a] = ((R)1 - (R)0.5 * om) * ((R)qa[-e] - (R)qa[e]) * (R)0.5;
    }
  } else {
    const A* a_q = (const A*)d.aux + 2 * d.PN;
    const long long sy = d.px, sz = (long long)d.px * d.py;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const A* qa = a_q + a * d.PN;
      const long long e = a == 0 ? 1 : (a == 1 ? sy : sz);
      Phi[a] = ((R)1 - (R)0.5 * om) * ((R)qa[bc_pnode(d, pc - e)] - (R)qa[bc_pnode(d, pc + e)]) * (R)0.5;
    }
  }
  if (kStaged) {
    // the block is done with the q boxes (a block-wide vote on the copy's arrival)
    if (__syncthreads_or(!tile_ok)) {
      if (tid == 0) atomicOr(d.flags, 2u);
      mbar_wait_bounded(bar, phase, kTileWaitPolls);
      return false;
    }
    hooks.aux();
    if (!active) return true;
  }

  collide_relax<D, R, NT>(d, ph, n, m, inv_rho, u, F, Phi, om, fp, fs, s_h, tid);

  // ---- float16-deviation storage: encode against this node's density, which the
  //      next step reads back as the writer density of every slot written here
  if constexpr (DevStorage<S>::value) {
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
        fp[k][ix] = fma2(fp[k][ix], both<R>(inv_rho * (R)(1.0 / wq<D>(RP::pop(k, 0, ix)))), both<R>((R)-1));
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) fs[ix] = fs[ix] * (inv_rho * (R)(1.0 / wq<D>(RP::single(ix)))) - (R)1;
    d.rho_w[1 - P][n] = (float)rho;
  }

  // ---- stream: A-A write
  const XBase xb = xbase<S>(d, x, n);
  auto store = [&](bool in) {
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        st_pop<S, R>(dst_ptr<D, P, S>(d, in, xb, x, y, z, n, RP::pop(k, 0, ix)), fp[k][ix].x);
        st_pop<S, R>(dst_ptr<D, P, S>(d, in, xb, x, y, z, n, RP::pop(k, 1, ix)), fp[k][ix].y);
      }
      st_pop<S, R>(dst_ptr<D, P, S>(d, in, xb, x, y, z, n, RP::single(ix)), fs[ix]);
    }
  };
  if (fast) store(true);
  else store(false);
  return true;
}

// Pass 1b on one tile of interior nodes of extents EX x EY x EZ whose origin is
// (x0, y0, z0), run by TX x TY threads, each walking TK nodes (along z in 3-D,
// along y in 2-D): q_a = rho v_a^3 (Eq. (correction) with P0/rho = cs^2) with v =
// (j + F/2)/rho the fluid velocity of the exact-difference forcing, F the force of
// Eq. (Kforce_final) from the staged (rho, psi) halo tile s_aux, j (loaded by
// qflux_load_j) and rho those pass 1 wrote for the node.  The node's q also goes to
// the ghost nodes that image it (negated across a wall: the no-slip image of pass
// 1's fields).  F itself is written over the node's j (read by this thread alone,
// before): pass 2 takes the force from there instead of evaluating the stencil again.
template <int D, int TX, int TY, int TK> struct QTileShape {
  static constexpr int EY = D == 3 ? TY : TY * TK, EZ = D == 3 ? TK : 1;
  static constexpr int HX = TX + 4, HY = EY + 4, HZ = D == 3 ? EZ + 4 : 1;
};

// The momenta j of this thread's TK nodes of the tile at (x0, y0, z0) (0 outside).
template <int D, int TX, int TY, int TK, typename A>
__device__ __forceinline__ void qflux_load_j(const DevDomain& d, int x0, int y0, int z0, A (&jn)[TK][D]) {
  const A* aux = (const A*)d.aux;
  const int x = x0 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < TK; ++k) {
    const int y = y0 + (D == 3 ? (int)threadIdx.y : (int)threadIdx.y + TY * k), z = z0 + (D == 3 ? k : 0);
    const bool in = x < d.nx && y < d.ny && z < d.nz;
    const long long pn = in ? bc_pnode(d, pnode_of<D>(d, x, y, z)) : 0;
#pragma unroll
    for (int a = 0; a < D; ++a) jn[k][a] = in ? aux[(2 + D + a) * d.PN + pn] : (A)0;
  }
}

// q and F of one interior node to the auxiliary planes (F over the node's j), and
// q to the ghost nodes imaging the node: every combination of its own or its ghost
// coordinate on each axis that has a ghost, other than its own on all of them.
template <int D, typename R, typename A>
__device__ __forceinline__ void qflux_store(const DevDomain& d, int x, int y, int z, int gx, bool gw_x, R rho,
                                            const A (&j)[3], const R (&F)[3]) {
  A* aux = (A*)d.aux;
  const long long pn = bc_pnode(d, pnode_of<D>(d, x, y, z));
  const R inv = (R)1 / rho;
  A q[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const R v = ((R)j[a] + (R)0.5 * F[a]) * inv;
    q[a] = (A)(rho * v * v * v);
    aux[(2 + a) * d.PN + pn] = q[a];
    aux[(2 + D + a) * d.PN + pn] = (A)F[a];  // F replaces j: pass 2 reads it at the node
  }
  bool gw_y = false, gw_z = false;
  const int gy = ghost_of(y, d.ny, d.wall_lo[1], d.wall_hi[1], &gw_y);
  const int gz = D == 3 ? ghost_of(z, d.nz, d.wall_lo[2], d.wall_hi[2], &gw_z) : -1;
  if (gx < 0 && gy < 0 && gz < 0) return;
#pragma unroll 1
  for (int m = 1; m < (1 << D); ++m) {
    if (((m & 1) && gx < 0) || ((m & 2) && gy < 0) || ((m & 4) && gz < 0)) continue;
    const int cx = (m & 1) ? gx : x + 2, cy = (m & 2) ? gy : y + 2, cz = D == 3 ? ((m & 4) ? gz : z + 2) : 0;
    const bool flip = ((m & 1) && gw_x) || ((m & 2) && gw_y) || ((m & 4) && gw_z);
    const long long g = bc_pnode(d, (long long)cx + (long long)d.px * ((long long)cy + (long long)d.py * cz));
#pragma unroll
    for (int a = 0; a < D; ++a) aux[(2 + a) * d.PN + g] = flip ? -q[a] : q[a];
  }
}

// Pass 1b node by node (the 2-D kernels): each of the thread's TK nodes evaluates
// the stencil of Eq. (Kforce_final) from the staged tile on its own.
template <int D, int TX, int TY, int TK, typename R, typename A>
__device__ __forceinline__ void qflux_nodes(const DevDomain& d, int x0, int y0, int z0, const Two<A>* s_aux,
                                            const A (&jn)[TK][D]) {
  using SH = QTileShape<D, TX, TY, TK>;
  const int x = x0 + threadIdx.x;
  bool gw_x = false;
  const int gx = ghost_of(x, d.nx, d.wall_lo[0], d.wall_hi[0], &gw_x);
#pragma unroll
  for (int k = 0; k < TK; ++k) {
    const int ly = D == 3 ? threadIdx.y : threadIdx.y + TY * k, lz = D == 3 ? k : 0;
    const int y = y0 + ly, z = z0 + lz;
    if (!(x < d.nx && y < d.ny && z < d.nz)) continue;
    const int sc = (threadIdx.x + 2) + SH::HX * ((ly + 2) + SH::HY * (D == 3 ? lz + 2 : 0));
    const R rho = (R)s_aux[sc].x;
    R F[3];
    stencil_force<D, R, A>(phys<R>(d), rho,
                           [&](int dx, int dy, int dz) { return s_aux[sc + dx + SH::HX * (dy + SH::HY * dz)]; }, F);
    const A j[3] = {jn[k][0], jn[k][1], D == 3 ? jn[k][D - 1] : (A)0};
    qflux_store<D, R, A>(d, x, y, z, gx, gw_x, rho, j, F);
  }
}

// Pass 1b in 3-D, plane by plane.  A thread walks the TK + 4 z planes of its column
// of the halo tile once.  Of each plane it reads the 17 (rho, psi) pairs that the
// radius-2 stencil of Eq. (Kforce_final) touches there (offsets in {-1, 0, 1}^2 and
// in {-2, 0, 2}^2) and adds the plane's share of the link sums to the nodes within
// two planes of it; a node's sums are complete, and the node is stored, once plane
// z + 2 is in.  The sums are stencil_force's, regrouped: a link row (cy, cz) takes
// its near points r + c from plane z + cz and its far points r + 2c from plane
// z + 2 cz, and both enter linearly.  Shared-memory reads per node fall from 53 to
// 17 (TK + 4) / TK.
template <int TX, int TY, int TK, typename R, typename A>
__device__ __forceinline__ void qflux_nodes_zwalk(const DevDomain& d, int x0, int y0, int z0, const Two<A>* s_aux) {
  using SH = QTileShape<3, TX, TY, TK>;
  using R2 = Two<R>;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (!(x < d.nx && y < d.ny)) return;
  const Phys<R>& ph = phys<R>(d);
  bool gw_x = false;
  const int gx = ghost_of(x, d.nx, d.wall_lo[0], d.wall_hi[0], &gw_x);
  // class weights w_yz / 6 (centre 4/3, edge 1/3, corner 1/12, over 6), and the same
  // times the far points' (-1/2, -1/8)
  constexpr double wc = 4.0 / 18.0, we = 1.0 / 18.0, wk = 1.0 / 72.0;
  const R2 Wc = both<R>((R)wc), We = both<R>((R)we), Wk = both<R>((R)wk);
  const R2 WcF = two<R>((R)(-0.5 * wc), (R)(-0.125 * wc)), WeF = two<R>((R)(-0.5 * we), (R)(-0.125 * we));
  const R2 WkF = two<R>((R)(-0.5 * wk), (R)(-0.125 * wk));
  const R2 four = both<R>((R)4), zero2 = both<R>((R)0);
  const Two<A>* col = s_aux + (threadIdx.x + 2) + SH::HX * (threadIdx.y + 2);  // this column, plane 0
  auto P = [&](int hz, int dx, int dy) {
    const Two<A> v = col[dx + SH::HX * (dy + SH::HY * hz)];
    return two<R>((R)v.x, (R)v.y);
  };
  const long long pj = pnode_of<3>(d, x, y, z0);
  const long long plane = (long long)d.px * d.py;
  const A* aj = (const A*)d.aux + 5 * d.PN;  // the j planes, (2 + D) PN
  R2 G[TK][3];
  Two<A> c[TK];
  A j[TK][3];
#pragma unroll
  for (int hz = 0; hz < TK + 4; ++hz) {
    // node k has its centre in plane k + 2; this plane is its dz = hz - k - 2
    if (hz < TK) {
      // the momenta of the node whose first plane this is, four planes before use
      const bool in = z0 + hz < d.nz;
#pragma unroll
      for (int a = 0; a < 3; ++a) j[hz][a] = in ? aj[a * d.PN + bc_pnode(d, pj + hz * plane)] : (A)0;
#pragma unroll
      for (int a = 0; a < 3; ++a) G[hz][a] = zero2;
    }
    const int k_up2 = hz - 4, k_dn2 = hz, k_up1 = hz - 3, k_dn1 = hz - 1, k_c = hz - 2;
    const bool r_up2 = k_up2 >= 0 && k_up2 < TK, r_dn2 = k_dn2 < TK, r_up1 = k_up1 >= 0 && k_up1 < TK;
    const bool r_dn1 = k_dn1 >= 0 && k_dn1 < TK, r_c = k_c >= 0 && k_c < TK;
    const R2 p00 = P(hz, 0, 0);
    if (r_c) c[k_c] = col[SH::HX * SH::HY * hz];
    if (r_up2 || r_dn2 || r_c) {
      // far points: row sums DF = t(+2) - t(-2), UF = 4 t(0) + t(+2) + t(-2) at dy = 2 cy
      R2 DF[3], UF[3];
#pragma unroll
      for (int cy = -1; cy <= 1; ++cy) {
        const R2 fm = P(hz, -2, 2 * cy), fp = P(hz, 2, 2 * cy);
        DF[cy + 1] = sub2(fp, fm);
        UF[cy + 1] = fma2(four, cy == 0 ? p00 : P(hz, 0, 2 * cy), add2(fp, fm));
      }
      if (r_up2 || r_dn2) {
        const R2 X = fma2(WeF, DF[1], mul2(WkF, add2(DF[0], DF[2])));
        const R2 Y = mul2(WkF, sub2(UF[2], UF[0]));
        const R2 Z = fma2(WeF, UF[1], mul2(WkF, add2(UF[0], UF[2])));
        if (r_up2) { G[k_up2][0] = add2(G[k_up2][0], X); G[k_up2][1] = add2(G[k_up2][1], Y); G[k_up2][2] = add2(G[k_up2][2], Z); }
        if (r_dn2) { G[k_dn2][0] = add2(G[k_dn2][0], X); G[k_dn2][1] = add2(G[k_dn2][1], Y); G[k_dn2][2] = sub2(G[k_dn2][2], Z); }
      }
      if (r_c) {
        G[k_c][0] = fma2(WcF, DF[1], fma2(WeF, add2(DF[0], DF[2]), G[k_c][0]));
        G[k_c][1] = fma2(WeF, sub2(UF[2], UF[0]), G[k_c][1]);
      }
    }
    if (r_up1 || r_dn1 || r_c) {
      // near points: DN = t(+1) - t(-1), UN = 4 t(0) + t(+1) + t(-1) at dy = cy
      R2 DN[3], UN[3];
#pragma unroll
      for (int cy = -1; cy <= 1; ++cy) {
        const R2 nm = P(hz, -1, cy), np = P(hz, 1, cy);
        DN[cy + 1] = sub2(np, nm);
        UN[cy + 1] = fma2(four, cy == 0 ? p00 : P(hz, 0, cy), add2(np, nm));
      }
      if (r_up1 || r_dn1) {
        const R2 X = fma2(We, DN[1], mul2(Wk, add2(DN[0], DN[2])));
        const R2 Y = mul2(Wk, sub2(UN[2], UN[0]));
        const R2 Z = fma2(We, UN[1], mul2(Wk, add2(UN[0], UN[2])));
        if (r_up1) { G[k_up1][0] = add2(G[k_up1][0], X); G[k_up1][1] = add2(G[k_up1][1], Y); G[k_up1][2] = add2(G[k_up1][2], Z); }
        if (r_dn1) { G[k_dn1][0] = add2(G[k_dn1][0], X); G[k_dn1][1] = add2(G[k_dn1][1], Y); G[k_dn1][2] = sub2(G[k_dn1][2], Z); }
      }
      if (r_c) {
        G[k_c][0] = fma2(Wc, DN[1], fma2(We, add2(DN[0], DN[2]), G[k_c][0]));
        G[k_c][1] = fma2(We, sub2(UN[2], UN[0]), G[k_c][1]);
      }
    }
    // node hz - 4 has all five of its planes
    if (r_up2 && z0 + k_up2 < d.nz) {
      const R rho = (R)c[k_up2].x;
      R F[3];
      force_from_gradients<3, R, A>(ph, rho, c[k_up2], G[k_up2][0], G[k_up2][1], G[k_up2][2], F);
      qflux_store<3, R, A>(d, x, y, z0 + k_up2, gx, gw_x, rho, j[k_up2], F);
    }
  }
}

// Pass 1b on one tile with warp-staged halo rows (the batched kernel's form).
template <int D, int TX, int TY, int TK, typename R, typename A>
__device__ __forceinline__ void qflux_tile_staged(const DevDomain& d, int x0, int y0, int z0, Two<A>* s_aux) {
  using SH = QTileShape<D, TX, TY, TK>;
  constexpr int NT = TX * TY;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const Two<A>* a2 = (const Two<A>*)d.aux;
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < SH::HY * SH::HZ; r += NT / 32) {
    const int yp = y0 + r % SH::HY, zp = z0 + r / SH::HY;
    const bool row_ok = yp < d.py && zp < d.pz;
    const long long base = (long long)d.px * ((long long)yp + (long long)d.py * zp) + x0;
    for (int hx = lane; hx < SH::HX; hx += 32) {
      const bool ok = row_ok && x0 + hx < d.px;
      s_aux[r * SH::HX + hx] = ok ? a2[base + hx] : two<A>((A)1, (A)0);
    }
  }
  __syncthreads();
  A jn[TK][D];
  qflux_load_j<D, TX, TY, TK, A>(d, x0, y0, z0, jn);
  qflux_nodes<D, TX, TY, TK, R, A>(d, x0, y0, z0, s_aux, jn);
}

// Pass 1b, one QTile tile per block: the halo tile comes from one TMA copy while
// the threads load their nodes' momenta.  (A persistent form with two halo buffers,
// the next tile's copy in flight during the current one, was slower: its two
// 41 KB buffers leave two blocks per SM, and the stencil's shared-memory reads,
// not the copy latency, set the pace.)  A wait that gives up sets bit 1 of the
// error word; the block then waits (bounded) for the copy and stops.
// Resident blocks per SM asked of the register allocator for pass 1b in float32:
// three (80 registers, 8 bytes spilled in the 3-D walk of TK = 8; float64 takes
// what it needs, 84).  On the 512x512x256
// impact, passes 1 + 1b take 2.06-2.10 ms so, against 2.34 ms with TK = 4 at 76
// registers, 2.18 ms with TK = 4 at 64 and 2.21 ms with TK = 8 at 64 (spills); a
// deeper walk, fewer halo planes per node, was slower too: TK = 16 at 114 registers
// (two 256-thread or four 128-thread blocks per SM, no spills) 2.14 and 2.20 ms,
// TK = 16 or 12 at 80 registers (three blocks, ~20 bytes spilled) 2.19 and 2.16 ms.
#ifndef LBM_QFLUX_MINBLOCKS
#define LBM_QFLUX_MINBLOCKS 3
#endif
template <int D, typename R, typename A>
__global__ void __launch_bounds__(QTile<D, 2 * sizeof(A)>::TX * QTile<D, 2 * sizeof(A)>::TY,
                                  sizeof(A) == 4 ? LBM_QFLUX_MINBLOCKS : 1)
qflux_tile_kernel(DevDomain d, const __grid_constant__ TileMaps maps) {
  using T = QTile<D, 2 * sizeof(A)>;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  Two<A>* s_aux = (Two<A>*)smem_dyn;  // [z][y][x] (rho, psi)
  unsigned long long* bar = (unsigned long long*)(smem_dyn + ((T::HN * sizeof(Two<A>) + 15) / 16) * 16);
  const int tid = threadIdx.x + T::TX * threadIdx.y;
  const int x0 = blockIdx.x * T::EX, y0 = blockIdx.y * T::EY, z0 = D == 3 ? blockIdx.z * T::EZ : 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, (uint32_t)(T::HN * sizeof(Two<A>)));
    tma_load_tile<D, A>(s_aux, &maps.aux_q, bar, x0, y0, z0);
  }
  __syncthreads();
  auto arrived = [&]() {
    if (mbar_wait_bounded(bar, 0, kTileWaitPolls)) return true;
    // every thread waits, so that the block cannot retire while the copy is in flight
    if (tid == 0) atomicOr(d.flags, 2u);
    mbar_wait_bounded(bar, 0, kTileWaitPolls);
    return false;
  };
  if constexpr (D == 3) {
    // the walk loads each node's j itself, four planes ahead of its use
    if (arrived()) qflux_nodes_zwalk<T::TX, T::TY, T::TK, R, A>(d, x0, y0, z0, s_aux);
  } else {
    // 2-D stays node by node: a row walk of the same kind ran no faster on the
    // L2-resident 2048x1024 impact (pass 1 + 1b 42.7 us against 42.4)
    A jn[T::TK][D];
    qflux_load_j<D, T::TX, T::TY, T::TK, A>(d, x0, y0, z0, jn);
    if (arrived()) qflux_nodes<D, T::TX, T::TY, T::TK, R, A>(d, x0, y0, z0, s_aux, jn);
  }
}

// Dynamic shared memory of the pass-1b kernel: the halo tile and its mbarrier.
template <int D, typename A>
constexpr size_t qflux_dyn_smem() {
  return ((QTile<D, 2 * sizeof(A)>::HN * sizeof(Two<A>) + 15) / 16) * 16 + 16;
}

template <int D, int P, typename S, typename R, typename A>
__global__ void __launch_bounds__(Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz, LBM_K2_MINBLOCKS(R, D))
collide_stream_kernel(DevDomain d, const __grid_constant__ TileMaps maps) {
  constexpr int BX = Blocks<D>::bx, BY = Blocks<D>::by, BZ = Blocks<D>::bz;
  using H = Halo<D, BX, BY, BZ>;
  __shared__ __align__(128) A s_q[D * H::template qstride<A>()];     // [a][z][y][x] q_a
  __shared__ __align__(8) unsigned long long tile_bar;
  // higher-order part h_i of every node of the tile, [i][thread] (dynamic: above 48 KB in float64)
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  if (tid == 0) mbar_init(&tile_bar, 1);
  __syncthreads();
  collide_tile<D, BX, BY, BZ, P, S, R, A, true>(d, &maps, blockIdx.x * BX, blockIdx.y * BY,
                                                 D == 3 ? blockIdx.z * BZ : 0, s_q, (R*)smem_dyn, &tile_bar, 0);
}

// Start the copies of the pre-collision populations of node (x, y, z) into the
// staging buffer s_f ([i][thread]); nothing for a node outside the domain.
template <int D, int P, typename S, int NT>
__device__ __forceinline__ void stage_populations(const DevDomain& d, int x, int y, int z, S* s_f, int tid) {
  constexpr int Q = Lattice<D>::Q;
  if (!(x < d.nx && y < d.ny && z < d.nz)) return;
  const long long n = node_of(d, x, y, z);
  const XBase xb = xbase<S>(d, x, n);
  if (P == 0 || fast_links<D>(d, x, y, z)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) cp_async_word<sizeof(S)>(s_f + i * NT + tid, src_ptr<D, P, S>(d, true, xb, x, y, z, n, i));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) cp_async_word<sizeof(S)>(s_f + i * NT + tid, src_ptr<D, P, S>(d, false, xb, x, y, z, n, i));
  }
}

// Persistent form of pass 2: a block walks the tiles t = blockIdx.x, + gridDim.x,
// ... (x fastest).  While it computes tile t the copies of tile t + gridDim.x are in
// flight: its populations (cp.async, started as soon as tile t's have been read
// into registers; the A-A pattern makes that safe, since a node's read slots are
// written by that node alone within the step) and, once the q boxes of tile t have
// been read, its q boxes (TMA).
template <int D, int P, typename S, typename R, typename A>
__global__ void __launch_bounds__(Blocks<D>::bx * Blocks<D>::by * Blocks<D>::bz, LBM_K2_MINBLOCKS(R, D))
collide_stream_persistent_kernel(DevDomain d, const __grid_constant__ TileMaps maps, int ntx, int nty, int ntiles) {
  constexpr int BX = Blocks<D>::bx, BY = Blocks<D>::by, BZ = Blocks<D>::bz;
  constexpr int NT = BX * BY * BZ;
  using H = Halo<D, BX, BY, BZ>;
  __shared__ __align__(128) A s_q[D * H::template qstride<A>()];  // [a][z][y][x] q_a
  __shared__ __align__(8) unsigned long long tile_bar;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  R* s_h = (R*)smem_dyn;                                            // [Q][NT] h
  S* s_f = (S*)(smem_dyn + (size_t)Lattice<D>::Q * NT * sizeof(R));  // [Q][NT] staged populations
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  if (tid == 0) mbar_init(&tile_bar, 1);
  __syncthreads();
  int t = blockIdx.x;
  if (t >= ntiles) return;
  auto origin = [&](int tt, int& ox, int& oy, int& oz) {
    ox = (tt % ntx) * BX;
    oy = ((tt / ntx) % nty) * BY;
    oz = D == 3 ? (tt / (ntx * nty)) * BZ : 0;
  };
  int x0, y0, z0;
  origin(t, x0, y0, z0);
  stage_populations<D, P, S, NT>(d, x0 + threadIdx.x, y0 + threadIdx.y, z0 + threadIdx.z, s_f, tid);
  cp_async_commit();
  if (tid == 0) tma_load_q_boxes<D, BX, BY, BZ, A>(&maps, s_q, &tile_bar, x0, y0, z0);
  for (uint32_t it = 0;; ++it) {
    const int tn = t + (int)gridDim.x;
    int nx0 = 0, ny0 = 0, nz0 = 0;
    if (tn < ntiles) origin(tn, nx0, ny0, nz0);
    struct Next {
      const DevDomain& d;
      const TileMaps* maps;
      A* s_q;
      unsigned long long* bar;
      S* s_f;
      int tid, x0, y0, z0;
      bool valid;
      __device__ void prefetch() const {
        if (valid) stage_populations<D, P, S, NT>(d, x0 + threadIdx.x, y0 + threadIdx.y, z0 + threadIdx.z, s_f, tid);
        cp_async_commit();
      }
      __device__ void aux() const {
        if (valid && tid == 0) {
          fence_proxy_async_smem();
          tma_load_q_boxes<D, BX, BY, BZ, A>(maps, s_q, bar, x0, y0, z0);
        }
      }
    } next{d, &maps, s_q, &tile_bar, s_f, tid, nx0, ny0, nz0, tn < ntiles};
    cp_async_wait_all();  // this thread's populations of tile t are in s_f
    if (!collide_tile<D, BX, BY, BZ, P, S, R, A, true, true, Next>(d, &maps, x0, y0, z0, s_q, s_h, &tile_bar,
                                                                     it & 1u, s_f, next))
      break;
    if (tn >= ntiles) break;
    t = tn;
    x0 = nx0; y0 = ny0; z0 = nz0;
  }
  cp_async_wait_all();  // no copy of this block still in flight at exit
}

}  // namespace lbm
