// Device-side building blocks of the entropic MRT two-phase lattice Boltzmann
// step (Hosseini, Dorschner & Karlin, arXiv:2201.12404) for sm_103a.
//
// Data layout in HBM (one domain):
//   populations  f[i * N + node]          SoA, node = x + nx*(y + ny*z), one A-A buffer
//   auxiliary    aux2[pnode] = (rho, psi) interleaved pairs, then q_a[pnode] planes
//                                         (element offset (2 + a) * PN), then D planes
//                                         at offset (2 + D + a) * PN that hold the bare
//                                         momentum j_a after pass 1 and the force F_a
//                                         after pass 1b (interior nodes); padded by a
//                                         2-node ghost layer on every axis (2-D: z not
//                                         padded)
// The A-A pattern keeps one population buffer: an even step (parity 0) reads and
// writes the node's own slots (writing direction i into slot Q-1-i), an odd step
// (parity 1) reads the neighbours' slots and writes back into them, so that after
// each odd step slot i of node r holds f_i(r) again.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---- lattice: velocities c_i in {-1,0,1}^D, i = (cx+1) + 3(cy+1) + 9(cz+1) (Sec. 2.1) ----
__host__ __device__ constexpr int cxi(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cyi(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int czi(int i) { return i / 9 - 1; }
template <int D> __host__ __device__ constexpr int cq(int i, int a) {
  return a == 0 ? cxi(i) : (a == 1 ? cyi(i) : (D == 3 ? czi(i) : 0));
}
template <int D> struct Lattice { static constexpr int Q = D == 2 ? 9 : 27; static constexpr int REST = (Q - 1) / 2; };

// One-dimensional weight Psi_c(0, cs^2): 2/3 at rest, 1/6 moving (Eq. wi).
__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
template <int D> __host__ __device__ constexpr double wq(int i) {
  return w1d(cxi(i)) * w1d(cyi(i)) * (D == 3 ? w1d(czi(i)) : 1.0);
}

// Block shape of the per-node kernels (x fastest); the force+collide+stream pass
// stages the q planes of a tile of this shape plus a 1-node halo (2 along x).
template <int D> struct Blocks;
template <> struct Blocks<2> { static constexpr int bx = 64, by = 4, bz = 1; };
// D3Q27: 64-thread blocks of 32x2x1 nodes, which retire and refill an SM in finer
// steps than 256-thread blocks: at 80 registers (24 warps per SM) pass 2 took
// 3.03 ms per launch on the 512x512x256 impact against 3.18 with 32x4x2, 3.06 with
// 32x2x2 and 3.08 with 32x4x1 blocks; at 96 registers (LBM_K2_MINBLOCKS_F32) 2.72
// against 2.75 with 32x2x2 and 2.78 with 32x1x1 blocks.
#ifndef LBM_BLOCK3_Y
#define LBM_BLOCK3_Y 2
#endif
#ifndef LBM_BLOCK3_Z
#define LBM_BLOCK3_Z 1
#endif
template <> struct Blocks<3> { static constexpr int bx = 32, by = LBM_BLOCK3_Y, bz = LBM_BLOCK3_Z; };

// Physical parameters in the arithmetic type of a path (filled on the host, so
// that kernels never convert float64 parameters on the slow float64 pipe).
template <typename R> struct Phys {
  R kappa, g[3];
  R nu_v, dnu, rho_v, inv_drho;  // nu(rho) = nu_v + clamp((rho - rho_v) inv_drho, 0, 1) dnu
  R RT, b, aalpha;               // Peng-Robinson: P = rho RT/(1 - b rho) - aalpha rho^2/(1 + 2 b rho - b^2 rho^2)
  R gamma_value;
  R band_lo, band_hi;            // interface band of densities (float64 EOS inside it when eos_fp64 == 1)
  // Sign s of P(rho) - rho cs^2: sgn0 below every threshold, flipped once for every
  // threshold t <= rho.  The thresholds are the smallest values of R above the roots
  // of P(rho) = rho cs^2 on (0, 1/b) (at most three), +inf where unused.
  R sgn_t[3];
  R sgn0;
};

// ---- two lanes of the arithmetic type ----
// float32 pairs are one packed FFMA2/FADD2/FMUL2 instruction for both lanes
// (round to nearest, each lane exactly the scalar operation); float64 pairs are
// two scalar operations.
template <typename R> struct TwoOf;
template <> struct TwoOf<float> { using T = float2; };
template <> struct TwoOf<double> { using T = double2; };
template <typename R> using Two = typename TwoOf<R>::T;

template <typename R> __device__ __forceinline__ Two<R> two(R a, R b) { return Two<R>{a, b}; }
template <typename R> __device__ __forceinline__ Two<R> both(R a) { return Two<R>{a, a}; }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, exact as a subtraction (b * -1 is exact, one rounding)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return double2{a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return double2{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
}
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return double2{a.x - b.x, a.y - b.y}; }

// ---- what a kernel needs to know about a domain (passed by value) ----
struct DevDomain {
  void* f;             // populations (storage type)
  void* aux;           // padded auxiliary fields (float64 in the FP64 path, float32 otherwise)
  float* gamma_out;    // per-node (gamma, omega) pairs of the last step, or nullptr
  unsigned int* flags; // bit 0: non-finite or non-positive density seen; bit 1: a bounded
                       // wait gave up; bit 2: an out-of-range index (bounds-checked builds)
  unsigned long long* guards; // nodes where f*_i <= 0 forced gamma = 2
  long long N, PN;     // interior and padded node counts
  int nx, ny, nz;      // nz = 1 in 2-D
  int px, py, pz;      // padded extents (pz = 1 in 2-D)
  int wall_lo[3], wall_hi[3];
  int gamma_mode;
  int eos_fp64;
  Phys<double> pd;     // parameters for the float64 path and the float64 islands
  Phys<float> pf;      // the same rounded to float32
  // Byte offsets, relative to node r's own slot 0, of the slot population i is
  // read from (src) and written to (dst) at an interior node, per A-A parity, in
  // elements: src[0][i] = i N, src[1][i] = (Q-1-i) N - off(c_i); dst[0][i] = (Q-1-i) N,
  // dst[1][i] = i N + off(c_i), off(c) = cx + nx cy + nx ny cz; times the size of a
  // stored population.
  long long src_boff[2][27], dst_boff[2][27];
  // Element offset of the upstream node r - c_i of an interior node: the node that
  // wrote the slot population i of r is read from, in either parity.
  long long up_off[27];
  // float16-deviation storage only: density of the writer of every slot, by
  // parity (a step of parity P decodes with rho_w[P] and records its own
  // densities in rho_w[1 - P]); nullptr otherwise.
  float* rho_w[2];
};

// The tensor maps of the collide kernel's TMA loads (passed as a kernel parameter).
struct TileMaps {
  CUtensorMap q;      // q_a boxes of pass 2
  CUtensorMap aux_q;  // (rho, psi) halo tile of pass 1b (QTile)
};

// Tile of pass 1b (the q kernel): TX x TY threads; in 3-D each thread walks TK
// nodes along z (tile TX x TY x TK), in 2-D along y (tile TX x TY*TK).  Taller
// tiles than pass 2's keep the staged halo small against the tile: pass 1b does
// little arithmetic per node, so the halo traffic would dominate.  kPairBytes is
// the size of one staged (rho, psi) pair.  In float32 3-D, 32x8 threads with TK = 8:
// a 41 KB tile, three blocks per SM (see LBM_QFLUX_MINBLOCKS).  Passes 1 + 1b on the
// 512x512x256 impact: 2.06 ms, against 2.08 with 32x4 threads (six blocks per SM),
// 2.16 with 32x2 (ten) and 2.19 with 32x4 threads and TK = 16.
#ifndef LBM_QTILE_TK3_F32
#define LBM_QTILE_TK3_F32 8
#endif
#ifndef LBM_QTILE_TY3
#define LBM_QTILE_TY3 8
#endif
template <int D, int kPairBytes> struct QTile {
  static constexpr int TX = D == 3 ? 32 : 64, TY = D == 3 ? LBM_QTILE_TY3 : 4;
  static constexpr int TK = D == 3 ? (kPairBytes == 8 ? LBM_QTILE_TK3_F32 : 4) : 4;
  static constexpr int EX = TX, EY = D == 3 ? TY : TY * TK, EZ = D == 3 ? TK : 1;  // tile extents
  static constexpr int HX = EX + 4, HY = EY + 4, HZ = D == 3 ? EZ + 4 : 1;         // with the halo
  static constexpr int HN = HX * HY * HZ;
};

// float16-deviation storage: a slot holds delta = f/(w_i rho_w) - 1 in half
// precision, rho_w being the density of the node that wrote it.
template <typename S> struct DevStorage { static constexpr bool value = false; };
template <> struct DevStorage<__half> { static constexpr bool value = true; };

template <typename R> __device__ __forceinline__ const Phys<R>& phys(const DevDomain& d);
template <> __device__ __forceinline__ const Phys<double>& phys<double>(const DevDomain& d) { return d.pd; }
template <> __device__ __forceinline__ const Phys<float>& phys<float>(const DevDomain& d) { return d.pf; }

// ---- storage conversion ----
template <typename S, typename R> __device__ __forceinline__ R ld_pop(const S* p) { return (R)(*p); }
template <typename S, typename R> __device__ __forceinline__ void st_pop(S* p, R v) { *p = (S)v; }
template <> __device__ __forceinline__ float ld_pop<__half, float>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ double ld_pop<__half, double>(const __half* p) { return (double)__half2float(*p); }
template <> __device__ __forceinline__ void st_pop<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }
// Post-collision populations are not read again within the step: streaming
// (evict-first) stores keep the auxiliary fields in L2 instead.
template <> __device__ __forceinline__ void st_pop<float, float>(float* p, float v) { __stcs(p, v); }
template <> __device__ __forceinline__ void st_pop<double, double>(double* p, double v) { __stcs(p, v); }

__device__ __forceinline__ long long node_of(const DevDomain& d, int x, int y, int z) {
  return (long long)x + (long long)d.nx * ((long long)y + (long long)d.ny * (long long)z);
}
template <int D>
__device__ __forceinline__ long long pnode_of(const DevDomain& d, int x, int y, int z) {
  return (long long)(x + 2) + (long long)d.px * ((long long)(y + 2) + (long long)d.py * (long long)(D == 3 ? z + 2 : 0));
}

// A node whose links leave the domain only across a periodic x boundary: every
// y and z neighbour inside, every x neighbour inside or wrapped periodically.  The
// lanes of a warp share y and z (a warp is one x row), so with periodic x they all
// take the same path.
template <int D>
__device__ __forceinline__ bool fast_links(const DevDomain& d, int x, int y, int z) {
  return y >= 1 && y <= d.ny - 2 && (D == 2 || (z >= 1 && z <= d.nz - 2)) &&
         ((x >= 1 && x <= d.nx - 2) || (d.wall_lo[0] == 0 && d.wall_hi[0] == 0));
}

// Padded coordinate of the ghost node that images interior coordinate x along an
// axis of n >= 5 nodes, or -1 when no ghost does (x more than 1 node from both
// faces); *wall is set when that ghost mirrors x across a bounce-back wall.  The
// ghost layers are 2 nodes wide: a periodic ghost sits n nodes away, a wall ghost
// is the mirror image across the half-way wall (the inverse of ghost_image).
__device__ __forceinline__ int ghost_of(int x, int n, int wlo, int whi, bool* wall) {
  if (x <= 1) {
    if (wlo) { *wall = true; return 1 - x; }
    return x + n + 2;
  }
  if (x >= n - 2) {
    if (whi) { *wall = true; return 2 * n + 1 - x; }
    return x - n + 2;
  }
  return -1;
}

// Node index n of (x, y, z) corrected for the periodic x wrap of the neighbour
// r - c along x: b[c + 1], c = -1, 0, +1 (used by fast_links nodes only), and the
// byte address of slot 0 of each in the population array (elements of S).
struct XBase {
  long long b[3];
  char* p[3];
};
template <typename S>
__device__ __forceinline__ XBase xbase(const DevDomain& d, int x, long long n) {
  XBase r;
  r.b[0] = x == d.nx - 1 ? n - d.nx : n;  // x + 1 wraps to 0
  r.b[1] = n;
  r.b[2] = x == 0 ? n + d.nx : n;         // x - 1 wraps to nx - 1
#pragma unroll
  for (int k = 0; k < 3; ++k) r.p[k] = (char*)((S*)d.f + r.b[k]);
  return r;
}

// Bounds-checked builds (-DLBM_BOUNDS_CHECK, the stand-in for a memory checker):
// every computed population address and auxiliary-field index is checked against
// its buffer; one outside it sets bit 2 of the error word (LBM_ERR_BOUNDS) and is
// replaced by the buffer's first element, so that the access stays in bounds.
// Regular builds compile the checks away.
__device__ __forceinline__ long long bc_index(const DevDomain& d, long long i, long long n) {
#ifdef LBM_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    atomicOr(d.flags, 4u);
    return 0;
  }
#endif
  return i;
}
// A padded auxiliary node index (a (rho, psi) pair or one element of a plane).
__device__ __forceinline__ long long bc_pnode(const DevDomain& d, long long pn) { return bc_index(d, pn, d.PN); }
// A population slot address in d.f.
template <int D, typename S>
__device__ __forceinline__ S* bc_pop(const DevDomain& d, S* p) {
#ifdef LBM_BOUNDS_CHECK
  return (S*)d.f + bc_index(d, (long long)(p - (S*)d.f), (long long)Lattice<D>::Q * d.N);
#else
  return p;
#endif
}

// Neighbour coordinate along one axis: periodic wrap, or wall = true when the
// link crosses a bounce-back wall.
__device__ __forceinline__ int step_axis(int x, int c, int n, int wlo, int whi, bool& wall) {
  int t = x + c;
  if (t < 0) { if (wlo) wall = true; else t += n; }
  else if (t >= n) { if (whi) wall = true; else t -= n; }
  return t;
}

// Slot holding the pre-collision population i of node (x,y,z) at parity P:
// P = 0: slot i of the node; P = 1: slot Q-1-i of the upstream node r - c_i, or
// slot i of the node itself when the upstream link crosses a wall.
template <int D, int P, typename S>
__device__ __forceinline__ S* src_ptr(const DevDomain& d, bool fast, const XBase& xb, int x, int y, int z, long long n,
                                      int i) {
  constexpr int Q = Lattice<D>::Q;
  S* F = (S*)d.f;
  if (P == 0) return bc_pop<D>(d, (S*)(xb.p[1] + d.src_boff[0][i]));
  if (fast) return bc_pop<D>(d, (S*)(xb.p[cxi(i) + 1] + d.src_boff[1][i]));
  bool wall = false;
  const int sx = step_axis(x, -cxi(i), d.nx, d.wall_lo[0], d.wall_hi[0], wall);
  const int sy = step_axis(y, -cyi(i), d.ny, d.wall_lo[1], d.wall_hi[1], wall);
  const int sz = D == 3 ? step_axis(z, -czi(i), d.nz, d.wall_lo[2], d.wall_hi[2], wall) : 0;
  return bc_pop<D>(d, F + (wall ? (long long)i * d.N + n : (long long)(Q - 1 - i) * d.N + node_of(d, sx, sy, sz)));
}

// Slot receiving the post-collision population i of node (x,y,z) at parity P:
// streaming f_i(r + c_i) <- f'_i(r); half-way bounce-back f_{Q-1-i}(r) <- f'_i(r)
// when r + c_i lies beyond a wall.
template <int D, int P, typename S>
__device__ __forceinline__ S* dst_ptr(const DevDomain& d, bool fast, const XBase& xb, int x, int y, int z, long long n,
                                      int i) {
  constexpr int Q = Lattice<D>::Q;
  S* F = (S*)d.f;
  if (P == 0) return bc_pop<D>(d, (S*)(xb.p[1] + d.dst_boff[0][i]));
  if (fast) return bc_pop<D>(d, (S*)(xb.p[1 - cxi(i)] + d.dst_boff[1][i]));
  bool wall = false;
  const int tx = step_axis(x, cxi(i), d.nx, d.wall_lo[0], d.wall_hi[0], wall);
  const int ty = step_axis(y, cyi(i), d.ny, d.wall_lo[1], d.wall_hi[1], wall);
  const int tz = D == 3 ? step_axis(z, czi(i), d.nz, d.wall_lo[2], d.wall_hi[2], wall) : 0;
  return bc_pop<D>(d, F + (wall ? (long long)(Q - 1 - i) * d.N + n : (long long)i * d.N + node_of(d, tx, ty, tz)));
}

// Node that wrote the slot population i of node (x,y,z) is read from: the
// upstream node r - c_i, or the node itself when that link crosses a wall.
template <int D>
__device__ __forceinline__ long long upstream_node(const DevDomain& d, bool fast, const XBase& xb, int x, int y, int z,
                                                   long long n, int i) {
  if (fast) return bc_index(d, xb.b[cxi(i) + 1] + d.up_off[i], d.N);
  bool wall = false;
  const int sx = step_axis(x, -cxi(i), d.nx, d.wall_lo[0], d.wall_hi[0], wall);
  const int sy = step_axis(y, -cyi(i), d.ny, d.wall_lo[1], d.wall_hi[1], wall);
  const int sz = D == 3 ? step_axis(z, -czi(i), d.nz, d.wall_lo[2], d.wall_hi[2], wall) : 0;
  return bc_index(d, wall ? n : node_of(d, sx, sy, sz), d.N);
}

template <int D, int P, typename S, typename R>
__device__ __forceinline__ void gather(const DevDomain& d, int x, int y, int z, R* f) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = node_of(d, x, y, z);
  const XBase xb = xbase<S>(d, x, n);
  if constexpr (DevStorage<S>::value) {
    // f_i = w_i rho_w (1 + delta_i)
    const float* rw = d.rho_w[P];
    if (fast_links<D>(d, x, y, z)) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        f[i] = (R)wq<D>(i) * (R)rw[upstream_node<D>(d, true, xb, x, y, z, n, i)] *
               ((R)1 + ld_pop<S, R>(src_ptr<D, P, S>(d, true, xb, x, y, z, n, i)));
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        f[i] = (R)wq<D>(i) * (R)rw[upstream_node<D>(d, false, xb, x, y, z, n, i)] *
               ((R)1 + ld_pop<S, R>(src_ptr<D, P, S>(d, false, xb, x, y, z, n, i)));
    }
  } else if (P == 0 || fast_links<D>(d, x, y, z)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = ld_pop<S, R>(src_ptr<D, P, S>(d, true, xb, x, y, z, n, i));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = ld_pop<S, R>(src_ptr<D, P, S>(d, false, xb, x, y, z, n, i));
  }
}

// Runtime-parity form for the field I/O kernels.
template <int D, typename S, typename R>
__device__ __forceinline__ void gather(const DevDomain& d, int parity, int x, int y, int z, R* f) {
  if (parity == 0) gather<D, 0, S, R>(d, x, y, z, f);
  else gather<D, 1, S, R>(d, x, y, z, f);
}

// rho = sum_i f_i (ascending i), j = sum_i c_i f_i, Pi_ab = sum_i c_ia c_ib f_i.
// Pi order: xx, yy, zz, xy, xz, yz.
template <int D, typename R>
__device__ __forceinline__ void moments(const R* f, R& rho, R* j, R* Pi) {
  constexpr int Q = Lattice<D>::Q;
  rho = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) rho += f[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) j[a] = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) Pi[k] = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int c0 = cq<D>(i, 0), c1 = cq<D>(i, 1), c2 = cq<D>(i, 2);
    if (c0 > 0) j[0] += f[i]; else if (c0 < 0) j[0] -= f[i];
    if (c1 > 0) j[1] += f[i]; else if (c1 < 0) j[1] -= f[i];
    if (c2 > 0) j[2] += f[i]; else if (c2 < 0) j[2] -= f[i];
    if (c0 != 0) Pi[0] += f[i];
    if (c1 != 0) Pi[1] += f[i];
    if (c2 != 0) Pi[2] += f[i];
    if (c0 * c1 > 0) Pi[3] += f[i]; else if (c0 * c1 < 0) Pi[3] -= f[i];
    if (c0 * c2 > 0) Pi[4] += f[i]; else if (c0 * c2 < 0) Pi[4] -= f[i];
    if (c1 * c2 > 0) Pi[5] += f[i]; else if (c1 * c2 < 0) Pi[5] -= f[i];
  }
}

// Peng-Robinson pressure, Eq. (PREoS).
template <typename T>
__device__ __forceinline__ T pr_pressure(const Phys<T>& p, T rho) {
  return rho * p.RT / ((T)1 - p.b * rho) - p.aalpha * rho * rho / ((T)1 + (T)2 * p.b * rho - p.b * p.b * rho * rho);
}

// Pseudo-potential psi = sqrt|P - P0|, P0 = rho cs^2 (Sec. 2.3); its sign s comes
// from psi_sign.
template <typename R>
__device__ __forceinline__ R psi_of(const DevDomain& d, R rho) {
  if (sizeof(R) == 8 || d.eos_fp64 == 2 ||
      (d.eos_fp64 == 1 && rho > phys<R>(d).band_lo && rho < phys<R>(d).band_hi)) {
    const double r = (double)rho;
    return (R)sqrt(fabs(pr_pressure<double>(d.pd, r) - r * (1.0 / 3.0)));
  }
  const float r = (float)rho;
  return (R)sqrtf(fabsf(pr_pressure<float>(d.pf, r) - r * (1.0f / 3.0f)));
}

// s = +1 where P(rho) > rho cs^2, else -1 (Sec. 2.3), from the host-computed
// densities where P(rho) - rho cs^2 changes sign.
template <typename R>
__device__ __forceinline__ R psi_sign(const Phys<R>& p, R rho) {
  R s = p.sgn0;
#pragma unroll
  for (int k = 0; k < 3; ++k) s = rho >= p.sgn_t[k] ? -s : s;
  return s;
}

template <typename R>
__device__ __forceinline__ R omega_of(const Phys<R>& p, R rho) {
  R phi = (rho - p.rho_v) * p.inv_drho;
  phi = phi < (R)0 ? (R)0 : (phi > (R)1 ? (R)1 : phi);
  const R nu = p.nu_v + phi * p.dnu;
  return (R)1 / ((R)3 * nu + (R)0.5);
}

}  // namespace lbm
