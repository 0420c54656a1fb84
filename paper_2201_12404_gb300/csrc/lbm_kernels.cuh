// Kernels of one time step and of the field I/O, templated on the lattice
// dimension D, the population storage type S and the arithmetic type R.
//
//  moments_eos_kernel    (pass 1)  gather f, form rho and j, evaluate the
//                                  Peng-Robinson pseudo-potential; writes (rho, psi) and
//                                  j to the padded auxiliary fields, ghosts included.
//  qflux_tile_kernel     (pass 1b) F from the (rho, psi) halo tile (Eq. Kforce_final)
//                                  and q = rho v^3, v = (j + F/2)/rho the fluid
//                                  velocity; q to the node and the ghosts imaging it,
//                                  F over the node's j.
//  collide_stream_kernel (pass 2)  gather f, the node's F from pass 1b, Phi from the
//                                  staged q boxes (Eq. correction), f^eq and
//                                  f* (Eqs. LBMeq, LBMstar), k/s/h split (Appendix A),
//                                  gamma (Sec. 2.4), relaxation (Eq. LBGK), A-A write.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Pass 1: one thread per interior node; the node also writes the ghost nodes
// that image it (periodic wrap or mirror across a half-way wall).
// ---------------------------------------------------------------------------
// Interior coordinate that padded coordinate cp (ghost layers of 2) images along
// an axis of n nodes: periodic wrap, or the mirror across a half-way wall (which
// sets *flip).
__device__ __forceinline__ int ghost_image(int cp, int n, int wlo, int whi, bool* flip) {
  int t = cp - 2;
  if (t < 0) { if (wlo) { t = -1 - t; *flip = true; } else t += n; }
  else if (t >= n) { if (whi) { t = 2 * n - 1 - t; *flip = true; } else t -= n; }
  return t;
}

// Pass 1 at interior node (x, y, z): rho and j from the gathered populations, psi
// from the Peng-Robinson pressure.  The (rho, psi) pair goes to the node's padded
// position and to every ghost node imaging it (each combination of its own or its
// ghost coordinate on the axes that have one), so that the later passes index
// their stencils without wrap logic; j goes to the node alone (pass 1b reads it
// there).  A warp is one aligned x row of 32 interior nodes, so each of its 27
// population loads is one 128-byte line.
template <int D, int P, typename S, typename R, typename A>
__device__ __forceinline__ void moments_eos_node(const DevDomain& d, int x, int y, int z) {
  constexpr int Q = Lattice<D>::Q;
  if (x >= d.nx || y >= d.ny || z >= d.nz) return;
  R f[Q];
  gather<D, P, S, R>(d, x, y, z, f);
  R rho, j[3], Pi[6];
  moments<D, R>(f, rho, j, Pi);
  if (!(rho > (R)0) || !(rho < (R)INFINITY)) atomicOr(d.flags, 1u);

  A* aux = (A*)d.aux;
  Two<A>* a2 = (Two<A>*)d.aux;
  const long long pn = bc_pnode(d, pnode_of<D>(d, x, y, z));
  const Two<A> pair = two<A>((A)rho, (A)psi_of<R>(d, rho));
  a2[pn] = pair;
#pragma unroll
  for (int a = 0; a < D; ++a) aux[(2 + D + a) * d.PN + pn] = (A)j[a];
  bool wall = false;
  const int gx = ghost_of(x, d.nx, d.wall_lo[0], d.wall_hi[0], &wall);
  const int gy = ghost_of(y, d.ny, d.wall_lo[1], d.wall_hi[1], &wall);
  const int gz = D == 3 ? ghost_of(z, d.nz, d.wall_lo[2], d.wall_hi[2], &wall) : -1;
  if (gx < 0 && gy < 0 && gz < 0) return;
#pragma unroll 1
  for (int m = 1; m < (1 << D); ++m) {
    if (((m & 1) && gx < 0) || ((m & 2) && gy < 0) || ((m & 4) && gz < 0)) continue;
    const int cx = (m & 1) ? gx : x + 2, cy = (m & 2) ? gy : y + 2, cz = D == 3 ? ((m & 4) ? gz : z + 2) : 0;
    a2[bc_pnode(d, (long long)cx + (long long)d.px * ((long long)cy + (long long)d.py * cz))] = pair;
  }
}

// The (rho, psi) pairs of every padded node straight from a density field
// (device, float64, N values), ghosts included: what pass 1 writes for a state
// whose density is that field, without forming populations first.  q is left
// alone (the next pass 1 writes it).
template <int D, typename R, typename A>
__global__ void __launch_bounds__(256) aux_density_kernel(DevDomain d, const double* rho_in) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x, yp = blockIdx.y * blockDim.y + threadIdx.y;
  const int zp = blockIdx.z * blockDim.z + threadIdx.z;
  if (xp >= d.nx + 4 || yp >= d.py || zp >= d.pz) return;
  bool flip = false;
  const int x = ghost_image(xp, d.nx, d.wall_lo[0], d.wall_hi[0], &flip);
  const int y = ghost_image(yp, d.ny, d.wall_lo[1], d.wall_hi[1], &flip);
  const int z = D == 3 ? ghost_image(zp, d.nz, d.wall_lo[2], d.wall_hi[2], &flip) : 0;
  const R rho = (R)rho_in[node_of(d, x, y, z)];
  if (!(rho > (R)0) || !(rho < (R)INFINITY)) atomicOr(d.flags, 1u);
  const long long pn = (long long)xp + (long long)d.px * ((long long)yp + (long long)d.py * (long long)zp);
  ((Two<A>*)d.aux)[pn] = two<A>((A)rho, (A)psi_of<R>(d, rho));
}

template <int D, int P, typename S, typename R, typename A>
__global__ void __launch_bounds__(256) moments_eos_kernel(DevDomain d) {
  moments_eos_node<D, P, S, R, A>(d, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
                                  blockIdx.z * blockDim.z + threadIdx.z);
}

}  // namespace lbm

#include "lbm_collide.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// f := f^eq(rho, u) at every node (natural layout, parity 0).
// ---------------------------------------------------------------------------
template <int D, typename S, typename R>
__global__ void init_equilibrium_kernel(DevDomain d, const double* rho, const double* ux,
                                        const double* uy, const double* uz) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  const R r = (R)rho[n];
  const R u[3] = {(R)ux[n], (R)uy[n], D == 3 ? (R)uz[n] : (R)0};
  R X[3][3];
  for (int a = 0; a < 3; ++a) {
    const R u2 = u[a] * u[a];
    X[a][1] = a < D ? (R)1 - (R)(1.0 / 3.0) - u2 : (R)1;
    X[a][2] = a < D ? (R)0.5 * ((R)(1.0 / 3.0) + u2 + u[a]) : (R)0;
    X[a][0] = a < D ? (R)0.5 * ((R)(1.0 / 3.0) + u2 - u[a]) : (R)0;
  }
  S* F = (S*)d.f;
  if constexpr (DevStorage<S>::value) {
    // each slot is encoded against the density of its upstream (writer) node; the
    // next step (even parity) decodes with rho_w[0] of that node
    const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
    const bool fast = fast_links<D>(d, x, y, z);
    const XBase xb = xbase<S>(d, x, n);
    d.rho_w[0][n] = (float)r;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R rw = (R)(float)rho[upstream_node<D>(d, fast, xb, x, y, z, n, i)];
      const R feq = r * X[0][cxi(i) + 1] * X[1][cyi(i) + 1] * X[2][D == 3 ? czi(i) + 1 : 1];
      F[(long long)i * d.N + n] = __float2half_rn((float)(feq / ((R)wq<D>(i) * rw) - (R)1));
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      st_pop<S, R>(F + (long long)i * d.N + n, r * X[0][cxi(i) + 1] * X[1][cyi(i) + 1] * X[2][D == 3 ? czi(i) + 1 : 1]);
  }
}

// ---------------------------------------------------------------------------
// Canonical (post-stream, pre-collision) populations <-> float64 buffer.
// ---------------------------------------------------------------------------
template <int D, typename S>
__global__ void canonical_read_kernel(DevDomain d, int parity, double* out) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
  double f[Q];
  gather<D, S, double>(d, parity, x, y, z, f);
  for (int i = 0; i < Q; ++i) out[(long long)i * d.N + n] = f[i];
}

// The same for the nodes of a box: window node (i, j, k) is domain node
// ((ox + i) mod nx, (oy + j) mod ny, (oz + k) mod nz); the host checks 0 <= o < n
// and 1 <= e <= n per axis, so o + i < 2n never overflows.
template <int D, typename S>
__global__ void canonical_window_kernel(DevDomain d, int parity, int ox, int oy, int oz, int ex, int ey, int ez,
                                        double* out) {
  constexpr int Q = Lattice<D>::Q;
  const long long m = (long long)ex * ey * ez;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int i = (int)(k % ex), j = (int)((k / ex) % ey), l = (int)(k / ((long long)ex * ey));
  int x = ox + i, y = oy + j, z = oz + l;
  if (x >= d.nx) x -= d.nx;
  if (y >= d.ny) y -= d.ny;
  if (z >= d.nz) z -= d.nz;
  double f[Q];
  gather<D, S, double>(d, parity, x, y, z, f);
  for (int q = 0; q < Q; ++q) out[(long long)q * m + k] = f[q];
}

template <int D, typename S>
__global__ void canonical_write_kernel(DevDomain d, const double* in) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  S* F = (S*)d.f;
  if constexpr (DevStorage<S>::value) {
    // rho_w[0] holds every node's density (canonical_density_kernel, launched before)
    const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
    const bool fast = fast_links<D>(d, x, y, z);
    const XBase xb = xbase<S>(d, x, n);
    for (int i = 0; i < Q; ++i) {
      const double rw = (double)d.rho_w[0][upstream_node<D>(d, fast, xb, x, y, z, n, i)];
      F[(long long)i * d.N + n] = __float2half_rn((float)(in[(long long)i * d.N + n] / (wq<D>(i) * rw) - 1.0));
    }
  } else {
    for (int i = 0; i < Q; ++i) st_pop<S, double>(F + (long long)i * d.N + n, in[(long long)i * d.N + n]);
  }
}

// float16-deviation storage: density of every node of a canonical state into rho_w[0].
template <int D>
__global__ void canonical_density_kernel(DevDomain d, const double* in) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  double r = 0.0;
  for (int i = 0; i < Q; ++i) r += in[(long long)i * d.N + n];
  d.rho_w[0][n] = (float)r;
}

// ---------------------------------------------------------------------------
// Force density F at node (x, y, z) from the auxiliary fields of the current
// state (Eq. Kforce_final with the sign of reading R1), rho the node's density:
// the link-by-link form of the stencil pass 2 evaluates row by row.
// ---------------------------------------------------------------------------
template <int D, typename R, typename A>
__device__ __forceinline__ void aux_force(const DevDomain& d, int x, int y, int z, R rho, R* F) {
  constexpr int Q = Lattice<D>::Q;
  const Two<A>* a2 = (const Two<A>*)d.aux;  // (rho, psi)
  const long long pc = pnode_of<D>(d, x, y, z);
  const long long sy = d.px, sz = (long long)d.px * d.py;
  R g4[3] = {0, 0, 0}, g3[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    if (i == Lattice<D>::REST) continue;
    const long long o = cxi(i) + sy * cyi(i) + (D == 3 ? sz * czi(i) : 0);
    const R t4 = (R)(4.0 / 3.0) * (R)a2[pc + o].y - (R)(1.0 / 6.0) * (R)a2[pc + 2 * o].y;
    const R t3 = (R)2 * (R)a2[pc + o].x - (R)a2[pc + 2 * o].x;
    const R W = (R)(3.0 * wq<D>(i));
    for (int a = 0; a < D; ++a) {
      const int c = cq<D>(i, a);
      g4[a] += W * (R)c * t4;
      g3[a] += W * (R)c * t3;
    }
  }
  const R spsi_c = psi_sign<R>(phys<R>(d), (R)a2[pc].x) * (R)a2[pc].y;
  for (int a = 0; a < 3; ++a)
    F[a] = a < D ? -((R)2 * spsi_c * g4[a] + phys<R>(d).kappa * rho * g3[a]) + rho * phys<R>(d).g[a] : (R)0;
}

// ---------------------------------------------------------------------------
// Density and exact-difference-method velocity u + F/(2 rho); the auxiliary
// fields must describe the current state (pass 1 run just before).
// ---------------------------------------------------------------------------
template <int D, typename S, typename R, typename A>
__global__ void macroscopic_kernel(DevDomain d, int parity, double* rho_out, double* u_out) {
  constexpr int Q = Lattice<D>::Q;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
  R f[Q];
  gather<D, S, R>(d, parity, x, y, z, f);
  R rho, j[3], Pi[6];
  moments<D, R>(f, rho, j, Pi);
  R F[3];
  aux_force<D, R, A>(d, x, y, z, rho, F);
  rho_out[n] = (double)rho;
  for (int a = 0; a < D; ++a) u_out[a * d.N + n] = (double)((j[a] + (R)0.5 * F[a]) / rho);
}

// ---------------------------------------------------------------------------
// Largest speed |u + F/(2 rho)| of the reported velocity (the velocity
// macroscopic_kernel writes), one partial maximum per block in field 4 of the
// [block][5] layout that diag_final_kernel reduces (fields 0-3 zero).  The
// auxiliary fields must describe the current state.
// ---------------------------------------------------------------------------
template <int D, typename S, typename R, typename A>
__global__ void __launch_bounds__(256) max_speed_partial_kernel(DevDomain d, int parity, double* partial) {
  constexpr int Q = Lattice<D>::Q;
  __shared__ double sh[256];
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double um = 0;
  if (n < d.N) {
    const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
    R f[Q];
    gather<D, S, R>(d, parity, x, y, z, f);
    R rho, j[3], Pi[6];
    moments<D, R>(f, rho, j, Pi);
    R F[3];
    aux_force<D, R, A>(d, x, y, z, rho, F);
    double u2 = 0;
    for (int a = 0; a < D; ++a) {
      const double ua = (double)((j[a] + (R)0.5 * F[a]) / rho);
      u2 += ua * ua;
    }
    um = sqrt(u2);
    if (!(um == um)) um = INFINITY;  // a non-finite state reports an infinite speed
  }
  sh[threadIdx.x] = um;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) partial[blockIdx.x * 5 + k] = 0.0;
    partial[blockIdx.x * 5 + 4] = sh[0];
  }
}

// ---------------------------------------------------------------------------
// Drop-on-film initial fields (float64, natural layout): see lbm_init_drop_on_film.
// The white noise draws from SplitMix64 (Steele, Lea & Flood 2014) keyed by
// (seed, node, component), two uniforms per value, normal by Box-Muller.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_open(unsigned long long z) {  // (0, 1]
  return ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

template <int D>
__global__ void drop_on_film_kernel(DevDomain d, double R, double film, double gap, double U, double W, double noise,
                                    unsigned long long seed, double rho_l, double rho_v, double* rho, double* u) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
  const double vert = D == 3 ? (double)z : (double)y;
  const double cv = film + R + gap;
  const double dx = x - 0.5 * (d.nx - 1);
  const double dy = D == 3 ? y - 0.5 * (d.ny - 1) : vert - cv;
  const double dz = D == 3 ? vert - cv : 0.0;
  const double d_drop = sqrt(dx * dx + dy * dy + dz * dz) - R;
  const double d_film = film > 0 ? vert - (film - 0.5) : INFINITY;
  const double dist = fmin(d_drop, d_film);
  rho[n] = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * tanh(2.0 * dist / W);
  const double liq = 0.5 - 0.5 * tanh(2.0 * d_drop / W);
  for (int a = 0; a < D; ++a) {
    double v = a == D - 1 ? -U * liq : 0.0;
    if (noise > 0) {
      const unsigned long long key = seed ^ ((unsigned long long)n * (unsigned long long)(2 * D) + 2ull * a) * 0xD1B54A32D192ED03ull;
      const double u1 = unit_open(splitmix64(key)), u2 = unit_open(splitmix64(key + 1));
      v += noise * U * liq * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
    u[a * d.N + n] = v;
  }
}

// ---------------------------------------------------------------------------
// Largest |grad rho| of the auxiliary density (second-order central differences;
// the ghost layer supplies the wrapped or mirrored neighbours), one partial
// maximum per block in field 4 of the diag layout.
// ---------------------------------------------------------------------------
template <int D, typename A>
__global__ void __launch_bounds__(256) grad_partial_kernel(DevDomain d, double* partial) {
  __shared__ double sh[256];
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double gm = 0;
  if (n < d.N) {
    const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
    const Two<A>* a2 = (const Two<A>*)d.aux;
    const long long pc = pnode_of<D>(d, x, y, z);
    const long long e[3] = {1, d.px, (long long)d.px * d.py};
    double g2 = 0;
    for (int a = 0; a < D; ++a) {
      const double ga = 0.5 * ((double)a2[pc + e[a]].x - (double)a2[pc - e[a]].x);
      g2 += ga * ga;
    }
    gm = sqrt(g2);
  }
  sh[threadIdx.x] = gm;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) partial[blockIdx.x * 5 + k] = 0.0;
    partial[blockIdx.x * 5 + 4] = sh[0];
  }
}

// ---------------------------------------------------------------------------
// Crown radius: over the nodes of one layer (index `layer` along the last axis),
// the largest distance from the vertical axis through the domain centre of a
// node whose auxiliary density exceeds rho_mid; one partial maximum per block in
// field 4 of the diag layout (0 where no node qualifies).
// ---------------------------------------------------------------------------
template <int D, typename A>
__global__ void __launch_bounds__(256) crown_partial_kernel(DevDomain d, int layer, double rho_mid, double* partial) {
  __shared__ double sh[256];
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nl = D == 3 ? (long long)d.nx * d.ny : d.nx;
  double rm = 0;
  if (k < nl) {
    const int x = (int)(k % d.nx);
    const int y = D == 3 ? (int)(k / d.nx) : layer;
    const int z = D == 3 ? layer : 0;
    const Two<A>* a2 = (const Two<A>*)d.aux;
    if ((double)a2[pnode_of<D>(d, x, y, z)].x > rho_mid) {
      const double dx = x - 0.5 * (d.nx - 1), dy = D == 3 ? y - 0.5 * (d.ny - 1) : 0.0;
      rm = sqrt(dx * dx + dy * dy);
    }
  }
  sh[threadIdx.x] = rm;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) partial[blockIdx.x * 5 + q] = 0.0;
    partial[blockIdx.x * 5 + 4] = sh[0];
  }
}

// ---------------------------------------------------------------------------
// Bare velocity of a state at rest in the reported sense: u -= F dt/(2 rho) in
// place, F from the auxiliary fields of the current (equilibrium) state.
// ---------------------------------------------------------------------------
template <int D, typename R, typename A>
__global__ void bare_velocity_kernel(DevDomain d, const double* rho_in, double* u) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.N) return;
  const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
  const R rho = (R)((const Two<A>*)d.aux)[pnode_of<D>(d, x, y, z)].x;
  R F[3];
  aux_force<D, R, A>(d, x, y, z, rho, F);
  for (int a = 0; a < D; ++a) u[a * d.N + n] -= (double)F[a] / (2.0 * rho_in[n]);
}

// ---------------------------------------------------------------------------
// Deterministic totals: per-block partial sums (fixed order), then one block.
// partial layout: [block][5] = mass, jx, jy, jz, max|u|.
// ---------------------------------------------------------------------------
template <int D, typename S>
__global__ void __launch_bounds__(256) diag_partial_kernel(DevDomain d, int parity, double* partial) {
  constexpr int Q = Lattice<D>::Q;
  __shared__ double sh[5][256];
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0, jj[3] = {0, 0, 0}, um = 0;
  if (n < d.N) {
    const int x = (int)(n % d.nx), y = (int)((n / d.nx) % d.ny), z = (int)(n / ((long long)d.nx * d.ny));
    double f[Q];
    gather<D, S, double>(d, parity, x, y, z, f);
    double Pi[6];
    moments<D, double>(f, m, jj, Pi);
    const double u2 = (jj[0] * jj[0] + jj[1] * jj[1] + jj[2] * jj[2]) / (m * m);
    um = sqrt(u2);
  }
  sh[0][threadIdx.x] = m; sh[1][threadIdx.x] = jj[0]; sh[2][threadIdx.x] = jj[1];
  sh[3][threadIdx.x] = jj[2]; sh[4][threadIdx.x] = um;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
      sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partial[blockIdx.x * 5 + k] = sh[k][0];
}

static __global__ void diag_final_kernel(const double* partial, int nblocks, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    for (int k = 0; k < 4; ++k) acc[k] += partial[b * 5 + k];
    acc[4] = fmax(acc[4], partial[b * 5 + 4]);
  }
  for (int k = 0; k < 5; ++k) out[k] = acc[k];
}

}  // namespace lbm
