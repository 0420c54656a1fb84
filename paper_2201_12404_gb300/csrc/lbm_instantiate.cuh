// Instantiates the launch table for one lattice dimension (included once per
// lattice translation unit so that the two lattices compile in parallel).
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_ops.h"

namespace lbm {

template <int D, typename S, typename R, typename A>
struct Launch {
  static dim3 node_grid(const DevDomain& d) {
    return dim3((d.nx + Blocks<D>::bx - 1) / Blocks<D>::bx, (d.ny + Blocks<D>::by - 1) / Blocks<D>::by,
                (d.nz + Blocks<D>::bz - 1) / Blocks<D>::bz);
  }
  static void moments_eos(const DevDomain& d, int parity, cudaStream_t s) {
    dim3 blk(Blocks<D>::bx, Blocks<D>::by, Blocks<D>::bz);
    if (parity == 0) moments_eos_kernel<D, 0, S, R, A><<<node_grid(d), blk, 0, s>>>(d);
    else moments_eos_kernel<D, 1, S, R, A><<<node_grid(d), blk, 0, s>>>(d);
  }
  static void qflux(const DevDomain& d, const TileMaps& maps, cudaStream_t s) {
    using T = QTile<D, 2 * sizeof(A)>;
    constexpr size_t smem = qflux_dyn_smem<D, A>();
    auto k = qflux_tile_kernel<D, R, A>;
    constexpr int kMaxDev = 64;
    static bool opted_in[kMaxDev] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024 && (dev < 0 || dev >= kMaxDev || !opted_in[dev])) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (dev >= 0 && dev < kMaxDev) opted_in[dev] = true;
    }
    const dim3 grd((d.nx + T::EX - 1) / T::EX, (d.ny + T::EY - 1) / T::EY, (d.nz + T::EZ - 1) / T::EZ);
    k<<<grd, dim3(T::TX, T::TY), smem, s>>>(d, maps);
  }
  static void collide_stream(const DevDomain& d, const TileMaps& maps, int parity, cudaStream_t s) {
    dim3 blk(Blocks<D>::bx, Blocks<D>::by, Blocks<D>::bz);
    if constexpr (sizeof(S) == 8) {
      // float64: one block per SM, so the persistent form keeps the next tile's
      // loads in flight; float32 and float16 keep one tile per block (three blocks
      // per SM overlap each other's loads, and the staging copies would only add
      // shared-memory traffic)
      constexpr size_t smem = persistent_dyn_smem<D, S, R>();
      auto k = parity == 0 ? collide_stream_persistent_kernel<D, 0, S, R, A>
                           : collide_stream_persistent_kernel<D, 1, S, R, A>;
      const dim3 tiles = node_grid(d);
      const long long ntiles = (long long)tiles.x * tiles.y * tiles.z;
      const int slots = resident_slots((const void*)k, blk.x * blk.y * blk.z, smem);
      const int grid = (int)(ntiles < slots ? ntiles : slots);
      k<<<grid, blk, smem, s>>>(d, maps, (int)tiles.x, (int)tiles.y, (int)ntiles);
    } else {
      constexpr size_t smem = collide_dyn_smem<D, R>();
      auto k = parity == 0 ? collide_stream_kernel<D, 0, S, R, A> : collide_stream_kernel<D, 1, S, R, A>;
      // static (staged fields) plus dynamic (h) shared memory exceeds the 48 KB default
      constexpr int kMaxDev = 64;
      static bool opted_in[2][kMaxDev] = {};
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= kMaxDev || !opted_in[parity][dev]) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < kMaxDev) opted_in[parity][dev] = true;
      }
      k<<<node_grid(d), blk, smem, s>>>(d, maps);
    }
  }
  // Blocks of kernel k resident on the whole device at once (SMs x blocks per SM),
  // with the dynamic shared memory attributes set; computed once per kernel and device.
  static int resident_slots(const void* k, int threads, size_t smem) {
    constexpr int kMaxDev = 64;
    static int cache[2][kMaxDev] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int which = k == (const void*)collide_stream_persistent_kernel<D, 0, S, R, A> ? 0 : 1;
    int* slot = dev >= 0 && dev < kMaxDev ? &cache[which][dev] : nullptr;
    if (slot && *slot > 0) return *slot;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int n = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (slot) *slot = n;
    return n;
  }
  static unsigned blocks1d(const DevDomain& d) { return (unsigned)((d.N + 255) / 256); }
  static void init_equilibrium(const DevDomain& d, const double* rho, const double* ux, const double* uy,
                               const double* uz, cudaStream_t s) {
    init_equilibrium_kernel<D, S, R><<<blocks1d(d), 256, 0, s>>>(d, rho, ux, uy, uz);
  }
  static void aux_density(const DevDomain& d, const double* rho, cudaStream_t s) {
    dim3 blk(Blocks<D>::bx, Blocks<D>::by, Blocks<D>::bz);
    dim3 grd((d.px + blk.x - 1) / blk.x, (d.py + blk.y - 1) / blk.y, (d.pz + blk.z - 1) / blk.z);
    aux_density_kernel<D, R, A><<<grd, blk, 0, s>>>(d, rho);
  }
  static void canonical_read(const DevDomain& d, int parity, double* out, cudaStream_t s) {
    canonical_read_kernel<D, S><<<blocks1d(d), 256, 0, s>>>(d, parity, out);
  }
  static void canonical_window(const DevDomain& d, int parity, const int o[3], const int e[3], double* out,
                               cudaStream_t s) {
    const long long m = (long long)e[0] * e[1] * e[2];
    canonical_window_kernel<D, S><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d, parity, o[0], o[1], o[2], e[0], e[1],
                                                                              e[2], out);
  }
  static void canonical_write(const DevDomain& d, const double* in, cudaStream_t s) {
    if constexpr (DevStorage<S>::value) canonical_density_kernel<D><<<blocks1d(d), 256, 0, s>>>(d, in);
    canonical_write_kernel<D, S><<<blocks1d(d), 256, 0, s>>>(d, in);
  }
  static void macroscopic(const DevDomain& d, int parity, double* rho, double* u, cudaStream_t s) {
    macroscopic_kernel<D, S, R, A><<<blocks1d(d), 256, 0, s>>>(d, parity, rho, u);
  }
  static void bare_velocity(const DevDomain& d, const double* rho, double* u, cudaStream_t s) {
    bare_velocity_kernel<D, R, A><<<blocks1d(d), 256, 0, s>>>(d, rho, u);
  }
  static int diag_partial(const DevDomain& d, int parity, double* partial, cudaStream_t s) {
    diag_partial_kernel<D, S><<<blocks1d(d), 256, 0, s>>>(d, parity, partial);
    return (int)blocks1d(d);
  }
  static int max_speed_partial(const DevDomain& d, int parity, double* partial, cudaStream_t s) {
    max_speed_partial_kernel<D, S, R, A><<<blocks1d(d), 256, 0, s>>>(d, parity, partial);
    return (int)blocks1d(d);
  }
  static void drop_on_film(const DevDomain& d, const lbm_drop_on_film& g, double rho_l, double rho_v, double* rho,
                           double* u, cudaStream_t s) {
    drop_on_film_kernel<D><<<blocks1d(d), 256, 0, s>>>(d, g.radius, g.film, g.gap, g.speed, g.width, g.noise,
                                                       (unsigned long long)g.seed, rho_l, rho_v, rho, u);
  }
  static int grad_partial(const DevDomain& d, double* partial, cudaStream_t s) {
    grad_partial_kernel<D, A><<<blocks1d(d), 256, 0, s>>>(d, partial);
    return (int)blocks1d(d);
  }
  static int crown_partial(const DevDomain& d, int layer, double rho_mid, double* partial, cudaStream_t s) {
    const long long nl = D == 3 ? (long long)d.nx * d.ny : d.nx;
    const unsigned nb = (unsigned)((nl + 255) / 256);
    crown_partial_kernel<D, A><<<nb, 256, 0, s>>>(d, layer, rho_mid, partial);
    return (int)nb;
  }
  static Ops table() {
    return Ops{D, Lattice<D>::Q, sizeof(S), sizeof(A), &moments_eos, &qflux, &collide_stream, &init_equilibrium, &aux_density,
               &canonical_read, &canonical_write, &canonical_window, &macroscopic, &bare_velocity, &diag_partial,
               &max_speed_partial, &drop_on_film, &grad_partial, &crown_partial};
  }
};

}  // namespace lbm
