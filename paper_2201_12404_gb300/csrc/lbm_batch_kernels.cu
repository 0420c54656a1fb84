// Persistent kernel that advances a batch of D2Q9 domains of uneven sizes by
// nsteps time steps in one launch.  The blocks of a cooperative launch walk the
// work list of tiles (every job's interior) three times per step, for pass 1,
// pass 1b and pass 2, with a grid barrier after each.  The per-tile work is the
// same code as the single-domain kernels (moments_eos_node, qflux_tile_staged,
// collide_tile), with pass 1b's halo tile staged by warps.
#include "../../include/lbm.h"
#include "lbm_batch.h"
#include "lbm_kernels.cuh"

namespace lbm {

// Bounded grid barrier for a cooperative launch (all blocks co-resident).  The
// generation is read before arriving; the last block to arrive resets the
// arrival count and advances the generation.  A wait gives up after `limit`
// polls (each sleeps ~0.1 us; the default limit is far above any real wait).
// Returns false when the wait gave up or another block already reported a
// timeout.  skip (a test switch) makes block 0 pass without arriving or waiting,
// so that the other blocks' waits run out: the timeout path, with no fault.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int* error, unsigned int limit, int skip) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    int ok = 1;
    if (skip && blockIdx.x == 0) {
      ok = (*(volatile unsigned int*)error & 2u) ? 0 : 1;
    } else if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned int polls = 0;
      while (*vgen == gen) {
        if (++polls > limit || (*(volatile unsigned int*)error & 2u)) { ok = 0; break; }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (!ok) atomicOr(error, 2u);
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Minimum resident blocks per SM for the float32/float16 batch kernel.  Five
// (51 registers, a few spilled) beat four (64, none) on the 16-job coexistence
// batch: 17.7 against 16.7 GLUPS.
#ifndef LBM_BATCH_MINBLOCKS_F32
#define LBM_BATCH_MINBLOCKS_F32 5
#endif
template <int BX, int BY, typename S, typename R, typename A>
__global__ void __launch_bounds__(BX * BY, sizeof(R) == 4 ? LBM_BATCH_MINBLOCKS_F32 : 1) batch_persistent_kernel(BatchArgs a) {
  __shared__ __align__(128) Two<A> s_aux[Halo<2, BX, BY, 1>::HN];
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  R* s_h = (R*)smem_dyn;
  for (int s = 0; s < a.nsteps; ++s) {
    // pass 1 over the interior tiles (each node also writes its ghost images)
    for (int it = blockIdx.x; it < a.n_k2; it += gridDim.x) {
      const BatchItem w = a.k2[it];
      const DevDomain& d = a.jobs[w.job];
      const int x = w.tx * BX + threadIdx.x, y = w.ty * BY + threadIdx.y;
      if (((a.parity[w.job] + s) & 1) == 0) moments_eos_node<2, 0, S, R, A>(d, x, y, 0);
      else moments_eos_node<2, 1, S, R, A>(d, x, y, 0);
    }
    if (!grid_barrier(a.barrier, a.error, a.poll_limit, a.skip_arrival)) return;
    // pass 1b: q over the interior tiles (and the ghosts imaging them)
    for (int it = blockIdx.x; it < a.n_k2; it += gridDim.x) {
      __syncthreads();  // the previous tile's threads are done with s_aux
      const BatchItem w = a.k2[it];
      qflux_tile_staged<2, BX, BY, 1, R, A>(a.jobs[w.job], w.tx * BX, w.ty * BY, 0, s_aux);
    }
    if (!grid_barrier(a.barrier, a.error, a.poll_limit, a.skip_arrival)) return;
    // pass 2: nothing staged is shared between threads (each uses its own column
    // of s_h), so the tiles need no block barrier
    for (int it = blockIdx.x; it < a.n_k2; it += gridDim.x) {
      const BatchItem w = a.k2[it];
      const DevDomain& d = a.jobs[w.job];
      if (((a.parity[w.job] + s) & 1) == 0)
        collide_tile<2, BX, BY, 1, 0, S, R, A, false>(d, nullptr, w.tx * BX, w.ty * BY, 0, nullptr, s_h, nullptr, 0);
      else
        collide_tile<2, BX, BY, 1, 1, S, R, A, false>(d, nullptr, w.tx * BX, w.ty * BY, 0, nullptr, s_h, nullptr, 0);
    }
    if (!grid_barrier(a.barrier, a.error, a.poll_limit, a.skip_arrival)) return;
  }
  // every block is past the last barrier: block 0 records the jobs' new parities
  if (blockIdx.x == 0 && (a.nsteps & 1)) {
    const int tid = threadIdx.x + BX * threadIdx.y;
    for (int j = tid; j < a.njobs; j += BX * BY) a.parity[j] ^= 1;
  }
}

template <int BX, int BY, typename S, typename R, typename A>
BatchVariant variant() {
  return BatchVariant{BX, BY, (const void*)&batch_persistent_kernel<BX, BY, S, R, A>,
                      (size_t)Lattice<2>::Q * BX * BY * sizeof(R)};
}

int batch_variants(int precision, const BatchVariant** out) {
  static const BatchVariant fp32[] = {variant<64, 4, float, float, float>(), variant<32, 8, float, float, float>(),
                                      variant<128, 2, float, float, float>()};
  static const BatchVariant fp16[] = {variant<64, 4, __half, float, float>(), variant<32, 8, __half, float, float>(),
                                      variant<128, 2, __half, float, float>()};
  static const BatchVariant fp64[] = {variant<64, 4, double, double, double>(), variant<32, 8, double, double, double>()};
  if (precision == LBM_FP64) { *out = fp64; return 2; }
  if (precision == LBM_FP16DEV) { *out = fp16; return 3; }
  *out = fp32;
  return 3;
}

}  // namespace lbm
