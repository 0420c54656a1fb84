// Batched persistent stepping of many D2Q9 domains (internal interface between
// the batch host code and its kernels).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// One tile of work: job index and tile coordinates in tile units.
struct BatchItem {
  int job, tx, ty;
};

struct BatchArgs {
  const DevDomain* jobs;  // device array, one per job
  int* parity;            // device array: A-A parity of every job; flipped by the kernel at the end
  int njobs;
  const BatchItem* k2;    // tiles over the interior of every job (all three passes)
  int n_k2;
  unsigned int* barrier;  // [0] arrivals, [1] generation
  unsigned int* error;    // bit 1: a bounded grid-barrier wait gave up
  int nsteps;
  unsigned int poll_limit;  // polls (each ~0.1 us) before a grid-barrier wait gives up
  int skip_arrival;         // test switch: block 0 does not arrive at the grid barriers
};

// Default poll limit of the grid barrier: far above any real wait (~3 s).
constexpr unsigned int kBarrierPollsDefault = 1u << 25;

// A compiled tile shape of the persistent kernel for one storage precision.
struct BatchVariant {
  int bx, by;
  const void* kernel;  // __global__ void (BatchArgs)
  size_t dyn_smem;     // dynamic shared memory per block
};

// Tile-shape variants compiled for a precision (lbm_precision value); returns their count.
int batch_variants(int precision, const BatchVariant** out);

}  // namespace lbm
