// lbm_step_noalloc: time steps without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// framework that owns the whole device memory pool, a memory-capped process,
// or a host thread that must not touch the allocator while other work is in
// flight.  They hand in the populations they own; the auxiliary fields that the
// step needs between its passes (density, signed pseudo-potential, q, j) live
// in a fixed scratch array compiled into this library instead of a cudaMalloc.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_ops.h"
#include "lbm_phys.h"

namespace {

// 16 MiB of scratch on every GPU that loads the library, held until exit.  The
// first 256 bytes hold the error flags and the gamma-guard counter; the
// auxiliary fields follow.
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr size_t kHeaderBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side handle, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
lbm_status scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LBM_ERR_CUDA;
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_params* p, void* populations, int64_t nsteps) {
  using lbm::DevDomain;
  using lbm::Ops;
  if (!p || !populations || nsteps < 0 || (nsteps & 1)) return LBM_ERR_INVALID_ARG;
  if (lbm_footprint_bytes(p) == 0) return LBM_ERR_INVALID_ARG;  // same checks as lbm_create_domain
  if (p->precision == LBM_FP16DEV) return LBM_ERR_INVALID_ARG;   // needs per-node writer densities

  const int D = p->lattice == LBM_D3Q27 ? 3 : 2;
  const Ops* ops = p->lattice == LBM_D2Q9 ? (p->precision == LBM_FP64 ? &lbm::ops_d2q9_fp64 : &lbm::ops_d2q9_fp32)
                                          : (p->precision == LBM_FP64 ? &lbm::ops_d3q27_fp64 : &lbm::ops_d3q27_fp32);
  // every population access is one aligned word of the storage type
  if ((uintptr_t)populations % ops->pop_bytes != 0) return LBM_ERR_INVALID_ARG;
  DevDomain d{};
  lbm::fill_geometry(d, *p, D, ops->pop_bytes);
  const double aux_bytes = (double)lbm::aux_fields_per_node(D) * (double)d.PN * (double)ops->aux_bytes;
  if (aux_bytes > (double)(kScratchBytes - kHeaderBytes)) return LBM_ERR_INVALID_ARG;  // beyond the scratch maximum
  if (nsteps == 0) return LBM_OK;
  // an error the caller left pending is theirs: report it without doing any work
  // (and without clearing it)
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ERR_CUDA;
  lbm::fill_phys(d, *p, D);

  unsigned char* scratch = nullptr;
  lbm_status st = scratch_address(&scratch);
  if (st != LBM_OK) return st;
  d.f = populations;
  d.flags = (unsigned int*)scratch;
  d.guards = (unsigned long long*)(scratch + 8);
  d.aux = scratch + kHeaderBytes;
  d.gamma_out = nullptr;

  lbm::TileMaps maps;
  const char* why = nullptr;
  if (!lbm::make_tile_maps(&maps, d, D, ops->aux_bytes, &why)) return LBM_ERR_CUDA;

  cudaStream_t stream = (cudaStream_t)p->stream;
  // the scratch keeps the previous call's contents: clear the flags and the counter
  if (cudaMemsetAsync(scratch, 0, 16, stream) != cudaSuccess) return LBM_ERR_CUDA;
  int parity = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    ops->moments_eos(d, parity, stream);
    ops->qflux(d, maps, stream);
    ops->collide_stream(d, maps, parity, stream);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    parity ^= 1;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_noalloc_status(void) {
  unsigned char* scratch = nullptr;
  lbm_status st = scratch_address(&scratch);
  if (st != LBM_OK) return st;
  unsigned int flags = 0;
  // a pageable host word: the copy allocates nothing
  if (cudaMemcpy(&flags, scratch, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
  if (flags & 4u) return LBM_ERR_BOUNDS;
  if (flags & 2u) return LBM_ERR_TIMEOUT;
  if (flags & 1u) return LBM_ERR_UNSTABLE;
  return LBM_OK;
}
