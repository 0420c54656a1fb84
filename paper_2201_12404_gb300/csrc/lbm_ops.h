// Launch table of one (lattice, precision) instantiation of the kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

struct Ops {
  int D, Q;
  size_t pop_bytes;  // bytes per stored population
  size_t aux_bytes;  // bytes per auxiliary value
  void (*moments_eos)(const DevDomain&, int parity, cudaStream_t);
  void (*collide_stream)(const DevDomain&, int parity, cudaStream_t);
  void (*init_equilibrium)(const DevDomain&, const double* rho, const double* ux, const double* uy,
                           const double* uz, cudaStream_t);
  void (*canonical_read)(const DevDomain&, int parity, double* out, cudaStream_t);
  void (*canonical_write)(const DevDomain&, const double* in, cudaStream_t);
  void (*macroscopic)(const DevDomain&, int parity, double* rho, double* u, cudaStream_t);
  // returns the number of partial blocks written to partial (5 doubles each)
  int (*diag_partial)(const DevDomain&, int parity, double* partial, cudaStream_t);
};

// Defined in lbm_d2q9.cu and lbm_d3q27.cu.
extern const Ops ops_d2q9_fp64, ops_d2q9_fp32, ops_d3q27_fp64, ops_d3q27_fp32;

// Fill the interior-node slot offset tables of d (needs d.N, d.nx, d.ny set).
inline void fill_slot_offsets(DevDomain& d, int D) {
  const int Q = D == 3 ? 27 : 9;
  for (int i = 0; i < 27; ++i) {
    const long long off = (long long)cxi(i) + (long long)d.nx * cyi(i) + (D == 3 ? (long long)d.nx * d.ny * czi(i) : 0ll);
    const bool live = i < Q;
    d.src_off[0][i] = live ? (long long)i * d.N : 0;
    d.src_off[1][i] = live ? (long long)(Q - 1 - i) * d.N - off : 0;
    d.dst_off[0][i] = live ? (long long)(Q - 1 - i) * d.N : 0;
    d.dst_off[1][i] = live ? (long long)i * d.N + off : 0;
  }
}

// Final fixed-order reduction of the diagnostic partial sums (lbm_d2q9.cu).
void launch_diag_final(const double* partial, int nblocks, double* out, cudaStream_t s);

}  // namespace lbm
