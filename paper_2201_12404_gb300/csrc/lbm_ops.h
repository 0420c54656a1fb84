// Launch table of one (lattice, precision) instantiation of the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

struct Ops {
  int D, Q;
  size_t pop_bytes;  // bytes per stored population
  size_t aux_bytes;  // bytes per auxiliary value
  void (*moments_eos)(const DevDomain&, int parity, cudaStream_t);
  void (*collide_stream)(const DevDomain&, const CUtensorMap& aux_map, int parity, cudaStream_t);
  void (*init_equilibrium)(const DevDomain&, const double* rho, const double* ux, const double* uy,
                           const double* uz, cudaStream_t);
  void (*canonical_read)(const DevDomain&, int parity, double* out, cudaStream_t);
  void (*canonical_write)(const DevDomain&, const double* in, cudaStream_t);
  void (*macroscopic)(const DevDomain&, int parity, double* rho, double* u, cudaStream_t);
  // u[a*N + n] -= F_a/(2 rho[n]), F from the current auxiliary fields
  void (*bare_velocity)(const DevDomain&, const double* rho, double* u, cudaStream_t);
  // returns the number of partial blocks written to partial (5 doubles each)
  int (*diag_partial)(const DevDomain&, int parity, double* partial, cudaStream_t);
};

// Defined in lbm_d2q9.cu and lbm_d3q27.cu.
extern const Ops ops_d2q9_fp64, ops_d2q9_fp32, ops_d3q27_fp64, ops_d3q27_fp32;
extern const Ops ops_d2q9_fp16dev, ops_d3q27_fp16dev;

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
    d.up_off[i] = live ? -off : 0;
  }
}

// Padded x extent of the auxiliary fields: nx plus the two 2-node ghost layers,
// rounded up to a multiple of 4 so that every row starts on a 16-byte boundary
// (a tensor-map stride requirement); the extra columns are never read.
inline int padded_x(int nx) { return (nx + 4 + 3) / 4 * 4; }

// Tensor map over the first two auxiliary fields (rho, s*psi) of d: a
// (px, py[, pz], 2) tensor of float32 or float64 with a box of one halo tile,
// (Blocks::bx + 4, Blocks::by + 4[, Blocks::bz + 4], 2).  Returns false with a
// message when the driver refuses it.
inline bool make_aux_map(CUtensorMap* map, const DevDomain& d, int D, size_t elem_bytes, const char** why) {
  typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static encode_fn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      *why = "cuTensorMapEncodeTiled is not available from the driver";
      return false;
    }
    encode = (encode_fn)fn;
  }
  const CUtensorMapDataType type = elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  cuuint32_t rank;
  if (D == 3) {
    rank = 4;
    dims[0] = d.px; dims[1] = d.py; dims[2] = d.pz; dims[3] = 2;
    strides[0] = (cuuint64_t)d.px * elem_bytes;
    strides[1] = (cuuint64_t)d.px * d.py * elem_bytes;
    strides[2] = (cuuint64_t)d.PN * elem_bytes;
    box[0] = Blocks<3>::bx + 4; box[1] = Blocks<3>::by + 4; box[2] = Blocks<3>::bz + 4; box[3] = 2;
  } else {
    rank = 3;
    dims[0] = d.px; dims[1] = d.py; dims[2] = 2;
    strides[0] = (cuuint64_t)d.px * elem_bytes;
    strides[1] = (cuuint64_t)d.PN * elem_bytes;
    box[0] = Blocks<2>::bx + 4; box[1] = Blocks<2>::by + 4; box[2] = 2;
  }
  const CUresult r = encode(map, type, rank, d.aux, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled rejected the auxiliary-field tensor map";
    return false;
  }
  return true;
}

// Final fixed-order reduction of the diagnostic partial sums (lbm_d2q9.cu).
void launch_diag_final(const double* partial, int nblocks, double* out, cudaStream_t s);

}  // namespace lbm
