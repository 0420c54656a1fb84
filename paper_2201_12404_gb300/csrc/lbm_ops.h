// Launch table of one (lattice, precision) instantiation of the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

struct Ops {
  int D, Q;
  size_t pop_bytes;  // bytes per stored population
  size_t aux_bytes;  // bytes per auxiliary value
  void (*moments_eos)(const DevDomain&, int parity, cudaStream_t);
  // q planes, ghosts included, from the (rho, psi) pairs and j planes pass 1 wrote
  void (*qflux)(const DevDomain&, const TileMaps& maps, cudaStream_t);
  void (*collide_stream)(const DevDomain&, const TileMaps& maps, int parity, cudaStream_t);
  void (*init_equilibrium)(const DevDomain&, const double* rho, const double* ux, const double* uy,
                           const double* uz, cudaStream_t);
  // (rho, psi) pairs of every padded node from a density field (device, float64)
  void (*aux_density)(const DevDomain&, const double* rho, cudaStream_t);
  void (*canonical_read)(const DevDomain&, int parity, double* out, cudaStream_t);
  void (*canonical_write)(const DevDomain&, const double* in, cudaStream_t);
  // canonical populations of the box origin + [0, extent) (coordinates wrapped
  // modulo the domain) into out[Q][ez][ey][ex]
  void (*canonical_window)(const DevDomain&, int parity, const int origin[3], const int extent[3], double* out,
                           cudaStream_t);
  void (*macroscopic)(const DevDomain&, int parity, double* rho, double* u, cudaStream_t);
  // u[a*N + n] -= F_a/(2 rho[n]), F from the current auxiliary fields
  void (*bare_velocity)(const DevDomain&, const double* rho, double* u, cudaStream_t);
  // returns the number of partial blocks written to partial (5 doubles each)
  int (*diag_partial)(const DevDomain&, int parity, double* partial, cudaStream_t);
  // the same layout, field 4 = largest |u + F/(2 rho)| of the block (auxiliary fields current)
  int (*max_speed_partial)(const DevDomain&, int parity, double* partial, cudaStream_t);
  // drop-on-film initial fields into rho[N], u[D*N] (device, float64)
  void (*drop_on_film)(const DevDomain&, const lbm_drop_on_film& g, double rho_l, double rho_v, double* rho, double* u,
                       cudaStream_t);
  // the same layout, field 4 = largest |grad rho| of the block (auxiliary fields current)
  int (*grad_partial)(const DevDomain&, double* partial, cudaStream_t);
  // the same layout, field 4 = crown radius of the block's nodes of one layer
  int (*crown_partial)(const DevDomain&, int layer, double rho_mid, double* partial, cudaStream_t);
};

// Defined in lbm_d2q9.cu and lbm_d3q27.cu.
extern const Ops ops_d2q9_fp64, ops_d2q9_fp32, ops_d3q27_fp64, ops_d3q27_fp32;
extern const Ops ops_d2q9_fp16dev, ops_d3q27_fp16dev;

// Fill the interior-node slot offset tables of d (needs d.N, d.nx, d.ny set) for
// populations stored in elem_bytes bytes.
inline void fill_slot_offsets(DevDomain& d, int D, size_t elem_bytes) {
  const int Q = D == 3 ? 27 : 9;
  const long long e = (long long)elem_bytes;
  for (int i = 0; i < 27; ++i) {
    const long long off = (long long)cxi(i) + (long long)d.nx * cyi(i) + (D == 3 ? (long long)d.nx * d.ny * czi(i) : 0ll);
    const bool live = i < Q;
    d.src_boff[0][i] = live ? e * ((long long)i * d.N) : 0;
    d.src_boff[1][i] = live ? e * ((long long)(Q - 1 - i) * d.N - off) : 0;
    d.dst_boff[0][i] = live ? e * ((long long)(Q - 1 - i) * d.N) : 0;
    d.dst_boff[1][i] = live ? e * ((long long)i * d.N + off) : 0;
    d.up_off[i] = live ? -off : 0;
  }
}

// Padded x extent of the auxiliary fields: nx plus the two 2-node ghost layers,
// rounded up to a multiple of 4 so that every row starts on a 16-byte boundary
// (a tensor-map stride requirement); the extra columns are never read.
inline int padded_x(int nx) { return (nx + 4 + 3) / 4 * 4; }

// cuTensorMapEncodeTiled from the driver (no link against libcuda).
typedef CUresult (*tensor_map_encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                         const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                         CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline tensor_map_encode_fn tensor_map_encoder(const char** why) {
  static tensor_map_encode_fn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      *why = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    encode = (tensor_map_encode_fn)fn;
  }
  return encode;
}

// Tensor map over the interleaved (rho, psi) pairs at the start of d.aux, with a
// box of one halo tile of `tile` pairs per axis.
// float32 pairs are single 8-byte elements of a (px, py[, pz]) tensor; float64
// pairs are the 16-byte innermost dimension of a (2, px, py[, pz]) tensor (a box's
// innermost extent must be a multiple of 16 bytes).  Returns false with a message
// when the driver refuses it.
inline bool make_aux_map(CUtensorMap* map, const DevDomain& d, int D, size_t elem_bytes, const cuuint32_t tile[3],
                         const char** why) {
  const tensor_map_encode_fn encode = tensor_map_encoder(why);
  if (!encode) return false;
  const size_t pair_bytes = 2 * elem_bytes;
  const cuuint64_t ext[3] = {(cuuint64_t)d.px, (cuuint64_t)d.py, (cuuint64_t)d.pz};
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  cuuint32_t rank = 0;
  CUtensorMapDataType type;
  if (elem_bytes == 4) {
    type = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    for (int a = 0; a < D; ++a) { dims[rank] = ext[a]; box[rank] = tile[a]; ++rank; }
  } else {
    type = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    dims[0] = 2; box[0] = 2; rank = 1;
    for (int a = 0; a < D; ++a) { dims[rank] = ext[a]; box[rank] = tile[a]; ++rank; }
  }
  // byte strides of dimensions 1..rank-1
  cuuint64_t stride = elem_bytes == 4 ? pair_bytes : elem_bytes;
  for (cuuint32_t k = 1; k < rank; ++k) {
    stride *= dims[k - 1];
    strides[k - 1] = stride;
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

// Tensor map over the q_a planes (element offset 2 PN of d.aux, one plane per
// axis): a (px, py[, pz], D) tensor with a box of (Blocks::bx + 4, Blocks::by + 2
// [, Blocks::bz + 2], 1), which holds q_a at the tile's nodes and their +-1
// neighbours along every axis (x starts 2 nodes early so that the box starts on a
// 16-byte boundary).
inline bool make_q_map(CUtensorMap* map, const DevDomain& d, int D, size_t elem_bytes, const char** why) {
  const tensor_map_encode_fn encode = tensor_map_encoder(why);
  if (!encode) return false;
  const cuuint64_t e = elem_bytes;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  const cuuint32_t rank = (cuuint32_t)D + 1;
  dims[0] = d.px; dims[1] = d.py;
  strides[0] = d.px * e;
  box[0] = (D == 3 ? Blocks<3>::bx : Blocks<2>::bx) + 4;
  box[1] = (D == 3 ? Blocks<3>::by : Blocks<2>::by) + 2;
  if (D == 3) {
    dims[2] = d.pz; dims[3] = 3;
    strides[1] = (cuuint64_t)d.px * d.py * e;
    strides[2] = (cuuint64_t)d.PN * e;
    box[2] = Blocks<3>::bz + 2; box[3] = 1;
  } else {
    dims[2] = 2;
    strides[1] = (cuuint64_t)d.PN * e;
    box[2] = 1;
  }
  void* base = (char*)d.aux + 2 * (size_t)d.PN * elem_bytes;
  const CUresult r = encode(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                            rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled rejected the q tensor map";
    return false;
  }
  return true;
}

// Auxiliary values per padded node: the (rho, psi) pair, the D q planes and the D
// j planes.
inline int aux_fields_per_node(int D) { return 2 + 2 * D; }

// Extents, walls and slot offsets of the domain p describes, with populations
// stored in pop_bytes bytes (the physical parameters come from fill_phys).
// Shared by lbm_create_domain and lbm_step_noalloc.
inline void fill_geometry(DevDomain& d, const lbm_params& p, int D, size_t pop_bytes) {
  d.nx = p.nx; d.ny = p.ny; d.nz = D == 3 ? p.nz : 1;
  d.N = (long long)d.nx * d.ny * d.nz;
  d.px = padded_x(p.nx); d.py = p.ny + 4; d.pz = D == 3 ? p.nz + 4 : 1;
  d.PN = (long long)d.px * d.py * d.pz;
  for (int a = 0; a < 3; ++a) {
    d.wall_lo[a] = a < D && p.bc[2 * a] == LBM_BC_BOUNCEBACK;
    d.wall_hi[a] = a < D && p.bc[2 * a + 1] == LBM_BC_BOUNCEBACK;
  }
  fill_slot_offsets(d, D, pop_bytes);
}

// The halo box of QTile<D, pair bytes> for pass 1b.
template <int D, int kPairBytes>
inline void qtile_box(cuuint32_t box[3]) {
  using T = QTile<D, kPairBytes>;
  box[0] = T::HX; box[1] = T::HY; box[2] = T::HZ;
}

inline bool make_tile_maps(TileMaps* m, const DevDomain& d, int D, size_t elem_bytes, const char** why) {
  // pass 1b: a QTile tile with a 2-node halo
  cuuint32_t qbox[3];
  if (D == 3) {
    if (elem_bytes == 4) qtile_box<3, 8>(qbox); else qtile_box<3, 16>(qbox);
  } else {
    if (elem_bytes == 4) qtile_box<2, 8>(qbox); else qtile_box<2, 16>(qbox);
  }
  return make_aux_map(&m->aux_q, d, D, elem_bytes, qbox, why) && make_q_map(&m->q, d, D, elem_bytes, why);
}

// Final fixed-order reduction of the diagnostic partial sums (lbm_d2q9.cu).
void launch_diag_final(const double* partial, int nblocks, double* out, cudaStream_t s);

}  // namespace lbm
