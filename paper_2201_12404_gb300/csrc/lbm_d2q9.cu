// D2Q9 instantiations: float64 reference path, float32 path, float16-deviation storage.
#include "lbm_instantiate.cuh"

namespace lbm {
const Ops ops_d2q9_fp64 = Launch<2, double, double, double>::table();
const Ops ops_d2q9_fp32 = Launch<2, float, float, float>::table();
const Ops ops_d2q9_fp16dev = Launch<2, __half, float, float>::table();

void launch_diag_final(const double* partial, int nblocks, double* out, cudaStream_t s) {
  diag_final_kernel<<<1, 32, 0, s>>>(partial, nblocks, out);
}
}  // namespace lbm
