// D3Q27 instantiations: float64 reference path, float32 path, float16-deviation storage.
#include "lbm_instantiate.cuh"

namespace lbm {
const Ops ops_d3q27_fp64 = Launch<3, double, double, double>::table();
const Ops ops_d3q27_fp32 = Launch<3, float, float, float>::table();
const Ops ops_d3q27_fp16dev = Launch<3, __half, float, float>::table();
}  // namespace lbm
