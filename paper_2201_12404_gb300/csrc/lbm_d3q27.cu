// D3Q27 instantiations: float64 reference path and float32 path.
#include "lbm_instantiate.cuh"

namespace lbm {
const Ops ops_d3q27_fp64 = Launch<3, double, double, double>::table();
const Ops ops_d3q27_fp32 = Launch<3, float, float, float>::table();
}  // namespace lbm
