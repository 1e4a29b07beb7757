// Explicit instantiation of every kernel for the D3Q19 stencil with F16S storage
// (one translation unit per pair so that the build compiles them in parallel).
#include "lbm_ops.cuh"

namespace lbm {
OpsTable ops_table_d3q19_f16s() { return make_table<D3Q19, StF16S>(); }
}  // namespace lbm
