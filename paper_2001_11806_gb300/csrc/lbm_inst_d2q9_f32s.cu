// Explicit instantiation of every kernel for the D2Q9 stencil with F32S storage
// (one translation unit per pair so that the build compiles them in parallel).
#include "lbm_ops.cuh"

namespace lbm {
OpsTable ops_table_d2q9_f32s() { return make_table<D2Q9, StF32S>(); }
}  // namespace lbm
