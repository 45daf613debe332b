// Explicit instantiation of the pass kernels and their orchestration for double.
#include "sbec_kernels.cuh"

namespace sbec {
template struct Ops<double>;
}  // namespace sbec
