// Explicit instantiation of the pass kernels and their orchestration for float.
#include "sbec_kernels.cuh"

namespace sbec {
template struct Ops<float>;
}  // namespace sbec
