// FP32 instantiation of the string-method kernels (FP32 spins, fields and FFTs; FP64 reductions).
#include "ss_kernels.cuh"

namespace ss {
SS_INSTANTIATE(float)
}  // namespace ss
