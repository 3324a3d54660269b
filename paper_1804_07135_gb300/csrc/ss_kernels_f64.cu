// FP64 instantiation of the string-method kernels (the plain FP64 GPU method) and the FP64 setup
// kernels of the dipole-tensor spectrum.
#define SS_COMMON_LAUNCHERS
#include "ss_kernels.cuh"

namespace ss {
SS_INSTANTIATE(double)
}  // namespace ss
