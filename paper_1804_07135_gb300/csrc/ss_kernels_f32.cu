// FP32 instantiation of the string-method kernels (FP32 spins, fields and FFTs; FP64 reductions).
#include "ss_kernels.cuh"

namespace ss {
SS_INSTANTIATE(float)

// one thread: the condition of a WHILE graph node over attempt rounds, nonzero while some system of the
// group is inside its interval (*active, cleared by rk_finish and set again by rk_control); precision-free,
// so it lives in this translation unit only
__global__ void rk_condition_kernel(cudaGraphConditionalHandle h, const int* active) {
    cudaGraphSetConditional(h, *active != 0 ? 1u : 0u);
}

void launch_rk_condition(cudaGraphConditionalHandle h, const int* active, cudaStream_t st) {
    rk_condition_kernel<<<1, 1, 0, st>>>(h, active);
}
}  // namespace ss
