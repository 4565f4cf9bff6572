// FP32 (mixed precision) instantiation of the step and rebuild kernels.
#include "md_kernels.cuh"

#define REAL float
#include "md_launch.inc"
#undef REAL

// Sets the IF-node condition of the first rebuild of a captured block from the device flag.
__global__ void k_arm(const Ctrl *ctrl, cudaGraphConditionalHandle h) {
    const int on = *(volatile const int *)&ctrl->need_any && !*(volatile const int *)&ctrl->halt;
    cudaGraphSetConditional(h, on ? 1u : 0u);
}

cudaError_t launch_arm(const Ctrl *ctrl, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_arm<<<1, 1, 0, s>>>(ctrl, h);
    return cudaGetLastError();
}
