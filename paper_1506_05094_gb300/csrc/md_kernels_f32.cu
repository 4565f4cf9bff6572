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

// ---- replica-resident kernel: tp in {1,2,4,8,16,32}, list-build lanes in {8, 32}
namespace {
template <int TP, bool SINGLE, int TPB> void *rep_fn() {
    return (void *)md::k_rep<float, TP, SINGLE, TPB>;
}
template <bool SINGLE, int TPB> void *rep_fn_tp(int tp) {
    switch (tp) {
    case 1: return rep_fn<1, SINGLE, TPB>();
    case 2: return rep_fn<2, SINGLE, TPB>();
    case 4: return rep_fn<4, SINGLE, TPB>();
    case 8: return rep_fn<8, SINGLE, TPB>();
    case 16: return rep_fn<16, SINGLE, TPB>();
    case 32: return rep_fn<32, SINGLE, TPB>();
    default: return nullptr;
    }
}
void *rep_kernel(int tp, int tpb, bool single) {
    if (tpb >= 32) return single ? rep_fn_tp<true, 32>(tp) : rep_fn_tp<false, 32>(tp);
    return single ? rep_fn_tp<true, 8>(tp) : rep_fn_tp<false, 8>(tp);
}
}  // namespace

cudaError_t prepare_rep(int tp, int tpb, bool single, size_t smem) {
    void *f = rep_kernel(tp, tpb, single);
    if (!f) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_rep(const StepArgs<float> &a, const RebuildArgs<float> &b, int tp, int block,
                       int grid, size_t smem, cudaStream_t s) {
    void *f = rep_kernel(tp, b.tpb, a.ntypes == 1);
    if (!f) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a, (void *)&b};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

// ---- grid step kernel with staged replica positions
namespace {
template <bool SINGLE> void *staged_fn(int tp) {
    switch (tp) {
    case 1: return (void *)md::k_step<float, 1, SINGLE, true>;
    case 2: return (void *)md::k_step<float, 2, SINGLE, true>;
    case 4: return (void *)md::k_step<float, 4, SINGLE, true>;
    case 8: return (void *)md::k_step<float, 8, SINGLE, true>;
    case 16: return (void *)md::k_step<float, 16, SINGLE, true>;
    case 32: return (void *)md::k_step<float, 32, SINGLE, true>;
    default: return nullptr;
    }
}
}  // namespace

cudaError_t prepare_step_staged(int tp, bool single, size_t smem) {
    void *f = single ? staged_fn<true>(tp) : staged_fn<false>(tp);
    if (!f) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_step_staged(const StepArgs<float> &a, int tp, int block, int ntiles,
                               size_t smem, cudaStream_t s) {
    void *f = a.ntypes == 1 ? staged_fn<true>(tp) : staged_fn<false>(tp);
    if (!f) return cudaErrorInvalidValue;
    if (ntiles <= 0) return cudaSuccess;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3(ntiles), dim3(block), args, smem, s);
}
