// The 512-thread shape of the solve kernels (128 registers a thread), in a
// translation unit of its own so that it compiles beside the 1024-thread
// shape in rgdbek_kernels.cu.
#include "rgdbek_solve.cuh"

namespace rgd {

const void *solve_kernel_fn_small(bool fp32) {
    return fp32 ? (const void *)refine_kernel<kSolveSmallThreads>
                : (const void *)solve_kernel<kSolveSmallThreads>;
}

const void *batched_kernel_fn_small(bool fp32) {
    return fp32 ? (const void *)batched_solve_kernel<true, kSolveSmallThreads>
                : (const void *)batched_solve_kernel<false, kSolveSmallThreads>;
}

}  // namespace rgd
