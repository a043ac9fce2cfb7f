// The batched solve kernels (FP64 and FP32 form, both shapes),
// in a translation unit of its own so that the solve kernels compile in
// parallel (the device code is in rgdbek_solve.cuh).
#include "rgdbek_solve.cuh"

namespace rgd {

const void *batched_fn(bool fp32, bool small) {
    if (small)
        return fp32 ? (const void *)batched_solve_kernel<true, kSolveSmallThreads>
                    : (const void *)batched_solve_kernel<false, kSolveSmallThreads>;
    return fp32 ? (const void *)batched_solve_kernel<true, kSolveMaxThreads>
                : (const void *)batched_solve_kernel<false, kSolveMaxThreads>;
}

}  // namespace rgd
