// The 1024-thread kernel of the FP32 form (FP64 refinement around FP32
// inner solves),
// in a translation unit of its own so that the solve kernels compile in
// parallel (the device code is in rgdbek_solve.cuh).
#include "rgdbek_solve.cuh"

namespace rgd {

const void *refine_fn_1024() { return (const void *)refine_kernel<kSolveMaxThreads>; }

}  // namespace rgd
