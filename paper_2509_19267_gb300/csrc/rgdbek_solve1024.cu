// The 1024-thread FP64 solve kernel,
// in a translation unit of its own so that the solve kernels compile in
// parallel (the device code is in rgdbek_solve.cuh).
#include "rgdbek_solve.cuh"

namespace rgd {

const void *solve_fn_1024() { return (const void *)solve_kernel<kSolveMaxThreads>; }

}  // namespace rgd
