// Internal interface between the host side of the library (rgdbek_api.cu)
// and the kernel translation units (rgdbek_kernels.cu, rgdbek_setup.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rgdbek_phases.cuh"

namespace rgd {

constexpr int kSolveMaxThreads = 1024;  // launch bound of the component kernels and the sampler
// The solve kernels come in two shapes: 512 threads (128 registers a thread,
// no spills; fastest while each CTA's share of the vectors fits its shared
// memory) and 1024 threads (64 registers; faster on large vectors, where the
// element-wise loops of the inner solves run from global memory).  The
// automatic choice takes 1024 threads when max(m, n) exceeds
// kSolveVecPerCta elements per CTA.
constexpr int kSolveSmallThreads = 512;
constexpr long long kSolveVecPerCta = 2048;
inline int auto_solve_block(long long m, long long n, int ctas) {
    const long long v = m > n ? m : n;
    return v > kSolveVecPerCta * (long long)(ctas > 0 ? ctas : 1) ? kSolveMaxThreads
                                                                   : kSolveSmallThreads;
}
// dynamic shared memory of a CTA of the batched solve (its chunk of the
// inner-solve block); the single solve takes what the device allows, or the
// option smem_per_cta
constexpr int kSolveDsmemBytes = 96 * 1024;

// One system of a batch: its FP64 view and (for the FP32 form) its FP32 view.
struct SysPair {
    Params p;
    ParamsF f;
};

// control block to its pre-launch state (status = kStatusRunning)
cudaError_t launch_reset_ctrl(Ctrl *c, cudaStream_t s);
// persistent solve (cooperative launch); returns the launch error.  FP64
// solve, or (P.precision == RGDBEK_PRECISION_FP32_INNER) the FP64 refinement
// loop around FP32 inner solves on the FP32 view F.
cudaError_t launch_solve(const Params &P, const ParamsF &F, int grid, int block, cudaStream_t s);
// batched solve: nteams * team CTAs (cooperative launch); sys_dev holds one
// SysPair per system (team already set), plan_dev[t * stride + q] the q-th
// system of team t (-1 ends a team's list)
cudaError_t launch_solve_batched(const SysPair *sys_dev, const int *plan_dev, int stride, int team,
                                 int nteams, bool fp32, int block, cudaStream_t s);
// the solve kernels of one shape (small: the 512-thread launch bound); fp32:
// the refinement kernel of the FP32 form
const void *solve_kernel_fn(bool fp32, bool small);
const void *batched_kernel_fn(bool fp32, bool small);
const void *solve_fn_512();     // rgdbek_solve512.cu
const void *solve_fn_1024();    // rgdbek_solve1024.cu
const void *refine_fn_512();    // rgdbek_refine512.cu
const void *refine_fn_1024();   // rgdbek_refine1024.cu
const void *batched_fn(bool fp32, bool small);  // rgdbek_batched.cu
// control blocks of a batch: reset before the launch, gathered after it
cudaError_t launch_reset_ctrls(const SysPair *sys_dev, int nsys, cudaStream_t s);
cudaError_t launch_gather_ctrls(const SysPair *sys_dev, int nsys, Ctrl *out, cudaStream_t s);
// out[i] = (float)in[i], round to nearest
cudaError_t launch_to_float(const double *in, long long len, float *out, cudaStream_t s);
// standalone sampler on given weights (cooperative launch)
cudaError_t launch_sample(const Params &P, int grid, int block, const double *eps, long long len,
                          long long s, unsigned long long seed, unsigned long long sysid,
                          unsigned long long k, unsigned long long phase, int *idx, bool greedy,
                          double eta, cudaStream_t st);
cudaError_t launch_spmv(const Params &P, int grid, int block, const double *x, double *y,
                        cudaStream_t s);
cudaError_t launch_spmv_t(const Params &P, int grid, int block, const double *z, double *g,
                          cudaStream_t s);
// FP32 products with the float copy of A (the FP32 form's passes): y = A x,
// or with transposed g = A^T z
cudaError_t launch_spmv_f32(const ParamsF &F, int grid, int block, const float *x, float *y,
                            bool transposed, cudaStream_t s);
// gv[e] = (b_i - ax_i) v_j - w_i x_j [+ u_i (g_j - q_j) when u != nullptr]
// over the stored entries e = (i, j) of P's CSR form
cudaError_t launch_adjoint_vals(const Params &P, int grid, int block, const double *b,
                                const double *ax, const double *w, const double *v,
                                const double *x, const double *u, const double *g,
                                const double *q, double *gv, cudaStream_t s);
cudaError_t launch_weights(const double *v, const double *norm2, long long len, double *eps,
                           Ctrl *ctrl, int grid, int block, cudaStream_t s);
// dynamic shared memory the single-solve kernels may use on the current
// device (set as their limit; 0 on error)
int solve_dsmem_max();
// CTAs of `block` threads of the persistent kernels that fit on one SM
int solve_blocks_per_sm(int block, int dsmem);
int batched_blocks_per_sm(int block);
int sample_blocks_per_sm(int block);

// ---- set-up (rgdbek_setup.cu) ----------------------------------------------
// Checks the CSR arrays on the device; *err_host receives 0 or a status code.
cudaError_t validate_csr(long long m, long long n, long long nnz, const long long *rp,
                         const int *ci, const double *av, int *err_dev, int *err_host,
                         cudaStream_t s);
// Builds the CSC form (col_ptr n+1, row_idx, vals; rows ascending within a
// column) from a valid CSR.  tmp_* are scratch of the stated sizes.
cudaError_t build_csc(long long m, long long n, long long nnz, const long long *rp, const int *ci,
                      const double *av, long long *cp, int *ri, double *cv, long long *key_a,
                      long long *key_b, int *row_of, long long *cursor, long long *blk_sums,
                      cudaStream_t s);
// Squared norms of the lines of a compressed matrix (CSR rows or CSC columns).
cudaError_t line_norms2(long long nlines, const long long *ptr, const double *val, double *out,
                        cudaStream_t s);

}  // namespace rgd
