// Kernels of the library besides the solve kernels (rgdbek_solve.cuh,
// instantiated in their own translation units): the batch control kernels,
// the component kernels that reuse the solve's phases (SpMV, A^T z, weights,
// sampler, adjoint entry gradients), and the host-side launchers.
#include <cmath>

#include "rgdbek_internal.h"
#include "rgdbek_solve.cuh"

namespace rgd {

// Resets the control blocks of a batch (one thread each).
__global__ void reset_ctrls_kernel(const SysPair *sys, int nsys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsys) return;
    Ctrl *c = sys[i].p.ctrl;
    c->bar_count = 0;
    c->abort = 0;
    c->status = kStatusRunning;
    c->stop_req = 0;
    for (int k = 0; k < RGDBEK_NUM_PHASES; ++k) c->zphase_ns[k] = 0;
}

// Copies the control blocks of a batch into one array (for one host copy).
__global__ void gather_ctrls_kernel(const SysPair *sys, int nsys, Ctrl *out) {
    const int i = blockIdx.x;
    if (i >= nsys) return;
    const int *src = reinterpret_cast<const int *>(sys[i].p.ctrl);
    int *dst = reinterpret_cast<int *>(out + i);
    for (int w = threadIdx.x; w < (int)(sizeof(Ctrl) / sizeof(int)); w += blockDim.x)
        dst[w] = src[w];
}

// ---------------------------------------------------------------------------
// Component kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSolveMaxThreads) spmv_kernel(const Params P, const double *x,
                                                                double *y) {
    enter_team(P);
    rows_matvec(P, x, y);
}
__global__ void __launch_bounds__(kSolveMaxThreads) spmv_t_kernel(const Params P, const double *z,
                                                                  double *g) {
    enter_team(P);
    cols_matvec(P, z, g);
}
__global__ void __launch_bounds__(kSolveMaxThreads) spmv_f32_kernel(const ParamsF F, const float *x,
                                                                    float *y) {
    enter_team(F);
    rows_matvec(F, x, y);
}
__global__ void __launch_bounds__(kSolveMaxThreads) spmv_t_f32_kernel(const ParamsF F,
                                                                      const float *z, float *g) {
    enter_team(F);
    cols_matvec(F, z, g);
}

// Gradient of a loss with respect to the stored entries of A (the implicit
// adjoint of x = A^+ b; Golub-Pereyra derivative of the pseudo-inverse):
//   gv[e] = (b_i - (Ax)_i) v_j - w_i x_j  [+ u_i (g_j - q_j)]  for entry e = (i, j).
// Each product and difference is rounded on its own (no contraction), in
// that order.  L lanes per row stream the row's column indices once.
__global__ void __launch_bounds__(kSolveMaxThreads)
    adjoint_vals_kernel(const Params P, const double *b, const double *ax, const double *w,
                        const double *v, const double *x, const double *u, const double *g,
                        const double *q, double *gv) {
    enter_team(P);
    const Grp G(P.ipr);
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        if (i >= P.m) continue;
        const double ri = __dsub_rn(b[i], ax[i]);
        const double wi = w[i];
        const double ui = u ? u[i] : 0.0;
        const long long e1 = __ldg(P.rp + i + 1);
        for (long long e = __ldg(P.rp + i) + G.sl; e < e1; e += G.L) {
            const int j = __ldg(P.ci + e);
            double d = __dsub_rn(__dmul_rn(ri, v[j]), __dmul_rn(wi, x[j]));
            if (u) d = __dadd_rn(d, __dmul_rn(ui, __dsub_rn(g[j], q[j])));
            gv[e] = d;
        }
    }
}

__global__ void __launch_bounds__(kSolveMaxThreads) weights_kernel(const double *v,
                                                                   const double *norm2,
                                                                   long long len, double *eps,
                                                                   Ctrl *C) {
    __shared__ BlockScratch bs;
    double emax = 0.0;
    long long bad = 0;
    for (long long j = gthread(); j < len; j += nthreads()) {
        const double c = norm2[j];
        const double x = v[j];
        const double e = c > 0.0 ? __ddiv_rn(__dmul_rn(x, x), c) : 0.0;
        eps[j] = e;
        if (!isfinite(e)) bad = 1;
        else emax = max_nonneg(emax, e);
    }
    emax = block_max(emax, bs);
    bad = block_sum(bad, bs);
    if (threadIdx.x == 0) {
        // nonnegative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long *>(&C->emax_out),
                  (unsigned long long)__double_as_longlong(emax));
        if (bad) atomicOr(&C->bad_out, 1);
    }
}

__global__ void __launch_bounds__(kSolveMaxThreads, 1)
    sample_kernel(const Params P, const double *eps, long long len, long long s,
                  unsigned long long seed, unsigned long long sysid, unsigned long long k,
                  unsigned long long phase, int *idx, bool greedy, double eta) {
    enter_team(P);
    __shared__ SolveSmem S;
    BlockScratch &bs = S.bs;
    const int nct = tsize(P);
    if (threadIdx.x == 0) S.epoch = 0;
    double emax = 0.0;
    long long bad = 0;
    for (long long j = tthread(P); j < len; j += tthreads(P)) {
        const double e = eps[j];
        if (!isfinite(e) || e < 0.0) bad = 1;
        else emax = max_nonneg(emax, e);
    }
    emax = block_max(emax, bs);
    bad = block_sum(bad, bs);
    if (threadIdx.x == 0) {
        P.pd[D_EMAX_C * nct + trank(P)] = emax;
        P.pi[I_BAD_C * nct + trank(P)] = bad;
    }
#define SAMPLE_SYNC(dm, dx, im)                                         \
    do {                                                                \
        if (!sync_collect(P, S, (dm), (dx), (im), S.red_d)) return;     \
    } while (0)
    SAMPLE_SYNC(DS(D_EMAX_C), DS(D_EMAX_C), DS(I_BAD_C));
    emax = S.red_d[D_EMAX_C];
    bad = S.red_i[I_BAD_C];
    long long count = 0;
    if (bad == 0 && emax > 0.0) {
        phase_quantize(P, eps, len, emax, greedy, eta, bs);
        SAMPLE_SYNC(0, 0, 0);
        if (!greedy) {
            phase_draw(P, len, s, seed, sysid, k, phase, S.tab, bs);
            SAMPLE_SYNC(0, 0, 0);
        }
        phase_compact_count<double>(P, len, eps, eps, nullptr, bs);
        SAMPLE_SYNC(0, 0, 0);
        count = phase_compact_write(P, len, P.rowpos, idx, S.tab, bs);
    }
    if (trank(P) == 0 && threadIdx.x == 0) {
        P.ctrl->sample_count = bad ? -1 : count;
        __threadfence();
        atomicCAS(&P.ctrl->status, kStatusRunning, RGDBEK_OK);
    }
}

#undef SAMPLE_SYNC
#undef DS

__global__ void to_float_kernel(const double *in, long long len, float *out) {
    for (long long i = gthread(); i < len; i += nthreads()) out[i] = __double2float_rn(in[i]);
}

__global__ void reset_ctrl_kernel(Ctrl *c) {
    c->bar_count = 0;
    c->abort = 0;
    c->status = kStatusRunning;
    c->stop_req = 0;
    c->iters = c->inner_u = c->inner_j = 0;
    c->sum_nu = c->sum_nj = c->sum_nnzu = c->sum_nnzj = 0;
    c->lsqr_nnzu = c->lsqr_nnzj = c->lsqr_nu = c->lsqr_nj = 0;
    for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) c->phase_ns[i] = 0;
    c->rel_res = c->normal_res = c->rse = 0.0;
    c->sample_count = 0;
    c->emax_out = 0.0;
    c->bad_out = 0;
    c->refinements = 0;
    c->bar_x = c->bar_z = 0;
    c->lk_zready = c->lk_zused = c->lk_tready = c->lk_colpass = c->lk_stop = 0;
    for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) c->zphase_ns[i] = 0;
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
cudaError_t launch_reset_ctrl(Ctrl *c, cudaStream_t s) {
    reset_ctrl_kernel<<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

// the solve kernels live in translation units of their own
const void *solve_kernel_fn(bool fp32, bool small) {
    if (fp32) return small ? refine_fn_512() : refine_fn_1024();
    return small ? solve_fn_512() : solve_fn_1024();
}
const void *batched_kernel_fn(bool fp32, bool small) { return batched_fn(fp32, small); }

cudaError_t launch_solve(const Params &P, const ParamsF &F, int grid, int block, cudaStream_t s) {
    Params p = P;
    p.team = grid;
    ParamsF f = F;
    f.team = grid;
    const bool fp32 = P.precision == RGDBEK_PRECISION_FP32_INNER;
    void *args1[] = {&p};
    void *args2[] = {&p, &f};
    const void *fn = solve_kernel_fn(fp32, block <= kSolveSmallThreads);
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), fp32 ? args2 : args1,
                                       (size_t)P.dsmem_bytes, s);
}

cudaError_t launch_sample(const Params &P, int grid, int block, const double *eps, long long len,
                          long long s, unsigned long long seed, unsigned long long sysid,
                          unsigned long long k, unsigned long long phase, int *idx, bool greedy,
                          double eta, cudaStream_t st) {
    Params p = P;
    p.team = grid;
    void *args[] = {&p, &eps, &len, &s, &seed, &sysid, &k, &phase, &idx, &greedy, &eta};
    return cudaLaunchCooperativeKernel((const void *)sample_kernel, dim3(grid), dim3(block), args, 0,
                                       st);
}

cudaError_t launch_spmv(const Params &P, int grid, int block, const double *x, double *y,
                        cudaStream_t s) {
    Params p = P;
    p.team = grid;
    spmv_kernel<<<grid, block, 0, s>>>(p, x, y);
    return cudaGetLastError();
}

cudaError_t launch_spmv_t(const Params &P, int grid, int block, const double *z, double *g,
                          cudaStream_t s) {
    Params p = P;
    p.team = grid;
    spmv_t_kernel<<<grid, block, 0, s>>>(p, z, g);
    return cudaGetLastError();
}

cudaError_t launch_spmv_f32(const ParamsF &F, int grid, int block, const float *x, float *y,
                            bool transposed, cudaStream_t s) {
    ParamsF f = F;
    f.team = grid;
    if (transposed) spmv_t_f32_kernel<<<grid, block, 0, s>>>(f, x, y);
    else spmv_f32_kernel<<<grid, block, 0, s>>>(f, x, y);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_vals(const Params &P, int grid, int block, const double *b,
                                const double *ax, const double *w, const double *v,
                                const double *x, const double *u, const double *g,
                                const double *q, double *gv, cudaStream_t s) {
    Params p = P;
    p.team = grid;
    adjoint_vals_kernel<<<grid, block, 0, s>>>(p, b, ax, w, v, x, u, g, q, gv);
    return cudaGetLastError();
}

cudaError_t launch_to_float(const double *in, long long len, float *out, cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    long long g = (len + 255) / 256;
    if (g > 4096) g = 4096;
    to_float_kernel<<<(int)g, 256, 0, s>>>(in, len, out);
    return cudaGetLastError();
}

cudaError_t launch_weights(const double *v, const double *norm2, long long len, double *eps,
                           Ctrl *ctrl, int grid, int block, cudaStream_t s) {
    weights_kernel<<<grid, block, 0, s>>>(v, norm2, len, eps, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_solve_batched(const SysPair *sys_dev, const int *plan_dev, int stride, int team,
                                 int nteams, bool fp32, int block, cudaStream_t s) {
    void *args[] = {&sys_dev, &plan_dev, &stride, &team};
    const void *fn = batched_kernel_fn(fp32, block <= kSolveSmallThreads);
    return cudaLaunchCooperativeKernel(fn, dim3(nteams * team), dim3(block), args,
                                       (size_t)kSolveDsmemBytes, s);
}

cudaError_t launch_reset_ctrls(const SysPair *sys_dev, int nsys, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    reset_ctrls_kernel<<<(nsys + 255) / 256, 256, 0, s>>>(sys_dev, nsys);
    return cudaGetLastError();
}

cudaError_t launch_gather_ctrls(const SysPair *sys_dev, int nsys, Ctrl *out, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    gather_ctrls_kernel<<<nsys, 128, 0, s>>>(sys_dev, nsys, out);
    return cudaGetLastError();
}

// Largest dynamic shared memory of a CTA of the single-solve kernels on the
// current device: the opt-in limit per block less the largest static shared
// memory of those kernels (1 KB granules).  Every single-solve kernel is
// allowed that much; the batched kernels get kSolveDsmemBytes.  0 on error.
int solve_dsmem_max() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    size_t stat = 0;
    for (int sh = 0; sh < 2; ++sh)
        for (int f32 = 0; f32 < 2; ++f32) {
            cudaFuncAttributes a{};
            if (cudaFuncGetAttributes(&a, solve_kernel_fn(f32 != 0, sh != 0)) != cudaSuccess)
                return 0;
            if (a.sharedSizeBytes > stat) stat = a.sharedSizeBytes;
        }
    const int avail = (int)(((long long)optin - (long long)stat) & ~1023ll);
    if (avail < kSolveDsmemBytes) return 0;
    for (int sh = 0; sh < 2; ++sh)
        for (int f32 = 0; f32 < 2; ++f32)
            if (cudaFuncSetAttribute(solve_kernel_fn(f32 != 0, sh != 0),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     avail) != cudaSuccess)
                return 0;
    return avail;
}

// CTAs of `block` threads of the single-solve kernels with dsmem bytes of
// dynamic shared memory that fit on one SM (the smaller of the FP64 and FP32
// form's kernel); solve_dsmem_max must have run.
int solve_blocks_per_sm(int block, int dsmem) {
    const bool small = block <= kSolveSmallThreads;
    int best = 1 << 30;
    for (int f32 = 0; f32 < 2; ++f32) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel_fn(f32 != 0, small),
                                                          block, dsmem) != cudaSuccess)
            return 0;
        if (nb < best) best = nb;
    }
    return best;
}

// The same for the batched kernels (kSolveDsmemBytes each; both shapes are
// given it, as a batch may run the other shape than its first handle).
int batched_blocks_per_sm(int block) {
    for (int sh = 0; sh < 2; ++sh)
        for (int f32 = 0; f32 < 2; ++f32)
            if (cudaFuncSetAttribute(batched_kernel_fn(f32 != 0, sh != 0),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kSolveDsmemBytes) != cudaSuccess)
                return 0;
    const bool small = block <= kSolveSmallThreads;
    int best = 1 << 30;
    for (int f32 = 0; f32 < 2; ++f32) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel_fn(f32 != 0, small),
                                                          block, kSolveDsmemBytes) != cudaSuccess)
            return 0;
        if (nb < best) best = nb;
    }
    return best;
}

int sample_blocks_per_sm(int block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel, block, 0) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace rgd
