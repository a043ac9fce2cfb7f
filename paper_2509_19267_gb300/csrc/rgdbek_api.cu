// Host side of the C ABI declared in include/rgdbek.h: handle life cycle,
// option checks, device memory layout, and the launches of the persistent
// solve kernel and of the component kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "rgdbek_internal.h"

using namespace rgd;

// The read-only matrix arrays (CSR, CSC, squared norms) of a handle, shared
// by the handles made from it with rgdbek_create_like; freed with the last.
struct MatrixStore {
    void *mem = nullptr;
    size_t bytes = 0;
    std::atomic<int> refs{1};
    // A's values and squared norms rounded to float, for the FP32 form: made
    // by the first FP32 solve on any handle that shares this matrix, complete
    // (its stream synchronised) before mem32 is published under the mutex
    std::mutex mu32;
    void *mem32 = nullptr;
    float *av32 = nullptr, *cv32 = nullptr, *rn2f = nullptr, *cn2f = nullptr;
};

struct rgdbek_s {
    int device = 0, num_sms = 0;
    MatrixStore *mat = nullptr;
    cudaStream_t stream = nullptr;
    rgdbek_options opt{};
    long long m = 0, n = 0, nnz = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    Ctrl *ctrl_host = nullptr;  // page-locked copy of the control block
    // A
    long long *rp = nullptr, *cp = nullptr;
    int *ci = nullptr, *ri = nullptr;
    double *av = nullptr, *cv = nullptr, *rn2 = nullptr, *cn2 = nullptr;
    // work
    double *z, *t, *r, *g, *epsc, *epsr, *uu, *vv, *ww, *yy, *dx, *xt;
    unsigned long long *Q;
    unsigned char *flag;
    int *colpos, *rowpos, *ulist, *jlist;
    int *srn, *scn;
    int *sci, *sri;
    double *sav, *scv;
    double *dots, *dots2;
    double *vvs, *dsc, *yh, *uus, *dsr;
    double *pd;
    long long *pi;
    // float work vectors of the FP32 form's inner solves (each max(m, n) long;
    // f_z holds the (z_i, t_i) pairs); the extracted block values share the
    // FP64 arrays sav / scv, which the FP32 form does not otherwise use
    float *f_z, *f_r, *f_g, *f_epsc, *f_epsr, *f_uu, *f_vv, *f_ww, *f_yy, *f_dx, *f_xt, *f_x, *f_b;
    float *f_dots, *f_dots2, *f_vvs, *f_dsc, *f_yh, *f_uus, *f_dsr, *f_pd;
    // the FP32 form's refinement loop: FP64 residual, and the right-hand side and
    // solution of its FP64 inner solves
    double *ref_t, *ref_b, *ref_x;
    // the column team's buffers of the two-team schedule (FP64 and FP32 views)
    double *uu_z, *vv_z, *ww_z, *dots_z, *dots2_z, *pd_z;
    float *f_uu_z, *f_vv_z, *f_ww_z, *f_dots_z, *f_dots2_z, *f_pd_z;
    long long *pi_z;
    unsigned long long *Q_z;
    unsigned char *flag_z;
    int *ulist2;
    Ctrl *ctrl;
    double *b_stage, *x_stage;
    // implicit adjoint scratch, allocated by the first rgdbek_backward call:
    // A x, w, v, u (length m or n, whichever the transposed solves need) and
    // A g, q
    double *adj = nullptr;
    double *adj_ax, *adj_w, *adj_v, *adj_u, *adj_ag, *adj_q;
    // launch shape
    int grid = 0, block = 0, sample_grid = 0, tpr = 1, tpc = 1, ipr = 1, ipc = 1;
    int lpr = 1, lpc = 1;  // lanes of the full-matrix passes (rgdbek_tune_spmv)
    int dsmem = kSolveDsmemBytes;  // dynamic shared memory per CTA of the single solve
    int tuned_team = 0;   // team size found by rgdbek_tune_batched (0 = none yet)
    int tuned_block = 0;  // block of the batched solve found by it (0 = automatic)
    // trace
    long long *tr_counts = nullptr;
    long long tr_count_cap = 0;
    int *tr_lists = nullptr;
    long long tr_list_cap = 0;
    double *tr_g = nullptr, *tr_r = nullptr;
    long long tr_vec_cap = 0;
};

namespace {

// Bump allocator over one device allocation; every sub-buffer 256-byte aligned.
struct Layout {
    size_t off = 0;
    char *base = nullptr;
    template <typename T>
    T *take(long long count) {
        const size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    }
};

// The matrix arrays, in their own allocation (shared by derived handles).
void carve_matrix(rgdbek_s *h, Layout &L) {
    const long long m = h->m, n = h->n, nnz = h->nnz;
    h->rp = L.take<long long>(m + 1);
    h->ci = L.take<int>(nnz);
    h->av = L.take<double>(nnz);
    h->cp = L.take<long long>(n + 1);
    h->ri = L.take<int>(nnz);
    h->cv = L.take<double>(nnz);
    h->rn2 = L.take<double>(m);
    h->cn2 = L.take<double>(n);
}

// The workspace of one handle.
void carve(rgdbek_s *h, Layout &L) {
    const long long m = h->m, n = h->n, nnz = h->nnz, mx = m > n ? m : n;
    // Work vectors indexed by rows or by columns are all max(m, n) long, so
    // that the same workspace serves the solves on A^T of rgdbek_backward.
    h->z = L.take<double>(2 * mx);  // (z_i, t_i) pairs
    h->t = h->z + 1;
    h->r = L.take<double>(mx);
    h->epsr = L.take<double>(mx);
    h->uu = L.take<double>(mx);
    h->g = L.take<double>(mx);
    h->epsc = L.take<double>(mx);
    h->vv = L.take<double>(mx);
    h->ww = L.take<double>(mx);
    h->yy = L.take<double>(mx);
    h->dx = L.take<double>(mx);
    h->xt = L.take<double>(mx);
    h->Q = L.take<unsigned long long>(mx);
    h->flag = L.take<unsigned char>(mx);
    h->colpos = L.take<int>(mx);
    h->rowpos = L.take<int>(mx);
    h->ulist = L.take<int>(mx);
    h->jlist = L.take<int>(mx);
    h->srn = L.take<int>(mx);
    h->sci = L.take<int>(nnz);
    h->sav = L.take<double>(nnz);
    h->scn = L.take<int>(mx);
    h->sri = L.take<int>(nnz);
    h->scv = L.take<double>(nnz);
    h->dots = L.take<double>(mx);
    h->dots2 = L.take<double>(mx);
    h->vvs = L.take<double>(mx);
    h->dsc = L.take<double>(mx);
    h->yh = L.take<double>(mx);
    h->uus = L.take<double>(mx);
    h->dsr = L.take<double>(mx);
    h->pd = L.take<double>((long long)D_NSLOTS * kMaxGrid);
    h->pi = L.take<long long>((long long)I_NSLOTS * kMaxGrid);
    h->f_z = L.take<float>(2 * mx);
    float **fv[] = {&h->f_r,  &h->f_g,    &h->f_epsc, &h->f_epsr, &h->f_uu,  &h->f_vv,
                    &h->f_ww, &h->f_yy,   &h->f_dx,   &h->f_xt,   &h->f_x,   &h->f_b,
                    &h->f_dots, &h->f_dots2, &h->f_vvs, &h->f_dsc, &h->f_yh, &h->f_uus,
                    &h->f_dsr};
    for (float **p : fv) *p = L.take<float>(mx);
    h->f_pd = L.take<float>((long long)D_NSLOTS * kMaxGrid);
    h->ref_t = L.take<double>(mx);
    h->ref_b = L.take<double>(mx);
    h->ref_x = L.take<double>(mx);
    double **zv[] = {&h->uu_z, &h->vv_z, &h->ww_z, &h->dots_z, &h->dots2_z};
    for (double **p : zv) *p = L.take<double>(mx);
    h->pd_z = L.take<double>((long long)D_NSLOTS * kMaxGrid);
    float **zf[] = {&h->f_uu_z, &h->f_vv_z, &h->f_ww_z, &h->f_dots_z, &h->f_dots2_z};
    for (float **p : zf) *p = L.take<float>(mx);
    h->f_pd_z = L.take<float>((long long)D_NSLOTS * kMaxGrid);
    h->pi_z = L.take<long long>((long long)I_NSLOTS * kMaxGrid);
    h->Q_z = L.take<unsigned long long>(mx);
    h->flag_z = L.take<unsigned char>(mx);
    h->ulist2 = L.take<int>(mx);
    h->ctrl = L.take<Ctrl>(1);
    h->b_stage = L.take<double>(m);
    h->x_stage = L.take<double>(n);
}

int check_options(const rgdbek_options &o) {
    if (!(o.eta_col > 0.0 && o.eta_col <= 1.0) || !(o.eta_row > 0.0 && o.eta_row <= 1.0))
        return RGDBEK_ERR_INVALID_ARG;
    if (o.selection != RGDBEK_SELECT_RANDOM && o.selection != RGDBEK_SELECT_GREEDY)
        return RGDBEK_ERR_INVALID_ARG;
    if (!(o.inner_tol >= 0.0) || o.inner_max < 1) return RGDBEK_ERR_INVALID_ARG;
    if (o.stop_rule < 0 || o.stop_rule > 3) return RGDBEK_ERR_INVALID_ARG;
    if (!(o.time_budget_s >= 0.0)) return RGDBEK_ERR_INVALID_ARG;
    if (o.blocks_per_sm < 0 || o.threads_per_block < 0) return RGDBEK_ERR_INVALID_ARG;
    if (o.precision != RGDBEK_PRECISION_FP64 && o.precision != RGDBEK_PRECISION_FP32_INNER)
        return RGDBEK_ERR_INVALID_ARG;
    if (o.batch_team < 0 || o.batch_team > kMaxGrid) return RGDBEK_ERR_INVALID_ARG;
    if (o.warm_start != 0 && o.warm_start != 1) return RGDBEK_ERR_INVALID_ARG;
    if (!(o.inner_adapt >= 0.0)) return RGDBEK_ERR_INVALID_ARG;
    if (o.col_team < -1 || o.col_team > kMaxGrid) return RGDBEK_ERR_INVALID_ARG;
    if (o.smem_per_cta != 0 && (o.smem_per_cta < 32768 || o.smem_per_cta % 1024 != 0))
        return RGDBEK_ERR_INVALID_ARG;
    if (o.threads_per_block != 0 &&
        (o.threads_per_block % 32 != 0 || o.threads_per_block < 64 ||
         o.threads_per_block > kSolveMaxThreads))
        return RGDBEK_ERR_INVALID_ARG;
    return RGDBEK_OK;
}

// launch shape of the persistent kernels for the handle's options
int configure_launch(rgdbek_s *h) {
    const int block = h->opt.threads_per_block ? h->opt.threads_per_block
                                               : auto_solve_block(h->m, h->n, h->num_sms);
    const int dmax = solve_dsmem_max();
    if (dmax <= 0) return RGDBEK_ERR_CUDA;
    // 96 KB unless asked: more shared memory shrinks the L1 cache, and the
    // full-matrix passes then lose more than the inner solves gain (measured)
    const int want = h->opt.smem_per_cta ? h->opt.smem_per_cta : kSolveDsmemBytes;
    const int dsmem = want < dmax ? want : dmax;
    int fit = solve_blocks_per_sm(block, dsmem);
    int fit_s = sample_blocks_per_sm(block);
    if (fit < 1 || fit_s < 1) return RGDBEK_ERR_CUDA;
    int bps = h->opt.blocks_per_sm ? h->opt.blocks_per_sm : fit;
    if (bps > fit) bps = fit;
    long long grid = (long long)bps * h->num_sms;
    if (grid > kMaxGrid) grid = kMaxGrid;
    long long sgrid = (long long)(fit_s < bps ? fit_s : bps) * h->num_sms;
    if (sgrid > kMaxGrid) sgrid = kMaxGrid;
    h->block = block;
    h->grid = (int)grid;
    h->sample_grid = (int)sgrid;
    h->dsmem = dsmem;
    return RGDBEK_OK;
}

// Kernel parameters for A (transposed = false) or for A^T (transposed =
// true): the CSC arrays of A are the CSR arrays of A^T and vice versa, and
// row and column norms trade places.  The trace is recorded for A only.
Params make_params(const rgdbek_s *h, bool transposed = false) {
    Params P{};
    P.m = h->m;
    P.n = h->n;
    P.nnz = h->nnz;
    P.rp = h->rp;
    P.ci = h->ci;
    P.av = h->av;
    P.cp = h->cp;
    P.ri = h->ri;
    P.cv = h->cv;
    P.rn2 = h->rn2;
    P.cn2 = h->cn2;
    P.z = h->z;
    P.t = h->t;
    P.r = h->r;
    P.g = h->g;
    P.epsc = h->epsc;
    P.epsr = h->epsr;
    P.uu = h->uu;
    P.vv = h->vv;
    P.ww = h->ww;
    P.yy = h->yy;
    P.dx = h->dx;
    P.xt = h->xt;
    P.Q = h->Q;
    P.flag = h->flag;
    P.colpos = h->colpos;
    P.rowpos = h->rowpos;
    P.ulist = h->ulist;
    P.jlist = h->jlist;
    P.srn = h->srn;
    P.sci = h->sci;
    P.sav = h->sav;
    P.scn = h->scn;
    P.sri = h->sri;
    P.scv = h->scv;
    P.dots = h->dots;
    P.dots2 = h->dots2;
    P.pd = h->pd;
    P.pi = h->pi;
    P.ctrl = h->ctrl;
    P.tr_counts = h->tr_counts;
    P.tr_count_cap = h->tr_count_cap;
    P.tr_lists = h->tr_lists;
    P.tr_list_cap = h->tr_list_cap;
    P.tr_g = h->tr_g;
    P.tr_r = h->tr_r;
    P.tr_vec_cap = h->tr_vec_cap;
    P.eta_col = h->opt.eta_col;
    P.eta_row = h->opt.eta_row;
    P.precision = h->opt.precision;
    P.warm = h->opt.warm_start != 0;
    P.inner_adapt = h->opt.inner_adapt;
    P.inner_tol = h->opt.inner_tol;
    P.k0 = 0;
    P.vvs = h->vvs;
    P.dsc = h->dsc;
    P.yh = h->yh;
    P.uus = h->uus;
    P.dsr = h->dsr;
    P.ref_t = h->ref_t;
    P.ref_b = h->ref_b;
    P.ref_x = h->ref_x;
    P.inner_max = h->opt.inner_max;
    P.stop_rule = h->opt.stop_rule;
    P.selection = h->opt.selection;
    P.sysid = h->opt.system_id;
    P.time_budget_ns = h->opt.time_budget_s * 1e9;
    P.tpr = h->tpr;
    P.tpc = h->tpc;
    P.lpr = h->lpr;
    P.lpc = h->lpc;
    P.ipr = h->ipr;
    P.ipc = h->ipc;
    P.dsmem_bytes = h->dsmem;
    P.team = h->grid;
    P.zteam = 0;  // one team unless the solve chooses two (run_solve)
    P.uu_z = h->uu_z;
    P.vv_z = h->vv_z;
    P.ww_z = h->ww_z;
    P.dots_z = h->dots_z;
    P.dots2_z = h->dots2_z;
    P.pd_z = h->pd_z;
    P.pi_z = h->pi_z;
    P.Q_z = h->Q_z;
    P.flag_z = h->flag_z;
    P.ulist2 = h->ulist2;
    P.bar = nullptr;
    if (transposed) {
        P.m = h->n;
        P.n = h->m;
        P.rp = h->cp;
        P.ci = h->ri;
        P.av = h->cv;
        P.cp = h->rp;
        P.ri = h->ci;
        P.cv = h->av;
        P.rn2 = h->cn2;
        P.cn2 = h->rn2;
        P.tpr = h->tpc;
        P.tpc = h->tpr;
        P.lpr = h->lpc;
        P.lpc = h->lpr;
        P.ipr = h->ipc;
        P.ipc = h->ipr;
        P.tr_counts = nullptr;
        P.tr_count_cap = 0;
        P.tr_lists = nullptr;
        P.tr_list_cap = 0;
        P.tr_g = nullptr;
        P.tr_r = nullptr;
        P.tr_vec_cap = 0;
    }
    return P;
}

// The FP32 view of the same system for the inner solves of the FP32 form:
// A's values and norms rounded to float (the matrix store's copies, which
// ensure_f32_matrix makes), float work vectors, and everything else shared
// with the FP64 view P (indices, selection scratch, int64 partials, control
// block, trace).  The inner solves start from d = 0 on their own right-hand
// side f_b and take the inner LSQR tolerance no lower than
// RGDBEK_FP32_INNER_TOL.
ParamsF make_params_f(const rgdbek_s *h, const Params &P, bool transposed) {
    ParamsF F{};
    const MatrixStore *M = h->mat;
    F.m = P.m;
    F.n = P.n;
    F.nnz = P.nnz;
    F.rp = P.rp;
    F.ci = P.ci;
    F.cp = P.cp;
    F.ri = P.ri;
    F.av = transposed ? M->cv32 : M->av32;
    F.cv = transposed ? M->av32 : M->cv32;
    F.rn2 = transposed ? M->cn2f : M->rn2f;
    F.cn2 = transposed ? M->rn2f : M->cn2f;
    F.b = h->f_b;
    F.x = h->f_x;
    F.z = h->f_z;
    F.t = h->f_z + 1;
    F.r = h->f_r;
    F.g = h->f_g;
    F.epsc = h->f_epsc;
    F.epsr = h->f_epsr;
    F.uu = h->f_uu;
    F.vv = h->f_vv;
    F.ww = h->f_ww;
    F.yy = h->f_yy;
    F.dx = h->f_dx;
    F.xt = h->f_xt;
    F.Q = P.Q;
    F.flag = P.flag;
    F.colpos = P.colpos;
    F.rowpos = P.rowpos;
    F.ulist = P.ulist;
    F.jlist = P.jlist;
    F.srn = P.srn;
    F.sci = P.sci;
    F.sav = reinterpret_cast<float *>(h->sav);
    F.scn = P.scn;
    F.sri = P.sri;
    F.scv = reinterpret_cast<float *>(h->scv);
    F.dots = h->f_dots;
    F.dots2 = h->f_dots2;
    F.pd = h->f_pd;
    F.pi = P.pi;
    F.ctrl = P.ctrl;
    F.tr_counts = P.tr_counts;
    F.tr_count_cap = P.tr_count_cap;
    F.tr_lists = P.tr_lists;
    F.tr_list_cap = P.tr_list_cap;
    F.tr_g = P.tr_g;
    F.tr_r = P.tr_r;
    F.tr_vec_cap = P.tr_vec_cap;
    F.tol = P.tol;
    F.inner_tol = P.inner_tol < RGDBEK_FP32_INNER_TOL ? RGDBEK_FP32_INNER_TOL : P.inner_tol;
    F.eta_col = P.eta_col;
    F.eta_row = P.eta_row;
    F.inner_adapt = P.inner_adapt;
    F.time_budget_ns = P.time_budget_ns;
    F.max_iter = P.max_iter;
    F.s_col = P.s_col;
    F.s_row = P.s_row;
    F.k0 = 0;
    F.seed = P.seed;
    F.sysid = P.sysid;
    F.inner_max = P.inner_max;
    F.stop_rule = P.stop_rule;
    F.selection = P.selection;
    F.precision = P.precision;
    F.team = P.team;
    F.warm = 0;
    F.vvs = h->f_vvs;
    F.dsc = h->f_dsc;
    F.yh = h->f_yh;
    F.uus = h->f_uus;
    F.dsr = h->f_dsr;
    F.tpr = P.tpr;
    F.tpc = P.tpc;
    F.lpr = P.lpr;
    F.lpc = P.lpc;
    F.ipr = P.ipr;
    F.ipc = P.ipc;
    F.dsmem_bytes = P.dsmem_bytes;
    F.zteam = P.zteam;
    F.uu_z = h->f_uu_z;
    F.vv_z = h->f_vv_z;
    F.ww_z = h->f_ww_z;
    F.dots_z = h->f_dots_z;
    F.dots2_z = h->f_dots2_z;
    F.pd_z = h->f_pd_z;
    F.pi_z = P.pi_z;
    F.Q_z = P.Q_z;
    F.flag_z = P.flag_z;
    F.ulist2 = P.ulist2;
    F.bar = nullptr;
    return F;
}

// The float copies of A's values and squared norms for the FP32 form, made
// once per matrix (and shared by the handles that share it).  The copies are
// complete before they are published: another handle on another stream may
// use them as soon as it sees them.
int ensure_f32_matrix(rgdbek_s *h) {
    MatrixStore *M = h->mat;
    std::lock_guard<std::mutex> lock(M->mu32);
    if (M->mem32) return RGDBEK_OK;
    Layout L;
    void *p = nullptr;
    float *av32 = nullptr, *cv32 = nullptr, *rn2f = nullptr, *cn2f = nullptr;
    for (int pass = 0; pass < 2; ++pass) {
        av32 = L.take<float>(h->nnz);
        cv32 = L.take<float>(h->nnz);
        rn2f = L.take<float>(h->m);
        cn2f = L.take<float>(h->n);
        if (pass == 0) {
            const cudaError_t e = cudaMalloc(&p, L.off);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RGDBEK_ERR_OOM : RGDBEK_ERR_CUDA;
            L = Layout();
            L.base = static_cast<char *>(p);
        }
    }
    cudaError_t e = launch_to_float(h->av, h->nnz, av32, h->stream);
    if (e == cudaSuccess) e = launch_to_float(h->cv, h->nnz, cv32, h->stream);
    if (e == cudaSuccess) e = launch_to_float(h->rn2, h->m, rn2f, h->stream);
    if (e == cudaSuccess) e = launch_to_float(h->cn2, h->n, cn2f, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaFree(p);
        return RGDBEK_ERR_CUDA;
    }
    M->av32 = av32;
    M->cv32 = cv32;
    M->rn2f = rn2f;
    M->cn2f = cn2f;
    M->mem32 = p;
    return RGDBEK_OK;
}

// ceil(eta * len) draws, at least one (Algorithm 1 selects eta*n columns)
long long num_draws(double eta, long long len) {
    if (len <= 0) return 0;
    double s = std::ceil(eta * (double)len);
    if (s < 1.0) s = 1.0;
    return (long long)s;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RGDBEK_OK;
    if (e == cudaErrorMemoryAllocation) return RGDBEK_ERR_OOM;
    return RGDBEK_ERR_CUDA;
}

// Copies the control block back and waits for the stream.
int read_ctrl(rgdbek_s *h) {
    cudaError_t e = cudaMemcpyAsync(h->ctrl_host, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

void fill_stats(const Ctrl &c, int status, rgdbek_stats *st);

// One persistent-kernel solve of A x = b (or of A^T x = b when transposed),
// x0 = 0; reads the control block back into *st.
// CTAs of the column team of a single solve (0: one team), option col_team;
// `transposed`: the solve runs on A^T (rows and columns swap roles).
//
// Automatic: two teams only where the row step dominates an outer iteration.
// With equal eta the two blocks hold about the same number of nonzeros, but
// for m >> n the row block (about eta m rows of n columns) is much closer to
// square than the column block (m rows, eta n columns), so its LSQR needs
// many more steps (47.6 against 7.5 per iteration on the 200000 x 50000
// benchmark, where a quarter of the grid on the column steps was measured
// fastest).  Where the two steps cost about the same (square or 2:1 systems,
// fat systems, blocks at the inner step cap) a column team of a quarter of
// the grid would become the critical path, so m < 4n runs one team.
int choose_zteam(const rgdbek_s *h, bool transposed) {
    const int c = h->opt.col_team;
    if (c < 0 || h->opt.inner_adapt > 0.0 || h->grid < 8) return 0;
    if (c > 0) return c < h->grid / 2 ? c : h->grid / 2;
    const long long rows = transposed ? h->n : h->m, cols = transposed ? h->m : h->n;
    if (rows < 4 * cols) return 0;
    const int a = h->grid / 4;
    return a > 1 ? a : 1;
}

int run_solve(rgdbek_s *h, bool transposed, const double *b, double *x, double tol,
              long long max_iter, uint64_t seed, rgdbek_stats *st, bool from_zero = false) {
    Params P = make_params(h, transposed);
    P.zteam = choose_zteam(h, transposed);
    if (from_zero) P.warm = 0;  // the adjoint's inner solves and the tuner's probes
    P.b = b;
    P.x = x;
    P.tol = tol;
    P.max_iter = max_iter;
    P.seed = seed;
    P.s_col = num_draws(h->opt.eta_col, P.n);
    P.s_row = num_draws(h->opt.eta_row, P.m);
    ParamsF F{};
    if (P.precision == RGDBEK_PRECISION_FP32_INNER) {
        const int st32 = ensure_f32_matrix(h);
        if (st32 != RGDBEK_OK) return st32;
        P.team = h->grid;
        F = make_params_f(h, P, transposed);
    }
    cudaError_t e = launch_reset_ctrl(h->ctrl, h->stream);
    if (e == cudaSuccess) e = launch_solve(P, F, h->grid, h->block, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int rs = read_ctrl(h);
    if (rs != RGDBEK_OK) return rs;
    const Ctrl &c = *h->ctrl_host;
    const int status = c.status == kStatusRunning ? RGDBEK_ERR_CUDA : c.status;
    fill_stats(c, status, st);
    return status;
}

void fill_stats(const Ctrl &c, int status, rgdbek_stats *st) {
    if (st) {
        st->iters = c.iters;
        st->inner_u = c.inner_u;
        st->inner_j = c.inner_j;
        st->sum_nu = c.sum_nu;
        st->sum_nj = c.sum_nj;
        st->sum_nnz_u = c.sum_nnzu;
        st->sum_nnz_j = c.sum_nnzj;
        st->lsqr_nnz_u = c.lsqr_nnzu;
        st->lsqr_nnz_j = c.lsqr_nnzj;
        st->lsqr_n_u = c.lsqr_nu;
        st->lsqr_n_j = c.lsqr_nj;
        st->rel_res = c.rel_res;
        st->normal_res = c.normal_res;
        st->rse = c.rse;
        st->status = status;
        for (int i = 0; i < RGDBEK_NUM_PHASES; ++i)
            st->phase_ms[i] = 1e-6 * ((double)c.phase_ns[i] + (double)c.zphase_ns[i]);
        st->refinements = c.refinements;
    }
}

// Team sizes the batched solve and its tuner consider (CTAs per system).
constexpr int kNumTeamCandidates = RGDBEK_BATCH_TEAM_CANDIDATES;
constexpr int kTeamCandidates[kNumTeamCandidates] = {1, 2, 4, 8, 19, 38, 76, 152};

// Without a tuned or requested size: about one system per team, i.e. the
// candidate nearest grid / nsys (at least 1).
int default_team(const rgdbek_s *h, int nsys) {
    if (!h) return 1;
    const double want = (double)h->grid / (double)nsys;
    int best = 1;
    for (int c = 0; c < kNumTeamCandidates; ++c)
        if (kTeamCandidates[c] <= h->grid && kTeamCandidates[c] <= want) best = kTeamCandidates[c];
    return best;
}

// Largest-first list scheduling (LPT) of the systems onto nteams teams, by a
// work estimate of nnz + m + n per outer iteration.  plan[t * stride + q] is
// the q-th system of team t, -1 after the last.
void plan_batch(int nsys, rgdbek_t *hs, int nteams, std::vector<int> &plan, int &stride) {
    std::vector<int> order(nsys);
    for (int i = 0; i < nsys; ++i) order[i] = i;
    auto cost = [&](int i) { return (double)(hs[i]->nnz + hs[i]->m + hs[i]->n); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
    std::vector<double> load(nteams, 0.0);
    std::vector<std::vector<int>> lists(nteams);
    for (int i : order) {
        int t = 0;
        for (int u = 1; u < nteams; ++u)
            if (load[u] < load[t]) t = u;
        load[t] += cost(i);
        lists[t].push_back(i);
    }
    stride = 1;
    for (const auto &l : lists) stride = std::max(stride, (int)l.size() + 1);
    plan.assign((size_t)nteams * stride, -1);
    for (int t = 0; t < nteams; ++t)
        for (size_t q = 0; q < lists[t].size(); ++q) plan[(size_t)t * stride + q] = lists[t][q];
}

// One cooperative launch solving all systems with `team` CTAs each.
// Optionally times the launch (ms).  Statuses: the most negative error, else
// NOT_CONVERGED if any system hit its cap.
int run_batched(int nsys, rgdbek_t *hs, const double *const *b, double *const *x,
                const double *tol, long long max_iter, uint64_t seed, rgdbek_stats *st, int team,
                float *ms, int block_req = 0) {
    rgdbek_s *h0 = hs[0];
    if (!h0 || team < 1) return RGDBEK_ERR_INVALID_ARG;
    for (int i = 0; i < nsys; ++i) {
        if (!hs[i] || !b[i] || !x[i] || !(tol[i] >= 0.0) || max_iter < 0) return RGDBEK_ERR_INVALID_ARG;
        if (hs[i]->device != h0->device || hs[i]->opt.precision != h0->opt.precision)
            return RGDBEK_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return RGDBEK_ERR_INVALID_ARG;  // one workspace per system
    }
    // block: hs[0]'s option, else by the largest system's share per CTA; the
    // grid: as many CTAs of that block as are co-resident
    int block = block_req ? block_req : h0->opt.threads_per_block;
    if (block == 0 && h0->tuned_block > 0) block = h0->tuned_block;
    if (block == 0) {
        long long vmax = 0;
        for (int i = 0; i < nsys; ++i) vmax = std::max(vmax, std::max(hs[i]->m, hs[i]->n));
        block = auto_solve_block(vmax, 0, team);
    }
    const int fit = batched_blocks_per_sm(block);
    if (fit < 1) return RGDBEK_ERR_CUDA;
    const long long gmax = std::min((long long)kMaxGrid, (long long)fit * h0->num_sms);
    if (team > gmax) return RGDBEK_ERR_INVALID_ARG;
    const int nteams = (int)(gmax / team);
    const bool f32 = h0->opt.precision == RGDBEK_PRECISION_FP32_INNER;
    std::vector<SysPair> sys(nsys);
    for (int i = 0; i < nsys; ++i) {
        if (f32) {
            const int st32 = ensure_f32_matrix(hs[i]);
            if (st32 != RGDBEK_OK) return st32;
        }
        Params P = make_params(hs[i]);
        P.b = b[i];
        P.x = x[i];
        P.tol = tol[i];
        P.max_iter = max_iter;
        P.seed = seed;
        P.sysid = (unsigned long long)i;
        P.s_col = num_draws(hs[i]->opt.eta_col, P.n);
        P.s_row = num_draws(hs[i]->opt.eta_row, P.m);
        P.team = team;
        P.dsmem_bytes = kSolveDsmemBytes;  // the batched kernel's launch size
        P.tr_counts = nullptr;
        P.tr_count_cap = 0;
        P.tr_lists = nullptr;
        P.tr_list_cap = 0;
        P.tr_g = nullptr;
        P.tr_r = nullptr;
        P.tr_vec_cap = 0;
        sys[i].p = P;
        sys[i].f = f32 ? make_params_f(hs[i], P, false) : ParamsF{};
    }
    std::vector<int> plan;
    int stride = 1;
    plan_batch(nsys, hs, nteams, plan, stride);
    const size_t sys_bytes = (sizeof(SysPair) * nsys + 255) & ~(size_t)255;
    const size_t plan_bytes = (sizeof(int) * plan.size() + 255) & ~(size_t)255;
    const size_t ctrl_bytes = sizeof(Ctrl) * nsys;
    char *dev = nullptr;
    Ctrl *host = nullptr;
    cudaStream_t s = h0->stream;
    cudaError_t e = cudaMalloc(&dev, sys_bytes + plan_bytes + ctrl_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&host, ctrl_bytes);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess && ms) {
        e = cudaEventCreate(&ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    }
    SysPair *sys_dev = reinterpret_cast<SysPair *>(dev);
    int *plan_dev = reinterpret_cast<int *>(dev + sys_bytes);
    Ctrl *ctrl_dev = reinterpret_cast<Ctrl *>(dev + sys_bytes + plan_bytes);
    // the handles' own streams must have finished their earlier work
    for (int i = 0; e == cudaSuccess && i < nsys; ++i)
        if (hs[i]->stream != s) e = cudaStreamSynchronize(hs[i]->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sys_dev, sys.data(), sizeof(SysPair) * nsys, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan_dev, plan.data(), sizeof(int) * plan.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_reset_ctrls(sys_dev, nsys, s);
    if (e == cudaSuccess && ms) e = cudaEventRecord(ev0, s);
    if (e == cudaSuccess)
        e = launch_solve_batched(sys_dev, plan_dev, stride, team, nteams, f32, block, s);
    if (e == cudaSuccess && ms) e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = launch_gather_ctrls(sys_dev, nsys, ctrl_dev, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, ctrl_dev, ctrl_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, ev0, ev1);
    int worst = RGDBEK_OK;
    if (e == cudaSuccess) {
        for (int i = 0; i < nsys; ++i) {
            const Ctrl &c = host[i];
            const int status = c.status == kStatusRunning ? RGDBEK_ERR_CUDA : c.status;
            fill_stats(c, status, st ? st + i : nullptr);
            if (status < 0 && (worst >= 0 || status < worst)) worst = status;
            else if (status == RGDBEK_NOT_CONVERGED && worst == RGDBEK_OK) worst = status;
        }
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (host) cudaFreeHost(host);
    if (dev) cudaFree(dev);
    return e == cudaSuccess ? worst : cuda_status(e);
}

void release(rgdbek_s *h) {
    if (!h) return;
    if (h->adj) cudaFree(h->adj);
    if (h->arena) cudaFree(h->arena);
    if (h->mat && h->mat->refs.fetch_sub(1) == 1) {
        if (h->mat->mem) cudaFree(h->mat->mem);
        if (h->mat->mem32) cudaFree(h->mat->mem32);
        delete h->mat;
    }
    if (h->ctrl_host) cudaFreeHost(h->ctrl_host);
    delete h;
}

}  // namespace

extern "C" {

void rgdbek_default_options(rgdbek_options *opt) {
    if (!opt) return;
    opt->eta_col = 0.5;
    opt->eta_row = 0.5;
    opt->selection = RGDBEK_SELECT_RANDOM;
    opt->inner_tol = 1e-10;
    opt->inner_max = 200;
    opt->stop_rule = RGDBEK_STOP_AUTO;
    opt->time_budget_s = 0.0;
    opt->system_id = 0;
    opt->blocks_per_sm = 0;
    opt->threads_per_block = 0;
    opt->precision = RGDBEK_PRECISION_FP64;
    opt->batch_team = 0;
    opt->warm_start = 0;
    opt->inner_adapt = 0.0;
    opt->col_team = 0;
    opt->smem_per_cta = 0;
}

int rgdbek_create(rgdbek_t *out, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, int ptr_is_device,
                  const rgdbek_options *opt, void *stream) {
    if (!out) return RGDBEK_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || nnz < 0 || m >= (1ll << 31) || n >= (1ll << 31) || nnz >= (1ll << 50))
        return RGDBEK_ERR_INVALID_ARG;
    if (!row_ptr || (nnz > 0 && (!col_idx || !vals))) return RGDBEK_ERR_INVALID_ARG;
    rgdbek_options o;
    rgdbek_default_options(&o);
    if (opt) o = *opt;
    int st = check_options(o);
    if (st != RGDBEK_OK) return st;

    rgdbek_s *h = new (std::nothrow) rgdbek_s();
    if (!h) return RGDBEK_ERR_OOM;
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    h->opt = o;
    h->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&h->device);
    int coop = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (e != cudaSuccess || !coop) {
        release(h);
        return RGDBEK_ERR_CUDA;
    }
    if ((st = configure_launch(h)) != RGDBEK_OK) {
        release(h);
        return st;
    }
    h->tpr = pick_lanes_fp64(nnz, m);
    h->tpc = pick_lanes_fp64(nnz, n);
    h->lpr = h->tpr;
    h->lpc = h->tpc;
    h->ipr = pick_lanes_int(nnz, m);
    h->ipc = pick_lanes_int(nnz, n);

    h->mat = new (std::nothrow) MatrixStore();
    if (!h->mat) {
        release(h);
        return RGDBEK_ERR_OOM;
    }
    Layout M;
    carve_matrix(h, M);
    h->mat->bytes = M.off;
    Layout L;
    carve(h, L);
    h->arena_bytes = L.off;
    if ((e = cudaMalloc(&h->mat->mem, h->mat->bytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->arena, h->arena_bytes)) != cudaSuccess ||
        (e = cudaMallocHost(&h->ctrl_host, sizeof(Ctrl))) != cudaSuccess) {
        release(h);
        return cuda_status(e);
    }
    M = Layout();
    M.base = static_cast<char *>(h->mat->mem);
    carve_matrix(h, M);
    L = Layout();
    L.base = static_cast<char *>(h->arena);
    carve(h, L);

    // set-up scratch, freed before returning
    const long long keys = nnz > n ? nnz : n;
    Layout S;
    long long *key_a = S.take<long long>(keys);
    long long *key_b = S.take<long long>(keys);
    int *row_of = S.take<int>(nnz);
    long long *cursor = S.take<long long>(n);
    long long *blk = S.take<long long>(n / 1024 + 2);
    int *err = S.take<int>(1);
    (void)key_a; (void)key_b; (void)row_of; (void)cursor; (void)blk; (void)err;
    void *scratch = nullptr;
    if ((e = cudaMalloc(&scratch, S.off)) != cudaSuccess) {
        release(h);
        return cuda_status(e);
    }
    S = Layout();
    S.base = static_cast<char *>(scratch);
    key_a = S.take<long long>(keys);
    key_b = S.take<long long>(keys);
    row_of = S.take<int>(nnz);
    cursor = S.take<long long>(n);
    blk = S.take<long long>(n / 1024 + 2);
    err = S.take<int>(1);

    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t s = h->stream;
    int verdict = RGDBEK_OK;
    do {
        if ((e = cudaMemcpyAsync(h->rp, row_ptr, (size_t)(m + 1) * sizeof(long long), kind, s)) !=
            cudaSuccess)
            break;
        if (nnz > 0) {
            if ((e = cudaMemcpyAsync(h->ci, col_idx, (size_t)nnz * sizeof(int), kind, s)) !=
                cudaSuccess)
                break;
            if ((e = cudaMemcpyAsync(h->av, vals, (size_t)nnz * sizeof(double), kind, s)) !=
                cudaSuccess)
                break;
        }
        if ((e = validate_csr(m, n, nnz, h->rp, h->ci, h->av, err, &verdict, s)) != cudaSuccess)
            break;
        if (verdict != RGDBEK_OK) break;
        if ((e = build_csc(m, n, nnz, h->rp, h->ci, h->av, h->cp, h->ri, h->cv, key_a, key_b,
                           row_of, cursor, blk, s)) != cudaSuccess)
            break;
        if ((e = line_norms2(m, h->rp, h->av, h->rn2, s)) != cudaSuccess) break;
        if ((e = line_norms2(n, h->cp, h->cv, h->cn2, s)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
    } while (0);
    cudaFree(scratch);
    if (e != cudaSuccess) verdict = cuda_status(e);
    if (verdict != RGDBEK_OK) {
        release(h);
        return verdict;
    }
    *out = h;
    return RGDBEK_OK;
}

int rgdbek_create_like(rgdbek_t base, const rgdbek_options *opt, void *stream, rgdbek_t *out) {
    if (!out) return RGDBEK_ERR_INVALID_ARG;
    *out = nullptr;
    if (!base || !base->mat) return RGDBEK_ERR_INVALID_ARG;
    rgdbek_options o = base->opt;
    if (opt) o = *opt;
    int st = check_options(o);
    if (st != RGDBEK_OK) return st;
    rgdbek_s *h = new (std::nothrow) rgdbek_s();
    if (!h) return RGDBEK_ERR_OOM;
    h->device = base->device;
    h->num_sms = base->num_sms;
    h->m = base->m;
    h->n = base->n;
    h->nnz = base->nnz;
    h->opt = o;
    h->stream = (cudaStream_t)stream;
    h->tpr = base->tpr;
    h->tpc = base->tpc;
    h->lpr = base->lpr;
    h->lpc = base->lpc;
    h->ipr = base->ipr;
    h->ipc = base->ipc;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
        delete h;
        return RGDBEK_ERR_INVALID_ARG;  // the matrix lives on another device
    }
    if ((st = configure_launch(h)) != RGDBEK_OK) {
        delete h;
        return st;
    }
    // share the matrix (pointers into the base's matrix allocation)
    h->mat = base->mat;
    h->mat->refs.fetch_add(1);
    h->rp = base->rp;
    h->ci = base->ci;
    h->av = base->av;
    h->cp = base->cp;
    h->ri = base->ri;
    h->cv = base->cv;
    h->rn2 = base->rn2;
    h->cn2 = base->cn2;
    Layout L;
    carve(h, L);
    h->arena_bytes = L.off;
    cudaError_t e;
    if ((e = cudaMalloc(&h->arena, h->arena_bytes)) != cudaSuccess ||
        (e = cudaMallocHost(&h->ctrl_host, sizeof(Ctrl))) != cudaSuccess) {
        release(h);
        return cuda_status(e);
    }
    L = Layout();
    L.base = static_cast<char *>(h->arena);
    carve(h, L);
    // the base's set-up (CSC, norms) must be complete before this handle uses it
    if ((e = cudaStreamSynchronize(base->stream)) != cudaSuccess) {
        release(h);
        return cuda_status(e);
    }
    *out = h;
    return RGDBEK_OK;
}

void rgdbek_destroy(rgdbek_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
}

int rgdbek_set_options(rgdbek_t h, const rgdbek_options *opt) {
    if (!h || !opt) return RGDBEK_ERR_INVALID_ARG;
    const int st = check_options(*opt);
    if (st != RGDBEK_OK) return st;
    const rgdbek_options old = h->opt;
    h->opt = *opt;
    const int cs = configure_launch(h);
    if (cs != RGDBEK_OK) {
        h->opt = old;
        configure_launch(h);
    }
    return cs;
}

int rgdbek_set_stream(rgdbek_t h, void *stream) {
    if (!h) return RGDBEK_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return RGDBEK_OK;
}

int rgdbek_get_info(rgdbek_t h, rgdbek_info_t *info) {
    if (!h || !info) return RGDBEK_ERR_INVALID_ARG;
    info->m = h->m;
    info->n = h->n;
    info->nnz = h->nnz;
    info->grid = h->grid;
    info->threads_per_block = h->block;
    info->lanes_per_row = h->lpr;
    info->lanes_per_col = h->lpc;
    info->num_sms = h->num_sms;
    info->device_bytes = (int64_t)(h->arena_bytes + (h->mat ? h->mat->bytes : 0));
    info->col_team = choose_zteam(h, false);
    info->smem_per_cta = h->dsmem;
    return RGDBEK_OK;
}

int rgdbek_set_trace(rgdbek_t h, int64_t *counts, int64_t count_cap, int32_t *lists,
                     int64_t list_cap) {
    if (!h || count_cap < 0 || list_cap < 0) return RGDBEK_ERR_INVALID_ARG;
    h->tr_counts = counts ? (long long *)counts : nullptr;
    h->tr_count_cap = counts ? count_cap : 0;
    h->tr_lists = lists;
    h->tr_list_cap = lists ? list_cap : 0;
    return RGDBEK_OK;
}

int rgdbek_set_trace_vectors(rgdbek_t h, double *g, double *r, int64_t iters_cap) {
    if (!h || iters_cap < 0 || ((g || r) && iters_cap == 0)) return RGDBEK_ERR_INVALID_ARG;
    h->tr_g = g;
    h->tr_r = r;
    h->tr_vec_cap = (g || r) ? iters_cap : 0;
    return RGDBEK_OK;
}

int rgdbek_solve(rgdbek_t h, const double *b, double *x, double tol, int64_t max_iter,
                 uint64_t seed, rgdbek_stats *st) {
    if (!h || !b || !x || !(tol >= 0.0) || max_iter < 0) return RGDBEK_ERR_INVALID_ARG;
    return run_solve(h, false, b, x, tol, max_iter, seed, st);
}

int rgdbek_solve_host(rgdbek_t h, const double *b_host, double *x_host, double tol,
                      int64_t max_iter, uint64_t seed, rgdbek_stats *st) {
    if (!h || !b_host || !x_host) return RGDBEK_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(h->b_stage, b_host, (size_t)h->m * sizeof(double),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->opt.warm_start)  // x_0 from the host buffer
        e = cudaMemcpyAsync(h->x_stage, x_host, (size_t)h->n * sizeof(double),
                            cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int status = rgdbek_solve(h, h->b_stage, h->x_stage, tol, max_iter, seed, st);
    if (status < 0 && status != RGDBEK_ERR_NONFINITE && status != RGDBEK_ERR_TIMEOUT) return status;
    e = cudaMemcpyAsync(x_host, h->x_stage, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? status : cuda_status(e);
}

int rgdbek_solve_batched(int nsys, rgdbek_t *hs, const double *const *b, double *const *x,
                         const double *tol, int64_t max_iter, uint64_t seed, rgdbek_stats *st) {
    if (nsys < 0 || (nsys > 0 && (!hs || !b || !x || !tol))) return RGDBEK_ERR_INVALID_ARG;
    if (nsys == 0) return RGDBEK_OK;
    int team = hs[0] ? hs[0]->opt.batch_team : 0;
    if (team == 0 && hs[0]) team = hs[0]->tuned_team;
    if (team == 0) team = default_team(hs[0], nsys);
    return run_batched(nsys, hs, b, x, tol, max_iter, seed, st, team, nullptr);
}

// Time budgets of the given handles switched off for the life of the object
// (a tuner's probes run their full length), then restored.
struct BudgetsOff {
    std::vector<std::pair<rgdbek_s *, double>> saved;
    BudgetsOff(int n, rgdbek_t *hs) {
        for (int i = 0; i < n; ++i)
            if (hs[i]) {
                saved.emplace_back(hs[i], hs[i]->opt.time_budget_s);
                hs[i]->opt.time_budget_s = 0.0;
            }
    }
    ~BudgetsOff() {
        for (auto &p : saved) p.first->opt.time_budget_s = p.second;
    }
};

int rgdbek_tune_batched(int nsys, rgdbek_t *hs, const double *const *b, double *const *x,
                        const double *tol, int64_t probe_iters, uint64_t seed, int *team_out,
                        int *block_out, double *ms_out) {
    if (nsys < 1 || !hs || !b || !x || !tol || probe_iters < 1 || !team_out || !hs[0])
        return RGDBEK_ERR_INVALID_ARG;
    const BudgetsOff budgets_off(nsys, hs);
    rgdbek_s *h0 = hs[0];
    const int grid = h0->grid;
    h0->tuned_block = 0;
    int best = 0;
    float best_ms = 0.f;
    // team sizes, with the automatic block
    for (int c = 0; c < kNumTeamCandidates; ++c) {
        const int T = kTeamCandidates[c];
        if (ms_out) ms_out[c] = -1.0;
        if (T > grid) continue;
        float ms = 0.f;
        const int s0 = run_batched(nsys, hs, b, x, tol, probe_iters, seed, nullptr, T, &ms);
        if (s0 < 0) return s0;
        if (ms_out) ms_out[c] = ms;
        if (best == 0 || ms < best_ms) {
            best = T;
            best_ms = ms;
        }
    }
    if (best == 0) return RGDBEK_ERR_INVALID_ARG;
    // then the solve kernel's other shape at that team size
    int best_block = 0;
    if (h0->opt.threads_per_block == 0) {
        for (int blk : {kSolveSmallThreads, kSolveMaxThreads}) {
            float ms = 0.f;
            const int s0 =
                run_batched(nsys, hs, b, x, tol, probe_iters, seed, nullptr, best, &ms, blk);
            if (s0 < 0) return s0;
            if (ms_out) ms_out[kNumTeamCandidates + (blk == kSolveMaxThreads ? 1 : 0)] = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best_block = blk;
            }
        }
    }
    h0->tuned_team = best;
    h0->tuned_block = best_block;
    *team_out = best;
    if (block_out) *block_out = best_block;
    return RGDBEK_OK;
}

int rgdbek_tune(rgdbek_t h, const double *b, double *x, int64_t probe_iters, uint64_t seed,
                int *block_out, double *ms_out) {
    if (!h || !b || !x || probe_iters < 1) return RGDBEK_ERR_INVALID_ARG;
    const rgdbek_options saved = h->opt;
    int best = 0;
    float best_ms = 0.f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    h->opt.time_budget_s = 0.0;  // the probes run their full length
    for (int c = 0; e == cudaSuccess && c < 2; ++c) {
        const int blk = c == 0 ? kSolveSmallThreads : kSolveMaxThreads;
        h->opt.threads_per_block = blk;
        int st = configure_launch(h);
        if (st != RGDBEK_OK) {
            h->opt = saved;
            configure_launch(h);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        float ms = 0.f;
        // the probe solves run from x0 = 0 with a zero tolerance: probe_iters
        // outer iterations each
        e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) st = run_solve(h, false, b, x, 0.0, probe_iters, seed, nullptr, true);
        if (e == cudaSuccess && st < 0 && st != RGDBEK_ERR_NONFINITE) {
            h->opt = saved;
            configure_launch(h);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) ms_out[c] = ms;
        if (e == cudaSuccess && (best == 0 || ms < best_ms)) {
            best = blk;
            best_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->opt = saved;
    if (e != cudaSuccess) {
        configure_launch(h);
        return cuda_status(e);
    }
    h->opt.threads_per_block = best;
    const int st = configure_launch(h);
    if (block_out) *block_out = best;
    return st;
}

int rgdbek_tune_teams(rgdbek_t h, const double *b, double *x, int64_t probe_iters,
                      uint64_t seed, int *col_team_out, double *ms_out) {
    if (!h || !b || !x || probe_iters < 1) return RGDBEK_ERR_INVALID_ARG;
    // candidates: one team, then 2/16 .. 5/16 of the grid
    int cand[RGDBEK_COL_TEAM_CANDIDATES];
    cand[0] = -1;
    for (int c = 1; c < RGDBEK_COL_TEAM_CANDIDATES; ++c) {
        int t = ((c + 1) * h->grid + 8) / 16;
        if (t < 1) t = 1;
        if (t > h->grid / 2) t = h->grid / 2;
        cand[c] = t;
    }
    const rgdbek_options saved = h->opt;
    int best = 0;
    bool have = false;
    float best_ms = 0.f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    h->opt.time_budget_s = 0.0;  // the probes run their full length
    for (int c = 0; e == cudaSuccess && c < RGDBEK_COL_TEAM_CANDIDATES; ++c) {
        if (ms_out) ms_out[c] = -1.0;
        // a team size the grid cannot take (grid below 8 CTAs: one team only)
        if (c > 0 && (h->grid < 8 || cand[c] < 1)) continue;
        h->opt.col_team = cand[c];
        float ms = 0.f;
        int st = RGDBEK_OK;
        e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) st = run_solve(h, false, b, x, 0.0, probe_iters, seed, nullptr, true);
        if (e == cudaSuccess && st < 0 && st != RGDBEK_ERR_NONFINITE) {
            h->opt = saved;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out && e == cudaSuccess) ms_out[c] = ms;
        if (e == cudaSuccess && (!have || ms < best_ms)) {
            best = cand[c];
            best_ms = ms;
            have = true;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->opt = saved;
    if (e != cudaSuccess) return cuda_status(e);
    h->opt.col_team = best;
    if (col_team_out) *col_team_out = best;
    return RGDBEK_OK;
}

int rgdbek_tune_eta(rgdbek_t h, const double *b, double *x, const double *candidates,
                    int ncand, int64_t probe_iters, uint64_t seed, double *eta_out,
                    double *rate_out) {
    static const double kDefault[RGDBEK_ETA_CANDIDATES] = {0.05, 0.1, 0.2, 0.3, 0.5};
    if (!h || !b || !x || probe_iters < 1 || ncand < 0 || (ncand > 0 && !candidates))
        return RGDBEK_ERR_INVALID_ARG;
    if (ncand == 0) {
        candidates = kDefault;
        ncand = RGDBEK_ETA_CANDIDATES;
    }
    for (int c = 0; c < ncand; ++c)
        if (!(candidates[c] > 0.0 && candidates[c] <= 1.0)) return RGDBEK_ERR_INVALID_ARG;
    const rgdbek_options saved = h->opt;
    int best = -1;
    double best_rate = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    h->opt.time_budget_s = 0.0;  // the probes run their full length
    for (int c = 0; e == cudaSuccess && c < ncand; ++c) {
        h->opt.eta_col = candidates[c];
        h->opt.eta_row = candidates[c];
        rgdbek_stats st{};
        float ms = 0.f;
        // probe_iters outer iterations from x0 = 0 with a zero tolerance
        e = cudaEventRecord(e0, h->stream);
        int rs = RGDBEK_OK;
        if (e == cudaSuccess) rs = run_solve(h, false, b, x, 0.0, probe_iters, seed, &st, true);
        if (e == cudaSuccess && rs < 0) {
            h->opt = saved;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rs;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        // the stopping rule's measure of x_K (it is 1 at x_0 = 0): its decrease
        // in natural-log units per second of device time
        const double r = h->opt.stop_rule == RGDBEK_STOP_REL_RES
                             ? st.rel_res
                             : (h->opt.stop_rule == RGDBEK_STOP_RSE ? st.rse : st.normal_res);
        const double t = ms > 0.f ? 1e-3 * ms : 1e-9;
        const double rate = r > 0.0 ? -std::log(r) / t : HUGE_VAL;
        if (rate_out) rate_out[c] = rate;
        if (best < 0 || rate > best_rate) {
            best = c;
            best_rate = rate;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->opt = saved;
    if (e != cudaSuccess) return cuda_status(e);
    h->opt.eta_col = candidates[best];
    h->opt.eta_row = candidates[best];
    if (eta_out) *eta_out = candidates[best];
    return RGDBEK_OK;
}

int rgdbek_backward(rgdbek_t h, const double *b, const double *x, const double *grad_x,
                    double *grad_b, double *grad_vals, double tol, int64_t max_iter,
                    uint64_t seed, int flags, rgdbek_stats *st) {
    if (!h || !b || !x || !grad_x || !(tol >= 0.0) || max_iter < 0 ||
        (flags & ~RGDBEK_ADJ_RANK_TERM) != 0)
        return RGDBEK_ERR_INVALID_ARG;
    const bool rank_term = (flags & RGDBEK_ADJ_RANK_TERM) != 0;
    const long long m = h->m, n = h->n;
    cudaError_t e = cudaSuccess;
    if (!h->adj) {
        Layout L;
        for (int pass = 0; pass < 2; ++pass) {
            h->adj_ax = L.take<double>(m);
            h->adj_w = L.take<double>(m);
            h->adj_v = L.take<double>(n);
            h->adj_u = L.take<double>(m);
            h->adj_ag = L.take<double>(m);
            h->adj_q = L.take<double>(n);
            if (pass == 0) {
                void *p = nullptr;
                if ((e = cudaMalloc(&p, L.off)) != cudaSuccess) return cuda_status(e);
                h->adj = static_cast<double *>(p);
                L = Layout();
                L.base = static_cast<char *>(p);
            }
        }
    }
    rgdbek_stats local[4];
    rgdbek_stats *S = st ? st : local;
    std::memset(S, 0, 4 * sizeof(rgdbek_stats));
    int worst = RGDBEK_OK;
    auto fold = [&](int s) {
        if (s < 0 && (worst >= 0 || s < worst)) worst = s;
        else if (s == RGDBEK_NOT_CONVERGED && worst == RGDBEK_OK) worst = s;
    };
    // w = A^+T g: the minimum-norm solution of A^T w = g
    int s0 = run_solve(h, true, grad_x, h->adj_w, tol, max_iter, seed, S + 0, true);
    fold(s0);
    if (s0 < 0) return s0;
    if (grad_b) {
        e = cudaMemcpyAsync(grad_b, h->adj_w, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice,
                            h->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (!grad_vals) {
        e = cudaStreamSynchronize(h->stream);
        return e == cudaSuccess ? worst : cuda_status(e);
    }
    // v = A^+ w
    int s1 = run_solve(h, false, h->adj_w, h->adj_v, tol, max_iter, seed + 1, S + 1, true);
    fold(s1);
    if (s1 < 0) return s1;
    const Params P = make_params(h);
    if (rank_term) {
        // u = A^+T x and q = A^+ (A g), so that p = g - q = (I - A^+ A) g
        int s2 = run_solve(h, true, x, h->adj_u, tol, max_iter, seed + 2, S + 2, true);
        fold(s2);
        if (s2 < 0) return s2;
        if ((e = launch_spmv(P, h->num_sms, kSolveMaxThreads, grad_x, h->adj_ag, h->stream)) != cudaSuccess)
            return cuda_status(e);
        int s3 = run_solve(h, false, h->adj_ag, h->adj_q, tol, max_iter, seed + 3, S + 3, true);
        fold(s3);
        if (s3 < 0) return s3;
    }
    e = launch_spmv(P, h->num_sms, kSolveMaxThreads, x, h->adj_ax, h->stream);
    if (e == cudaSuccess)
        e = launch_adjoint_vals(P, h->num_sms, kSolveMaxThreads, b, h->adj_ax, h->adj_w, h->adj_v, x,
                                rank_term ? h->adj_u : nullptr, grad_x,
                                rank_term ? h->adj_q : nullptr, grad_vals, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? worst : cuda_status(e);
}

int rgdbek_tune_spmv(rgdbek_t h, int reps, int *lanes_row, int *lanes_col, double *us_out) {
    if (!h || reps < 1) return RGDBEK_ERR_INVALID_ARG;
    static const int kCand[RGDBEK_SPMV_LANE_CANDIDATES] = {1, 2, 4, 8, 16, 32};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // input and output vectors from the handle's workspace (zeros: the time of
    // a pass does not depend on the values)
    double *xin = h->ref_x, *zin = h->ref_b, *out = h->ref_t;
    const long long mx = h->m > h->n ? h->m : h->n;
    if (e == cudaSuccess) e = cudaMemsetAsync(xin, 0, (size_t)mx * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(zin, 0, (size_t)mx * sizeof(double), h->stream);
    int best[2] = {h->lpr, h->lpc};
    for (int side = 0; side < 2 && e == cudaSuccess; ++side) {
        float best_us = 0.f;
        for (int c = 0; c < RGDBEK_SPMV_LANE_CANDIDATES && e == cudaSuccess; ++c) {
            Params P = make_params(h);
            if (side == 0) P.lpr = kCand[c];
            else P.lpc = kCand[c];
            std::vector<float> ts;
            for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
                e = cudaEventRecord(e0, h->stream);
                if (e == cudaSuccess)
                    e = side == 0 ? launch_spmv(P, h->num_sms, kSolveMaxThreads, xin, out, h->stream)
                                  : launch_spmv_t(P, h->num_sms, kSolveMaxThreads, zin, out, h->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) ts.push_back(1e3f * ms);  // the first launch warms up
            }
            if (e != cudaSuccess) break;
            std::sort(ts.begin(), ts.end());
            const float us = ts[ts.size() / 2];
            if (us_out) us_out[side * RGDBEK_SPMV_LANE_CANDIDATES + c] = us;
            if (c == 0 || us < best_us) {
                best_us = us;
                best[side] = kCand[c];
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    h->lpr = best[0];
    h->lpc = best[1];
    if (lanes_row) *lanes_row = best[0];
    if (lanes_col) *lanes_col = best[1];
    return RGDBEK_OK;
}

int rgdbek_set_pass_lanes(rgdbek_t h, int lanes_row, int lanes_col) {
    auto ok = [](int L) { return L >= 1 && L <= 32 && (L & (L - 1)) == 0; };
    if (!h || !ok(lanes_row) || !ok(lanes_col)) return RGDBEK_ERR_INVALID_ARG;
    h->lpr = lanes_row;
    h->lpc = lanes_col;
    return RGDBEK_OK;
}

int rgdbek_spmv(rgdbek_t h, const double *x, double *y) {
    if (!h || !x || !y) return RGDBEK_ERR_INVALID_ARG;
    return cuda_status(launch_spmv(make_params(h), h->num_sms, kSolveMaxThreads, x, y, h->stream));
}

int rgdbek_spmv_f32(rgdbek_t h, int transposed, const float *x, float *y) {
    if (!h || !x || !y || (transposed != 0 && transposed != 1)) return RGDBEK_ERR_INVALID_ARG;
    const int st = ensure_f32_matrix(h);
    if (st != RGDBEK_OK) return st;
    const Params P = make_params(h);
    const ParamsF F = make_params_f(h, P, false);
    return cuda_status(launch_spmv_f32(F, h->num_sms, kSolveMaxThreads, x, y, transposed != 0,
                                       h->stream));
}

int rgdbek_spmv_t(rgdbek_t h, const double *z, double *g) {
    if (!h || !z || !g) return RGDBEK_ERR_INVALID_ARG;
    return cuda_status(launch_spmv_t(make_params(h), h->num_sms, kSolveMaxThreads, z, g, h->stream));
}

int rgdbek_weights(rgdbek_t h, int which, const double *v, double *eps, double *eps_max) {
    if (!h || !v || !eps || !eps_max || (which != 0 && which != 1)) return RGDBEK_ERR_INVALID_ARG;
    const long long len = which == 0 ? h->n : h->m;
    cudaError_t e = launch_reset_ctrl(h->ctrl, h->stream);
    if (e == cudaSuccess)
        e = launch_weights(v, which == 0 ? h->cn2 : h->rn2, len, eps, h->ctrl, h->num_sms, kSolveMaxThreads,
                           h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int rs = read_ctrl(h);
    if (rs != RGDBEK_OK) return rs;
    *eps_max = h->ctrl_host->emax_out;
    return h->ctrl_host->bad_out ? RGDBEK_ERR_NONFINITE : RGDBEK_OK;
}

int rgdbek_sample(rgdbek_t h, const double *eps, int64_t len, int64_t s, uint64_t seed,
                  uint64_t sysid, int64_t k, int phase, int32_t *idx, int64_t *count) {
    const long long mx = h ? (h->m > h->n ? h->m : h->n) : 0;
    if (!h || !eps || !idx || !count || len < 1 || len > mx || s < 0 ||
        s > (long long)RGDBEK_MAX_DRAWS_PER_ENTRY * len || k < 0 || (phase != 0 && phase != 1))
        return RGDBEK_ERR_INVALID_ARG;
    const bool greedy = h->opt.selection == RGDBEK_SELECT_GREEDY;
    const double eta = phase == 0 ? h->opt.eta_col : h->opt.eta_row;
    cudaError_t e = launch_reset_ctrl(h->ctrl, h->stream);
    if (e == cudaSuccess)
        e = launch_sample(make_params(h), h->sample_grid, h->block, eps, len, s, seed, sysid,
                          (unsigned long long)k, (unsigned long long)phase, idx, greedy, eta,
                          h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int rs = read_ctrl(h);
    if (rs != RGDBEK_OK) return rs;
    if (h->ctrl_host->status != RGDBEK_OK) return RGDBEK_ERR_TIMEOUT;
    if (h->ctrl_host->sample_count < 0) return RGDBEK_ERR_NONFINITE;
    *count = h->ctrl_host->sample_count;
    return RGDBEK_OK;
}

int rgdbek_get_norms(rgdbek_t h, double *row_norms2, double *col_norms2) {
    if (!h) return RGDBEK_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (row_norms2)
        e = cudaMemcpyAsync(row_norms2, h->rn2, (size_t)h->m * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && col_norms2)
        e = cudaMemcpyAsync(col_norms2, h->cn2, (size_t)h->n * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

int rgdbek_get_csc(rgdbek_t h, int64_t *col_ptr, int32_t *row_idx, double *vals) {
    if (!h || !col_ptr || (h->nnz > 0 && (!row_idx || !vals))) return RGDBEK_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(col_ptr, h->cp, (size_t)(h->n + 1) * sizeof(long long),
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && h->nnz > 0)
        e = cudaMemcpyAsync(row_idx, h->ri, (size_t)h->nnz * sizeof(int), cudaMemcpyDeviceToDevice,
                            h->stream);
    if (e == cudaSuccess && h->nnz > 0)
        e = cudaMemcpyAsync(vals, h->cv, (size_t)h->nnz * sizeof(double), cudaMemcpyDeviceToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

const char *rgdbek_status_string(int status) {
    switch (status) {
    case RGDBEK_OK: return "ok";
    case RGDBEK_NOT_CONVERGED: return "not converged (iteration cap reached)";
    case RGDBEK_ERR_INVALID_ARG: return "invalid argument";
    case RGDBEK_ERR_NONFINITE: return "non-finite value in the input or a residual weight";
    case RGDBEK_ERR_CUDA: return "CUDA runtime error";
    case RGDBEK_ERR_OOM: return "out of device memory";
    case RGDBEK_ERR_TIMEOUT: return "time budget or device wait limit exceeded";
    case RGDBEK_ERR_BAD_CSR: return "malformed CSR matrix";
    default: return "unknown status";
    }
}

}  // extern "C"
