// Device code of the persistent solve: the inner LSQR, the phases of one
// outer iteration (solve_body) and the single and batched solve kernels,
// templated on the inner precision (F32) and the launch bound (NT threads).
// Two translation units include it, each instantiating one launch bound, so
// that the two shapes compile in parallel.
//
// One outer iteration k of Algorithm 1, phase by phase (| = grid barrier):
//   col:  x_k = x_{k-1} + dx; g = A^T z_k; h = A^T (b - A x_k); eps^z  |
//         stopping test on x_k (every CTA decides identically)
//   column block (skipped if eps^z == 0):
//         quantise eps^z | Philox draws | count marks | compact -> U_k |
//         count nnz of A_U | extract A_U as CSR, start LSQR on A_U D (unit
//         columns; v~ = D g_U/||z||) | LSQR steps (2 phases each) ...
//   z:    z_{k+1} = z_k - A_U y; r = (b - A x_k) - z_{k+1}; eps^x             |
//   row block (skipped if eps^x == 0):
//         quantise | draws | count | compact -> J_k | count nnz(A^J) |
//         extract A^J as CSC, u~ = D r_J | v~ = (D A^J)^T u~ / ||D r_J|| |
//         LSQR steps on D A^J (unit rows; again unscaled if the block is
//         found inconsistent); the solution accumulates in dx ...
//   t:    t_{k+1} = b - A (x_k + dx)                                          |
// The stopping test of x_{k+1} is taken in the next col phase, which also
// applies x_{k+1} = x_k + dx, so the returned x is exactly the tested one.
#pragma once

#include <cmath>

#include "rgdbek_internal.h"

namespace rgd {

// Scalars of the LSQR recurrences.  GB300's FP64 rate is low, so they are
// computed by thread 0 of each CTA only (every CTA gets bit-identical values
// from the identically reduced partials) and broadcast through shared memory.
struct LsqrState {
    double alpha, beta, rhobar, phibar, beta1, fro;
    double irho, cs, sn;         // plane rotation of the current step (1/rho, c, s)
    double inv_a, ab, wcoef;     // coefficients of the next rows phase
    double inv_b, ba, phi_rho;   // coefficients of the next cols phase
    double itol;                 // inner tolerance of this solve
    int mv, done;
    int fit;                     // at the end: 1 = the residual met the tolerance (a
                                 // consistent block), 2 = step cap, 0 = otherwise
};

// Scalars of the outer iteration, also computed by thread 0 only.
struct OuterState {
    double bb, tt, zz, atb2, rel, nrm, emax_c, emax_r;
    double beta1, alpha1, fro2, inv_beta1;
    double beta1s, fro2s;        // row step: the same for the row-scaled block
    double itol;                 // inner tolerance of this iteration
    int verdict;                 // status to finish with, or kStatusRunning to go on
};

// per-solve counters, kept by thread 0 (only CTA 0's copy is reported)
struct Acc {
    long long inner_u, inner_j, sum_nu, sum_nj, sum_nnzu, sum_nnzj;
    long long lsqr_nnzu, lsqr_nnzj, lsqr_nu, lsqr_nj;
};

struct SolveSmem {
    BlockScratch bs;
    Acc acc;
    long long tab[kMaxGrid];
    double red_d[D_NSLOTS];                          // reduced partials of the last barrier
    long long red_i[I_NSLOTS];
    LsqrState lsqr;                                  // LSQR scalars (written by thread 0)
    OuterState o;                                    // outer-loop scalars (thread 0)
    unsigned long long epoch;                        // grid barriers passed (thread 0 copy)
    int leader;                                      // this CTA has rank 0 in its team
    unsigned long long tlast;                        // phase timers (CTA 0, thread 0)
    unsigned long long tphase[RGDBEK_NUM_PHASES];
};

enum PhaseId { PH_SETUP = 0, PH_COL, PH_COL_SEL, PH_COL_EXT, PH_COL_LSQR, PH_ZUPD, PH_ROW_SEL,
               PH_ROW_EXT, PH_ROW_LSQR, PH_RESID };

// charges the time since the previous mark to phase `id` (team rank 0 only)
__device__ __forceinline__ void mark(SolveSmem &S, int id) {
    if (S.leader && threadIdx.x == 0) {
        const unsigned long long now = globaltimer_ns();
        S.tphase[id] += now - S.tlast;
        S.tlast = now;
    }
}

#define DS(x) (1u << (x))

// Grid barrier, then the requested partial slots reduced into S.red_*.
// Returns false if the barrier was abandoned.
__device__ __forceinline__ bool sync_collect(const Params &P, SolveSmem &S, unsigned dmask,
                                             unsigned dmax, unsigned imask) {
    if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return false;
    if (dmask | imask)
        collect_partials(P.pd, P.pi, tsize(P), dmask, dmax, imask, S.red_d, S.red_i);
    return true;
}

__device__ __forceinline__ void finish(const Params &P, int status, long long k, double rel,
                                       double nrm, const SolveSmem &S) {
    if (trank(P) == 0 && threadIdx.x == 0) {
        const Acc &a = S.acc;
        Ctrl *C = P.ctrl;
        for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) C->phase_ns[i] = S.tphase[i];
        C->iters = k;
        C->inner_u = a.inner_u;
        C->inner_j = a.inner_j;
        C->sum_nu = a.sum_nu;
        C->sum_nj = a.sum_nj;
        C->sum_nnzu = a.sum_nnzu;
        C->sum_nnzj = a.sum_nnzj;
        C->lsqr_nnzu = a.lsqr_nnzu;
        C->lsqr_nnzj = a.lsqr_nnzj;
        C->lsqr_nu = a.lsqr_nu;
        C->lsqr_nj = a.lsqr_nj;
        C->rel_res = rel;
        C->normal_res = nrm;
        C->rse = rel * rel;
        __threadfence();
        atomicCAS(&C->status, kStatusRunning, status);
    }
}

// ---------------------------------------------------------------------------
// LSQR (Paige & Saunders 1982) on a block B, the inner solver of Remark 3.1.
//
// B is given by its two sides in contiguous line order: R, the lines of B
// (u-space), and C, the lines of B^T (v-space).  CTA b owns the contiguous
// chunk b of R's lines and of C's lines for the whole inner solve; at the
// start it copies its chunks (line pointers, indices, values) and its slices
// of u~ (previous value), v~, w and y into shared memory, so that each phase
// reads the block from shared memory and only gathers the other side's
// vector from L2.  A chunk that does not fit stays in global memory.
//
// Vectors are kept unnormalised, u~ = beta u and v~ = alpha v, and each step
// is two grid phases:
//   rows:  w = v~/alpha - (theta/rho_prev) w   (own columns; the w update of
//          the previous step), u~_new = B v~ / alpha - (alpha/beta) u~
//   cols:  v~_new = B^T u~_new / beta_new - (beta_new/alpha) v~,
//          y += (phi/rho) w
// ---------------------------------------------------------------------------
// One side of a block: n lines, line l spanning idx/val[b, e) with
//   b = ptr[src], e = cnt ? b + cnt[src] : ptr[src + 1],  src = list ? list[l] : l
// (an extracted block keeps its lines in place with counts; a block made of
// selected rows/columns of A reads them through the selection list).
struct SideC {
    const long long *ptr;
    const int *cnt;
    const int *list;
    const int *idx;        // indices into the other space
    const double *val;
    long long n;           // lines
    int L;                 // lanes per line
};

__device__ __forceinline__ void line_span(const SideC &S, long long l, long long &b, long long &e) {
    const long long src = S.list ? S.list[l] : l;
    b = __ldg(S.ptr + src);
    e = S.cnt ? b + S.cnt[src] : __ldg(S.ptr + src + 1);
}

// This CTA's chunk [lo, lo + nl) of a side.  Cached: local line li spans
// idx/val[ptr[li], ptr[li+1]) in shared memory.  Otherwise the lines are read
// from the global arrays through line_span.
struct CtaSide {
    const long long *ptr;
    const int *idx;
    const double *val;   // cached values (FP64 inner products)
    const float *valf;   // cached values (FP32 inner products)
    int nl;
    long long lo;
    int L;               // lanes per line, FP64 products
    int Lf;              // lanes per line, FP32 products
    bool cached;
    SideC g;
};

// bump allocation in dynamic shared memory (16-byte granules)
struct SmemArena {
    unsigned char *base;
    long long left, used;
    template <typename T>
    __device__ __forceinline__ T *take(long long count) {
        const long long bytes = ((count * (long long)sizeof(T)) + 15) & ~15ll;
        if (bytes > left) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        left -= bytes;
        return p;
    }
};

// Copies this CTA's chunk of a side into shared memory (compacting the
// lines), if it fits; with fp32 the values are stored as float.  All threads
// of the CTA call it.
template <bool fp32>
__device__ __forceinline__ CtaSide cache_side(const SideC &S, SmemArena &A, BlockScratch &bs,
                                              int rank, int nct) {
    const Chunk C(S.n, rank, nct);
    CtaSide out;
    out.nl = (int)(C.hi - C.lo);
    out.lo = C.lo;
    out.L = S.L;
    out.Lf = S.L;
    out.g = S;
    out.cached = false;
    out.ptr = nullptr;
    out.idx = nullptr;
    out.val = nullptr;
    out.valf = nullptr;
    const SmemArena save = A;
    long long *ps = A.take<long long>(out.nl + 1);
    long long *gs = ps ? A.take<long long>(out.nl) : nullptr;  // global start of each line
    if (!gs) {
        A = save;
        return out;
    }
    // line lengths -> local offsets (exclusive scan in line order)
    long long run = 0;
    for (int base = 0; base < out.nl; base += blockDim.x) {
        const int li = base + threadIdx.x;
        long long len = 0;
        if (li < out.nl) {
            long long b, e;
            line_span(S, C.lo + li, b, e);
            len = e - b;
            gs[li] = b;
        }
        long long tot;
        const long long ex = block_excl_scan<long long>(len, bs, &tot);
        if (li < out.nl) ps[li] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) ps[out.nl] = run;
    // FP32 products are cheap to reduce across lanes, so they spread each line
    // over enough lanes for about four entries per lane (one round of
    // gathers), as far as warps 1.. cover all lines in one pass
    int Lf = 1;
    {
        const long long per_line = out.nl > 0 ? (run + out.nl - 1) / out.nl : 0;
        const long long lanes = (long long)((blockDim.x >> 5) - 1) * 32;
        while (Lf < 32 && 4ll * Lf < per_line) Lf *= 2;
        while (Lf > 1 && (long long)out.nl * Lf > lanes) Lf >>= 1;
    }
    int *is = A.take<int>(run);
    double *vs = (is && !fp32) ? A.take<double>(run) : nullptr;
    float *vf = (is && fp32) ? A.take<float>(run) : nullptr;
    if (!vs && !vf) {
        A = save;
        __syncthreads();
        return out;
    }
    __syncthreads();
    // a group of L lanes per line (one thread per line for short lines)
    {
        const Grp G(S.L);
        const int per = (blockDim.x >> 5) * G.rpw;
        for (int base = 0; base < out.nl; base += per) {
            const int li = base + (threadIdx.x >> 5) * G.rpw + G.sub;
            if (li < out.nl) {
                const long long b = gs[li], o = ps[li], len = ps[li + 1] - o;
                for (long long k = G.sl; k < len; k += G.L) {
                    is[o + k] = S.idx[b + k];
                    if (fp32) vf[o + k] = (float)S.val[b + k];
                    else vs[o + k] = S.val[b + k];
                }
            }
        }
    }
    __syncthreads();
    out.cached = true;
    out.Lf = Lf;
    out.ptr = ps;
    out.idx = is;
    out.val = vs;
    out.valf = vf;
    return out;
}

// This lane's share of an FP32 dot product over entries e, e + L, ... < e1,
// Kahan-compensated (Kahan 1965): c carries the rounding error of the running
// sum into the next term; the lane returns s - c.  Four entries per trip,
// their gathers issued together.
__device__ __forceinline__ float lane_dot_kahan(int e, int e1, int L, const int *idx,
                                                const float *val, const float *vec) {
    float s = 0.f, c = 0.f;
    for (; e < e1; e += 4 * L) {
        int ix[4];
        float a[4], x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok = e + q * L < e1;
            ix[q] = ok ? idx[e + q * L] : -1;
            a[q] = ok ? val[e + q * L] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = ix[q] >= 0 ? vec[ix[q]] : 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (ix[q] >= 0) {
                const float y = fmaf(a[q], x[q], -c);
                const float t = s + y;
                c = (t - s) - y;
                s = t;
            }
        }
    }
    return s - c;
}

// Dot products of this CTA's lines with a gathered vector, into dots[li].
// Warp 0 is left out: it reduces the partials of the previous barrier and
// computes the LSQR scalars meanwhile.
// FP32 form of cta_dots for a cached side.
__device__ __forceinline__ void cta_dots_f32(const long long *ptr, const int *idx, const float *valf,
                                          int nl, int Lf, const float *vec32, double *dots) {
    const int warp = threadIdx.x >> 5;
    const Grp G(Lf);
    const int per = ((blockDim.x >> 5) - 1) * G.rpw;
    for (int base = 0; base < nl; base += per) {
        const int li = base + (warp - 1) * G.rpw + G.sub;
        float s = 0.f;
        if (li < nl) s = lane_dot_kahan((int)ptr[li] + G.sl, (int)ptr[li + 1], G.L, idx, valf, vec32);
        s = group_sum(s, G.L);
        if (li < nl && G.sl == 0) dots[li] = (double)s;
    }
}

template <bool F32>
__device__ __forceinline__ void cta_dots(const CtaSide &C, const double *vec, const float *vec32,
                                         double *dots) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) return;
    if (F32 && C.cached) {
        cta_dots_f32(C.ptr, C.idx, C.valf, C.nl, C.Lf, vec32, dots);
        return;
    }
    const Grp G(C.L);
    const int per = ((blockDim.x >> 5) - 1) * G.rpw;
    const auto gat = [&](int j) { return vec[j]; };
    for (int base = 0; base < C.nl; base += per) {
        const int li = base + (warp - 1) * G.rpw + G.sub;
        double s = 0.0;
        if (li < C.nl) {
            if (C.cached) {
                s = lane_dot<false>(C.ptr[li] + G.sl, C.ptr[li + 1], G.L, C.idx, C.val, gat);
            } else {
                long long b, e;
                line_span(C.g, C.lo + li, b, e);
                s = lane_dot<false>(b + G.sl, e, G.L, C.g.idx, C.g.val, gat);
            }
        }
        s = group_sum(s, G.L);
        if (li < C.nl && G.sl == 0) dots[li] = s;
    }
}

// Warp 0: sum of the per-CTA partials of one slot (fixed order), for lane 0.
__device__ __forceinline__ double warp0_collect(const double *pd, int slot, int nb) {
    const double *p = pd + slot * nb;
    double s = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < nb; i += 32) s += __ldcg(p + i);
    return warp_sum(s);
}

// LSQR from y = 0 on the block (R, C) with right-hand side c0 (u-space,
// global, element i at c0[i * c0s]; without v_given c0s must be 1), beta1 = ||c0||.  With v_given, v~_1 = B^T c0 / beta1 is already in
// P.vv and alpha1 is passed; otherwise it is computed first (one more
// phase).  fro2 = ||B||_F^2.  y_g (v-space) receives the solution; with xt
// given (the row step, v-space = x-space) also xt = x + y, so the residual
// pass gathers x_{k+1} without an addition per nonzero.  With csc (the column
// step; requires v_given) the solve runs on B D, D = diag(csc) over the
// v-space (unit columns): the rows phase gathers D v~, the cols phase scales
// B^T u~ by D, and y_g receives y = D y^, so B y_g is the projection of c0
// whatever the scaling.  Returns the number of steps (0 if alpha1 == 0), or
// -1 if a grid barrier was abandoned.
//
// Per phase: grid barrier | warp 0 reduces the partials and updates the
// scalars while warps 1.. compute the dot products of the CTA's lines |
// __syncthreads | all threads combine element-wise and form the partial.
template <bool f32>
__device__ __forceinline__ int run_lsqr(const Params &P, const SideC &Rs, const SideC &Cs,
                                        const double *c0, int c0s, const float *c0_32, double *y_g,
                                        double *xt, const double *csc, const double *rsc,
                                        bool v_given,
                                        double alpha1, double beta1, double fro2,
                                        unsigned char *dsmem, long long dsmem_bytes,
                                        SolveSmem &S) {
    LsqrState &L = S.lsqr;
    SmemArena A{dsmem, dsmem_bytes, 0};
    const Chunk RC(Rs.n, trank(P), tsize(P)), CC(Cs.n, trank(P), tsize(P));
    const int nrl = (int)(RC.hi - RC.lo), ncl = (int)(CC.hi - CC.lo);
    // per-CTA vector slices and dot buffers
    double *uold = A.take<double>(nrl);
    double *dr = uold ? A.take<double>(nrl) : nullptr;
    double *vown = dr ? A.take<double>(ncl) : nullptr;
    double *wown = vown ? A.take<double>(ncl) : nullptr;
    double *yown = wown ? A.take<double>(ncl) : nullptr;
    double *dc = yown ? A.take<double>(ncl) : nullptr;
    // column scaling D of the v-space (column step), row scaling of the
    // u-space (row step): their slices
    double *sown = (dc && csc) ? A.take<double>(ncl) : nullptr;
    double *rown = (dc && rsc) ? A.take<double>(nrl) : nullptr;
    const bool st_smem = dc != nullptr && (sown != nullptr || csc == nullptr) &&
                         (rown != nullptr || rsc == nullptr);
    if (!st_smem) {
        A = SmemArena{dsmem, dsmem_bytes, 0};
        uold = nullptr;
        dr = P.dots + RC.lo;
        vown = P.vv + CC.lo;
        wown = P.ww + CC.lo;
        yown = (csc ? P.yh : y_g) + CC.lo;  // scaled: y^ apart from y = D y^
        dc = P.dots2 + CC.lo;
        for (int i = threadIdx.x; i < ncl; i += blockDim.x) yown[i] = 0.0;
    } else {
        for (int i = threadIdx.x; i < nrl; i += blockDim.x) {
            uold[i] = c0[(RC.lo + i) * c0s];
            if (rown) rown[i] = rsc[RC.lo + i];
        }
        for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
            vown[i] = v_given ? P.vv[CC.lo + i] : 0.0;
            yown[i] = 0.0;
            if (sown) sown[i] = csc[CC.lo + i];
        }
    }
    const double *dloc = csc ? (sown ? sown : csc + CC.lo) : nullptr;
    const double *rloc = rsc ? (rown ? rown : rsc + RC.lo) : nullptr;
    // the cols phase gathers D u~ when the u-space is scaled
    const double *usrc = rsc ? P.uus : P.uu;
    // the rows phase gathers D v~ when the v-space is scaled
    const double *vsrc = csc ? P.vvs : P.vv;
    const CtaSide R = cache_side<f32>(Rs, A, S.bs, trank(P), tsize(P));
    const CtaSide C = cache_side<f32>(Cs, A, S.bs, trank(P), tsize(P));
    if (threadIdx.x == 0) {
        L.inv_b = 1.0 / beta1;
        L.done = 0;
        L.fit = 0;
        L.itol = S.o.itol;
    }
    __syncthreads();

    if (!v_given) {
        // v~_1 = B^T c0 / beta1 (warp 0 has no scalars to update in this phase)
        cta_dots<f32>(C, rsc ? P.uus : c0, c0_32, dc);
        __syncthreads();
        double acc = 0.0;
        for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
            const double v = dc[li] * L.inv_b;
            vown[li] = v;
            P.vv[CC.lo + li] = v;
            if (f32) P.vv32[CC.lo + li] = (float)v;
            acc = fma(v, v, acc);
        }
        acc = block_sum(acc, S.bs);
        if (threadIdx.x == 0) P.pd[D_VV * tsize(P) + trank(P)] = acc;
        if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return -1;
        if (threadIdx.x < 32) {
            const double vv = warp0_collect(P.pd, D_VV, tsize(P));
            if (threadIdx.x == 0) L.alpha = sqrt(vv);
        }
        __syncthreads();
        alpha1 = L.alpha;
        if (!(alpha1 > 0.0)) return 0;
    }
    if (threadIdx.x == 0) {
        L.alpha = alpha1;
        L.beta = beta1;
        L.rhobar = alpha1;
        L.phibar = beta1;
        L.beta1 = beta1;
        L.fro = sqrt(fro2);
        L.inv_a = 1.0 / alpha1;
        L.ab = alpha1 / beta1;
        L.wcoef = 0.0;
    }
    __syncthreads();
    for (int it = 1;; ++it) {
        const bool first = it == 1;
        // ---- rows phase: u~_new = B v~ / alpha - (alpha/beta) u~, w update
        cta_dots<f32>(R, vsrc, P.vv32, dr);
        if (threadIdx.x < 32 && !first) {
            // scalars from ||v~||^2 of the previous cols phase
            const double vv = warp0_collect(P.pd, D_VV, tsize(P));
            if (threadIdx.x == 0) {
                // alpha_{i+1} = ||v~||; the divisions of the recurrence are
                // multiplications by reciprocals formed with rsqrt, which keeps
                // the dependent FP64 chain of this single thread short
                const double cs = L.cs, sn = L.sn, bn = L.beta;
                const double an = bn > 0.0 ? sqrt(vv) : 0.0;
                const double ian = an > 0.0 ? rsqrt(vv) : 0.0;
                L.rhobar = -cs * an;
                L.wcoef = sn * an * L.irho;   // theta / rho
                const double rnorm = L.phibar;
                const double arnorm = L.phibar * an * fabs(cs);
                const bool resid = rnorm <= L.itol * L.beta1 || bn == 0.0;
                const bool other = arnorm <= L.itol * L.fro * rnorm || an == 0.0;
                const bool cap = it - 1 >= P.inner_max;
                L.done = resid || other || cap;
                L.fit = resid ? 1 : (other ? 0 : (cap ? 2 : 0));
                L.alpha = an;
                L.inv_a = ian;
                L.ab = an * L.inv_b;           // alpha / beta
            }
        }
        __syncthreads();
        if (L.done) return it - 1;
        {
            const double inv_a = L.inv_a, ab = L.ab, wcoef = L.wcoef;
            for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
                const double vn = vown[li] * inv_a;
                wown[li] = first ? vn : vn - wcoef * wown[li];
            }
            double acc = 0.0;
            for (int li = threadIdx.x; li < nrl; li += blockDim.x) {
                const double rl = rloc ? rloc[li] : 1.0;
                const double uo = st_smem ? uold[li]
                                          : (first ? c0[(RC.lo + li) * c0s] : P.uu[RC.lo + li]);
                const double u = (rloc ? dr[li] * rl : dr[li]) * inv_a - ab * uo;
                P.uu[RC.lo + li] = u;
                if (rloc) P.uus[RC.lo + li] = u * rl;
                if (f32) P.uu32[RC.lo + li] = (float)(rloc ? u * rl : u);
                if (st_smem) uold[li] = u;
                acc = fma(u, u, acc);
            }
            acc = block_sum(acc, S.bs);
            if (threadIdx.x == 0) P.pd[D_UU * tsize(P) + trank(P)] = acc;
        }
        if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return -1;

        // ---- cols phase: v~_new = B^T u~ / beta - (beta/alpha) v~, y update
        cta_dots<f32>(C, usrc, P.uu32, dc);
        if (threadIdx.x < 32) {
            const double uu = warp0_collect(P.pd, D_UU, tsize(P));
            if (threadIdx.x == 0) {
                // beta_{i+1} = ||u~||, rho = sqrt(rhobar^2 + beta^2); 1/rho from
                // rsqrt of rho^2 directly, in parallel with sqrt(||u~||^2)
                const double bn = sqrt(uu);
                const double irho = rsqrt(fma(L.rhobar, L.rhobar, uu));
                const double cs = L.rhobar * irho, sn = bn * irho;
                const double phi = cs * L.phibar;
                L.phibar = sn * L.phibar;
                L.mv = bn > 0.0;
                L.inv_b = bn > 0.0 ? rsqrt(uu) : 0.0;
                L.ba = bn * L.inv_a;           // beta / alpha
                L.phi_rho = phi * irho;
                L.beta = bn;
                L.irho = irho;
                L.cs = cs;
                L.sn = sn;
            }
        }
        __syncthreads();
        {
            const double inv_b = L.inv_b, ba = L.ba, phi_rho = L.phi_rho;
            const bool mv = L.mv != 0;
            double acc = 0.0;
            for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
                const double dl = dloc ? dloc[li] : 1.0;
                if (mv) {
                    const double v = (dloc ? dc[li] * dl : dc[li]) * inv_b - ba * vown[li];
                    vown[li] = v;
                    P.vv[CC.lo + li] = v;
                    if (dloc) P.vvs[CC.lo + li] = v * dl;
                    if (f32) P.vv32[CC.lo + li] = (float)(dloc ? v * dl : v);
                    acc = fma(v, v, acc);
                }
                const double y = fma(phi_rho, wown[li], yown[li]);
                yown[li] = y;
                y_g[CC.lo + li] = dloc ? y * dl : y;   // y = D y^ when scaled
                if (xt) xt[CC.lo + li] = P.x[CC.lo + li] + y;
            }
            acc = block_sum(acc, S.bs);
            if (threadIdx.x == 0) P.pd[D_VV * tsize(P) + trank(P)] = acc;
        }
        if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return -1;
    }
}

// z_{k+1} = z_k - A_U y (A_U as extracted CSR), r = t_k - z_{k+1},
// eps^x_i = r_i^2 / ||A^(i)||^2.  Partials: max eps^x, ||z_{k+1}||^2, bad.
__device__ __forceinline__ void phase_zupdate(const Params &P, bool hasU, int Lsub,
                                              BlockScratch &bs) {
    const Grp G(hasU ? Lsub : 1);
    double emax = 0.0, zz = 0.0;
    long long bad = 0;
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        double s = 0.0;
        if (hasU && i < P.m)
            s = lane_dot<false>(P.rp[i] + G.sl, P.rp[i] + P.srn[i], G.L, P.sci, P.sav,
                                [&](int p) { return P.yy[p]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) {
            const double zi = P.z[2 * i] - s;
            P.z[2 * i] = zi;
            const double ri = P.t[2 * i] - zi;
            P.r[i] = ri;
            const double c = __ldg(P.rn2 + i);
            const double e = c > 0.0 ? __ddiv_rn(__dmul_rn(ri, ri), c) : 0.0;
            P.epsr[i] = e;
            if (!isfinite(e)) bad = 1;
            else emax = max_nonneg(emax, e);
            zz = fma(zi, zi, zz);
        }
    }
    emax = block_max(emax, bs);
    zz = block_sum(zz, bs);
    bad = block_sum(bad, bs);
    if (threadIdx.x == 0) {
        P.pd[D_EMAX_R * tsize(P) + trank(P)] = emax;
        P.pd[D_ZZ * tsize(P) + trank(P)] = zz;
        P.pi[I_BAD_R * tsize(P) + trank(P)] = bad;
    }
}

#define RGD_SYNC(dm, dx, im)                                 \
    do {                                                     \
        if (!sync_collect(P, S, (dm), (dx), (im))) return;   \
    } while (0)

// One whole solve of Algorithm 1 by the CTAs of a team (after enter_team).
// F32: inner LSQR products in FP32 (RGDBEK_PRECISION_FP32_INNER); a separate
// instantiation, so the FP64 code's registers are unaffected.
template <bool F32>
__device__ __forceinline__ void solve_body(const Params &P, SolveSmem &S, unsigned char *dsmem) {
    BlockScratch &bs = S.bs;
    OuterState &O = S.o;
    const int nct = tsize(P);
    const bool greedy = P.selection == RGDBEK_SELECT_GREEDY;
    const unsigned long long t_start = globaltimer_ns();
    if (threadIdx.x == 0) {
        S.epoch = 0;
        S.leader = trank(P) == 0;
        S.acc = Acc{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        S.tlast = t_start;
        for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) S.tphase[i] = 0;
    }

    // ---- x_0 = 0, z_0 = b, t_0 = b - A x_0 = b, dx = 0
    {
        double bb = 0.0;
        long long bad = 0;
        for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
            const double bi = __ldg(P.b + i);
            P.z[2 * i] = bi;
            P.t[2 * i] = bi;
            bb = fma(bi, bi, bb);
            if (!isfinite(bi)) bad = 1;
        }
        // x_0 = 0, or the caller's x (warm start)
        for (long long j = tthread(P); j < P.n; j += tthreads(P)) {
            const double x0 = P.warm ? P.x[j] : 0.0;
            if (!isfinite(x0)) bad = 1;
            P.x[j] = x0;
            P.xt[j] = x0;
        }
        bb = block_sum(bb, bs);
        bad = block_sum(bad, bs);
        if (threadIdx.x == 0) {
            P.pd[D_BB * nct + trank(P)] = bb;
            P.pi[I_BAD_R * nct + trank(P)] = bad;
        }
    }
    RGD_SYNC(DS(D_BB), 0, DS(I_BAD_R));
    mark(S, PH_SETUP);
    if (P.warm) {
        // t_0 = b - A x_0 for the first stopping test
        phase_residual(P, bs);
        RGD_SYNC(DS(D_TT), 0, 0);
    }
    if (threadIdx.x == 0) {
        O.bb = S.red_d[D_BB];
        O.tt = P.warm ? S.red_d[D_TT] : O.bb;  // t_0 = b - A x_0 (= b from x_0 = 0)
        O.zz = O.bb;
        O.atb2 = 0.0;
        O.verdict = (S.red_i[I_BAD_R] != 0 || !isfinite(O.bb)) ? RGDBEK_ERR_NONFINITE
                                                                : kStatusRunning;
    }
    __syncthreads();
    if (O.verdict != kStatusRunning) {
        finish(P, O.verdict, 0, NAN, NAN, S);
        return;
    }
    long long tr_off = 0;
    bool tr_full = P.tr_lists == nullptr;

    for (long long k = 0;; ++k) {
        // ---- column pass and stopping test on x_k
        if (trank(P) == 0 && threadIdx.x == 0 && P.time_budget_ns > 0.0 &&
            (double)(globaltimer_ns() - t_start) > P.time_budget_ns)
            P.ctrl->stop_req = 1;
        phase_col(P, bs);
        RGD_SYNC(DS(D_EMAX_C) | DS(D_HH) | DS(D_GG), DS(D_EMAX_C), DS(I_BAD_C));
        mark(S, PH_COL);
        if (P.tr_g && k < P.tr_vec_cap)  // trace: g = A^T z_k, complete after the barrier
            for (long long j = tthread(P); j < P.n; j += tthreads(P)) P.tr_g[k * P.n + j] = P.g[j];
        if (threadIdx.x == 0) {
            const double hh = S.red_d[D_HH];
            O.emax_c = S.red_d[D_EMAX_C];
            if (k == 0) O.atb2 = S.red_d[D_GG];  // g = A^T z_0 = A^T b
            O.rel = O.bb > 0.0 ? sqrt(O.tt / O.bb) : 0.0;
            O.nrm = O.atb2 > 0.0 ? sqrt(hh / O.atb2) : 0.0;
            // inner tolerance of this iteration: fixed, or tied to how far x_k
            // is from the stopping rule (looser block solves while far away)
            O.itol = P.inner_tol;
            if (P.inner_adapt > 0.0) {
                const double rk = P.stop_rule == RGDBEK_STOP_REL_RES
                                      ? O.rel
                                      : (P.stop_rule == RGDBEK_STOP_RSE ? O.rel * O.rel : O.nrm);
                const double a = fmin(0.1, P.inner_adapt * rk);
                if (a > O.itol) O.itol = a;
            }
            int v = kStatusRunning;
            if (S.red_i[I_BAD_C] != 0 || !isfinite(hh) || !isfinite(O.tt)) v = RGDBEK_ERR_NONFINITE;
            else if (stop_rule_holds(P.stop_rule, P.tol, O.rel, O.nrm)) v = RGDBEK_OK;
            else if (k >= P.max_iter) v = RGDBEK_NOT_CONVERGED;
            else if (ld_volatile_i32(&P.ctrl->stop_req)) v = RGDBEK_ERR_TIMEOUT;
            O.verdict = v;
        }
        __syncthreads();
        if (O.verdict != kStatusRunning) {
            finish(P, O.verdict, k, O.rel, O.nrm, S);
            return;
        }

        // ---- column block U_k and z_{k+1} = z_k - A_U A_U^+ z_k
        long long nU = 0, nnzU = 0;
        int stepsU = 0, Lsub_u = 1;
        bool rec_u = !tr_full;
        if (O.emax_c > 0.0) {
            phase_quantize(P, P.epsc, P.n, O.emax_c, greedy, P.eta_col, bs);
            RGD_SYNC(0, 0, 0);
            if (!greedy) {
                phase_draw(P, P.n, P.s_col, P.seed, P.sysid, (unsigned long long)k, 0ull, S.tab, bs);
                RGD_SYNC(0, 0, 0);
            }
            phase_compact_count(P, P.n, P.cn2, P.g, P.epsc, bs);
            RGD_SYNC(DS(D_FRO_S) | DS(D_EXTRA_S), 0, 0);
            if (threadIdx.x == 0) {
                // LSQR start on B = A_U D (columns scaled to unit norm, D =
                // diag(1/||A_j||)) with c = z_k: beta1 = ||z_k||, alpha1 =
                // ||B^T z_k|| / beta1 = sqrt(sum of the selected eps^z) / beta1,
                // ||B||_F^2 = |U|
                O.fro2 = S.red_d[D_FRO_S];
                O.beta1 = sqrt(O.zz);
                O.inv_beta1 = O.beta1 > 0.0 ? 1.0 / O.beta1 : 0.0;
                O.alpha1 = sqrt(S.red_d[D_EXTRA_S]) * O.inv_beta1;
            }
            nU = phase_compact_write(P, P.n, P.colpos, P.ulist, S.tab, bs);
            RGD_SYNC(0, 0, 0);
            mark(S, PH_COL_SEL);
            rec_u = !tr_full && tr_off + nU <= P.tr_list_cap;
            const double inv_beta1 = O.inv_beta1;
            for (long long p = tthread(P); p < nU; p += tthreads(P)) {
                const int j = P.ulist[p];
                const double d = rsqrt(P.cn2[j]);       // selected: ||A_j|| > 0
                const double v1 = P.g[j] * d * inv_beta1;  // v~_1 = B^T z_k / beta1
                P.dsc[p] = d;
                P.vv[p] = v1;
                P.vvs[p] = v1 * d;
                if (F32) P.vv32[p] = (float)(v1 * d);
                P.yy[p] = 0.0;
                if (rec_u) P.tr_lists[tr_off + p] = j;
            }
            // A_U: the entries of every row of A that lie in U's columns
            // about ten entries per lane, as in the FP64 passes (measured: fewer
            // lanes per line keep more lines, and so more loads, in flight)
            const Lines Arows{P.rp, P.ci, P.av, P.m, P.tpr};
            phase_extract(P, Arows, P.colpos, P.srn, P.sci, P.sav, bs);
            RGD_SYNC(0, 0, DS(I_NNZ));
            mark(S, PH_COL_EXT);
            nnzU = S.red_i[I_NNZ];
            Lsub_u = pick_lanes_fp64(nnzU, P.m);
            if (O.beta1 > 0.0 && O.alpha1 > 0.0) {
                const SideC rows{P.rp, P.srn, nullptr, P.sci, P.sav, P.m, Lsub_u};
                const SideC cols{P.cp, nullptr, P.ulist, P.ri, P.cv, nU, P.tpc};
                stepsU = run_lsqr<F32>(P, rows, cols, P.z, 2, nullptr, P.yy, nullptr, P.dsc, nullptr, true, O.alpha1, O.beta1,
                                  O.fro2, dsmem, P.dsmem_bytes, S);
                if (stepsU < 0) return;
                mark(S, PH_COL_LSQR);
            }
        }

        // ---- z_{k+1}, row residual r = b - z_{k+1} - A x_k, row weights
        phase_zupdate(P, nU > 0, Lsub_u, bs);
        RGD_SYNC(DS(D_EMAX_R) | DS(D_ZZ), DS(D_EMAX_R), DS(I_BAD_R));
        mark(S, PH_ZUPD);
        if (P.tr_r && k < P.tr_vec_cap)  // trace: the row residual r = b - z_{k+1} - A x_k
            for (long long i = tthread(P); i < P.m; i += tthreads(P)) P.tr_r[k * P.m + i] = P.r[i];
        if (threadIdx.x == 0) {
            O.emax_r = S.red_d[D_EMAX_R];
            O.zz = S.red_d[D_ZZ];
            O.verdict = S.red_i[I_BAD_R] != 0 ? RGDBEK_ERR_NONFINITE : kStatusRunning;
        }
        __syncthreads();
        if (O.verdict != kStatusRunning) {
            finish(P, O.verdict, k, O.rel, O.nrm, S);
            return;
        }

        // ---- row block J_k and dx = (A^J)^+ r_J
        long long nJ = 0, nnzJ = 0;
        int stepsJ = 0;
        bool rec_j = false;
        if (O.emax_r > 0.0) {
            phase_quantize(P, P.epsr, P.m, O.emax_r, greedy, P.eta_row, bs);
            RGD_SYNC(0, 0, 0);
            if (!greedy) {
                phase_draw(P, P.m, P.s_row, P.seed, P.sysid, (unsigned long long)k, 1ull, S.tab, bs);
                RGD_SYNC(0, 0, 0);
            }
            phase_compact_count(P, P.m, P.rn2, P.r, P.epsr, bs);
            RGD_SYNC(DS(D_FRO) | DS(D_EXTRA) | DS(D_FRO_S) | DS(D_EXTRA_S), 0, 0);
            if (threadIdx.x == 0) {
                // LSQR start on A^J with c = r_J: beta1 = ||r_J||; on D A^J
                // (unit rows) with c = D r_J: beta1 = sqrt(sum of the weights)
                O.fro2 = S.red_d[D_FRO];
                O.beta1 = sqrt(S.red_d[D_EXTRA]);
                O.inv_beta1 = O.beta1 > 0.0 ? 1.0 / O.beta1 : 0.0;
                O.fro2s = S.red_d[D_FRO_S];
                O.beta1s = sqrt(S.red_d[D_EXTRA_S]);
            }
            nJ = phase_compact_write(P, P.m, P.rowpos, P.jlist, S.tab, bs);
            RGD_SYNC(0, 0, 0);
            mark(S, PH_ROW_SEL);
            rec_j = rec_u && tr_off + nU + nJ <= P.tr_list_cap;
            // |J| <= n: first on D A^J (rows scaled to unit norm, D =
            // diag(1/||A^(i)||)) with c = D r_J, which has the same minimum-norm
            // solution whenever the block system is consistent
            const bool rscale = nJ <= P.n;
            for (long long p = tthread(P); p < nJ; p += tthreads(P)) {
                const int i = P.jlist[p];
                const double ri = P.r[i];
                if (rscale) {
                    const double d = rsqrt(P.rn2[i]);  // selected: ||A^(i)|| > 0
                    const double u1 = ri * d;          // u~_1 = D r_J
                    P.dsr[p] = d;
                    P.uu[p] = u1;
                    P.uus[p] = u1 * d;
                    if (F32) P.uu32[p] = (float)(u1 * d);
                } else {
                    P.uu[p] = ri;  // u~_1 = r_J
                    if (F32) P.uu32[p] = (float)ri;
                }
                if (rec_j) P.tr_lists[tr_off + nU + p] = i;
            }
            // A^J: the entries of every column of A that lie in J's rows
            const Lines Acols{P.cp, P.ri, P.cv, P.n, P.tpc};
            phase_extract(P, Acols, P.rowpos, P.scn, P.sri, P.scv, bs);
            RGD_SYNC(0, 0, DS(I_NNZ));
            mark(S, PH_ROW_EXT);
            nnzJ = S.red_i[I_NNZ];
            if (O.beta1 > 0.0) {
                const SideC rows{P.rp, nullptr, P.jlist, P.ci, P.av, nJ, P.tpr};
                const SideC cols{P.cp, P.scn, nullptr, P.sri, P.scv, P.n,
                                 pick_lanes_fp64(nnzJ, P.n)};
                int fit = 0;
                if (rscale) {
                    stepsJ = run_lsqr<F32>(P, rows, cols, P.uu, 1, P.uu32, P.dx, P.xt, nullptr,
                                           P.dsr, false, 0.0, O.beta1s, O.fro2s, dsmem,
                                           P.dsmem_bytes, S);
                    if (stepsJ < 0) return;
                    fit = S.lsqr.fit;
                }
                if (!rscale || fit == 0) {
                    if (rscale) {
                        // found inconsistent: (A^J)^+ r_J needs the unscaled block;
                        // the scaled attempt's x + y is undone first
                        for (long long p = tthread(P); p < nJ; p += tthreads(P)) {
                            const double ri = P.r[P.jlist[p]];
                            P.uu[p] = ri;
                            if (F32) P.uu32[p] = (float)ri;
                        }
                        for (long long j = tthread(P); j < P.n; j += tthreads(P)) P.xt[j] = P.x[j];
                        RGD_SYNC(0, 0, 0);
                    }
                    const int s2 = run_lsqr<F32>(P, rows, cols, P.uu, 1, P.uu32, P.dx, P.xt,
                                                 nullptr, nullptr, false, 0.0, O.beta1, O.fro2,
                                                 dsmem, P.dsmem_bytes, S);
                    if (s2 < 0) return;
                    stepsJ += s2;
                }
                mark(S, PH_ROW_LSQR);
            }
        }

        if (threadIdx.x == 0) {
            Acc &acc = S.acc;
            acc.inner_u += stepsU;
            acc.inner_j += stepsJ;
            acc.sum_nu += nU;
            acc.sum_nj += nJ;
            acc.sum_nnzu += nnzU;
            acc.sum_nnzj += nnzJ;
            acc.lsqr_nnzu += (long long)stepsU * nnzU;
            acc.lsqr_nnzj += (long long)stepsJ * nnzJ;
            acc.lsqr_nu += (long long)stepsU * nU;
            acc.lsqr_nj += (long long)stepsJ * nJ;
        }
        if (trank(P) == 0 && threadIdx.x == 0 && P.tr_counts && k < P.tr_count_cap) {
            P.tr_counts[4 * k + 0] = nU;
            P.tr_counts[4 * k + 1] = nJ;
            P.tr_counts[4 * k + 2] = stepsU;
            P.tr_counts[4 * k + 3] = stepsJ;
        }
        if (!tr_full) {
            const bool ok = rec_u && (nJ == 0 || rec_j) && tr_off + nU + nJ <= P.tr_list_cap;
            if (ok) tr_off += nU + nJ;
            else tr_full = true;
        }
        if (nU == 0 && nJ == 0) {
            // both blocks empty: x can no longer change
            finish(P, RGDBEK_OK, k, O.rel, O.nrm, S);
            return;
        }

        // ---- t_{k+1} = b - A x_{k+1}
        phase_residual(P, bs);
        RGD_SYNC(DS(D_TT), 0, 0);
        mark(S, PH_RESID);
        if (threadIdx.x == 0) O.tt = S.red_d[D_TT];
    }
}

// A single solve: the whole grid is one team.  NT: launch bound (threads).
template <bool F32, int NT>
__global__ void __launch_bounds__(NT, 1) solve_kernel(const Params P) {
    __shared__ SolveSmem S;
    extern __shared__ __align__(16) unsigned char dsmem[];
    enter_team(P);
    solve_body<F32>(P, S, dsmem);
}

// Many independent systems in one cooperative launch: the grid is cut into
// teams of `team` consecutive CTAs; team t solves the systems
// plan[t * stride], plan[t * stride + 1], ... (ending at -1) one after
// another, each to its own stopping rule (its Params and control block in
// sys[]), with barriers among the team's CTAs only.
template <bool F32, int NT>
__global__ void __launch_bounds__(NT, 1)
    batched_solve_kernel(const Params *sys, const int *plan, int stride, int team) {
    __shared__ SolveSmem S;
    __shared__ Params SP;
    extern __shared__ __align__(16) unsigned char dsmem[];
    const int t = (int)(blockIdx.x / (unsigned)team);
    for (int q = 0; q < stride; ++q) {
        const int i = plan[(long long)t * stride + q];
        if (i < 0) break;
        {
            const int *src = reinterpret_cast<const int *>(sys + i);
            int *dst = reinterpret_cast<int *>(&SP);
            for (int w = threadIdx.x; w < (int)(sizeof(Params) / sizeof(int)); w += blockDim.x)
                dst[w] = src[w];
        }
        __syncthreads();
        enter_team(SP);
        solve_body<F32>(SP, S, dsmem);
        __syncthreads();
    }
}

}  // namespace rgd
