// Device code of the persistent solve: the inner LSQR, the phases of one
// outer iteration (solve_body), the FP64 refinement loop of the FP32 form
// (refine_body) and the single and batched solve kernels, templated on the
// value type V of the iteration (double, or float for the inner solves of
// RGDBEK_PRECISION_FP32_INNER) and the launch bound (NT threads).  Each kernel
// and shape is instantiated in a translation unit of its own
// (rgdbek_solve512/1024.cu, rgdbek_refine512/1024.cu, rgdbek_batched.cu), so
// that they compile in parallel.
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
#include <type_traits>

#include "rgdbek_internal.h"

namespace rgd {

// Scalars of the LSQR recurrences.  GB300's FP64 rate is low, so they are
// computed by thread 0 of each CTA only (every CTA gets bit-identical values
// from the identically reduced partials) and broadcast through shared memory.
template <typename V>
struct LsqrStateT {
    V alpha, beta, rhobar, phibar, beta1, fro;
    V irho, cs, sn;         // plane rotation of the current step (1/rho, c, s)
    V inv_a, ab, wcoef;     // coefficients of the next rows phase
    V inv_b, ba, phi_rho;   // coefficients of the next cols phase
    V itol;                 // inner tolerance of this solve
    int mv, done;
    int fit;                // at the end: 1 = the residual met the tolerance (a
                            // consistent block), 2 = step cap, 0 = otherwise
};

// Scalars of the outer iteration, also computed by thread 0 only.
template <typename V>
struct OuterStateT {
    V bb, tt, zz, atb2, rel, nrm, emax_c, emax_r;
    V beta1, alpha1, fro2, inv_beta1;
    V beta1s, fro2s;        // row step: the same for the row-scaled block
    V itol;                 // inner tolerance of this iteration
    V best;                 // smallest stopping measure so far (stall test)
    long long kbest;        // iteration that reached it
    int verdict;            // status to finish with, or kStatusRunning to go on
};

// Scalars of the FP64 refinement loop of the FP32 form (thread 0 only).
struct RefineState {
    double bb, atb2, tt, hh, rel, nrm, best;
    double scale, inv_scale;  // ||t|| and its reciprocal: the inner rhs is t / ||t||
    double itol;              // target of the next inner solve
    long long refinements, kbest;
    int fp64;                 // the inner solves now run in FP64 (FP32 reached its floor)
    int verdict;
};

// per-solve counters, kept by thread 0 (only CTA 0's copy is reported)
struct Acc {
    long long inner_u, inner_j, sum_nu, sum_nj, sum_nnzu, sum_nnzj;
    long long lsqr_nnzu, lsqr_nnzj, lsqr_nu, lsqr_nj;
};

// Shared state of a solve.  It holds the scalars of both value types, so that
// one kernel can run FP64 and FP32 solves (the refinement loop of the FP32
// form does) with one barrier epoch and one set of counters.
struct SolveSmem {
    BlockScratch bs;
    Acc acc;
    long long tab[kMaxGrid];
    double red_d[D_NSLOTS];                          // reduced partials of the last barrier
    float red_f[D_NSLOTS];                           // (FP64 and FP32 slots)
    long long red_i[I_NSLOTS];
    LsqrStateT<double> lsqr_d;                       // LSQR scalars (written by thread 0)
    LsqrStateT<float> lsqr_f;
    OuterStateT<double> o_d;                         // outer-loop scalars (thread 0)
    OuterStateT<float> o_f;
    RefineState ref;                                 // refinement scalars (thread 0)
    unsigned long long epoch;                        // grid barriers passed (thread 0 copy)
    unsigned long long epoch_sub;                    // the same on the CTA's team counter of
                                                     // a two-team solve (kept between calls)
    unsigned long long split_calls;                  // two-team solves run by this kernel
    int leader;                                      // this CTA has rank 0 in its team
    unsigned long long tlast;                        // phase timers (CTA 0, thread 0)
    unsigned long long tphase[RGDBEK_NUM_PHASES];
    unsigned long long t_start;                      // globaltimer at the start of the solve
    long long tr_off;                                // trace: list entries written so far
    int tr_full;                                     // trace: lists full (or off)

    template <typename V>
    __device__ __forceinline__ V *red() {
        if constexpr (sizeof(V) == 8) return red_d;
        else return red_f;
    }
    template <typename V>
    __device__ __forceinline__ LsqrStateT<V> &lsqr() {
        if constexpr (sizeof(V) == 8) return lsqr_d;
        else return lsqr_f;
    }
    template <typename V>
    __device__ __forceinline__ OuterStateT<V> &o() {
        if constexpr (sizeof(V) == 8) return o_d;
        else return o_f;
    }
};

enum PhaseId { PH_SETUP = 0, PH_COL, PH_COL_SEL, PH_COL_EXT, PH_COL_LSQR, PH_ZUPD, PH_ROW_SEL,
               PH_ROW_EXT, PH_ROW_LSQR, PH_RESID, PH_REFINE };

// Status value of a solve that left because a grid barrier was abandoned: the
// barrier already recorded the error in the control block.
constexpr int kAbandoned = kStatusRunning;

// charges the time since the previous mark to phase `id` (team rank 0 only)
__device__ __forceinline__ void mark(SolveSmem &S, int id) {
    if (S.leader && threadIdx.x == 0) {
        const unsigned long long now = globaltimer_ns();
        S.tphase[id] += now - S.tlast;
        S.tlast = now;
    }
}

// Start-of-solve state of the shared block (every kernel calls it before
// solve_body / refine_body; a batched team calls it for each system).
template <typename PT>
__device__ __forceinline__ void init_solve_smem(SolveSmem &S, const PT &P) {
    if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer_ns();
        S.epoch = 0;
        S.epoch_sub = 0;
        S.split_calls = 0;
        S.leader = trank(P) == 0;
        S.acc = Acc{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        S.tlast = now;
        S.t_start = now;
        for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) S.tphase[i] = 0;
        S.tr_off = 0;
        S.tr_full = P.tr_lists == nullptr;
    }
    __syncthreads();
}

#define DS(x) (1u << (x))

// the barrier counter of the CTA's team
template <typename PT>
__device__ __forceinline__ unsigned long long *bar_of(const PT &P) {
    return P.bar ? P.bar : &P.ctrl->bar_count;
}

// Grid barrier, then the requested partial slots reduced into S.red_*.
// Returns false if the barrier was abandoned.
template <typename V>
__device__ __forceinline__ bool sync_collect(const ParamsT<V> &P, SolveSmem &S, unsigned dmask,
                                             unsigned dmax, unsigned imask, V *out_d) {
    if (!grid_barrier(P.ctrl, bar_of(P), S.epoch, tsize(P))) return false;
    if (dmask | imask)
        collect_partials<V>(P.pd, P.pi, tsize(P), dmask, dmax, imask, out_d, S.red_i);
    return true;
}

__device__ __forceinline__ void finish(const Params &P, int status, long long k, double rel,
                                       double nrm, long long refinements, const SolveSmem &S) {
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
        C->refinements = refinements;
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
template <typename V>
struct SideC {
    const long long *ptr;
    const int *cnt;
    const int *list;
    const int *idx;        // indices into the other space
    const V *val;
    long long n;           // lines
    int L;                 // lanes per line
};

template <typename V>
__device__ __forceinline__ void line_span(const SideC<V> &S, long long l, long long &b,
                                          long long &e) {
    const long long src = S.list ? S.list[l] : l;
    b = __ldg(S.ptr + src);
    e = S.cnt ? b + S.cnt[src] : __ldg(S.ptr + src + 1);
}

// This CTA's chunk [lo, lo + nl) of a side.  Cached: local line li spans
// idx/val[ptr[li], ptr[li+1]) in shared memory.  Otherwise the lines are read
// from the global arrays through line_span.
template <typename V>
struct CtaSide {
    const int *ptr;      // cached: chunk-local line offsets
    const int *idx;
    const V *val;        // cached values
    int nl;
    long long lo;
    int L;               // lanes per line (FP64 products, and uncached lines)
    int Lf;              // lanes per line of cached FP32 products
    bool cached;
    SideC<V> g;
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

// New places of the entries of one line, staged at ks/vs[0, len): the entry
// with index key goes to place (number of the line's indices below key),
// written to idx/val[0, len).  This lane takes entries first, first + step, ...
template <typename V>
__device__ __forceinline__ void rank_place(const int *ks, const V *vs, int len, int first, int step,
                                           int *idx, V *val) {
    for (int q = first; q < len; q += step) {
        const int key = ks[q];
        int r = 0;
        for (int t = 0; t < len; ++t) r += ks[t] < key;
        idx[r] = key;
        val[r] = vs[q];
    }
}

// Sorts by index, in place, the entries of lines [lo, hi) of a block side
// that phase_select_scatter wrote in arbitrary order (line l: idx/val[ptr[l],
// ptr[l] + cnt[l])), so that every product over a line sums in one fixed
// order, the ascending order of A's own lines.  The indices of a line are
// distinct (each selected line contributes at most one entry), so each
// entry's place is its rank.  The CTA's lines are staged in shared memory
// (arena A, released on return) and ranked there by groups of lanes sized to
// the average line (lines above eight entries per lane are ranked by a
// whole warp); a chunk that does not fit is sorted line by line in global
// memory.  All threads of the CTA call it.
template <typename V>
__device__ __forceinline__ void sort_scattered_lines(const long long *ptr, const int *cnt, int *idx,
                                                     V *val, long long lo, long long hi,
                                                     SmemArena A, BlockScratch &bs) {
    const int nl = (int)(hi - lo);
    long long *ps = A.take<long long>(nl + 1);
    long long run = 0, lmax = 0;
    for (int base = 0; base < nl; base += blockDim.x) {
        const int li = base + threadIdx.x;
        const long long len = li < nl ? cnt[lo + li] : 0;
        lmax = max(lmax, len);
        long long tot;
        const long long ex = block_excl_scan<long long>(len, bs, &tot);
        if (ps && li < nl) ps[li] = run + ex;
        run += tot;
    }
    lmax = block_max_ll(lmax, bs);
    if (lmax <= 1) return;  // nothing to order
    int *ks = ps ? A.take<int>(run) : nullptr;
    V *vs = ks ? A.take<V>(run) : nullptr;
    if (!vs) {
        // insertion sort of each line in global memory (chunks too large to stage)
        for (int li = threadIdx.x; li < nl; li += blockDim.x) {
            const long long b = ptr[lo + li];
            const int len = cnt[lo + li];
            for (int a = 1; a < len; ++a) {
                const int key = idx[b + a];
                const V v = val[b + a];
                int c = a - 1;
                while (c >= 0 && idx[b + c] > key) {
                    idx[b + c + 1] = idx[b + c];
                    val[b + c + 1] = val[b + c];
                    --c;
                }
                idx[b + c + 1] = key;
                val[b + c + 1] = v;
            }
        }
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0) ps[nl] = run;
    __syncthreads();
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const Grp G(8);
        for (int base = 0; base < nl; base += nw * G.rpw) {
            const int li = base + warp * G.rpw + G.sub;
            if (li < nl) {
                const long long o = ps[li], len = ps[li + 1] - o, b = ptr[lo + li];
                for (long long k = G.sl; k < len; k += G.L) {
                    ks[o + k] = idx[b + k];
                    vs[o + k] = val[b + k];
                }
            }
        }
    }
    __syncthreads();
    int Ls = 1;
    {
        const long long avg = (run + nl - 1) / nl;
        while (Ls < 32 && 2ll * Ls < avg) Ls *= 2;
    }
    const long long cap = 8ll * Ls;
    {
        const Grp G(Ls);
        for (int base = 0; base < nl; base += nw * G.rpw) {
            const int li = base + warp * G.rpw + G.sub;
            if (li < nl) {
                const long long o = ps[li], len = ps[li + 1] - o;
                if (len >= 2 && len <= cap)
                    rank_place(ks + o, vs + o, (int)len, G.sl, G.L, idx + ptr[lo + li],
                               val + ptr[lo + li]);
            }
        }
    }
    if (lmax > cap) {
        for (int li = warp; li < nl; li += nw) {
            const long long o = ps[li], len = ps[li + 1] - o;
            if (len > cap)
                rank_place(ks + o, vs + o, (int)len, lane, 32, idx + ptr[lo + li],
                           val + ptr[lo + li]);
        }
    }
    __syncthreads();
}

// Copies this CTA's chunk of a side into shared memory (compacting the
// lines), if it fits.  All threads of the CTA call it.
// With sort (a side phase_select_scatter wrote in arbitrary order), every
// line of the chunk is also sorted by index: each entry's place is its rank
// among the line's (distinct) indices, taken from the shared-memory copy; the
// entries are written back to the global arrays in that order and the copy
// is reloaded.  A chunk that does not fit is sorted in global memory
// (sort_scattered_lines) and read from there.
template <typename V>
__device__ __forceinline__ CtaSide<V> cache_side(const SideC<V> &S, SmemArena &A, BlockScratch &bs,
                                                 int rank, int nct, bool sort = false) {
    const Chunk C(S.n, rank, nct);
    CtaSide<V> out;
    out.nl = (int)(C.hi - C.lo);
    out.lo = C.lo;
    out.L = S.L;
    out.Lf = S.L;
    out.g = S;
    out.cached = false;
    out.ptr = nullptr;
    out.idx = nullptr;
    out.val = nullptr;
    const SmemArena save = A;
    // chunk-local offsets of the lines (the global starts are reread where
    // needed: shared memory is kept for the entries)
    int *ps = A.take<int>(out.nl + 1);
    if (!ps) {
        A = save;
        if (sort)
            sort_scattered_lines<V>(S.ptr, S.cnt, const_cast<int *>(S.idx), const_cast<V *>(S.val),
                                    C.lo, C.hi, A, bs);
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
        }
        long long tot;
        const long long ex = block_excl_scan<long long>(len, bs, &tot);
        if (li < out.nl) ps[li] = (int)(run + ex);
        run += tot;
    }
    if (threadIdx.x == 0) ps[out.nl] = (int)run;
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
    int *is = run < (1ll << 30) ? A.take<int>(run) : nullptr;
    V *vs = is ? A.take<V>(run) : nullptr;
    if (!vs) {
        A = save;
        __syncthreads();
        if (sort)
            sort_scattered_lines<V>(S.ptr, S.cnt, const_cast<int *>(S.idx), const_cast<V *>(S.val),
                                    C.lo, C.hi, A, bs);
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
                long long b, e;
                line_span(S, C.lo + li, b, e);
                const long long o = ps[li], len = ps[li + 1] - o;
                for (long long k = G.sl; k < len; k += G.L) {
                    is[o + k] = S.idx[b + k];
                    vs[o + k] = S.val[b + k];
                }
            }
        }
    }
    __syncthreads();
    if (sort) {
        // ranks from the copy, entries to their places in the global arrays
        int *gidx = const_cast<int *>(S.idx);
        V *gval = const_cast<V *>(S.val);
        const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int Ls = 1;
        {
            const long long avg = out.nl > 0 ? (run + out.nl - 1) / out.nl : 0;
            while (Ls < 32 && 2ll * Ls < avg) Ls *= 2;
        }
        const long long cap = 8ll * Ls;
        bool has_long = false;
        {
            const Grp G(Ls);
            for (int base = 0; base < out.nl; base += nw * G.rpw) {
                const int li = base + warp * G.rpw + G.sub;
                if (li < out.nl) {
                    const long long o = ps[li], len = ps[li + 1] - o;
                    if (len >= 2 && len <= cap) {
                        long long b, e;
                        line_span(S, C.lo + li, b, e);
                        rank_place(is + o, vs + o, (int)len, G.sl, G.L, gidx + b, gval + b);
                    }
                    has_long |= len > cap;
                }
            }
        }
        if (__syncthreads_or(has_long)) {
            for (int li = warp; li < out.nl; li += nw) {
                const long long o = ps[li], len = ps[li + 1] - o;
                if (len > cap) {
                    long long b, e;
                    line_span(S, C.lo + li, b, e);
                    rank_place(is + o, vs + o, (int)len, lane, 32, gidx + b, gval + b);
                }
            }
        }
        __syncthreads();
        // reload the rewritten lines
        const Grp G(Ls);
        for (int base = 0; base < out.nl; base += nw * G.rpw) {
            const int li = base + warp * G.rpw + G.sub;
            if (li < out.nl) {
                const long long o = ps[li], len = ps[li + 1] - o;
                long long b = 0, e;
                if (len >= 2) line_span(S, C.lo + li, b, e);
                if (len >= 2)
                    for (long long k = G.sl; k < len; k += G.L) {
                        is[o + k] = gidx[b + k];
                        vs[o + k] = gval[b + k];
                    }
            }
        }
        __syncthreads();
    }
    out.cached = true;
    out.Lf = Lf;
    out.ptr = ps;
    out.idx = is;
    out.val = vs;
    return out;
}

// Dot products of this CTA's lines with a gathered vector, into dots[li].
// Warp 0 is left out: it reduces the partials of the previous barrier and
// computes the LSQR scalars meanwhile.  FP32 lines accumulate with Kahan
// compensation (lane_dot).
template <typename V>
__device__ __forceinline__ void cta_dots(const CtaSide<V> &C, const V *vec, V *dots) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) return;
    const int L = (sizeof(V) == 4 && C.cached) ? C.Lf : C.L;
    if (!C.cached && L == 1) {
        // Short lines read from global memory (a chunk larger than shared
        // memory, e.g. the u-space of a column block on a small team): one
        // lane per line and four lines per lane at a time, their entries two
        // per round, so the loads of eight entries and their gathers are in
        // flight together.  Each line still sums in entry order from zero, as
        // lane_dot does, so the results are the same.
        const int per = ((blockDim.x >> 5) - 1) * 32;
        const int me = (warp - 1) * 32 + (threadIdx.x & 31);
        for (int base = 0; base < C.nl; base += 4 * per) {
            long long b[4], e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int li = base + q * per + me;
                b[q] = 0;
                e[q] = 0;
                if (li < C.nl) line_span(C.g, C.lo + li, b[q], e[q]);
            }
            V s[4] = {V(0), V(0), V(0), V(0)};
            KahanF kf[4];
            for (;;) {
                int j[4][2];
                V a[4][2];
                bool any = false;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const long long f = b[q] + t;
                        const bool v = f < e[q];
                        j[q][t] = v ? C.g.idx[f] : -1;
                        a[q][t] = v ? C.g.val[f] : V(0);
                        any |= v;
                    }
                if (!any) break;
                V x[4][2];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int t = 0; t < 2; ++t) x[q][t] = j[q][t] >= 0 ? vec[j[q][t]] : V(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (j[q][t] < 0) continue;
                        if constexpr (sizeof(V) == 8) s[q] = fma(a[q][t], x[q][t], s[q]);
                        else kf[q].add(a[q][t], x[q][t]);
                    }
                    b[q] += 2;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int li = base + q * per + me;
                if (li < C.nl) {
                    if constexpr (sizeof(V) == 8) dots[li] = s[q];
                    else dots[li] = kf[q].sum();
                }
            }
        }
        return;
    }
    const Grp G(L);
    const int per = ((blockDim.x >> 5) - 1) * G.rpw;
    const auto gat = [&](int j) { return vec[j]; };
    for (int base = 0; base < C.nl; base += per) {
        const int li = base + (warp - 1) * G.rpw + G.sub;
        V s = V(0);
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

// Warp 0: sum of the per-CTA partials of one slot, for lane 0.  FP64: the
// order-independent fixed-point sum (no FP64 adds on the critical path of the
// phase); FP32: float adds in a fixed order.
template <typename V>
__device__ __forceinline__ V warp0_collect(const V *pd, int slot, int nb) {
    if constexpr (sizeof(V) == 8) {
        return warp_sum_fixed(pd + slot * nb, nb);
    } else {
        const V *p = pd + slot * nb;
        V s = V(0);
#pragma unroll 8
        for (int i = threadIdx.x; i < nb; i += 32) s += __ldcg(p + i);
        return warp_sum(s);
    }
}

// CTA sum of the squares the LSQR combine forms (FP64: fixed point, as above).
template <typename V>
__device__ __forceinline__ V lsqr_block_sum(V v, BlockScratch &bs) {
    if constexpr (sizeof(V) == 8) return block_sum_fixed(v, bs);
    else return block_sum(v, bs);
}

// LSQR from y = 0 on the block (R, C) with right-hand side c0 (u-space,
// global, element i at c0[i * c0s]; without v_given c0s must be 1), beta1 =
// ||c0||.  With v_given, v~_1 = B^T c0 / beta1 is already in P.vv and alpha1
// is passed; otherwise it is computed first (one more phase).  fro2 =
// ||B||_F^2.  y_g (v-space) receives the solution; with xt given (the row
// step, v-space = x-space) also xt = x + y, so the residual pass gathers
// x_{k+1} without an addition per nonzero.  With csc (the column step;
// requires v_given) the solve runs on B D, D = diag(csc) over the v-space
// (unit columns): the rows phase gathers D v~, the cols phase scales B^T u~
// by D, and y_g receives y = D y^, so B y_g is the projection of c0 whatever
// the scaling.  Returns the number of steps (0 if alpha1 == 0), or -1 if a
// grid barrier was abandoned.  sort_side (1 = R, 2 = C): that side was
// written by phase_select_scatter, and each CTA sorts the lines of its chunk
// of it while caching them (cache_side); the CTA alone reads them before the
// first barrier.
//
// Per phase: grid barrier | warp 0 reduces the partials and updates the
// scalars while warps 1.. compute the dot products of the CTA's lines |
// __syncthreads | all threads combine element-wise and form the partial.
template <typename V>
__device__ __forceinline__ int run_lsqr(const ParamsT<V> &P, const SideC<V> &Rs,
                                        const SideC<V> &Cs, const V *c0, int c0s, V *y_g, V *xt,
                                        const V *csc, const V *rsc, bool v_given, V alpha1,
                                        V beta1, V fro2, unsigned char *dsmem,
                                        long long dsmem_bytes, SolveSmem &S, int sort_side = 0) {
    LsqrStateT<V> &L = S.lsqr<V>();
    SmemArena A{dsmem, dsmem_bytes, 0};
    const Chunk RC(Rs.n, trank(P), tsize(P)), CC(Cs.n, trank(P), tsize(P));
    const int nrl = (int)(RC.hi - RC.lo), ncl = (int)(CC.hi - CC.lo);
    // per-CTA vector slices and dot buffers
    V *uold = A.take<V>(nrl);
    V *dr = uold ? A.take<V>(nrl) : nullptr;
    V *vown = dr ? A.take<V>(ncl) : nullptr;
    V *wown = vown ? A.take<V>(ncl) : nullptr;
    V *yown = wown ? A.take<V>(ncl) : nullptr;
    V *dc = yown ? A.take<V>(ncl) : nullptr;
    // column scaling D of the v-space (column step), row scaling of the
    // u-space (row step): their slices
    V *sown = (dc && csc) ? A.take<V>(ncl) : nullptr;
    V *rown = (dc && rsc) ? A.take<V>(nrl) : nullptr;
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
        for (int i = threadIdx.x; i < ncl; i += blockDim.x) yown[i] = V(0);
    } else {
        for (int i = threadIdx.x; i < nrl; i += blockDim.x) {
            uold[i] = c0[(RC.lo + i) * c0s];
            if (rown) rown[i] = rsc[RC.lo + i];
        }
        for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
            vown[i] = v_given ? P.vv[CC.lo + i] : V(0);
            yown[i] = V(0);
            if (sown) sown[i] = csc[CC.lo + i];
        }
    }
    const V *dloc = csc ? (sown ? sown : csc + CC.lo) : nullptr;
    const V *rloc = rsc ? (rown ? rown : rsc + RC.lo) : nullptr;
    // the cols phase gathers D u~ when the u-space is scaled
    const V *usrc = rsc ? P.uus : P.uu;
    // the rows phase gathers D v~ when the v-space is scaled
    const V *vsrc = csc ? P.vvs : P.vv;
    const CtaSide<V> R = cache_side<V>(Rs, A, S.bs, trank(P), tsize(P), sort_side == 1);
    const CtaSide<V> C = cache_side<V>(Cs, A, S.bs, trank(P), tsize(P), sort_side == 2);
    if (threadIdx.x == 0) {
        L.inv_b = V(1) / beta1;
        L.done = 0;
        L.fit = 0;
        L.itol = S.o<V>().itol;
    }
    __syncthreads();

    if (!v_given) {
        // v~_1 = B^T c0 / beta1 (warp 0 has no scalars to update in this phase)
        cta_dots<V>(C, rsc ? P.uus : c0, dc);
        __syncthreads();
        V acc = V(0);
        for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
            const V v = dc[li] * L.inv_b;
            vown[li] = v;
            P.vv[CC.lo + li] = v;
            acc = vfma(v, v, acc);
        }
        acc = lsqr_block_sum(acc, S.bs);
        if (threadIdx.x == 0) P.pd[D_VV * tsize(P) + trank(P)] = acc;
        if (!grid_barrier(P.ctrl, bar_of(P), S.epoch, tsize(P))) return -1;
        if (threadIdx.x < 32) {
            const V vv = warp0_collect(P.pd, D_VV, tsize(P));
            if (threadIdx.x == 0) L.alpha = vsqrt(vv);
        }
        __syncthreads();
        alpha1 = L.alpha;
        if (!(alpha1 > V(0))) return 0;
    }
    if (threadIdx.x == 0) {
        L.alpha = alpha1;
        L.beta = beta1;
        L.rhobar = alpha1;
        L.phibar = beta1;
        L.beta1 = beta1;
        L.fro = vsqrt(fro2);
        L.inv_a = V(1) / alpha1;
        L.ab = alpha1 / beta1;
        L.wcoef = V(0);
    }
    __syncthreads();
    for (int it = 1;; ++it) {
        const bool first = it == 1;
        // ---- rows phase: u~_new = B v~ / alpha - (alpha/beta) u~, w update
        cta_dots<V>(R, vsrc, dr);
        if (threadIdx.x < 32 && !first) {
            // scalars from ||v~||^2 of the previous cols phase
            const V vv = warp0_collect(P.pd, D_VV, tsize(P));
            if (threadIdx.x == 0) {
                // alpha_{i+1} = ||v~||; the divisions of the recurrence are
                // multiplications by reciprocals formed with rsqrt, which keeps
                // the dependent chain of this single thread short
                // alpha = vv * rsqrt(vv): one reciprocal square root serves both
                const V cs = L.cs, sn = L.sn, bn = L.beta;
                const V ivv = vv > V(0) ? vrsqrt(vv) : V(0);
                const V an = bn > V(0) ? vv * ivv : V(0);
                const V ian = an > V(0) ? ivv : V(0);
                L.rhobar = -cs * an;
                L.wcoef = sn * an * L.irho;   // theta / rho
                const V rnorm = L.phibar;
                const V arnorm = L.phibar * an * fabs(cs);
                const bool resid = rnorm <= L.itol * L.beta1 || bn == V(0);
                const bool other = arnorm <= L.itol * L.fro * rnorm || an == V(0);
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
            const V inv_a = L.inv_a, ab = L.ab, wcoef = L.wcoef;
            for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
                const V vn = vown[li] * inv_a;
                wown[li] = first ? vn : vn - wcoef * wown[li];
            }
            V acc = V(0);
            for (int li = threadIdx.x; li < nrl; li += blockDim.x) {
                const V rl = rloc ? rloc[li] : V(1);
                const V uo = st_smem ? uold[li]
                                     : (first ? c0[(RC.lo + li) * c0s] : P.uu[RC.lo + li]);
                const V u = (rloc ? dr[li] * rl : dr[li]) * inv_a - ab * uo;
                P.uu[RC.lo + li] = u;
                if (rloc) P.uus[RC.lo + li] = u * rl;
                if (st_smem) uold[li] = u;
                acc = vfma(u, u, acc);
            }
            acc = lsqr_block_sum(acc, S.bs);
            if (threadIdx.x == 0) P.pd[D_UU * tsize(P) + trank(P)] = acc;
        }
        if (!grid_barrier(P.ctrl, bar_of(P), S.epoch, tsize(P))) return -1;

        // ---- cols phase: v~_new = B^T u~ / beta - (beta/alpha) v~, y update
        cta_dots<V>(C, usrc, dc);
        if (threadIdx.x < 32) {
            const V uu = warp0_collect(P.pd, D_UU, tsize(P));
            if (threadIdx.x == 0) {
                // beta_{i+1} = ||u~|| = uu * rsqrt(uu), rho = sqrt(rhobar^2 +
                // beta^2); 1/rho from rsqrt of rho^2 directly, in parallel
                const V iuu = uu > V(0) ? vrsqrt(uu) : V(0);
                const V bn = uu * iuu;
                const V irho = vrsqrt(vfma(L.rhobar, L.rhobar, uu));
                const V cs = L.rhobar * irho, sn = bn * irho;
                const V phi = cs * L.phibar;
                L.phibar = sn * L.phibar;
                L.mv = bn > V(0);
                L.inv_b = bn > V(0) ? iuu : V(0);
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
            const V inv_b = L.inv_b, ba = L.ba, phi_rho = L.phi_rho;
            const bool mv = L.mv != 0;
            V acc = V(0);
            for (int li = threadIdx.x; li < ncl; li += blockDim.x) {
                const V dl = dloc ? dloc[li] : V(1);
                if (mv) {
                    const V v = (dloc ? dc[li] * dl : dc[li]) * inv_b - ba * vown[li];
                    vown[li] = v;
                    P.vv[CC.lo + li] = v;
                    if (dloc) P.vvs[CC.lo + li] = v * dl;
                    acc = vfma(v, v, acc);
                }
                const V y = vfma(phi_rho, wown[li], yown[li]);
                yown[li] = y;
                y_g[CC.lo + li] = dloc ? y * dl : y;   // y = D y^ when scaled
                if (xt) xt[CC.lo + li] = P.x[CC.lo + li] + y;
            }
            acc = lsqr_block_sum(acc, S.bs);
            if (threadIdx.x == 0) P.pd[D_VV * tsize(P) + trank(P)] = acc;
        }
        if (!grid_barrier(P.ctrl, bar_of(P), S.epoch, tsize(P))) return -1;
    }
}

// z_{k+1} = z_k - A_U y (A_U as extracted CSR), r = t_k - z_{k+1},
// eps^x_i = r_i^2 / ||A^(i)||^2.  Partials: max eps^x, ||z_{k+1}||^2, bad.
// kMode 0: all of it.  kMode 1 (column team of a two-team solve): z_{k+1}
// and ||z_{k+1}||^2 only.  kMode 2 (row team): r and the row weights from the
// z_{k+1} the column team wrote (hasU ignored).
template <typename V, int kMode = 0>
__device__ __forceinline__ void phase_zupdate(const ParamsT<V> &P, bool hasU, int Lsub,
                                              BlockScratch &bs) {
    constexpr bool kZ = kMode != 2, kR = kMode != 1;
    const Grp G(kZ && hasU ? Lsub : 1);
    V emax = V(0), zz = V(0);
    long long bad = 0;
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        V s = V(0);
        if (kZ && hasU && i < P.m)
            s = lane_dot<false>(P.rp[i] + G.sl, P.rp[i] + P.srn[i], G.L, P.sci, P.sav,
                                [&](int p) { return P.yy[p]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) {
            V zi;
            if constexpr (kZ) {
                zi = P.z[2 * i] - s;
                P.z[2 * i] = zi;
                zz = vfma(zi, zi, zz);
            } else {
                zi = P.z[2 * i];
            }
            if constexpr (kR) {
                const V ri = P.t[2 * i] - zi;
                P.r[i] = ri;
                const V c = __ldg(P.rn2 + i);
                const V e = c > V(0) ? weight_of(ri, c) : V(0);
                P.epsr[i] = e;
                if (!isfinite(e)) bad = 1;
                else emax = max_nonneg(emax, e);
            }
        }
    }
    if (kR) emax = block_max(emax, bs);
    if (kZ) zz = block_sum(zz, bs);
    if (kR) bad = block_sum(bad, bs);
    if (threadIdx.x == 0) {
        if (kR) P.pd[D_EMAX_R * tsize(P) + trank(P)] = emax;
        if (kZ) P.pd[D_ZZ * tsize(P) + trank(P)] = zz;
        if (kR) P.pi[I_BAD_R * tsize(P) + trank(P)] = bad;
    }
}

// Sizes and inner steps of one block of an outer iteration.
struct BlockInfo {
    long long n, nnz;
    int steps, lanes;
};

#define RGD_SYNC_I(dm, dx, im)                                                   \
    do {                                                                         \
        if (!sync_collect(P, S, (dm), (dx), (im), red)) return -1;               \
    } while (0)

// Column block of iteration k (Algorithm 1, column step; Eq. 4 and Remark
// 3.1): U_k drawn from eps^z (P.epsc, maximum O.emax_c > 0) with Philox
// counter (k, 0), A_U scattered from the CSC columns of U into the rows of
// A_U, and LSQR on A_U D from z_k (beta1 = sqrt(O.zz)); y goes to P.yy for the
// z update.  ulist receives U_k; with tr_on it is also recorded at
// P.tr_lists[tr_base ..] if it fits.  Returns 0, or -1 if a barrier was
// abandoned.
template <typename V>
__device__ __forceinline__ int col_block(const ParamsT<V> &P, SolveSmem &S, unsigned char *dsmem,
                                         long long k, int *ulist, bool tr_on, long long tr_base,
                                         BlockInfo &U) {
    BlockScratch &bs = S.bs;
    OuterStateT<V> &O = S.o<V>();
    V *const red = S.red<V>();
    const int nct = tsize(P);
    const bool greedy = P.selection == RGDBEK_SELECT_GREEDY;
    // quantise (the row counts of A_U cleared) | draws, counted per chunk |
    // compaction + scatter of the selected columns into the rows of A_U
    phase_quantize(P, P.epsc, P.n, O.emax_c, greedy, P.eta_col, bs, true, P.srn, P.m);
    RGD_SYNC_I(0, 0, 0);
    if (!greedy) {
        phase_draw(P, P.n, P.s_col, P.seed, P.sysid, (unsigned long long)k, 0ull, S.tab, bs,
                   P.pi + I_CNT * nct);
        RGD_SYNC_I(0, 0, 0);
    }
    mark(S, PH_COL_SEL);
    if (threadIdx.x == 0) {
        O.beta1 = vsqrt(O.zz);
        O.inv_beta1 = O.beta1 > V(0) ? V(1) / O.beta1 : V(0);
    }
    __syncthreads();
    const V inv_beta1 = O.inv_beta1;
    // LSQR start on B = A_U D (columns scaled to unit norm, D =
    // diag(1/||A_j||)) with c = z_k: v~_1 = B^T z_k / beta1
    U.n = phase_select_scatter(
        P, P.n, P.cn2, P.g, P.epsc, nullptr, ulist, S.tab, bs, P.cp, P.ri, P.cv, P.rp,
        P.srn, P.sci, P.sav, [&](long long p, long long j, long long tot) {
            const V d = vrsqrt(P.cn2[j]);           // selected: ||A_j|| > 0
            const V v1 = P.g[j] * d * inv_beta1;
            P.dsc[p] = d;
            P.vv[p] = v1;
            P.vvs[p] = v1 * d;
            P.yy[p] = V(0);
            if (tr_on && tr_base + tot <= P.tr_list_cap) P.tr_lists[tr_base + p] = (int)j;
        });
    RGD_SYNC_I(DS(D_FRO_S) | DS(D_EXTRA_S), 0, DS(I_NNZ));
    mark(S, PH_COL_EXT);
    if (threadIdx.x == 0) {
        // beta1 = ||z_k||, alpha1 = ||B^T z_k|| / beta1 = sqrt(sum of the
        // selected eps^z) / beta1, ||B||_F^2 = |U|
        O.fro2 = red[D_FRO_S];
        O.alpha1 = vsqrt(red[D_EXTRA_S]) * O.inv_beta1;
    }
    __syncthreads();
    U.nnz = S.red_i[I_NNZ];
    U.lanes = pick_lanes_fp64(U.nnz, P.m);
    if (O.beta1 > V(0) && O.alpha1 > V(0)) {
        const SideC<V> rows{P.rp, P.srn, nullptr, P.sci, P.sav, P.m, U.lanes};
        const SideC<V> cols{P.cp, nullptr, ulist, P.ri, P.cv, U.n, P.tpc};
        U.steps = run_lsqr<V>(P, rows, cols, P.z, 2, P.yy, nullptr, P.dsc, nullptr, true,
                             O.alpha1, O.beta1, O.fro2, dsmem, P.dsmem_bytes, S, 1);
        if (U.steps < 0) return -1;
        mark(S, PH_COL_LSQR);
    }
    return 0;
}

// Row block of iteration k (Algorithm 1, row step): J_k drawn from eps^x
// (P.epsr, maximum O.emax_r > 0) with Philox counter (k, 1), A^J scattered from
// the CSR rows of J into the columns of A^J, and the minimum-norm solution of
// A^J d = r_J by LSQR (first on the row-scaled block, see below); d goes to
// P.dx and x + d to P.xt.  With tr_on, J_k is recorded at P.tr_lists[tr_base
// ..] if it fits.  Returns 0, or -1 if a barrier was abandoned.
template <typename V>
__device__ __forceinline__ int row_block(const ParamsT<V> &P, SolveSmem &S, unsigned char *dsmem,
                                         long long k, bool tr_on, long long tr_base,
                                         BlockInfo &J) {
    constexpr bool kF32 = sizeof(V) == 4;
    BlockScratch &bs = S.bs;
    OuterStateT<V> &O = S.o<V>();
    V *const red = S.red<V>();
    const int nct = tsize(P);
    const bool greedy = P.selection == RGDBEK_SELECT_GREEDY;
    // quantise (the column counts of A^J cleared) | draws | compaction +
    // scatter of the selected rows into the columns of A^J
    phase_quantize(P, P.epsr, P.m, O.emax_r, greedy, P.eta_row, bs, true, P.scn, P.n);
    RGD_SYNC_I(0, 0, 0);
    if (!greedy) {
        phase_draw(P, P.m, P.s_row, P.seed, P.sysid, (unsigned long long)k, 1ull, S.tab, bs,
                   P.pi + I_CNT * nct);
        RGD_SYNC_I(0, 0, 0);
    }
    mark(S, PH_ROW_SEL);
    // |J| <= n: first on D A^J (rows scaled to unit norm, D =
    // diag(1/||A^(i)||)) with c = D r_J, which has the same minimum-norm
    // solution whenever the block system is consistent
    J.n = phase_select_scatter(
        P, P.m, P.rn2, P.r, P.epsr, nullptr, P.jlist, S.tab, bs, P.rp, P.ci, P.av, P.cp,
        P.scn, P.sri, P.scv, [&](long long p, long long i, long long tot) {
            const V ri = P.r[i];
            if (tot <= P.n) {
                const V d = vrsqrt(P.rn2[i]);      // selected: ||A^(i)|| > 0
                const V u1 = ri * d;               // u~_1 = D r_J
                P.dsr[p] = d;
                P.uu[p] = u1;
                P.uus[p] = u1 * d;
            } else {
                P.uu[p] = ri;  // u~_1 = r_J
            }
            if (tr_on && tr_base + tot <= P.tr_list_cap) P.tr_lists[tr_base + p] = (int)i;
        });
    RGD_SYNC_I(DS(D_FRO) | DS(D_EXTRA) | DS(D_FRO_S) | DS(D_EXTRA_S), 0, DS(I_NNZ));
    mark(S, PH_ROW_EXT);
    if (threadIdx.x == 0) {
        // LSQR start on A^J with c = r_J: beta1 = ||r_J||; on D A^J
        // (unit rows) with c = D r_J: beta1 = sqrt(sum of the weights)
        O.fro2 = red[D_FRO];
        O.beta1 = vsqrt(red[D_EXTRA]);
        O.inv_beta1 = O.beta1 > V(0) ? V(1) / O.beta1 : V(0);
        O.fro2s = red[D_FRO_S];
        O.beta1s = vsqrt(red[D_EXTRA_S]);
    }
    __syncthreads();
    const bool rscale = J.n <= P.n;
    J.nnz = S.red_i[I_NNZ];
    if (O.beta1 > V(0)) {
        const SideC<V> rows{P.rp, nullptr, P.jlist, P.ci, P.av, J.n, P.tpr};
        const SideC<V> cols{P.cp, P.scn, nullptr, P.sri, P.scv, P.n,
                            pick_lanes_fp64(J.nnz, P.n)};
        int fit = 0;
        if (rscale) {
            J.steps = run_lsqr<V>(P, rows, cols, P.uu, 1, P.dx, P.xt, nullptr, P.dsr,
                                 false, V(0), O.beta1s, O.fro2s, dsmem, P.dsmem_bytes, S,
                                 2);
            if (J.steps < 0) return -1;
            fit = S.lsqr<V>().fit;
        }
        // The FP32 inner solve keeps the row-scaled step even when LSQR
        // finds the block inconsistent at FP32 rounding level: the step
        // still lies in range(A^T), and the FP64 refinement removes the
        // difference.  The FP64 solve takes (A^J)^+ r_J exactly.
        if (!rscale || (!kF32 && fit == 0)) {
            if (rscale) {
                // found inconsistent: (A^J)^+ r_J needs the unscaled block;
                // the scaled attempt's x + y is undone first
                for (long long p = tthread(P); p < J.n; p += tthreads(P))
                    P.uu[p] = P.r[P.jlist[p]];
                for (long long j = tthread(P); j < P.n; j += tthreads(P)) P.xt[j] = P.x[j];
                RGD_SYNC_I(0, 0, 0);
            }
            const int s2 = run_lsqr<V>(P, rows, cols, P.uu, 1, P.dx, P.xt, nullptr,
                                       nullptr, false, V(0), O.beta1, O.fro2, dsmem,
                                       P.dsmem_bytes, S, rscale ? 0 : 2);
            if (s2 < 0) return -1;
            J.steps += s2;
        }
        mark(S, PH_ROW_LSQR);
    }
    return 0;
}

#undef RGD_SYNC_I

// Result of one solve_body: the status to finish with (kAbandoned when a
// barrier was abandoned), the iteration reached and the measures of x_k.
template <typename V>
struct SolveOut {
    int status;
    long long k;
    V rel, nrm;
};

// Iterations without a new smallest stopping measure after which the FP32
// inner solve of the refinement loop stops (it has reached its rounding floor).
constexpr long long kInnerStallIters = 40;

#define RGD_SYNC(dm, dx, im)                                                     \
    do {                                                                         \
        if (!sync_collect(P, S, (dm), (dx), (im), red))                          \
            return SolveOut<V>{kAbandoned, 0, V(0), V(0)};                       \
    } while (0)

// One whole solve of Algorithm 1 by the CTAs of a team (after enter_team and
// init_solve_smem), from iteration P.k0.  V = double: the FP64 solve.  V =
// float: the inner solve of the refinement loop (x_0 = 0, its own right-hand
// side P.b and stopping test; it also stops when its measure has not reached a
// new minimum for kInnerStallIters iterations, reported as NOT_CONVERGED).
template <typename V>
__device__ __forceinline__ SolveOut<V> solve_body(const ParamsT<V> &P, SolveSmem &S,
                                                  unsigned char *dsmem) {
    constexpr bool kF32 = sizeof(V) == 4;
    BlockScratch &bs = S.bs;
    OuterStateT<V> &O = S.o<V>();
    V *const red = S.red<V>();
    const int nct = tsize(P);

    // ---- x_0 = 0, z_0 = b, t_0 = b - A x_0 = b, dx = 0
    {
        V bb = V(0);
        long long bad = 0;
        for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
            const V bi = ld_rhs(P.b + i);
            P.z[2 * i] = bi;
            P.t[2 * i] = bi;
            bb = vfma(bi, bi, bb);
            if (!isfinite(bi)) bad = 1;
        }
        // x_0 = 0, or the caller's x (warm start)
        for (long long j = tthread(P); j < P.n; j += tthreads(P)) {
            const V x0 = P.warm ? P.x[j] : V(0);
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
        O.bb = red[D_BB];
        O.tt = P.warm ? red[D_TT] : O.bb;  // t_0 = b - A x_0 (= b from x_0 = 0)
        O.zz = O.bb;
        O.atb2 = V(0);
        O.best = V(0);
        O.kbest = P.k0;
        O.verdict = (S.red_i[I_BAD_R] != 0 || !isfinite(O.bb)) ? RGDBEK_ERR_NONFINITE
                                                                : kStatusRunning;
    }
    __syncthreads();
    if (O.verdict != kStatusRunning) return SolveOut<V>{O.verdict, P.k0, V(NAN), V(NAN)};

    for (long long k = P.k0;; ++k) {
        // ---- column pass and stopping test on x_k
        if (trank(P) == 0 && threadIdx.x == 0 && P.time_budget_ns > 0.0 &&
            (double)(globaltimer_ns() - S.t_start) > P.time_budget_ns)
            P.ctrl->stop_req = 1;
        phase_col(P, bs);
        RGD_SYNC(DS(D_EMAX_C) | DS(D_HH) | DS(D_GG), DS(D_EMAX_C), DS(I_BAD_C));
        mark(S, PH_COL);
        if (P.tr_g && k < P.tr_vec_cap)  // trace: g = A^T z_k, complete after the barrier
            for (long long j = tthread(P); j < P.n; j += tthreads(P))
                P.tr_g[k * P.n + j] = (double)P.g[j];
        if (threadIdx.x == 0) {
            const V hh = red[D_HH];
            O.emax_c = red[D_EMAX_C];
            if (k == P.k0) O.atb2 = red[D_GG];  // g = A^T z_0 = A^T b
            O.rel = O.bb > V(0) ? vsqrt(O.tt / O.bb) : V(0);
            O.nrm = O.atb2 > V(0) ? vsqrt(hh / O.atb2) : V(0);
            const V meas = P.stop_rule == RGDBEK_STOP_REL_RES
                               ? O.rel
                               : (P.stop_rule == RGDBEK_STOP_RSE ? O.rel * O.rel : O.nrm);
            // inner tolerance of this iteration: fixed, or tied to how far x_k
            // is from the stopping rule (looser block solves while far away)
            O.itol = (V)P.inner_tol;
            if (P.inner_adapt > 0.0) {
                const V a = fmin(V(0.1), (V)P.inner_adapt * meas);
                if (a > O.itol) O.itol = a;
            }
            if (k == P.k0 || meas < O.best) {
                O.best = meas;
                O.kbest = k;
            }
            int v = kStatusRunning;
            if (S.red_i[I_BAD_C] != 0 || !isfinite(hh) || !isfinite(O.tt)) v = RGDBEK_ERR_NONFINITE;
            else if (stop_rule_holds(P.stop_rule, P.tol, O.rel, O.nrm)) v = RGDBEK_OK;
            else if (k >= P.max_iter) v = RGDBEK_NOT_CONVERGED;
            else if (ld_volatile_i32(&P.ctrl->stop_req)) v = RGDBEK_ERR_TIMEOUT;
            else if (kF32 && k - O.kbest >= kInnerStallIters) v = RGDBEK_NOT_CONVERGED;
            O.verdict = v;
        }
        __syncthreads();
        if (O.verdict != kStatusRunning) return SolveOut<V>{O.verdict, k, O.rel, O.nrm};

        // ---- column block U_k and z_{k+1} = z_k - A_U A_U^+ z_k
        BlockInfo U{0, 0, 0, 1};
        bool rec_u = !S.tr_full;
        if (O.emax_c > V(0)) {
            if (col_block<V>(P, S, dsmem, k, P.ulist, !S.tr_full, S.tr_off, U) < 0)
                return SolveOut<V>{kAbandoned, k, V(0), V(0)};
            rec_u = !S.tr_full && S.tr_off + U.n <= P.tr_list_cap;
        }

        // ---- z_{k+1}, row residual r = b - z_{k+1} - A x_k, row weights
        phase_zupdate(P, U.n > 0, U.lanes, bs);
        RGD_SYNC(DS(D_EMAX_R) | DS(D_ZZ), DS(D_EMAX_R), DS(I_BAD_R));
        mark(S, PH_ZUPD);
        if (P.tr_r && k < P.tr_vec_cap)  // trace: the row residual r = b - z_{k+1} - A x_k
            for (long long i = tthread(P); i < P.m; i += tthreads(P))
                P.tr_r[k * P.m + i] = (double)P.r[i];
        if (threadIdx.x == 0) {
            O.emax_r = red[D_EMAX_R];
            O.zz = red[D_ZZ];
            O.verdict = S.red_i[I_BAD_R] != 0 ? RGDBEK_ERR_NONFINITE : kStatusRunning;
        }
        __syncthreads();
        if (O.verdict != kStatusRunning) return SolveOut<V>{O.verdict, k, O.rel, O.nrm};

        // ---- row block J_k and dx = (A^J)^+ r_J
        BlockInfo J{0, 0, 0, 1};
        bool rec_j = false;
        if (O.emax_r > V(0)) {
            if (row_block<V>(P, S, dsmem, k, rec_u, S.tr_off + U.n, J) < 0)
                return SolveOut<V>{kAbandoned, k, V(0), V(0)};
            rec_j = rec_u && S.tr_off + U.n + J.n <= P.tr_list_cap;
        }
        const long long nU = U.n, nJ = J.n, nnzU = U.nnz, nnzJ = J.nnz;
        const int stepsU = U.steps, stepsJ = J.steps;

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
        if (!S.tr_full) {
            // every thread evaluates the same condition; thread 0 stores it
            const bool ok = rec_u && (nJ == 0 || rec_j) && S.tr_off + nU + nJ <= P.tr_list_cap;
            __syncthreads();
            if (threadIdx.x == 0) {
                if (ok) S.tr_off += nU + nJ;
                else S.tr_full = 1;
            }
            __syncthreads();
        }
        if (nU == 0 && nJ == 0) {
            // both blocks empty: x can no longer change
            return SolveOut<V>{RGDBEK_OK, k, O.rel, O.nrm};
        }

        // ---- t_{k+1} = b - A x_{k+1}
        phase_residual(P, bs);
        RGD_SYNC(DS(D_TT), 0, 0);
        mark(S, PH_RESID);
        if (threadIdx.x == 0) O.tt = red[D_TT];
    }
}

#undef RGD_SYNC

// ---------------------------------------------------------------------------
// Two-team schedule of one solve (P.zteam > 0).
//
// In Algorithm 1 the column step of iteration k maps z_k to z_{k+1} with
// weights, draws and projections that depend on z_k alone (z_0 = b), while
// the row step of iteration k needs z_{k+1} and x_k.  So the column step of
// iteration k+1 can run while the row step of iteration k runs.  The grid is
// cut into a row team (the first team - zteam CTAs) and a column team (the
// last zteam CTAs), each with its own barrier counter:
//   column team, iteration k:  g = A^T z_k, eps^z, and h = A^T t for the row
//                              team's stopping test | U_k, A_U, LSQR | (once
//                              the row team has read z_k) z_{k+1} = z_k - A_U y
//   row team, iteration k:     (once z_{k+1} is written) r = t_k - z_{k+1},
//                              eps^x | J_k, A^J, LSQR -> x_k + dx | stopping
//                              test of x_k | t_{k+1} = b - A x_{k+1}, x_{k+1}
//                              adopted
// Every quantity comes from the same inputs as in solve_body, so the iterates
// are those of Algorithm 1; only the partition of the reductions over CTAs
// differs (rounding level).  The test of x_k needs ||A^T t_k||, which the
// column team forms in the pass that forms g = A^T z_{k+1} (t_k is written at
// the end of row step k-1); so the row team tests x_k after its row step k,
// returns x_k if the test holds (that row step and its counters are then
// discarded), and otherwise adopts x_{k+1}.  x_{k0} is tested before the first
// row step, and x_k with k >= max_iter before its row step (that test stops).
//
// Link words (Ctrl::lk_*) hold (call << 32) | count, so the calls of one
// kernel (the inner solves of the refinement loop) never see an earlier
// call's words:
//   lk_colpass = c|j+1 after column pass k0 + j, with, in slot j & 1, its
//                ||A^T t||^2 (t_{k0} for j = 0, t_{k0+j-1} for j >= 2, none
//                for j = 1), the non-finite flag of eps^z and (j = 0)
//                ||A^T b||^2
//   lk_zready  = c|j+1 once z_{k0+j+1} is written; |U|, nnz(A_U) and the
//                LSQR steps in slot j & 1, U_{k0+j} in list j & 1
//   lk_zused   = c|j+1 once the row team has read z_{k0+j+1}
//   lk_tready  = c|j   once t_{k0+j} is written
//   lk_stop    = c     once the row team has finished
// The column team writes z_{k+1} over z_k only after the row team has read
// z_k; the row team writes t_{k+1} over t_k only after the column pass that
// reads t_k.  A slot or list of parity j is rewritten two iterations later,
// after its reader has passed a point its writer waits for.
// ---------------------------------------------------------------------------

// dst = src by all threads of the CTA (dst in shared memory), then a barrier
template <typename PT>
__device__ __forceinline__ void copy_params(PT &dst, const PT &src) {
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int w = threadIdx.x; w < (int)(sizeof(PT) / sizeof(int)); w += blockDim.x) d[w] = s[w];
    __syncthreads();
}

__device__ __forceinline__ unsigned long long lk_enc(unsigned long long call, long long n) {
    return (call << 32) | (unsigned long long)n;
}

#define X_SYNC(dm, dx, im)                                                        \
    do {                                                                          \
        if (!sync_collect(P, S, (dm), (dx), (im), red))                           \
            return SolveOut<V>{kAbandoned, 0, V(0), V(0)};                        \
    } while (0)
#define X_WAIT(word, target)                                                      \
    do {                                                                          \
        if (link_wait(C, &C->word, (target), 0ull) != 0)                          \
            return SolveOut<V>{kAbandoned, 0, V(0), V(0)};                        \
    } while (0)

// The row team's part of a two-team solve: the status, the iteration and the
// measures of the returned x (as solve_body).
template <typename V>
__device__ __forceinline__ SolveOut<V> xchain_body(const ParamsT<V> &P, SolveSmem &S,
                                                   unsigned char *dsmem, unsigned long long call,
                                                   int *const *ulists) {
    constexpr bool kF32 = sizeof(V) == 4;
    BlockScratch &bs = S.bs;
    OuterStateT<V> &O = S.o<V>();
    V *const red = S.red<V>();
    const int nct = tsize(P);
    Ctrl *const C = P.ctrl;
    const bool lead = trank(P) == 0 && threadIdx.x == 0;

    // ---- x_0 (0 or the caller's), xt = x_0, t_0 = b, ||b||^2, non-finite inputs
    {
        V bb = V(0);
        long long bad = 0;
        for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
            const V bi = ld_rhs(P.b + i);
            P.t[2 * i] = bi;
            bb = vfma(bi, bi, bb);
            if (!isfinite(bi)) bad = 1;
        }
        for (long long j = tthread(P); j < P.n; j += tthreads(P)) {
            const V x0 = P.warm ? P.x[j] : V(0);
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
    X_SYNC(DS(D_BB), 0, DS(I_BAD_R));
    if (P.warm) {
        phase_residual(P, bs);  // t_0 = b - A x_0
        X_SYNC(DS(D_TT), 0, 0);
    }
    mark(S, PH_SETUP);
    if (threadIdx.x == 0) {
        O.bb = red[D_BB];
        O.tt = P.warm ? red[D_TT] : O.bb;
        O.atb2 = V(0);
        O.best = V(0);
        O.kbest = P.k0;
        O.itol = (V)P.inner_tol;
        O.verdict = (S.red_i[I_BAD_R] != 0 || !isfinite(O.bb)) ? RGDBEK_ERR_NONFINITE
                                                                : kStatusRunning;
    }
    __syncthreads();
    if (O.verdict != kStatusRunning) return SolveOut<V>{O.verdict, P.k0, V(NAN), V(NAN)};
    if (lead) st_release_u64(&C->lk_tready, lk_enc(call, 0));

    // Stopping test of x_k (the rule of solve_body) from ||t_k||^2 (O.tt) and
    // the column team's ||A^T t_k||^2 and eps^z flag (link slots sh, sb).
    const auto verdict_of = [&](long long k, int sh, int sb) -> int {
        if (threadIdx.x == 0) {
            if (k == P.k0) O.atb2 = (V)__ldcg(&C->lk_gg);
            const V hh = (V)__ldcg(&C->lk_hh[sh]);
            const long long badc = __ldcg(&C->lk_badc[sb]);
            O.rel = O.bb > V(0) ? vsqrt(O.tt / O.bb) : V(0);
            O.nrm = O.atb2 > V(0) ? vsqrt(hh / O.atb2) : V(0);
            const V meas = P.stop_rule == RGDBEK_STOP_REL_RES
                               ? O.rel
                               : (P.stop_rule == RGDBEK_STOP_RSE ? O.rel * O.rel : O.nrm);
            if (k == P.k0 || meas < O.best) {
                O.best = meas;
                O.kbest = k;
            }
            int v = kStatusRunning;
            if (badc != 0 || !isfinite(hh) || !isfinite(O.tt)) v = RGDBEK_ERR_NONFINITE;
            else if (stop_rule_holds(P.stop_rule, P.tol, O.rel, O.nrm)) v = RGDBEK_OK;
            else if (k >= P.max_iter) v = RGDBEK_NOT_CONVERGED;
            else if (ld_volatile_i32(&C->stop_req)) v = RGDBEK_ERR_TIMEOUT;
            else if (kF32 && k - O.kbest >= kInnerStallIters) v = RGDBEK_NOT_CONVERGED;
            O.verdict = v;
        }
        __syncthreads();
        return O.verdict;
    };

    for (long long k = P.k0;; ++k) {
        const long long j = k - P.k0;
        const int sl = (int)(j & 1), sn = (int)((j + 1) & 1);
        // the time budget, checked before the barrier of the r phase: every CTA
        // reads the stop request at the test of x_k, after that barrier
        if (lead && j >= 1 && P.time_budget_ns > 0.0 &&
            (double)(globaltimer_ns() - S.t_start) > P.time_budget_ns)
            C->stop_req = 1;
        if (j == 0 || k >= P.max_iter) {
            // x_{k0}: its test needs column pass k0 only; at the cap the test
            // stops for certain, so it is taken before a row step is spent
            X_WAIT(lk_colpass, lk_enc(call, j == 0 ? 1 : j + 2));
            mark(S, PH_COL);
            const int v = verdict_of(k, j == 0 ? 0 : sn, sl);
            if (v != kStatusRunning) return SolveOut<V>{v, k, O.rel, O.nrm};
        }

        // ---- r = t_k - z_{k+1} and the row weights, once z_{k+1} is written
        X_WAIT(lk_zready, lk_enc(call, j + 1));
        mark(S, PH_COL);
        const long long nU = __ldcg(&C->lk_nu[sl]), nnzU = __ldcg(&C->lk_nnzu[sl]);
        const int stepsU = (int)__ldcg(&C->lk_stepsu[sl]);
        const bool rec_u = !S.tr_full && S.tr_off + nU <= P.tr_list_cap;
        if (rec_u) {
            const int *ul = ulists[sl];
            for (long long p = tthread(P); p < nU; p += tthreads(P))
                P.tr_lists[S.tr_off + p] = __ldcg(ul + p);
        }
        phase_zupdate<V, 2>(P, false, 1, bs);
        X_SYNC(DS(D_EMAX_R), DS(D_EMAX_R), DS(I_BAD_R));
        if (lead) st_release_u64(&C->lk_zused, lk_enc(call, j + 1));
        mark(S, PH_ZUPD);
        if (P.tr_r && k < P.tr_vec_cap)  // trace: the row residual r = b - z_{k+1} - A x_k
            for (long long i = tthread(P); i < P.m; i += tthreads(P))
                P.tr_r[k * P.m + i] = (double)P.r[i];
        if (threadIdx.x == 0) O.emax_r = red[D_EMAX_R];
        __syncthreads();
        if (S.red_i[I_BAD_R] != 0) {
            // the test of x_k comes first, as in solve_body
            if (j >= 1) {
                X_WAIT(lk_colpass, lk_enc(call, j + 2));
                const int v = verdict_of(k, sn, sl);
                if (v != kStatusRunning) return SolveOut<V>{v, k, O.rel, O.nrm};
            }
            return SolveOut<V>{RGDBEK_ERR_NONFINITE, k, O.rel, O.nrm};
        }

        // ---- row block J_k, xt = x_k + (A^J)^+ r_J
        BlockInfo J{0, 0, 0, 1};
        bool rec_j = false;
        if (O.emax_r > V(0)) {
            if (row_block<V>(P, S, dsmem, k, rec_u, S.tr_off + nU, J) < 0)
                return SolveOut<V>{kAbandoned, k, V(0), V(0)};
            rec_j = rec_u && S.tr_off + nU + J.n <= P.tr_list_cap;
        }

        // ---- stopping test of x_k (column pass k + 1 holds ||A^T t_k||^2)
        if (j >= 1) {
            X_WAIT(lk_colpass, lk_enc(call, j + 2));
            mark(S, PH_COL);
            const int v = verdict_of(k, sn, sl);
            if (v != kStatusRunning) return SolveOut<V>{v, k, O.rel, O.nrm};
        }

        // ---- iteration k stands: its counters and trace
        const long long nJ = J.n, nnzJ = J.nnz;
        const int stepsJ = J.steps;
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
        if (lead && P.tr_counts && k < P.tr_count_cap) {
            P.tr_counts[4 * k + 0] = nU;
            P.tr_counts[4 * k + 1] = nJ;
            P.tr_counts[4 * k + 2] = stepsU;
            P.tr_counts[4 * k + 3] = stepsJ;
        }
        if (!S.tr_full) {
            const bool ok = rec_u && (nJ == 0 || rec_j) && S.tr_off + nU + nJ <= P.tr_list_cap;
            __syncthreads();
            if (threadIdx.x == 0) {
                if (ok) S.tr_off += nU + nJ;
                else S.tr_full = 1;
            }
            __syncthreads();
        }
        if (nU == 0 && nJ == 0) return SolveOut<V>{RGDBEK_OK, k, O.rel, O.nrm};

        // ---- t_{k+1} = b - A x_{k+1}, x_{k+1} adopted (the column pass that
        // reads t_k has been waited for above)
        phase_residual(P, bs, true);
        X_SYNC(DS(D_TT), 0, 0);
        if (lead) st_release_u64(&C->lk_tready, lk_enc(call, j + 1));
        mark(S, PH_RESID);
        if (threadIdx.x == 0) O.tt = red[D_TT];
    }
}

#undef X_SYNC
#undef X_WAIT

#define Z_SYNC(dm, dx, im)                                                        \
    do {                                                                          \
        if (!sync_collect(P, S, (dm), (dx), (im), red)) return -1;                \
    } while (0)
#define Z_WAIT(word, target)                                                      \
    do {                                                                          \
        const int r_ = link_wait(C, &C->word, (target), call);                    \
        if (r_ != 0) return r_;                                                   \
    } while (0)

// The column team's part of a two-team solve.  Returns 1 once the row team
// has finished, -1 if a barrier or wait was abandoned.
template <typename V>
__device__ __forceinline__ int zchain_body(const ParamsT<V> &P, SolveSmem &S,
                                           unsigned char *dsmem, unsigned long long call,
                                           int *const *ulists) {
    BlockScratch &bs = S.bs;
    OuterStateT<V> &O = S.o<V>();
    V *const red = S.red<V>();
    const int nct = tsize(P);
    Ctrl *const C = P.ctrl;
    const bool lead = trank(P) == 0 && threadIdx.x == 0;

    // ---- z_0 = b, ||z_0||^2
    {
        V zz = V(0);
        for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
            const V bi = ld_rhs(P.b + i);
            P.z[2 * i] = bi;
            zz = vfma(bi, bi, zz);
        }
        zz = block_sum(zz, bs);
        if (threadIdx.x == 0) P.pd[D_ZZ * nct + trank(P)] = zz;
    }
    Z_SYNC(DS(D_ZZ), 0, 0);
    if (threadIdx.x == 0) {
        O.zz = red[D_ZZ];
        O.itol = (V)P.inner_tol;
    }
    __syncthreads();
    mark(S, PH_SETUP);

    for (long long k = P.k0;; ++k) {
        const long long j = k - P.k0;
        const int sl = (int)(j & 1);
        // ---- g = A^T z_k, eps^z, and h = A^T t for the row team's test:
        // t_{k0} at j = 0, t_{k-1} from j = 2 on (none is due at j = 1)
        const bool with_h = j != 1;
        if (with_h) Z_WAIT(lk_tready, lk_enc(call, j == 0 ? 0 : j - 1));
        phase_col(P, bs, false, with_h);
        // rank 0 reports whether the row team has finished: all CTAs then
        // leave after the barrier together
        if (threadIdx.x == 0)
            P.pi[I_STOP * nct + trank(P)] =
                (trank(P) == 0 && ld_acquire_u64(&C->lk_stop) >= call) ? 1 : 0;
        Z_SYNC(DS(D_EMAX_C) | DS(D_HH) | DS(D_GG), DS(D_EMAX_C), DS(I_BAD_C) | DS(I_STOP));
        mark(S, PH_COL);
        if (S.red_i[I_STOP] != 0) return 1;
        if (P.tr_g && k < P.tr_vec_cap)  // trace: g = A^T z_k
            for (long long c = tthread(P); c < P.n; c += tthreads(P))
                P.tr_g[k * P.n + c] = (double)P.g[c];
        if (lead) {
            C->lk_hh[sl] = (double)red[D_HH];
            C->lk_badc[sl] = S.red_i[I_BAD_C];
            if (j == 0) C->lk_gg = (double)red[D_GG];  // g = A^T z_0 = A^T b
            st_release_u64(&C->lk_colpass, lk_enc(call, j + 1));
        }
        if (threadIdx.x == 0) O.emax_c = red[D_EMAX_C];
        __syncthreads();

        // ---- column block U_k
        BlockInfo U{0, 0, 0, 1};
        if (O.emax_c > V(0)) {
            if (col_block<V>(P, S, dsmem, k, ulists[sl], false, 0, U) < 0) return -1;
        }

        // ---- z_{k+1} = z_k - A_U y, once the row team has read z_k
        if (j >= 1) Z_WAIT(lk_zused, lk_enc(call, j));
        phase_zupdate<V, 1>(P, U.n > 0, U.lanes, bs);
        Z_SYNC(DS(D_ZZ), 0, 0);
        mark(S, PH_ZUPD);
        if (threadIdx.x == 0) O.zz = red[D_ZZ];
        if (lead) {
            C->lk_nu[sl] = U.n;
            C->lk_nnzu[sl] = U.nnz;
            C->lk_stepsu[sl] = U.steps;
            st_release_u64(&C->lk_zready, lk_enc(call, j + 1));
        }
        __syncthreads();
    }
}

#undef Z_SYNC
#undef Z_WAIT

// A solve with P.zteam > 0, called by every CTA of the grid (after
// enter_team and init_solve_smem): the two teams of the two-team schedule
// run their parts on their own copies of the parameters (in shared memory;
// the column team with its own work buffers and partials), then every CTA
// learns the row team's result after a whole-grid barrier (the refinement
// loop goes on with the whole grid).
template <typename V>
__device__ __forceinline__ SolveOut<V> solve_split(const ParamsT<V> &P, SolveSmem &S,
                                                   unsigned char *dsmem) {
    __shared__ ParamsT<V> SP;
    __shared__ unsigned long long s_call;
    const int tz = P.zteam, tx = P.team - P.zteam;
    const bool isZ = (int)blockIdx.x >= tx;
    copy_params(SP, P);
    if (threadIdx.x == 0) {
        SP.zteam = 0;
        SP.team = isZ ? tz : tx;
        if (isZ) {
            SP.bar = &P.ctrl->bar_z;
            SP.pd = P.pd_z;
            SP.pi = P.pi_z;
            SP.Q = P.Q_z;
            SP.flag = P.flag_z;
            SP.uu = P.uu_z;
            SP.vv = P.vv_z;
            SP.ww = P.ww_z;
            SP.dots = P.dots_z;
            SP.dots2 = P.dots2_z;
        } else {
            SP.bar = &P.ctrl->bar_x;
        }
        s_team_rank = isZ ? (int)blockIdx.x - tx : (int)blockIdx.x;
        S.leader = s_team_rank == 0;
        S.tlast = globaltimer_ns();
        const unsigned long long e = S.epoch;
        S.epoch = S.epoch_sub;
        S.epoch_sub = e;
        s_call = ++S.split_calls;
    }
    __syncthreads();
    int *const ulists[2] = {P.ulist, P.ulist2};
    Ctrl *const C = P.ctrl;
    if (isZ) {
        zchain_body<V>(SP, S, dsmem, s_call, ulists);
        if (S.leader && threadIdx.x == 0)
            for (int i = 0; i < RGDBEK_NUM_PHASES; ++i) C->zphase_ns[i] = S.tphase[i];
    } else {
        const SolveOut<V> o = xchain_body<V>(SP, S, dsmem, s_call, ulists);
        if (S.leader && threadIdx.x == 0) {
            C->lk_res_k = o.k;
            C->lk_res_status = o.status;
            C->lk_res_rel = (double)o.rel;
            C->lk_res_nrm = (double)o.nrm;
            st_release_u64(&C->lk_stop, s_call);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_team_rank = (int)(blockIdx.x % (unsigned)P.team);
        S.leader = s_team_rank == 0;
        const unsigned long long e = S.epoch;
        S.epoch = S.epoch_sub;
        S.epoch_sub = e;
    }
    __syncthreads();
    if (!grid_barrier(C, S.epoch, P.team)) return SolveOut<V>{kAbandoned, 0, V(0), V(0)};
    return SolveOut<V>{__ldcg(&C->lk_res_status), __ldcg(&C->lk_res_k), (V)__ldcg(&C->lk_res_rel),
                       (V)__ldcg(&C->lk_res_nrm)};
}

// One solve by the whole grid: two-team schedule when P.zteam > 0.
template <typename V>
__device__ __forceinline__ SolveOut<V> solve_any(const ParamsT<V> &P, SolveSmem &S,
                                                 unsigned char *dsmem) {
    if (P.zteam > 0) return solve_split<V>(P, S, dsmem);
    return solve_body<V>(P, S, dsmem);
}

// ---------------------------------------------------------------------------
// RGDBEK_PRECISION_FP32_INNER: FP32 inner RGDBEK wrapped in FP64 iterative
// refinement.  Every update of x lies in range(A^T), so A^+ (b - A x) = x* - x
// for x* = A^+ b (Theorem 2.3's limit): solving A d = t, t = b - A x, for its
// minimum-norm least-squares solution and adding d to x is one exact step to
// x*.  The refinement loop does that with an approximate d from Algorithm 1
// run in FP32 on A's values rounded to float, with t scaled to unit norm:
//   t = b - A x (FP64 CSR pass), ||A^T t|| (FP64 CSC pass), stopping test
//   d = FP32 RGDBEK(A_f32, t / ||t||) to relative measure tau_j
//   x += ||t|| d (FP64)
// tau_j = clamp(0.5 tol / measure_j, kRefineTolMin, 0.5), so the last inner
// solve does no more than the outer tolerance needs; an inner solve also
// stops at its FP32 rounding floor (kInnerStallIters without progress).
// The rounding of t / ||t|| to float limits what an FP32 step can resolve:
// for a least-squares problem t is dominated by the residual r* = b - A x*,
// and the normal-equation measure of its FP32 image cannot fall much below
// about kappa(A) u_32 ||r*|| / ||b||.  When an FP32 step no longer halves the
// FP64 measure, the remaining steps solve the same system A d = t / ||t||
// with the FP64 iteration: its z starts at t, within a small multiple of the
// final r*, so those solves are short.  The outer measures, the stopping test
// and x are FP64 throughout.
// ---------------------------------------------------------------------------
constexpr double kRefineTolMin = RGDBEK_FP32_REFINE_TOL_MIN;
constexpr double kRefineTolMax = 0.5;
// refinement steps in a row without halving the outer measure after which the
// solve stops with NOT_CONVERGED (with FP64 inner solves: no more progress)
constexpr int kRefineStallSteps = 3;

// t_i = b_i - (A x)_i over the CSR rows in FP64, into t (m).  Partial: ||t||^2.
__device__ __forceinline__ void phase_outer_residual(const Params &P, double *t, BlockScratch &bs) {
    const Grp G(P.lpr);
    double tt = 0.0;
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        double s = 0.0;
        if (i < P.m)
            s = lane_dot<true>(__ldg(P.rp + i) + G.sl, __ldg(P.rp + i + 1), G.L, P.ci, P.av,
                               [&](int j) { return P.x[j]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) {
            const double ti = __ldg(P.b + i) - s;
            t[i] = ti;
            tt = fma(ti, ti, tt);
        }
    }
    tt = block_sum(tt, bs);
    if (threadIdx.x == 0) P.pd[D_TT * tsize(P) + trank(P)] = tt;
}

// ||A^T v||^2 over the CSC columns in FP64 (the vector itself is not kept),
// into partial slot `slot`.
__device__ __forceinline__ void phase_outer_normal(const Params &P, const double *v, int slot,
                                                   BlockScratch &bs) {
    const Grp G(P.lpc);
    double hh = 0.0;
    for (long long base = twarp(P) * G.rpw; base < P.n; base += twarps(P) * G.rpw) {
        const long long j = base + G.sub;
        double s = 0.0;
        if (j < P.n)
            s = lane_dot<true>(__ldg(P.cp + j) + G.sl, __ldg(P.cp + j + 1), G.L, P.ri, P.cv,
                               [&](int i) { return v[i]; });
        s = group_sum(s, G.L);
        if (j < P.n && G.sl == 0) hh = fma(s, s, hh);
    }
    hh = block_sum(hh, bs);
    if (threadIdx.x == 0) P.pd[slot * tsize(P) + trank(P)] = hh;
}

// The refinement loop by the CTAs of a team (after enter_team and
// init_solve_smem).  P: the FP64 view (A in FP64, b, x, the refinement
// buffers ref_t / ref_b / ref_x and the FP64 work vectors for FP64 inner
// solves); F: the FP32 view of the same system (A_f32, float work vectors, its
// own right-hand side F.b written here, solution F.x).
// kSplit: the inner solves may use the two-team schedule (single solves);
// the batched kernel runs one team per system and compiles without it.
template <bool kSplit = true>
__device__ __forceinline__ void refine_body(const Params &P, const ParamsF &F, SolveSmem &S,
                                            unsigned char *dsmem) {
    BlockScratch &bs = S.bs;
    RefineState &R = S.ref;
    double *const t64 = P.ref_t;  // the FP64 residual b - A x
    // the parameters of the inner solves (their tolerance and first iteration
    // set per solve), in shared memory
    __shared__ ParamsF s_fj;
    __shared__ Params s_pj;
    copy_params(s_fj, F);
    copy_params(s_pj, P);
    double *const red = S.red_d;
#define RGD_SYNC64(dm, im)                                                         \
    do {                                                                           \
        if (!sync_collect(P, S, (dm), 0u, (im), red)) return;                      \
    } while (0)

    // ---- x_0 (0 or the caller's), ||b||^2, non-finite inputs
    {
        double bb = 0.0;
        long long bad = 0;
        for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
            const double bi = __ldg(P.b + i);
            bb = fma(bi, bi, bb);
            if (!isfinite(bi)) bad = 1;
        }
        for (long long j = tthread(P); j < P.n; j += tthreads(P)) {
            const double x0 = P.warm ? P.x[j] : 0.0;
            if (!isfinite(x0)) bad = 1;
            P.x[j] = x0;
        }
        bb = block_sum(bb, bs);
        bad = block_sum(bad, bs);
        if (threadIdx.x == 0) {
            P.pd[D_BB * tsize(P) + trank(P)] = bb;
            P.pi[I_BAD_R * tsize(P) + trank(P)] = bad;
        }
    }
    RGD_SYNC64(DS(D_BB), DS(I_BAD_R));
    if (threadIdx.x == 0) {
        R.bb = red[D_BB];
        R.refinements = 0;
        R.best = 0.0;
        R.kbest = 0;
        R.fp64 = 0;
        R.verdict = (S.red_i[I_BAD_R] != 0 || !isfinite(R.bb)) ? RGDBEK_ERR_NONFINITE
                                                               : kStatusRunning;
    }
    __syncthreads();
    if (R.verdict != kStatusRunning) {
        finish(P, R.verdict, 0, NAN, NAN, 0, S);
        return;
    }
    // ||A^T b||^2 (the reference of the normal-equation measure) and t_0 = b - A x_0
    phase_outer_normal(P, P.b, D_GG, bs);
    phase_outer_residual(P, t64, bs);
    RGD_SYNC64(DS(D_GG) | DS(D_TT), 0);
    if (threadIdx.x == 0) {
        R.atb2 = red[D_GG];
        R.tt = red[D_TT];
    }
    // the time budget is checked by rank 0 before the barrier that ends each
    // refinement step, so that every CTA reads the same stop request after it
    const auto check_budget = [&]() {
        if (trank(P) == 0 && threadIdx.x == 0 && P.time_budget_ns > 0.0 &&
            (double)(globaltimer_ns() - S.t_start) > P.time_budget_ns)
            P.ctrl->stop_req = 1;
    };
    phase_outer_normal(P, t64, D_HH, bs);
    check_budget();
    RGD_SYNC64(DS(D_HH), 0);
    if (threadIdx.x == 0) R.hh = red[D_HH];
    mark(S, PH_REFINE);

    long long k = 0;  // outer iterations of all inner solves so far
    for (;;) {
        if (threadIdx.x == 0) {
            R.rel = R.bb > 0.0 ? sqrt(R.tt / R.bb) : 0.0;
            R.nrm = R.atb2 > 0.0 ? sqrt(R.hh / R.atb2) : 0.0;
            const double meas = P.stop_rule == RGDBEK_STOP_REL_RES
                                    ? R.rel
                                    : (P.stop_rule == RGDBEK_STOP_RSE ? R.rel * R.rel : R.nrm);
            if (R.refinements == 0 || meas <= 0.5 * R.best) {
                R.best = meas;
                R.kbest = R.refinements;
            } else if (!R.fp64) {
                // an FP32 step that did not halve the measure: FP32 has reached
                // its floor, the next steps run in FP64
                R.fp64 = 1;
                R.kbest = R.refinements;
            }
            int v = kStatusRunning;
            if (!isfinite(R.tt) || !isfinite(R.hh)) v = RGDBEK_ERR_NONFINITE;
            else if (stop_rule_holds(P.stop_rule, P.tol, R.rel, R.nrm)) v = RGDBEK_OK;
            else if (k >= P.max_iter) v = RGDBEK_NOT_CONVERGED;
            else if (ld_volatile_i32(&P.ctrl->stop_req)) v = RGDBEK_ERR_TIMEOUT;
            else if (R.refinements - R.kbest >= kRefineStallSteps) v = RGDBEK_NOT_CONVERGED;
            R.verdict = v;
            // the target of the next inner solve, and the scaling of its rhs
            double tau = meas > 0.0 ? 0.5 * P.tol / meas : kRefineTolMax;
            R.itol = fmin(kRefineTolMax, fmax(R.fp64 ? 0.0 : kRefineTolMin, tau));
            R.scale = sqrt(R.tt);
            R.inv_scale = R.scale > 0.0 ? 1.0 / R.scale : 0.0;
        }
        __syncthreads();
        if (R.verdict != kStatusRunning) {
            finish(P, R.verdict, k, R.rel, R.nrm, R.refinements, S);
            return;
        }
        const bool fp64 = R.fp64 != 0;
        // ---- the inner right-hand side t / ||t|| (FP32, or FP64 for FP64 steps)
        {
            const double is = R.inv_scale;
            float *bf = const_cast<float *>(F.b);
            for (long long i = tthread(P); i < P.m; i += tthreads(P)) {
                const double v = t64[i] * is;
                if (fp64) P.ref_b[i] = v;
                else bf[i] = (float)v;
            }
        }
        if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return;
        mark(S, PH_REFINE);
        int ist;
        if (!fp64) {
            // ---- d = FP32 RGDBEK(A_f32, t / ||t||)
            if (threadIdx.x == 0) {
                s_fj.tol = R.itol;
                s_fj.k0 = k;
            }
            __syncthreads();
            SolveOut<float> o;
            if constexpr (kSplit) o = solve_any<float>(s_fj, S, dsmem);
            else o = solve_body<float>(s_fj, S, dsmem);
            ist = o.status;
            k = o.k;
        } else {
            // ---- d = FP64 RGDBEK(A, t / ||t||)
            if (threadIdx.x == 0) {
                s_pj.b = P.ref_b;
                s_pj.x = P.ref_x;
                s_pj.warm = 0;
                s_pj.tol = R.itol;
                s_pj.k0 = k;
            }
            __syncthreads();
            SolveOut<double> o;
            if constexpr (kSplit) o = solve_any<double>(s_pj, S, dsmem);
            else o = solve_body<double>(s_pj, S, dsmem);
            ist = o.status;
            k = o.k;
        }
        if (ist == kAbandoned) return;
        if (ist < 0) {
            // NONFINITE inside the inner solve, or TIMEOUT between its iterations
            finish(P, ist, k, R.rel, R.nrm, R.refinements, S);
            return;
        }
        // ---- x += ||t|| d (FP64), then t = b - A x and ||A^T t||
        {
            const double sc = R.scale;
            for (long long j = tthread(P); j < P.n; j += tthreads(P))
                P.x[j] = fma(sc, fp64 ? P.ref_x[j] : (double)F.x[j], P.x[j]);
        }
        if (!grid_barrier(P.ctrl, S.epoch, tsize(P))) return;
        phase_outer_residual(P, t64, bs);
        RGD_SYNC64(DS(D_TT), 0);
        if (threadIdx.x == 0) R.tt = red[D_TT];
        phase_outer_normal(P, t64, D_HH, bs);
        check_budget();
        RGD_SYNC64(DS(D_HH), 0);
        if (threadIdx.x == 0) {
            R.hh = red[D_HH];
            ++R.refinements;
        }
        mark(S, PH_REFINE);
    }
#undef RGD_SYNC64
}

// A single solve: the whole grid is one team.  NT: launch bound (threads).
template <int NT>
__global__ void __launch_bounds__(NT, 1) solve_kernel(const Params P) {
    __shared__ SolveSmem S;
    extern __shared__ __align__(16) unsigned char dsmem[];
    enter_team(P);
    init_solve_smem(S, P);
    const SolveOut<double> o = solve_any<double>(P, S, dsmem);
    if (o.status != kAbandoned) finish(P, o.status, o.k, o.rel, o.nrm, 0, S);
}

// The FP32 form: FP64 refinement around FP32 inner solves, the whole grid one team.
template <int NT>
__global__ void __launch_bounds__(NT, 1) refine_kernel(const Params P, const ParamsF F) {
    __shared__ SolveSmem S;
    extern __shared__ __align__(16) unsigned char dsmem[];
    enter_team(P);
    init_solve_smem(S, P);
    refine_body<true>(P, F, S, dsmem);
}

// Many independent systems in one cooperative launch: the grid is cut into
// teams of `team` consecutive CTAs; team t solves the systems
// plan[t * stride], plan[t * stride + 1], ... (ending at -1) one after
// another, each to its own stopping rule (its parameters and control block in
// sys[]), with barriers among the team's CTAs only.
template <bool F32, int NT>
__global__ void __launch_bounds__(NT, 1)
    batched_solve_kernel(const SysPair *sys, const int *plan, int stride, int team) {
    __shared__ SolveSmem S;
    __shared__ Params SP;
    __shared__ ParamsF SF;
    extern __shared__ __align__(16) unsigned char dsmem[];
    const int t = (int)(blockIdx.x / (unsigned)team);
    for (int q = 0; q < stride; ++q) {
        const int i = plan[(long long)t * stride + q];
        if (i < 0) break;
        {
            const int *src = reinterpret_cast<const int *>(&sys[i].p);
            int *dst = reinterpret_cast<int *>(&SP);
            for (int w = threadIdx.x; w < (int)(sizeof(Params) / sizeof(int)); w += blockDim.x)
                dst[w] = src[w];
            if (F32) {
                const int *sf = reinterpret_cast<const int *>(&sys[i].f);
                int *df = reinterpret_cast<int *>(&SF);
                for (int w = threadIdx.x; w < (int)(sizeof(ParamsF) / sizeof(int));
                     w += blockDim.x)
                    df[w] = sf[w];
            }
        }
        __syncthreads();
        enter_team(SP);
        init_solve_smem(S, SP);
        if constexpr (F32) {
            refine_body<false>(SP, SF, S, dsmem);
        } else {
            const SolveOut<double> o = solve_body<double>(SP, S, dsmem);
            if (o.status != kAbandoned) finish(SP, o.status, o.k, o.rel, o.nrm, 0, S);
        }
        __syncthreads();
    }
}

}  // namespace rgd
