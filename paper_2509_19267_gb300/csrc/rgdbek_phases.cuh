// Phases of one RGDBEK outer iteration (Algorithm 1) as device functions.
//
// The persistent solve kernel runs them back to back with a grid barrier
// between phases; the component kernels (spmv, weights, sampler) run the
// same functions so that the component entry points test the solver's code.
//
// Work distribution:
//  * sparse rows/columns: a group of L lanes (power of two) per row/column,
//    warp-strided over the grid; the group sums in a fixed xor-tree order.
//  * scans (quantised weights, compaction, block extraction): the index range
//    is cut into gridDim.x contiguous chunks, one per CTA, each scanned in
//    thread order; CTA offsets come from an exclusive prefix of the per-CTA
//    totals, so every scan is exact (integers) and deterministic.
//  * reductions: per-CTA partials, then every CTA reduces the partials in
//    the same order, so all CTAs take identical branch decisions.
//
// Buffers that the kernel writes are read with ordinary loads (coherent after
// the grid barrier); only A, its norms and b, which never change during a
// solve, go through the read-only path.
#pragma once

#include "rgdbek_device.cuh"

namespace rgd {

struct Params {
    long long m, n, nnz;
    // A in CSR and CSC form, squared row/column norms
    const long long *__restrict__ rp;
    const int *__restrict__ ci;
    const double *__restrict__ av;
    const long long *__restrict__ cp;
    const int *__restrict__ ri;
    const double *__restrict__ cv;
    const double *__restrict__ rn2;
    const double *__restrict__ cn2;
    // right-hand side and solution
    const double *b;
    double *x;
    // work vectors: z (m) and t = b - A x (m), stored as (z_i, t_i) pairs
    // (z_i at z[2 i], t_i at t[2 i] = z[2 i + 1]: the column pass gathers both
    // with one 16-byte load), r (m), g = A^T z (n), weights, LSQR vectors u (m),
    // v, w, y (n), the row-step solution dx (n) and the trial iterate
    // xt = x + dx (n) that the next column pass adopts
    double *z, *t, *r, *g, *epsc, *epsr, *uu, *vv, *ww, *yy, *dx, *xt;
    unsigned long long *Q;  // chunk-local inclusive prefix of quantised weights
    unsigned char *flag;    // drawn / selected marks
    int *colpos, *rowpos;   // position of a column in U / of a row in J, or -1
    int *ulist, *jlist;     // U_k and J_k, ascending
    int *srn;               // A_U as CSR over all m rows: row i holds srn[i] entries
    int *sci;               // at sci/sav[rp[i] ..], columns renumbered 0..|U|-1
    double *sav;
    int *scn;               // A^J as CSC over all n columns: column j holds scn[j]
    int *sri;               // entries at sri/scv[cp[j] ..], rows renumbered 0..|J|-1
    double *scv;
    double *dots, *dots2;   // per-line dot products of the inner solve when a CTA's
                            // chunk does not fit in shared memory (max(m, n) each)
    double *pd;             // double partials [D_NSLOTS][grid]
    long long *pi;          // int64 partials [I_NSLOTS][grid]
    Ctrl *ctrl;
    long long *tr_counts;
    long long tr_count_cap;
    int *tr_lists;
    long long tr_list_cap;
    double *tr_g, *tr_r;    // per-iteration copies of g = A^T z_k and of r (or null)
    long long tr_vec_cap;   // iterations those buffers hold
    // options
    double tol, inner_tol, eta_col, eta_row;
    double inner_adapt;     // > 0: per-iteration inner tolerance tied to the outer residual
    double time_budget_ns;
    long long max_iter, s_col, s_row;
    unsigned long long seed, sysid;
    int inner_max, stop_rule, selection;
    int fp32_inner;         // inner LSQR products in FP32 (Kahan dots)
    int team;               // CTAs that work on this system (rank = blockIdx.x % team)
    int warm;               // x holds x_0 on entry (else x_0 = 0)
    float *vv32, *uu32;     // float copies of the LSQR vectors v~, u~ (fp32_inner)
    double *vvs, *dsc;      // column step: D v~ and D = 1/||A_j|| per column of U
    double *yh;             // column step: y^ of the scaled block (global fallback)
    double *uus, *dsr;      // row step: D u~ and D = 1/||A^(i)|| per row of J
    int tpr, tpc;           // lanes per row (CSR) / column (CSC) of A, FP64 passes
    int ipr, ipc;           // lanes per row / column of A, integer passes
    long long dsmem_bytes;  // dynamic shared memory per CTA of the solve kernel
};

// Lane geometry of a group of L lanes inside a warp.
struct Grp {
    int L, sub, sl, rpw, lead;
    unsigned gmask_shift;
    __device__ __forceinline__ explicit Grp(int L_) : L(L_) {
        const int lane = threadIdx.x & 31;
        const int lg = __ffs(L) - 1;
        sub = lane >> lg;
        sl = lane & (L - 1);
        rpw = 32 >> lg;
        lead = sub << lg;
        gmask_shift = (unsigned)lead;
    }
    // this group's bits of a warp ballot
    __device__ __forceinline__ unsigned mine(unsigned bal) const {
        return L == 32 ? bal : (bal >> gmask_shift) & ((1u << L) - 1u);
    }
};

__device__ __forceinline__ long long gwarp() {
    return (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
}
__device__ __forceinline__ long long nwarps() {
    return (long long)gridDim.x * (blockDim.x >> 5);
}
__device__ __forceinline__ long long gthread() {
    return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long nthreads() {
    return (long long)gridDim.x * blockDim.x;
}

// The CTAs that solve one system form a team: the whole grid for a single
// solve, `team` consecutive CTAs of a batched launch.  Phase code indexes by
// the CTA's rank in its team and by the team's size.
// The rank is computed once per kernel by enter_team (every kernel that runs
// phase code calls it first) and kept in shared memory.
__shared__ int s_team_rank;
__device__ __forceinline__ void enter_team(const Params &P) {
    if (threadIdx.x == 0) s_team_rank = (int)(blockIdx.x % (unsigned)P.team);
    __syncthreads();
}
__device__ __forceinline__ int trank(const Params &P) {
    (void)P;
    // re-read at each use (like a special register) rather than held live
    return *reinterpret_cast<volatile int *>(&s_team_rank);
}
__device__ __forceinline__ int tsize(const Params &P) { return P.team; }
__device__ __forceinline__ long long twarp(const Params &P) {
    return (long long)trank(P) * (blockDim.x >> 5) + (threadIdx.x >> 5);
}
__device__ __forceinline__ long long twarps(const Params &P) {
    return (long long)P.team * (blockDim.x >> 5);
}
__device__ __forceinline__ long long tthread(const Params &P) {
    return (long long)trank(P) * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long tthreads(const Params &P) {
    return (long long)P.team * blockDim.x;
}

// Loads through the read-only path (RO) for arrays that never change during
// a kernel, ordinary loads otherwise.
template <bool RO, typename T>
__device__ __forceinline__ T ldx(const T *p) {
    if constexpr (RO) return __ldg(p);
    else return *p;
}

// This lane's share of sum_e val[e] * f(idx[e]) over e = e, e + L, e + 2L, ...
// below e1, accumulated in exactly that order.  Four entries are handled per
// trip with all their loads issued before the multiply-adds, so four
// independent index/value loads and four gathers are in flight per lane.
template <bool RO, typename F>
__device__ __forceinline__ double lane_dot(long long e, long long e1, long long L, const int *idx,
                                           const double *val, F f) {
    double s = 0.0;
    for (; e < e1; e += 4 * L) {
        const bool v1 = e + L < e1, v2 = e + 2 * L < e1, v3 = e + 3 * L < e1;
        const int i0 = ldx<RO>(idx + e);
        const int i1 = v1 ? ldx<RO>(idx + e + L) : 0;
        const int i2 = v2 ? ldx<RO>(idx + e + 2 * L) : 0;
        const int i3 = v3 ? ldx<RO>(idx + e + 3 * L) : 0;
        const double a0 = ldx<RO>(val + e);
        const double a1 = v1 ? ldx<RO>(val + e + L) : 0.0;
        const double a2 = v2 ? ldx<RO>(val + e + 2 * L) : 0.0;
        const double a3 = v3 ? ldx<RO>(val + e + 3 * L) : 0.0;
        const double x0 = f(i0);
        const double x1 = v1 ? f(i1) : 0.0;
        const double x2 = v2 ? f(i2) : 0.0;
        const double x3 = v3 ? f(i3) : 0.0;
        s = fma(a0, x0, s);
        if (v1) s = fma(a1, x1, s);
        if (v2) s = fma(a2, x2, s);
        if (v3) s = fma(a3, x3, s);
    }
    return s;
}

// Two dot products sharing the index/value loads (A^T z and A^T t): the two
// vectors are stored as (z_i, t_i) pairs, so one 16-byte gather serves both.
__device__ __forceinline__ void lane_dot2(long long e, long long e1, long long L, const int *idx,
                                          const double *val, const double2 *zt, double &sf,
                                          double &sg) {
    for (; e < e1; e += 4 * L) {
        const bool v1 = e + L < e1, v2 = e + 2 * L < e1, v3 = e + 3 * L < e1;
        const int i0 = __ldg(idx + e);
        const int i1 = v1 ? __ldg(idx + e + L) : 0;
        const int i2 = v2 ? __ldg(idx + e + 2 * L) : 0;
        const int i3 = v3 ? __ldg(idx + e + 3 * L) : 0;
        const double a0 = __ldg(val + e);
        const double a1 = v1 ? __ldg(val + e + L) : 0.0;
        const double a2 = v2 ? __ldg(val + e + 2 * L) : 0.0;
        const double a3 = v3 ? __ldg(val + e + 3 * L) : 0.0;
        const double2 p0 = zt[i0];
        const double2 p1 = v1 ? zt[i1] : make_double2(0.0, 0.0);
        const double2 p2 = v2 ? zt[i2] : make_double2(0.0, 0.0);
        const double2 p3 = v3 ? zt[i3] : make_double2(0.0, 0.0);
        sf = fma(a0, p0.x, sf);
        sg = fma(a0, p0.y, sg);
        if (v1) { sf = fma(a1, p1.x, sf); sg = fma(a1, p1.y, sg); }
        if (v2) { sf = fma(a2, p2.x, sf); sg = fma(a2, p2.y, sg); }
        if (v3) { sf = fma(a3, p3.x, sf); sg = fma(a3, p3.y, sg); }
    }
}

// Number of entries e = e, e + L, ... below e1 with map[idx[e]] >= 0.
__device__ __forceinline__ int lane_count(long long e, long long e1, long long L, const int *idx,
                                          const int *map) {
    int c = 0;
    for (; e < e1; e += 4 * L) {
        const bool v1 = e + L < e1, v2 = e + 2 * L < e1, v3 = e + 3 * L < e1;
        const int i0 = __ldg(idx + e);
        const int i1 = v1 ? __ldg(idx + e + L) : 0;
        const int i2 = v2 ? __ldg(idx + e + 2 * L) : 0;
        const int i3 = v3 ? __ldg(idx + e + 3 * L) : 0;
        c += map[i0] >= 0;
        if (v1) c += map[i1] >= 0;
        if (v2) c += map[i2] >= 0;
        if (v3) c += map[i3] >= 0;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Full-matrix products
// ---------------------------------------------------------------------------

// y = A x (rows of the CSR form, L lanes per row).  Component entry point.
__device__ __forceinline__ void rows_matvec(const Params &P, const double *xin, double *y) {
    const Grp G(P.tpr);
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        double s = 0.0;
        if (i < P.m)
            s = lane_dot<true>(__ldg(P.rp + i) + G.sl, __ldg(P.rp + i + 1), G.L, P.ci, P.av,
                               [&](int j) { return xin[j]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) y[i] = s;
    }
}

// g = A^T z (columns of the CSC form, L lanes per column).  Component entry point.
__device__ __forceinline__ void cols_matvec(const Params &P, const double *zin, double *gout) {
    const Grp G(P.tpc);
    for (long long base = twarp(P) * G.rpw; base < P.n; base += twarps(P) * G.rpw) {
        const long long j = base + G.sub;
        double s = 0.0;
        if (j < P.n)
            s = lane_dot<true>(__ldg(P.cp + j) + G.sl, __ldg(P.cp + j + 1), G.L, P.ri, P.cv,
                               [&](int i) { return zin[i]; });
        s = group_sum(s, G.L);
        if (j < P.n && G.sl == 0) gout[j] = s;
    }
}

// Column pass of iteration k (Algorithm 1, first half; Section 2 weights):
//   x_k = xt (x_{k-1} plus the row update of the previous iteration),
//   g = A^T z_k, h = A^T t_k with t_k = b - A x_k (for the stopping test),
//   eps^z_j = g_j^2 / ||A_j||^2.
// Partials: max eps^z, ||h||^2, ||g||^2, non-finite flag.
__device__ __forceinline__ void phase_col(const Params &P, BlockScratch &bs) {
    const Grp G(P.tpc);
    double emax = 0.0, hh = 0.0, gg = 0.0;
    long long bad = 0;
    for (long long base = twarp(P) * G.rpw; base < P.n; base += twarps(P) * G.rpw) {
        const long long j = base + G.sub;
        double sg = 0.0, sh = 0.0;
        if (j < P.n)
            lane_dot2(__ldg(P.cp + j) + G.sl, __ldg(P.cp + j + 1), G.L, P.ri, P.cv,
                      reinterpret_cast<const double2 *>(P.z), sg, sh);
        sg = group_sum(sg, G.L);
        sh = group_sum(sh, G.L);
        if (j < P.n && G.sl == 0) {
            P.x[j] = P.xt[j];
            const double c = __ldg(P.cn2 + j);
            const double e = c > 0.0 ? __ddiv_rn(__dmul_rn(sg, sg), c) : 0.0;
            P.g[j] = sg;
            P.epsc[j] = e;
            if (!isfinite(e)) bad = 1;
            else emax = max_nonneg(emax, e);
            hh = fma(sh, sh, hh);
            gg = fma(sg, sg, gg);
        }
    }
    emax = block_max(emax, bs);
    hh = block_sum(hh, bs);
    gg = block_sum(gg, bs);
    bad = block_sum(bad, bs);
    if (threadIdx.x == 0) {
        P.pd[D_EMAX_C * tsize(P) + trank(P)] = emax;
        P.pd[D_HH * tsize(P) + trank(P)] = hh;
        P.pd[D_GG * tsize(P) + trank(P)] = gg;
        P.pi[I_BAD_C * tsize(P) + trank(P)] = bad;
    }
}

// t_{k+1} = b - A x_{k+1} over the CSR rows, x_{k+1} = xt.  Partial: ||t||^2.
__device__ __forceinline__ void phase_residual(const Params &P, BlockScratch &bs) {
    const Grp G(P.tpr);
    double tt = 0.0;
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        double s = 0.0;
        if (i < P.m)
            s = lane_dot<true>(__ldg(P.rp + i) + G.sl, __ldg(P.rp + i + 1), G.L, P.ci, P.av,
                               [&](int j) { return P.xt[j]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) {
            const double ti = __ldg(P.b + i) - s;
            P.t[2 * i] = ti;
            tt = fma(ti, ti, tt);
        }
    }
    tt = block_sum(tt, bs);
    if (threadIdx.x == 0) P.pd[D_TT * tsize(P) + trank(P)] = tt;
}

// ---------------------------------------------------------------------------
// Block selection (Section 2): quantise, draw, compact
// ---------------------------------------------------------------------------
struct Chunk {
    long long lo, hi, size;
    __device__ __forceinline__ Chunk(long long len, int cta, int nct) {
        size = (len + nct - 1) / nct;
        lo = min(len, (long long)cta * size);
        hi = min(len, lo + size);
    }
};

// Random rule: q_j = floor(2^K eps_j / eps_max), K = 62 - ceil(log2 len), and
// the chunk-local inclusive prefix of q into Q; clears the marks.  Partial:
// the chunk total.  Greedy rule: marks {j : eps_j >= eta eps_max, eps_j > 0}.
__device__ __forceinline__ void phase_quantize(const Params &P, const double *eps, long long len,
                                               double emax, bool greedy, double eta,
                                               BlockScratch &bs) {
    const Chunk C(len, trank(P), tsize(P));
    if (greedy) {
        const double thr = __dmul_rn(eta, emax);
        for (long long j = C.lo + threadIdx.x; j < C.hi; j += blockDim.x) {
            const double e = eps[j];
            P.flag[j] = (e >= thr && e > 0.0) ? 1 : 0;
        }
        return;
    }
    const int K = 62 - ceil_log2_ll(len);
    unsigned long long run = 0;
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        unsigned long long q = 0;
        if (j < C.hi) {
            const double ratio = __ddiv_rn(eps[j], emax);
            q = __double2ull_rz(floor(scalbn(ratio, K)));
            P.flag[j] = 0;
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<unsigned long long>(q, bs, &tot);
        if (j < C.hi) P.Q[j] = run + ex + q;
        run += tot;
    }
    if (threadIdx.x == 0) P.pi[I_TOT * tsize(P) + trank(P)] = (long long)run;
}

// s independent draws: R = word (t mod 4) of Philox4x64-10 with key
// (seed, sysid) and counter (k, phase, t div 4, 0); target = floor(R Q_tot /
// 2^64); the drawn index is the first j whose global inclusive prefix of q
// exceeds target (located through the per-CTA totals, then inside the chunk).
__device__ __forceinline__ void phase_draw(const Params &P, long long len, long long s,
                                           unsigned long long seed, unsigned long long sysid,
                                           unsigned long long k, unsigned long long phase,
                                           long long *tab, BlockScratch &bs) {
    const int nct = tsize(P);
    partials_prefix(P.pi + I_TOT * nct, nct, tab, bs);
    const unsigned long long qtot = (unsigned long long)tab[nct - 1];
    if (qtot == 0) return;
    const long long csize = (len + nct - 1) / nct;
    const long long nblk = (s + 3) >> 2;
    for (long long t4 = tthread(P); t4 < nblk; t4 += tthreads(P)) {
        const U64x4 R = philox4x64_10(seed, sysid, k, phase, (unsigned long long)t4, 0ull);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if (4 * t4 + w >= s) break;
            const unsigned long long target = __umul64hi(R.v[w], qtot);
            int lo = 0, hi = nct - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((unsigned long long)tab[mid] > target) hi = mid;
                else lo = mid + 1;
            }
            const unsigned long long local = target - (lo > 0 ? (unsigned long long)tab[lo - 1] : 0ull);
            long long a = (long long)lo * csize;
            long long e = min(len, a + csize) - 1;
            while (a < e) {
                const long long mid = a + ((e - a) >> 1);
                if (P.Q[mid] > local) e = mid;
                else a = mid + 1;
            }
            P.flag[a] = 1;
        }
    }
}

// Count of marked indices in the chunk, and over them the sums of norm2 (the
// block's squared Frobenius norm) and of vec^2 (for the LSQR start).
// Partials over the selected lines: their count, the sums of norm2 (squared
// Frobenius norm of the block) and of vec^2 (squared norm of the right-hand
// side, or of B^T c in the column step), and with unit (the weights eps =
// vec^2 / norm2) the same two sums for the block with its lines scaled to
// unit norm: the line count and the sum of the weights.
__device__ __forceinline__ void phase_compact_count(const Params &P, long long len,
                                                    const double *norm2, const double *vec,
                                                    const double *unit, BlockScratch &bs) {
    const Chunk C(len, trank(P), tsize(P));
    long long cnt = 0;
    double fro = 0.0, ext = 0.0, frs = 0.0, exs = 0.0;
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const bool f = j < C.hi && P.flag[j];
        cnt += __popc(__ballot_sync(kFull, f)) * ((threadIdx.x & 31) == 0);
        if (f) {
            fro += __ldg(norm2 + j);
            const double v = vec[j];
            ext = fma(v, v, ext);
            if (unit) {
                frs += 1.0;
                exs += unit[j];
            }
        }
    }
    cnt = block_sum(cnt, bs);
    fro = block_sum(fro, bs);
    ext = block_sum(ext, bs);
    if (unit) {
        frs = block_sum(frs, bs);
        exs = block_sum(exs, bs);
    }
    if (threadIdx.x == 0) {
        P.pi[I_CNT * tsize(P) + trank(P)] = cnt;
        P.pd[D_FRO * tsize(P) + trank(P)] = fro;
        P.pd[D_EXTRA * tsize(P) + trank(P)] = ext;
        P.pd[D_FRO_S * tsize(P) + trank(P)] = frs;
        P.pd[D_EXTRA_S * tsize(P) + trank(P)] = exs;
    }
}

// Exclusive rank of a predicate over the CTA in thread order (ballot/popc per
// warp, then the warp counts scanned); *total gets the CTA count.
__device__ __forceinline__ long long block_rank_pred(bool f, BlockScratch &bs, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(kFull, f);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) bs.i[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        long long s = lane < nw ? bs.i[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        bs.i[lane] = s;
    }
    __syncthreads();
    *total = bs.i[nw - 1];
    return (warp > 0 ? bs.i[warp - 1] : 0) + rank;
}

// Marked indices -> ascending list; pos[j] = position in the list or -1.
// Returns the list length.
__device__ __forceinline__ long long phase_compact_write(const Params &P, long long len, int *pos,
                                                         int *list, long long *tab,
                                                         BlockScratch &bs) {
    const int nct = tsize(P);
    partials_prefix(P.pi + I_CNT * nct, nct, tab, bs);
    const long long total = tab[nct - 1];
    const Chunk C(len, trank(P), nct);
    long long run = trank(P) > 0 ? tab[trank(P) - 1] : 0;
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const bool f = j < C.hi && P.flag[j];
        long long tot;
        const long long ex = block_rank_pred(f, bs, &tot);
        if (j < C.hi) {
            if (f) {
                pos[j] = (int)(run + ex);
                list[run + ex] = (int)j;
            } else {
                pos[j] = -1;
            }
        }
        run += tot;
    }
    return total;
}

// ---------------------------------------------------------------------------
// Block extraction in one pass: for each line (CSR row or CSC column) of A,
// the entries whose other index is selected (map[idx] >= 0) are written,
// renumbered through map, at the start of the line's own slot in A's arrays
// (oidx/oval[ptr[l] .. ptr[l] + ocnt[l])).  No scan over the grid is needed;
// the block products read each line as (ptr[l], ocnt[l]).  A_U keeps all m
// rows and A^J all n columns, so both block products are gathers.
// Partial: the number of extracted entries.
// ---------------------------------------------------------------------------
struct Lines {
    const long long *ptr;
    const int *idx;
    const double *val;
    long long n;
    int L;
};

__device__ __forceinline__ void phase_extract(const Params &P, const Lines &A, const int *map,
                                              int *ocnt, int *oidx, double *oval,
                                              BlockScratch &bs) {
    const Grp G(A.L);
    const long long L = G.L;
    long long total = 0;
    for (long long base = twarp(P) * G.rpw; base < A.n; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        const bool valid = i < A.n;
        const long long e0 = valid ? __ldg(A.ptr + i) : 0;
        const long long e1 = valid ? __ldg(A.ptr + i + 1) : 0;
        int nit = valid ? (int)((e1 - e0 + 4 * L - 1) / (4 * L)) : 0;
        nit = (int)__reduce_max_sync(kFull, (unsigned)nit);
        long long pos = e0;
        for (int it = 0; it < nit; ++it) {
            // four entries per lane per trip: index and value loads, then map gathers
            const long long e = e0 + (long long)it * 4 * L + G.sl;
            int p[4];
            double vq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long f = e + q * L;
                const bool in = valid && f < e1;
                p[q] = in ? __ldg(A.idx + f) : -1;
                vq[q] = in ? __ldg(A.val + f) : 0.0;   // with the index: one round trip less
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) p[q] = p[q] >= 0 ? map[p[q]] : -1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned gm = G.mine(__ballot_sync(kFull, p[q] >= 0));
                if (p[q] >= 0) {
                    const long long o = pos + __popc(gm & ((1u << G.sl) - 1u));
                    oidx[o] = p[q];
                    oval[o] = vq[q];
                }
                pos += __popc(gm);
            }
        }
        if (valid && G.sl == 0) {
            ocnt[i] = (int)(pos - e0);
            total += pos - e0;
        }
    }
    total = block_sum(total, bs);
    if (threadIdx.x == 0) P.pi[I_NNZ * tsize(P) + trank(P)] = total;
}

__device__ __forceinline__ bool stop_rule_holds(int rule, double tol, double rel, double nrm) {
    switch (rule) {
    case RGDBEK_STOP_REL_RES: return rel <= tol;
    case RGDBEK_STOP_RSE: return rel * rel <= tol;
    default: return nrm <= tol;
    }
}

}  // namespace rgd
