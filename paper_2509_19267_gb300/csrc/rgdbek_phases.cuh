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

// Kernel parameters of one system, for values of type V: double for the FP64
// solve (and the FP64 outer loop of the FP32 form), float for the FP32 inner
// solve of RGDBEK_PRECISION_FP32_INNER.  Index arrays, selection scratch and
// the control block are shared by both views of a system.
template <typename V>
struct ParamsT {
    long long m, n, nnz;
    // A in CSR and CSC form, squared row/column norms
    const long long *__restrict__ rp;
    const int *__restrict__ ci;
    const V *__restrict__ av;
    const long long *__restrict__ cp;
    const int *__restrict__ ri;
    const V *__restrict__ cv;
    const V *__restrict__ rn2;
    const V *__restrict__ cn2;
    // right-hand side and solution
    const V *b;
    V *x;
    // work vectors: z (m) and t = b - A x (m), stored as (z_i, t_i) pairs
    // (z_i at z[2 i], t_i at t[2 i] = z[2 i + 1]: the column pass gathers both
    // with one load), r (m), g = A^T z (n), weights, LSQR vectors u (m),
    // v, w, y (n), the row-step solution dx (n) and the trial iterate
    // xt = x + dx (n) that the next column pass adopts
    V *z, *t, *r, *g, *epsc, *epsr, *uu, *vv, *ww, *yy, *dx, *xt;
    unsigned long long *Q;  // chunk-local inclusive prefix of quantised weights
    unsigned char *flag;    // drawn / selected marks
    int *colpos, *rowpos;   // position of a column in U / of a row in J, or -1
    int *ulist, *jlist;     // U_k and J_k, ascending
    int *srn;               // A_U as CSR over all m rows: row i holds srn[i] entries
    int *sci;               // at sci/sav[rp[i] ..], columns renumbered 0..|U|-1
    V *sav;
    int *scn;               // A^J as CSC over all n columns: column j holds scn[j]
    int *sri;               // entries at sri/scv[cp[j] ..], rows renumbered 0..|J|-1
    V *scv;
    V *dots, *dots2;        // per-line dot products of the inner solve when a CTA's
                            // chunk does not fit in shared memory (max(m, n) each)
    V *pd;                  // value partials [D_NSLOTS][grid]
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
    long long k0;           // number of the first outer iteration (the Philox counter)
    unsigned long long seed, sysid;
    int inner_max, stop_rule, selection;
    int precision;          // RGDBEK_PRECISION_* of the solve
    int team;               // CTAs that work on this system (rank = blockIdx.x % team)
    int warm;               // x holds x_0 on entry (else x_0 = 0)
    V *vvs, *dsc;           // column step: D v~ and D = 1/||A_j|| per column of U
    V *yh;                  // column step: y^ of the scaled block (global fallback)
    V *uus, *dsr;           // row step: D u~ and D = 1/||A^(i)|| per row of J
    // refinement loop of the FP32 form (FP64 view only): the FP64 residual
    // b - A x (m), the scaled right-hand side (m) and solution (n) of an FP64
    // inner solve
    V *ref_t, *ref_b, *ref_x;
    int tpr, tpc;           // lanes per row (CSR) / column (CSC) of A: block extraction
                            // and the selected lines of the inner solves
    int lpr, lpc;           // lanes per row / column of A in the full-matrix passes
                            // (A^T z, b - A x, the component SpMVs; tunable)
    int ipr, ipc;           // lanes per row / column of A, integer passes
    long long dsmem_bytes;  // dynamic shared memory per CTA of the solve kernel
    // two-team schedule (solve_split): zteam > 0 CTAs of the grid run the
    // column steps, one outer iteration ahead of the row steps that the other
    // CTAs run (the z recurrence of Algorithm 1 does not depend on x); the
    // column team's own copies of the buffers both steps use, and the second
    // list of U (the row team records U_k while U_{k+1} is drawn)
    int zteam;
    V *uu_z, *vv_z, *ww_z, *dots_z, *dots2_z, *pd_z;
    long long *pi_z;
    unsigned long long *Q_z;
    unsigned char *flag_z;
    int *ulist2;
    unsigned long long *bar;  // this team's barrier counter (null: ctrl->bar_count)
};
using Params = ParamsT<double>;
using ParamsF = ParamsT<float>;

// Pairs of values loaded with one instruction.
template <typename V>
struct Vec2;
template <>
struct Vec2<double> {
    using type = double2;
};
template <>
struct Vec2<float> {
    using type = float2;
};

// Arithmetic of the two value types (the FP64 forms are the ones the FP64
// solve has always used, so its results do not change).
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float vsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double vrsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float vrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
// residual weight v^2 / c, each operation correctly rounded (Section 2)
__device__ __forceinline__ double weight_of(double v, double c) {
    return __ddiv_rn(__dmul_rn(v, v), c);
}
__device__ __forceinline__ float weight_of(float v, float c) {
    return __fdiv_rn(__fmul_rn(v, v), c);
}

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
template <typename PT>
__device__ __forceinline__ void enter_team(const PT &P) {
    if (threadIdx.x == 0) s_team_rank = (int)(blockIdx.x % (unsigned)P.team);
    __syncthreads();
}
template <typename PT>
__device__ __forceinline__ int trank(const PT &P) {
    (void)P;
    // re-read at each use (like a special register) rather than held live
    return *reinterpret_cast<volatile int *>(&s_team_rank);
}
template <typename PT>
__device__ __forceinline__ int tsize(const PT &P) { return P.team; }
template <typename PT>
__device__ __forceinline__ long long twarp(const PT &P) {
    return (long long)trank(P) * (blockDim.x >> 5) + (threadIdx.x >> 5);
}
template <typename PT>
__device__ __forceinline__ long long twarps(const PT &P) {
    return (long long)P.team * (blockDim.x >> 5);
}
template <typename PT>
__device__ __forceinline__ long long tthread(const PT &P) {
    return (long long)trank(P) * blockDim.x + threadIdx.x;
}
template <typename PT>
__device__ __forceinline__ long long tthreads(const PT &P) {
    return (long long)P.team * blockDim.x;
}

// Loads through the read-only path (RO) for arrays that never change during
// a kernel, ordinary loads otherwise.
template <bool RO, typename T>
__device__ __forceinline__ T ldx(const T *p) {
    if constexpr (RO) return __ldg(p);
    else return *p;
}

// The right-hand side b of a solve.  The FP64 solve never writes it during a
// kernel, so it goes through the read-only path; the FP32 inner solve's b is
// rewritten by the refinement loop of the same kernel, so it is loaded from L2
// (the non-coherent read-only cache could still hold the previous one).
__device__ __forceinline__ double ld_rhs(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_rhs(const float *p) { return __ldcg(p); }

// Kahan-compensated accumulation (Kahan 1965) of FP32 products: c carries the
// rounding error of the running sum into the next term, and the sum is
// returned as s - c.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float x) {
        const float y = fmaf(a, x, -c);
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float sum() const { return s - c; }
};

// This lane's share of sum_e val[e] * f(idx[e]) over e = e, e + L, e + 2L, ...
// below e1, accumulated in exactly that order (FP64: a chain of fused
// multiply-adds; FP32: Kahan-compensated).
//
// FP64: eight entries per trip, all their index/value loads and gathers
// issued before the multiply-adds; the last 1..7 entries likewise, their
// loads predicated, and their multiply-adds in a loop of exactly that count
// that shifts the operands down.  GB300 issues about two FP64 lane-operations
// per SM per clock, and a multiply-add predicated off still takes its issue
// slot, so no FP64 instruction is spent on an entry that does not exist.
//
// FP32: four entries per trip with all their loads issued before the
// arithmetic, so four independent index/value loads and four gathers are in
// flight per lane.
template <bool RO, typename V, typename F>
__device__ __forceinline__ V lane_dot(long long e, long long e1, long long L, const int *idx,
                                      const V *val, F f) {
    if constexpr (sizeof(V) == 8) {
        V s = V(0);
        for (; e + 7 * L < e1; e += 8 * L) {
            int j[8];
            V a[8], x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                j[q] = ldx<RO>(idx + e + q * L);
                a[q] = ldx<RO>(val + e + q * L);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = f(j[q]);
#pragma unroll
            for (int q = 0; q < 8; ++q) s = fma(a[q], x[q], s);
        }
        if (e < e1) {
            int rem = 0, j[7];
            V a[7], x[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const bool v = e + q * L < e1;
                rem += v ? 1 : 0;
                j[q] = v ? ldx<RO>(idx + e + q * L) : 0;
                a[q] = v ? ldx<RO>(val + e + q * L) : V(0);
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) x[q] = (e + q * L < e1) ? f(j[q]) : V(0);
#pragma unroll 1
            for (int q = 0; q < rem; ++q) {
                s = fma(a[0], x[0], s);
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    a[t] = a[t + 1];
                    x[t] = x[t + 1];
                }
            }
        }
        return s;
    }
    KahanF k;
    for (; e < e1; e += 4 * L) {
        const bool v1 = e + L < e1, v2 = e + 2 * L < e1, v3 = e + 3 * L < e1;
        const int i0 = ldx<RO>(idx + e);
        const int i1 = v1 ? ldx<RO>(idx + e + L) : 0;
        const int i2 = v2 ? ldx<RO>(idx + e + 2 * L) : 0;
        const int i3 = v3 ? ldx<RO>(idx + e + 3 * L) : 0;
        const V a0 = ldx<RO>(val + e);
        const V a1 = v1 ? ldx<RO>(val + e + L) : V(0);
        const V a2 = v2 ? ldx<RO>(val + e + 2 * L) : V(0);
        const V a3 = v3 ? ldx<RO>(val + e + 3 * L) : V(0);
        const V x0 = f(i0);
        const V x1 = v1 ? f(i1) : V(0);
        const V x2 = v2 ? f(i2) : V(0);
        const V x3 = v3 ? f(i3) : V(0);
        k.add(a0, x0);
        if (v1) k.add(a1, x1);
        if (v2) k.add(a2, x2);
        if (v3) k.add(a3, x3);
    }
    return k.sum();
}

// Two dot products sharing the index/value loads (A^T z and A^T t): the two
// vectors are stored as (z_i, t_i) pairs, so one gather serves both.
template <typename V>
__device__ __forceinline__ void lane_dot2(long long e, long long e1, long long L, const int *idx,
                                          const V *val, const typename Vec2<V>::type *zt, V &sf,
                                          V &sg) {
    using V2 = typename Vec2<V>::type;
    KahanF kf, kg;
    for (; e < e1; e += 4 * L) {
        const bool v1 = e + L < e1, v2 = e + 2 * L < e1, v3 = e + 3 * L < e1;
        const int i0 = __ldg(idx + e);
        const int i1 = v1 ? __ldg(idx + e + L) : 0;
        const int i2 = v2 ? __ldg(idx + e + 2 * L) : 0;
        const int i3 = v3 ? __ldg(idx + e + 3 * L) : 0;
        const V a0 = __ldg(val + e);
        const V a1 = v1 ? __ldg(val + e + L) : V(0);
        const V a2 = v2 ? __ldg(val + e + 2 * L) : V(0);
        const V a3 = v3 ? __ldg(val + e + 3 * L) : V(0);
        const V2 zero{V(0), V(0)};
        const V2 p0 = zt[i0];
        const V2 p1 = v1 ? zt[i1] : zero;
        const V2 p2 = v2 ? zt[i2] : zero;
        const V2 p3 = v3 ? zt[i3] : zero;
        if constexpr (sizeof(V) == 8) {
            sf = fma(a0, p0.x, sf);
            sg = fma(a0, p0.y, sg);
            if (v1) { sf = fma(a1, p1.x, sf); sg = fma(a1, p1.y, sg); }
            if (v2) { sf = fma(a2, p2.x, sf); sg = fma(a2, p2.y, sg); }
            if (v3) { sf = fma(a3, p3.x, sf); sg = fma(a3, p3.y, sg); }
        } else {
            kf.add(a0, p0.x);
            kg.add(a0, p0.y);
            if (v1) { kf.add(a1, p1.x); kg.add(a1, p1.y); }
            if (v2) { kf.add(a2, p2.x); kg.add(a2, p2.y); }
            if (v3) { kf.add(a3, p3.x); kg.add(a3, p3.y); }
        }
    }
    if constexpr (sizeof(V) == 4) {
        sf = kf.sum();
        sg = kg.sum();
    }
}

// ---------------------------------------------------------------------------
// Full-matrix products
// ---------------------------------------------------------------------------

// y = A x (rows of the CSR form, L lanes per row).  Component entry point;
// FP32: A's float values, Kahan-compensated lane sums (the FP32 form's passes).
template <typename V>
__device__ __forceinline__ void rows_matvec(const ParamsT<V> &P, const V *xin, V *y) {
    const Grp G(P.lpr);
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        V s = V(0);
        if (i < P.m)
            s = lane_dot<true>(__ldg(P.rp + i) + G.sl, __ldg(P.rp + i + 1), G.L, P.ci, P.av,
                               [&](int j) { return xin[j]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) y[i] = s;
    }
}

// g = A^T z (columns of the CSC form, L lanes per column).  Component entry point.
template <typename V>
__device__ __forceinline__ void cols_matvec(const ParamsT<V> &P, const V *zin, V *gout) {
    const Grp G(P.lpc);
    for (long long base = twarp(P) * G.rpw; base < P.n; base += twarps(P) * G.rpw) {
        const long long j = base + G.sub;
        V s = V(0);
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
// The column team of a two-team solve runs it with apply_x = false (the row
// team adopts x) and, where no t is due, with_h = false (h is not formed).
template <typename V>
__device__ __forceinline__ void phase_col(const ParamsT<V> &P, BlockScratch &bs,
                                          bool apply_x = true, bool with_h = true) {
    using V2 = typename Vec2<V>::type;
    const Grp G(P.lpc);
    V emax = V(0), hh = V(0), gg = V(0);
    long long bad = 0;
    for (long long base = twarp(P) * G.rpw; base < P.n; base += twarps(P) * G.rpw) {
        const long long j = base + G.sub;
        V sg = V(0), sh = V(0);
        if (j < P.n)
            lane_dot2<V>(__ldg(P.cp + j) + G.sl, __ldg(P.cp + j + 1), G.L, P.ri, P.cv,
                         reinterpret_cast<const V2 *>(P.z), sg, sh);
        sg = group_sum(sg, G.L);
        sh = group_sum(sh, G.L);
        if (j < P.n && G.sl == 0) {
            if (apply_x) P.x[j] = P.xt[j];
            const V c = __ldg(P.cn2 + j);
            const V e = c > V(0) ? weight_of(sg, c) : V(0);
            P.g[j] = sg;
            P.epsc[j] = e;
            if (!isfinite(e)) bad = 1;
            else emax = max_nonneg(emax, e);
            if (with_h) hh = vfma(sh, sh, hh);
            gg = vfma(sg, sg, gg);
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
// With apply_x (the row team of a two-team solve) x = xt is also adopted.
template <typename V>
__device__ __forceinline__ void phase_residual(const ParamsT<V> &P, BlockScratch &bs,
                                               bool apply_x = false) {
    const Grp G(P.lpr);
    V tt = V(0);
    if (apply_x)
        for (long long j = tthread(P); j < P.n; j += tthreads(P)) P.x[j] = P.xt[j];
    for (long long base = twarp(P) * G.rpw; base < P.m; base += twarps(P) * G.rpw) {
        const long long i = base + G.sub;
        V s = V(0);
        if (i < P.m)
            s = lane_dot<true>(__ldg(P.rp + i) + G.sl, __ldg(P.rp + i + 1), G.L, P.ci, P.av,
                               [&](int j) { return P.xt[j]; });
        s = group_sum(s, G.L);
        if (i < P.m && G.sl == 0) {
            const V ti = ld_rhs(P.b + i) - s;
            P.t[2 * i] = ti;
            tt = vfma(ti, ti, tt);
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

// q = floor(2^K * fl(eps / eps_max)), the quantised weight of the random rule.
// FP64: the correctly rounded FP64 ratio scaled by 2^K (exact) and floored.
__device__ __forceinline__ unsigned long long quantize_weight(double e, double emax, int K) {
    const double ratio = __ddiv_rn(e, emax);
    return __double2ull_rz(floor(scalbn(ratio, K)));
}
// FP32: the correctly rounded FP32 ratio r in [0, 1] is m * 2^(x - 150) for
// its 24-bit significand m and biased exponent x, so floor(2^K r) is m
// shifted left by x - 150 + K, or right by its negative (bits shifted out
// are the floor), computed exactly with integer operations.  Subnormal
// ratios (below 2^-126) give 0, as 2^(K - 126) < 1 for K <= 62.
__device__ __forceinline__ unsigned long long quantize_weight(float e, float emax, int K) {
    const unsigned bits = __float_as_uint(__fdiv_rn(e, emax));
    const int ex = (int)((bits >> 23) & 0xffu);
    if (ex == 0) return 0ull;
    const unsigned long long mant = (unsigned long long)((bits & 0x7fffffu) | 0x800000u);
    const int sh = ex - 150 + K;
    if (sh >= 0) return mant << sh;
    if (sh <= -24) return 0ull;
    return mant >> (-sh);
}

// Random rule: q_j = floor(2^K eps_j / eps_max), K = 62 - ceil(log2 len), and
// the chunk-local inclusive prefix of q into Q; clears the marks.  Partial:
// the chunk total.  Greedy rule: marks {j : eps_j >= eta eps_max, eps_j > 0}.
// For the solve (count_slot): the chunk's count of marks in slot I_CNT (0 for
// the random rule: the draws count them), and zero_cnt[0 .. zero_len) cleared
// (the line counts the scatter of the selected lines will fill).
template <typename V>
__device__ __forceinline__ void phase_quantize(const ParamsT<V> &P, const V *eps, long long len,
                                               V emax, bool greedy, double eta,
                                               BlockScratch &bs, bool count_slot = false,
                                               int *zero_cnt = nullptr, long long zero_len = 0) {
    const Chunk C(len, trank(P), tsize(P));
    for (long long i = tthread(P); i < zero_len; i += tthreads(P)) zero_cnt[i] = 0;
    if (greedy) {
        const V thr = (V)eta * emax;
        long long cnt = 0;
        for (long long base = C.lo; base < C.hi; base += blockDim.x) {
            const long long j = base + threadIdx.x;
            bool f = false;
            if (j < C.hi) {
                const V e = eps[j];
                f = e >= thr && e > V(0);
                P.flag[j] = f ? 1 : 0;
            }
            cnt += __popc(__ballot_sync(kFull, f)) * ((threadIdx.x & 31) == 0);
        }
        if (count_slot) {
            cnt = block_sum(cnt, bs);
            if (threadIdx.x == 0) P.pi[I_CNT * tsize(P) + trank(P)] = cnt;
        }
        return;
    }
    const int K = 62 - ceil_log2_ll(len);
    unsigned long long run = 0;
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        unsigned long long q = 0;
        if (j < C.hi) {
            q = quantize_weight(eps[j], emax, K);
            P.flag[j] = 0;
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<unsigned long long>(q, bs, &tot);
        if (j < C.hi) P.Q[j] = run + ex + q;
        run += tot;
    }
    if (threadIdx.x == 0) {
        P.pi[I_TOT * tsize(P) + trank(P)] = (long long)run;
        if (count_slot) P.pi[I_CNT * tsize(P) + trank(P)] = 0;
    }
}

// s independent draws: R = word (t mod 4) of Philox4x64-10 with key
// (seed, sysid) and counter (k, phase, t div 4, 0); target = floor(R Q_tot /
// 2^64); the drawn index is the first j whose global inclusive prefix of q
// exceeds target (located through the per-CTA totals, then inside the chunk).
// With cnt (the solve), each first mark of an index is also counted for the
// chunk that holds it (cnt[chunk], cleared by phase_quantize): the marks are
// set with an atomic OR on the 32-bit word that holds them, and only the
// draw that finds its byte clear adds one, so every chunk's count of
// distinct marks is exact whatever the order of the draws.
template <typename PT>
__device__ __forceinline__ void phase_draw(const PT &P, long long len, long long s,
                                           unsigned long long seed, unsigned long long sysid,
                                           unsigned long long k, unsigned long long phase,
                                           long long *tab, BlockScratch &bs,
                                           long long *cnt = nullptr) {
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
            if (cnt) {
                const unsigned sh = 8u * (unsigned)(a & 3);
                unsigned *w = reinterpret_cast<unsigned *>(P.flag + (a & ~3ll));
                const unsigned old = atomicOr(w, 1u << sh);
                if (((old >> sh) & 0xffu) == 0u)
                    atomicAdd(reinterpret_cast<unsigned long long *>(cnt + lo), 1ull);
            } else {
                P.flag[a] = 1;
            }
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
template <typename V>
__device__ __forceinline__ void phase_compact_count(const ParamsT<V> &P, long long len,
                                                    const V *norm2, const V *vec,
                                                    const V *unit, BlockScratch &bs) {
    const Chunk C(len, trank(P), tsize(P));
    long long cnt = 0;
    V fro = V(0), ext = V(0), frs = V(0), exs = V(0);
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const bool f = j < C.hi && P.flag[j];
        cnt += __popc(__ballot_sync(kFull, f)) * ((threadIdx.x & 31) == 0);
        if (f) {
            fro += __ldg(norm2 + j);
            const V v = vec[j];
            ext = vfma(v, v, ext);
            if (unit) {
                frs += V(1);
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
template <typename PT>
__device__ __forceinline__ long long phase_compact_write(const PT &P, long long len, int *pos,
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
// Compaction of the marks and extraction of the block in one phase.
//
// The marked indices of the CTA's chunk get their place in the ascending
// list (offsets from the prefix of the per-chunk counts of the draws), and
// the entries of each selected line of A (a CSC column for the column block,
// a CSR row for the row block) are scattered into the other side's lines:
// entry (l, o) goes to line o of the block at dptr[o] + (dcnt[o]++), with l
// renumbered to its place p in the list (pos[j] = p, or -1 where j is not
// selected, when pos is given).  Only the selected lines are read
// (about eta of A), not all of A.  The line counts come from atomic
// increments, so the entries of a line land in arbitrary order; the inner
// solve sorts them by index before its first product (sort_scattered_lines),
// which gives every line the order of A's own lines.
// init(p, j, total) runs once per selected index j (place p, list length
// total) before the scatter: the start vectors of the inner solve.
// Partials over the selected lines, summed per thread in the chunk's order:
// the sums of norm2 (squared Frobenius norm of the block) and of vec^2 (the
// LSQR right-hand side, or B^T c in the column step), with unit (the weights
// eps = vec^2 / norm2) the line count and the sum of the weights, and the
// number of scattered entries (nnz of the block).
// ---------------------------------------------------------------------------
template <typename V, typename Init>
__device__ __forceinline__ long long phase_select_scatter(
    const ParamsT<V> &P, long long len, const V *norm2, const V *vec, const V *unit, int *pos,
    int *list, long long *tab, BlockScratch &bs, const long long *sptr, const int *sidx,
    const V *sval, const long long *dptr, int *dcnt, int *didx, V *dval, Init init) {
    const int nct = tsize(P);
    partials_prefix(P.pi + I_CNT * nct, nct, tab, bs);
    const long long total = tab[nct - 1];
    const Chunk C(len, trank(P), nct);
    const long long first = trank(P) > 0 ? tab[trank(P) - 1] : 0;
    long long run = first;
    V fro = V(0), ext = V(0), frs = V(0), exs = V(0);
    for (long long base = C.lo; base < C.hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const bool f = j < C.hi && P.flag[j];
        long long tot;
        const long long ex = block_rank_pred(f, bs, &tot);
        if (j < C.hi) {
            if (f) {
                const long long p = run + ex;
                if (pos) pos[j] = (int)p;
                list[p] = (int)j;
                init(p, j, total);
                fro += __ldg(norm2 + j);
                const V v = vec[j];
                ext = vfma(v, v, ext);
                if (unit) {
                    frs += V(1);
                    exs += unit[j];
                }
            } else if (pos) {
                pos[j] = -1;
            }
        }
        run += tot;
    }
    __syncthreads();  // the CTA's list entries [first, run) are visible to all its threads
    // Scatter: the entries of the CTA's selected lines, numbered in line order,
    // are dealt to the threads in turn (four at a time, all loads and
    // increments in flight), so the work is even whatever the line lengths.
    // The line of an entry is found by a binary search of the chunk-local
    // prefix of the line lengths (bs.big, staged in rounds of blockDim lines).
    long long nnz = 0;
    long long *off = reinterpret_cast<long long *>(bs.big);
    for (long long r0 = first; r0 < run; r0 += blockDim.x) {
        const long long q = r0 + threadIdx.x;
        const int nq = (int)min((long long)blockDim.x, run - r0);
        long long e0 = 0, len = 0;
        if (q < run) {
            const long long l = list[q];
            e0 = __ldg(sptr + l);
            len = __ldg(sptr + l + 1) - e0;
        }
        long long tot;
        const long long ex = block_excl_scan<long long>(len, bs, &tot);
        __syncthreads();
        if (q < run) off[threadIdx.x] = ex;
        __syncthreads();
        nnz += tot;
        for (long long t0 = threadIdx.x; t0 < tot; t0 += 4ll * blockDim.x) {
            int o[4];
            V v[4];
            int qq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long t = t0 + (long long)u * blockDim.x;
                o[u] = -1;
                v[u] = V(0);
                qq[u] = 0;
                if (t < tot) {
                    int lo = 0, hi = nq - 1;  // last line whose offset is <= t
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (off[mid] <= t) lo = mid;
                        else hi = mid - 1;
                    }
                    const long long l = list[r0 + lo];
                    const long long f = __ldg(sptr + l) + (t - off[lo]);
                    o[u] = __ldg(sidx + f);
                    v[u] = __ldg(sval + f);
                    qq[u] = (int)(r0 + lo);
                }
            }
            long long d[4];
            int c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                d[u] = o[u] >= 0 ? __ldg(dptr + o[u]) : 0;
                c[u] = o[u] >= 0 ? atomicAdd(dcnt + o[u], 1) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (o[u] >= 0) {
                    didx[d[u] + c[u]] = qq[u];
                    dval[d[u] + c[u]] = v[u];
                }
            }
        }
        __syncthreads();
    }
    fro = block_sum(fro, bs);
    ext = block_sum(ext, bs);
    if (unit) {
        frs = block_sum(frs, bs);
        exs = block_sum(exs, bs);
    }
    if (threadIdx.x == 0) {
        P.pd[D_FRO * nct + trank(P)] = fro;
        P.pd[D_EXTRA * nct + trank(P)] = ext;
        P.pd[D_FRO_S * nct + trank(P)] = frs;
        P.pd[D_EXTRA_S * nct + trank(P)] = exs;
        P.pi[I_NNZ * nct + trank(P)] = nnz;
    }
    return total;
}

template <typename V>
__device__ __forceinline__ bool stop_rule_holds(int rule, double tol, V rel, V nrm) {
    switch (rule) {
    case RGDBEK_STOP_REL_RES: return rel <= (V)tol;
    case RGDBEK_STOP_RSE: return rel * rel <= (V)tol;
    default: return nrm <= (V)tol;
    }
}

}  // namespace rgd
