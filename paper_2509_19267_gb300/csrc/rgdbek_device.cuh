// Device-side building blocks of the RGDBEK library (sm_103a):
// the per-handle control block, a bounded grid barrier for the persistent
// cooperative kernels, deterministic warp/block reductions and scans, and a
// Philox4x64-10 generator written from its published definition (Salmon et
// al., SC'11).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rgdbek.h"

namespace rgd {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStatusRunning = 0x7fff;  // ctrl->status while a kernel runs
constexpr int kMaxGrid = 1024;    // CTAs of a persistent launch (prefix tables in smem)
constexpr int kMaxThreads = 1024;

// Wait limits of the grid barrier: after either, the waiting CTA records
// RGDBEK_ERR_TIMEOUT, raises the abort flag and returns, so no wait is endless.
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;  // 4 s
constexpr unsigned long long kBarrierMaxSpins = 1ull << 30;

// Slots of the per-CTA partial arrays (double and int64), [slot][grid].
// Two phases separated by one barrier never write the same slot, so a slow
// CTA still reading the previous phase's partials is never overwritten.
enum DSlot {
    D_BB = 0,     // ||b||^2
    D_EMAX_C,     // max column weight
    D_HH,         // ||A^T t||^2
    D_FRO,        // sum of squared norms over the block
    D_EXTRA,      // sum of squares of the LSQR right-hand side over the block
    D_UU,         // LSQR ||u~||^2
    D_VV,         // LSQR ||v~||^2
    D_EMAX_R,     // max row weight
    D_ZZ,         // ||z||^2
    D_TT,         // ||t||^2
    D_FRO_S,      // the block's squared Frobenius norm with unit lines (their count)
    D_EXTRA_S,    // ||D c||^2 of the line-scaled right-hand side (sum of the weights)
    D_GG,         // ||A^T z||^2 (at k = 0, z_0 = b: ||A^T b||^2)
    D_NSLOTS
};
enum ISlot {
    I_BAD_C = 0,  // non-finite column weight seen
    I_BAD_R,      // non-finite row weight / b entry seen
    I_TOT,        // chunk total of quantised weights
    I_CNT,        // chunk count of flagged indices
    I_NNZ,        // count of extracted nonzeros
    I_STOP,       // two-team schedule: the row team has finished (set by rank 0)
    I_NSLOTS
};

// Device control block, one per handle.  The barrier counter sits on its
// own 128-byte line.
struct Ctrl {
    unsigned long long bar_count;  // arrivals since the launch (monotonic)
    unsigned long long pad0[15];
    int abort;
    int status;
    int stop_req;
    int pad2[29];
    // results, written by CTA 0 at the end of a solve
    long long iters, inner_u, inner_j, sum_nu, sum_nj, sum_nnzu, sum_nnzj;
    long long lsqr_nnzu, lsqr_nnzj, lsqr_nu, lsqr_nj;
    unsigned long long phase_ns[RGDBEK_NUM_PHASES];
    double rel_res, normal_res, rse;
    long long sample_count;  // block size returned by the standalone sampler
    double emax_out;         // maximum returned by the standalone weights kernel
    int bad_out;
    int pad3[15];
    long long refinements;   // FP64 refinement steps of the FP32 form
    // ---- two-team schedule (the column steps of Algorithm 1 run one iteration
    // ahead of the row steps on a team of their own; see solve_split)
    alignas(128) unsigned long long bar_x;  // barrier counter of the row team
    alignas(128) unsigned long long bar_z;  // barrier counter of the column team
    // link words, each (call << 32) | count within the call, written with
    // release stores by the writing team's rank 0 after a team barrier:
    alignas(128) unsigned long long lk_zready;  // z_{k+1} written (column team)
    unsigned long long lk_zused;    // z_{k+1} read by the row team
    unsigned long long lk_tready;   // t_{k+1} written (row team)
    unsigned long long lk_colpass;  // column pass k done (its ||A^T t||^2 below)
    unsigned long long lk_stop;     // the row team has finished this call
    // values that travel with the link words (slot = iteration parity)
    double lk_hh[2], lk_gg;
    long long lk_badc[2], lk_nu[2], lk_nnzu[2], lk_stepsu[2];
    // the row team's result, for the CTAs of the column team
    long long lk_res_k;
    int lk_res_status, pad4;
    double lk_res_rel, lk_res_nrm;
    unsigned long long zphase_ns[RGDBEK_NUM_PHASES];  // the column team's phase times
};

// ---------------------------------------------------------------------------
// Memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long *p,
                                                                   unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;"
                 : "=l"(old)
                 : "l"(p), "l"(v)
                 : "memory");
    return old;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier of the nct CTAs of a team in a cooperative launch (all CTAs
// resident; the team is the whole grid for a single solve), on the team's own
// counter.  `epoch` (read and advanced by thread 0 only) counts the barriers
// this CTA has passed, the same number in every CTA of the team: barrier
// number e completes when the arrival counter reaches nct * (e + 1).
// Arrival is a release add by thread 0 after the CTA's __syncthreads (so the
// CTA's writes are published); the wait is an acquire load followed by a
// __syncthreads (so every thread sees the other CTAs' writes).  Returns false
// if the wait was abandoned: another CTA raised the abort flag, or the
// time/spin limit ran out (then this CTA records TIMEOUT and raises abort).
// cnt: the team's arrival counter (c->bar_count, or a counter of its own
// when two teams work on one system; abort and status stay c's).
__device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned long long *cnt,
                                             unsigned long long &epoch, int nct) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (unsigned long long)nct * (epoch + 1);
        atom_add_release_u64(cnt, 1ull);
        unsigned long long spins = 0;
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u64(cnt) < target) {
            ++spins;
            if ((spins & 1023) == 0) {
                if (ld_volatile_i32(&c->abort)) { ok = 0; break; }
                if (spins > kBarrierMaxSpins || globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                    atomicCAS(&c->status, kStatusRunning, RGDBEK_ERR_TIMEOUT);
                    atomicExch(&c->abort, 1);
                    ok = 0;
                    break;
                }
            }
            if (spins > 256) __nanosleep(20);
        }
        s_ok = ok;
        ++epoch;
    }
    __syncthreads();
    return s_ok != 0;
}
__device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned long long &epoch, int nct) {
    return grid_barrier(c, &c->bar_count, epoch, nct);
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Wait limits of a wait on the other team of a two-team solve: that team's
// progress is itself bounded by its barriers' limits (an abandoned barrier
// raises the abort flag seen here), so this limit only guards the protocol.
constexpr unsigned long long kLinkTimeoutNs = 30000000000ull;  // 30 s

// Thread 0 of the CTA waits until *word >= target (acquire), then the CTA
// synchronises.  With stop_call != 0 the wait also ends when the row team has
// finished call stop_call (c->lk_stop >= stop_call) while *word < target: the
// stop word is read before the awaited word, and the row team raises it only
// after its last link write, so every CTA of a team reaches the same
// decision.  Returns 0 (reached), 1 (stopped), -1 (abort flag, or the wait
// limit ran out: then TIMEOUT is recorded and the abort flag raised).
__device__ __forceinline__ int link_wait(Ctrl *c, const unsigned long long *word,
                                         unsigned long long target, unsigned long long stop_call) {
    __shared__ int s_r;
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = 0;
        unsigned long long spins = 0;
        const unsigned long long t0 = globaltimer_ns();
        for (;;) {
            const unsigned long long st = stop_call ? ld_acquire_u64(&c->lk_stop) : 0ull;
            if (ld_acquire_u64(word) >= target) break;
            if (stop_call && st >= stop_call) {
                r = 1;
                break;
            }
            ++spins;
            if ((spins & 1023) == 0) {
                if (ld_volatile_i32(&c->abort)) {
                    r = -1;
                    break;
                }
                if (spins > kBarrierMaxSpins || globaltimer_ns() - t0 > kLinkTimeoutNs) {
                    atomicCAS(&c->status, kStatusRunning, RGDBEK_ERR_TIMEOUT);
                    atomicExch(&c->abort, 1);
                    r = -1;
                    break;
                }
            }
            if (spins > 256) __nanosleep(64);
        }
        s_r = r;
    }
    __syncthreads();
    return s_r;
}

// ---------------------------------------------------------------------------
// Warp / group / block reductions (fixed order, so every CTA that reduces the
// same data gets bit-identical results)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
// running maximum of a nonnegative finite double, on bit patterns
__device__ __forceinline__ double max_nonneg(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

__device__ __forceinline__ float max_nonneg(float a, float b) {
    return __int_as_float(max(__float_as_int(a), __float_as_int(b)));
}

// maximum over the warp of nonnegative finite doubles (integer compare of the
// bit patterns, which order like the values; no FP64 instructions)
__device__ __forceinline__ double warp_max(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(kFull, b, o));
    return __longlong_as_double(b);
}
__device__ __forceinline__ float warp_max(float v) {
    int b = __float_as_int(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(kFull, b, o));
    return __int_as_float(b);
}
// sum over the L consecutive lanes of a group (L a power of two, <= 32); all
// 32 lanes must call it
template <typename T>
__device__ __forceinline__ T group_sum(T v, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

struct BlockScratch {
    double d[34];
    long long i[34];
    unsigned long long u[34];
    float f[34];
    double big[kMaxThreads];      // one partial per thread (FP64 block sums)
    double mid[kMaxThreads / 4];  // first level of the FP64 block-sum tree
};

template <typename T>
__device__ __forceinline__ T *scratch_of(BlockScratch &s);
template <>
__device__ __forceinline__ double *scratch_of<double>(BlockScratch &s) { return s.d; }
template <>
__device__ __forceinline__ long long *scratch_of<long long>(BlockScratch &s) { return s.i; }
template <>
__device__ __forceinline__ unsigned long long *scratch_of<unsigned long long>(BlockScratch &s) {
    return s.u;
}
template <>
__device__ __forceinline__ float *scratch_of<float>(BlockScratch &s) { return s.f; }

// Integer block sum: warp shuffles, then warp 0 over the warp totals.
template <typename T>
__device__ __forceinline__ T block_sum(T v, BlockScratch &bs) {
    T *sm = scratch_of<T>(bs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T r = lane < nw ? sm[lane] : T(0);
        r = warp_sum(r);
        if (lane == 0) sm[32] = r;
    }
    __syncthreads();
    return sm[32];
}

// FP64 block sum.  GB300 issues one warp-wide FP64 add per SM every ~17
// cycles, so a shuffle tree in every warp (5 adds x 32 warps) costs more than
// the work it reduces; instead the partials go through shared memory: blockDim/4
// threads add four each, then warp 0 adds the rest and finishes with one
// shuffle tree (about blockDim/32 + 13 warp-wide adds).  Fixed order, so every
// CTA reducing the same values gets the same bits.  blockDim % 64 == 0.
template <>
__device__ __forceinline__ double block_sum<double>(double v, BlockScratch &bs) {
    const int t = threadIdx.x, n = blockDim.x, c1 = n >> 2;
    __syncthreads();
    bs.big[t] = v;
    __syncthreads();
    if (t < c1) {
        const double *p = bs.big + 4 * t;
        bs.mid[t] = (p[0] + p[1]) + (p[2] + p[3]);
    }
    __syncthreads();
    if (t < 32) {
        double r = 0.0;
        for (int i = t; i < c1; i += 32) r += bs.mid[i];
        r = warp_sum(r);
        if (t == 0) bs.d[32] = r;
    }
    __syncthreads();
    return bs.d[32];
}

// Maximum of nonnegative finite doubles, taken on their bit patterns (which
// order like the values) with integer instructions.
__device__ __forceinline__ double block_max(double v, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(kFull, b, o));
    __syncthreads();
    if (lane == 0) bs.i[warp] = b;
    __syncthreads();
    if (warp == 0) {
        long long r = lane < nw ? bs.i[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(kFull, r, o));
        if (lane == 0) bs.i[32] = r;
    }
    __syncthreads();
    return __longlong_as_double(bs.i[32]);
}

// Maximum of one int64 per thread over the CTA; every thread returns it.
__device__ __forceinline__ long long block_max_ll(long long v, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    __syncthreads();
    if (lane == 0) bs.i[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long r = lane < nw ? bs.i[lane] : bs.i[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(kFull, r, o));
        if (lane == 0) bs.i[32] = r;
    }
    __syncthreads();
    return bs.i[32];
}

// The same for nonnegative finite floats (bit patterns compared as integers).
__device__ __forceinline__ float block_max(float v, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int b = __float_as_int(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(kFull, b, o));
    __syncthreads();
    if (lane == 0) bs.i[warp] = b;
    __syncthreads();
    if (warp == 0) {
        int r = lane < nw ? (int)bs.i[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(kFull, r, o));
        if (lane == 0) bs.i[32] = r;
    }
    __syncthreads();
    return __int_as_float((int)bs.i[32]);
}

// ---------------------------------------------------------------------------
// Sums of nonnegative doubles in fixed point (order-independent, no FP64 adds)
//
// On GB300 a dependent FP64 add costs 64 cycles, and several hundred while
// other warps of the SM issue FP64 work, so a tree of FP64 adds on the
// critical path of every inner-solver phase is slow.  These sums instead align
// every term to the largest exponent of the set and add the significands as
// 64-bit integers: exact integer arithmetic, so the result does not depend on
// the order of the terms, and each term is truncated to a multiple of
// 2^(e_max - 52 - h), h = the headroom bits left for the count of terms.  The
// relative error is below count * 2^-(52 + h) of the largest term, about 1e-14
// for a thousand terms, against about count * 2^-53 for an FP64 add tree.
// Inputs must be nonnegative (sums of squares); a NaN or infinite term gives
// a NaN result.  One integer-to-double conversion and one power-of-two
// multiply remain in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fx_headroom(int count) {
    // 63 bits hold count terms below 2^(53 + shift) when count <= 2^(10 - shift)
    int h = 0;
    while ((1 << h) < count) ++h;
    return h;
}
// significand of a nonnegative finite double aligned to exponent emax, with
// `shift` extra low bits (shift = 63 - 53 - headroom >= 0)
__device__ __forceinline__ unsigned long long fx_term(unsigned long long bits, int emax, int shift) {
    const int e = (int)(bits >> 52);
    if (e == 0) return 0ull;  // zero (subnormal terms are far below any nonzero sum here)
    const unsigned long long m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int d = emax - e;
    return d < 64 ? (m << shift) >> d : 0ull;
}
// the fixed-point sum back to a double: acc * 2^(emax - 1075 - shift)
__device__ __forceinline__ double fx_value(unsigned long long acc, int emax, int shift) {
    if (emax == 0x7ff) return __longlong_as_double(0x7ff8000000000000ll);  // NaN or Inf term
    if (emax == 0) return 0.0;
    const int e2 = emax - 52 - shift;  // biased exponent of the unit 2^(emax - 1075 - shift)
    if (e2 <= 0) return __ull2double_rn(acc) * 0.0;  // below the normal range: zero
    return __ull2double_rn(acc) * __longlong_as_double((long long)e2 << 52);
}

// Sum of the per-CTA partials p[0..nb) (nonnegative) by one warp, nb <=
// kMaxGrid; every lane returns it.  Up to 256 partials are held in registers
// (one load each); more are loaded twice.
__device__ __forceinline__ double warp_sum_fixed(const double *p, int nb) {
    const int lane = threadIdx.x & 31;
    const int shift = 10 - fx_headroom(nb);
    long long mx = 0;
    unsigned long long acc = 0;
    if (nb <= 256) {
        unsigned long long b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = lane + 32 * q;
            b[q] = i < nb ? (unsigned long long)__double_as_longlong(__ldcg(p + i)) : 0ull;
            mx = max(mx, (long long)b[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        const int emax = (int)((unsigned long long)mx >> 52);
        if (emax < 0x7ff) {
#pragma unroll
            for (int q = 0; q < 8; ++q) acc += fx_term(b[q], emax, shift);
        }
    } else {
        for (int i = lane; i < nb; i += 32) mx = max(mx, __double_as_longlong(__ldcg(p + i)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        const int emax = (int)((unsigned long long)mx >> 52);
        if (emax < 0x7ff)
            for (int i = lane; i < nb; i += 32)
                acc += fx_term((unsigned long long)__double_as_longlong(__ldcg(p + i)), emax, shift);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    return fx_value(acc, (int)((unsigned long long)mx >> 52), shift);
}

// Sum over the CTA of one nonnegative double per thread (blockDim <= 1024);
// every thread returns it.
__device__ __forceinline__ double block_sum_fixed(double v, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    long long mx = (long long)bits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    __syncthreads();
    if (lane == 0) bs.i[warp] = mx;
    __syncthreads();
    if (warp == 0) {
        long long r = lane < nw ? bs.i[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(kFull, r, o));
        if (lane == 0) bs.i[33] = r;
    }
    __syncthreads();
    const int emax = (int)((unsigned long long)bs.i[33] >> 52);
    const int shift = 10 - fx_headroom((int)blockDim.x);
    unsigned long long q = emax < 0x7ff ? fx_term(bits, emax, shift) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
    if (lane == 0) bs.u[warp] = q;
    __syncthreads();
    if (warp == 0) {
        unsigned long long r = lane < nw ? bs.u[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
        if (lane == 0) bs.d[33] = fx_value(r, emax, shift);
    }
    __syncthreads();
    return bs.d[33];
}

// Exclusive scan of one value per thread in thread order; *total gets the sum.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, BlockScratch &bs, T *total) {
    T *sm = scratch_of<T>(bs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? sm[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        sm[lane] = s;  // inclusive prefix over warps
    }
    __syncthreads();
    const T off = warp > 0 ? sm[warp - 1] : T(0);
    *total = sm[nw - 1];
    return off + x - v;
}

// All requested partial slots reduced at once: warp w of the CTA reduces the
// w-th requested slot (FP64 sums in fixed point, FP32 sums in a fixed order;
// maxima for slots in dmax), and
// the results land in out_d[slot] / out_i[slot] for every thread.  dmask /
// imask select double / int64 slots (bit = slot).
template <typename V>
__device__ __forceinline__ void collect_partials(const V *pd, const long long *pi, int nb,
                                                 unsigned dmask, unsigned dmax, unsigned imask,
                                                 V *out_d, long long *out_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int w = 0;
    for (int slot = 0; slot < D_NSLOTS; ++slot) {
        if (!(dmask >> slot & 1u)) continue;
        if (warp == w) {
            const V *p = pd + slot * nb;
            const bool mx = dmax >> slot & 1u;
            V s = V(0);
            if (sizeof(V) == 8 && !mx) {
                // FP64 sums (all of nonnegative terms) in fixed point
                s = (V)warp_sum_fixed(reinterpret_cast<const double *>(p), nb);
            } else {
#pragma unroll 8
                for (int i = lane; i < nb; i += 32) {
                    const V v = __ldcg(p + i);
                    s = mx ? max_nonneg(s, v) : s + v;
                }
                s = mx ? warp_max(s) : warp_sum(s);
            }
            if (lane == 0) out_d[slot] = s;
        }
        ++w;
    }
    for (int slot = 0; slot < I_NSLOTS; ++slot) {
        if (!(imask >> slot & 1u)) continue;
        if (warp == w) {
            const long long *p = pi + slot * nb;
            long long s = 0;
#pragma unroll 8
            for (int i = lane; i < nb; i += 32) s += __ldcg(p + i);
            s = warp_sum(s);
            if (lane == 0) out_i[slot] = s;
        }
        ++w;
    }
    __syncthreads();
}

// Inclusive prefix over the per-CTA int64 partials of one slot, into smem
// table tab[0..nb-1] (nb <= kMaxGrid).  Every thread may read tab afterwards.
__device__ __forceinline__ void partials_prefix(const long long *p, int nb, long long *tab,
                                                BlockScratch &bs) {
    long long run = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        long long v = i < nb ? __ldcg(p + i) : 0;
        long long tot;
        long long ex = block_excl_scan<long long>(v, bs, &tot);
        if (i < nb) tab[i] = run + ex + v;
        run += tot;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Philox4x64-10: ten rounds of the 4x64 S-box, key bumped by the two Weyl
// constants between rounds.  Constants from the Random123 publication.
// ---------------------------------------------------------------------------
struct U64x4 {
    unsigned long long v[4];
};
__device__ __forceinline__ U64x4 philox4x64_10(unsigned long long k0, unsigned long long k1,
                                              unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long c3) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0;
        const unsigned long long n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    U64x4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

__device__ __forceinline__ int ceil_log2_ll(long long v) {
    // smallest c with 2^c >= v, for v >= 1
    return v <= 1 ? 0 : 64 - __clzll((unsigned long long)(v - 1));
}

// Lanes to put on one row/column of a matrix with nnz nonzeros in `lines`
// rows/columns, integer arithmetic only.
// pick_lanes_int: for the adjoint's pass over the entries, where each lane
// does little per entry: the largest power of two L <= 32 with 2L <= nnz / lines.
// pick_lanes_fp64: for passes with FP64 multiply-adds, where GB300's low FP64
// issue rate makes idle lanes and group shuffle-adds expensive, and for the
// block extractions, where fewer lanes per line keep more lines in flight:
// about eight entries per lane (the largest power of two L <= 32 with
// 8L <= nnz / lines).
__host__ __device__ __forceinline__ int pick_lanes_int(long long nnz, long long lines) {
    int L = 1;
    while (L < 32 && 4ll * L * lines <= nnz) L *= 2;
    return L;
}
__host__ __device__ __forceinline__ int pick_lanes_fp64(long long nnz, long long lines) {
    int L = 1;
    while (L < 32 && 16ll * L * lines <= nnz) L *= 2;
    return L;
}

}  // namespace rgd
