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
constexpr unsigned long long kBarrierMaxSpins = 1ull << 28;

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
    D_NSLOTS
};
enum ISlot {
    I_BAD_C = 0,  // non-finite column weight seen
    I_BAD_R,      // non-finite row weight / b entry seen
    I_TOT,        // chunk total of quantised weights
    I_CNT,        // chunk count of flagged indices
    I_NNZ,        // chunk count of extracted nonzeros
    I_NSLOTS
};

// Device control block, one per handle.  Barrier words sit on their own
// 128-byte lines.
struct Ctrl {
    unsigned bar_count;
    unsigned pad0[31];
    unsigned bar_gen;
    unsigned pad1[31];
    int abort;
    int status;
    int stop_req;
    int pad2[29];
    // results, written by CTA 0 at the end of a solve
    long long iters, inner_u, inner_j, sum_nu, sum_nj, sum_nnzu, sum_nnzj;
    long long lsqr_nnzu, lsqr_nnzj, lsqr_nu, lsqr_nj;
    double rel_res, normal_res, rse;
    long long sample_count;  // block size returned by the standalone sampler
    double emax_out;         // maximum returned by the standalone weights kernel
    int bad_out;
    int pad3[15];
};

// ---------------------------------------------------------------------------
// Memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for cooperative launches (all CTAs resident).  Returns
// false if the wait was abandoned: another CTA raised the abort flag, or the
// time/spin limit ran out (then this CTA records TIMEOUT and raises abort).
__device__ __forceinline__ bool grid_barrier(Ctrl *c) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(&c->bar_gen);
        __threadfence();
        const unsigned prev = atomicAdd(&c->bar_count, 1u);
        if (prev == gridDim.x - 1) {
            c->bar_count = 0;
            __threadfence();
            st_release_u32(&c->bar_gen, gen + 1);
        } else {
            unsigned long long spins = 0;
            const unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_u32(&c->bar_gen) == gen) {
                ++spins;
                if ((spins & 255) == 0) {
                    if (ld_volatile_i32(&c->abort)) { ok = 0; break; }
                    if (spins > kBarrierMaxSpins || globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                        atomicCAS(&c->status, kStatusRunning, RGDBEK_ERR_TIMEOUT);
                        atomicExch(&c->abort, 1);
                        ok = 0;
                        break;
                    }
                }
                if (spins > 64) __nanosleep(32);
            }
        }
        __threadfence();
        if (ld_volatile_i32(&c->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
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

__device__ __forceinline__ double block_max(double v, BlockScratch &bs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) bs.d[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double r = lane < nw ? bs.d[lane] : 0.0;
        r = warp_max(r);
        if (lane == 0) bs.d[32] = r;
    }
    __syncthreads();
    return bs.d[32];
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

// Sum over the per-CTA partials of one slot, computed by warp 0 in a fixed
// order; the result is returned to every thread of the CTA.
__device__ __forceinline__ double reduce_partials_sum(const double *p, int nb, BlockScratch &bs) {
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += 32) s += __ldcg(p + i);
        s = warp_sum(s);
        if (threadIdx.x == 0) bs.d[33] = s;
    }
    __syncthreads();
    return bs.d[33];
}
__device__ __forceinline__ double reduce_partials_max(const double *p, int nb, BlockScratch &bs) {
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += 32) s = fmax(s, __ldcg(p + i));
        s = warp_max(s);
        if (threadIdx.x == 0) bs.d[33] = s;
    }
    __syncthreads();
    return bs.d[33];
}
__device__ __forceinline__ long long reduce_partials_isum(const long long *p, int nb,
                                                          BlockScratch &bs) {
    __syncthreads();
    if (threadIdx.x < 32) {
        long long s = 0;
        for (int i = threadIdx.x; i < nb; i += 32) s += __ldcg(p + i);
        s = warp_sum(s);
        if (threadIdx.x == 0) bs.i[33] = s;
    }
    __syncthreads();
    return bs.i[33];
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

// lanes to put on one row/column with `avg` nonzeros on average: the largest
// power of two L <= 32 with 2L <= avg (at least 1)
__host__ __device__ __forceinline__ int pick_lanes(double avg) {
    int L = 1;
    while (L < 32 && 4.0 * L <= avg) L *= 2;
    return L;
}

}  // namespace rgd
