// Set-up kernels of a solver handle: CSR validation, the CSC copy of A and
// the squared row/column norms (Section 2 divides every residual weight by
// them, so they are computed once per matrix).
//
// The CSC copy is built deterministically: entries are bucketed by column
// with integer atomics, then each column's bucket is sorted by CSR entry
// index (= by row), so the result does not depend on thread timing and the
// A^T products of every solve sum in the same order.
#include <climits>

#include "rgdbek_internal.h"

namespace rgd {

namespace {

constexpr int kSetupThreads = 256;

int setup_grid(long long work) {
    long long g = (work + kSetupThreads - 1) / kSetupThreads;
    if (g < 1) g = 1;
    if (g > 8192) g = 8192;
    return (int)g;
}

__global__ void check_row_ptr_kernel(long long m, long long nnz, const long long *rp, int *err) {
    for (long long i = gthread(); i < m; i += nthreads()) {
        const long long a = rp[i], b = rp[i + 1];
        if (a > b || a < 0 || b > nnz) atomicMax(err, 1);
        if (i == 0 && a != 0) atomicMax(err, 1);
        if (i == m - 1 && b != nnz) atomicMax(err, 1);
    }
}

// err: 1 = non-finite value, 2 = column index out of range or out of order
// (the larger code wins)
__global__ void check_entries_kernel(long long m, long long n, const long long *rp, const int *ci,
                                     const double *av, int *err) {
    for (long long i = gwarp(); i < m; i += nwarps()) {
        const long long e0 = rp[i], e1 = rp[i + 1];
        for (long long e = e0 + (threadIdx.x & 31); e < e1; e += 32) {
            const int c = ci[e];
            if (c < 0 || c >= n) atomicMax(err, 2);
            if (e > e0 && ci[e - 1] >= c) atomicMax(err, 2);
            if (!isfinite(av[e])) atomicMax(err, 1);
        }
    }
}

__global__ void row_of_kernel(long long m, const long long *rp, int *row_of) {
    for (long long i = gwarp(); i < m; i += nwarps()) {
        const long long e1 = rp[i + 1];
        for (long long e = rp[i] + (threadIdx.x & 31); e < e1; e += 32) row_of[e] = (int)i;
    }
}

__global__ void histogram_kernel(long long nnz, const int *ci, long long *cnt) {
    for (long long e = gthread(); e < nnz; e += nthreads())
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt + ci[e]), 1ull);
}

// exclusive scan of cnt[0..len) into out[0..len], out[len] = total; three passes
__global__ void scan_reduce_kernel(long long len, long long chunk, const long long *cnt,
                                   long long *blk) {
    __shared__ BlockScratch bs;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(len, lo + chunk);
    long long s = 0;
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) s += cnt[j];
    s = block_sum(s, bs);
    if (threadIdx.x == 0) blk[blockIdx.x] = s;
}
__global__ void scan_blocks_kernel(int nblk, long long *blk) {
    __shared__ BlockScratch bs;
    long long run = 0;
    for (int base = 0; base < nblk; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < nblk ? blk[i] : 0;
        long long tot;
        const long long ex = block_excl_scan<long long>(v, bs, &tot);
        if (i < nblk) blk[i] = run + ex;
        run += tot;
    }
}
__global__ void scan_apply_kernel(long long len, long long chunk, const long long *cnt,
                                  const long long *blk, long long *out, long long *cursor) {
    __shared__ BlockScratch bs;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(len, lo + chunk);
    long long run = blk[blockIdx.x];
    for (long long base = lo; base < hi; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const long long v = j < hi ? cnt[j] : 0;
        long long tot;
        const long long ex = block_excl_scan<long long>(v, bs, &tot);
        if (j < hi) {
            out[j] = run + ex;
            cursor[j] = run + ex;
        }
        run += tot;
    }
    if (hi == len && lo < hi && threadIdx.x == 0) out[len] = run;
}

__global__ void scatter_kernel(long long nnz, const int *ci, long long *cursor, long long *key) {
    for (long long e = gthread(); e < nnz; e += nthreads()) {
        const long long slot =
            (long long)atomicAdd(reinterpret_cast<unsigned long long *>(cursor + ci[e]), 1ull);
        key[slot] = e;
    }
}

// Sorts each column's bucket of CSR entry indices (all distinct) into dst:
// one warp per column; runs of 32 are ranked in registers, then runs are
// merged pairwise, each element finding its place by binary search in the
// other run.  Ping-pongs between a (the scattered input) and dst.
__global__ void sort_columns_kernel(long long n, const long long *cp, long long *a,
                                    long long *dst) {
    const int lane = threadIdx.x & 31;
    for (long long j = gwarp(); j < n; j += nwarps()) {
        const long long lo = cp[j], len = cp[j + 1] - lo;
        if (len == 0) continue;
        // runs of 32, a -> dst
        for (long long r = 0; r < len; r += 32) {
            const long long q = r + lane;
            const long long v = q < len ? a[lo + q] : LLONG_MAX;
            int rank = 0;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) rank += __shfl_sync(kFull, v, l) < v;
            if (q < len) dst[lo + r + rank] = v;
        }
        __syncwarp();
        long long *cur = dst, *nxt = a;
        for (long long w = 32; w < len; w <<= 1) {
            for (long long q = lane; q < len; q += 32) {
                const long long a0 = (q / (2 * w)) * (2 * w);
                const long long mid = min(len, a0 + w), end = min(len, a0 + 2 * w);
                const long long v = cur[lo + q];
                // count of elements of the other run smaller than v
                long long s, e;
                if (q < mid) { s = mid; e = end; }
                else { s = a0; e = mid; }
                long long l2 = s, h2 = e;
                while (l2 < h2) {
                    const long long md = (l2 + h2) >> 1;
                    if (cur[lo + md] < v) l2 = md + 1;
                    else h2 = md;
                }
                const long long smaller = l2 - s;
                const long long out = q < mid ? q + smaller : a0 + (q - mid) + smaller;
                nxt[lo + out] = v;
            }
            __syncwarp();
            long long *t = cur;
            cur = nxt;
            nxt = t;
        }
        if (cur != dst)
            for (long long q = lane; q < len; q += 32) dst[lo + q] = cur[lo + q];
        __syncwarp();
    }
}

__global__ void gather_csc_kernel(long long nnz, const long long *key, const int *row_of,
                                  const double *av, int *ri, double *cv) {
    for (long long s = gthread(); s < nnz; s += nthreads()) {
        const long long e = key[s];
        ri[s] = row_of[e];
        cv[s] = av[e];
    }
}

// one warp per line, lanes strided, fixed xor-tree sum
__global__ void line_norms_kernel(long long nlines, const long long *ptr, const double *val,
                                  double *out) {
    for (long long i = gwarp(); i < nlines; i += nwarps()) {
        double s = 0.0;
        const long long e1 = ptr[i + 1];
        for (long long e = ptr[i] + (threadIdx.x & 31); e < e1; e += 32) s = fma(val[e], val[e], s);
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) out[i] = s;
    }
}

}  // namespace

cudaError_t validate_csr(long long m, long long n, long long nnz, const long long *rp,
                         const int *ci, const double *av, int *err_dev, int *err_host,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(err_dev, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    check_row_ptr_kernel<<<setup_grid(m), kSetupThreads, 0, s>>>(m, nnz, rp, err_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int code = 0;
    if ((e = cudaMemcpyAsync(&code, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (code != 0) {
        *err_host = RGDBEK_ERR_BAD_CSR;
        return cudaSuccess;
    }
    if (nnz > 0) {
        check_entries_kernel<<<setup_grid(m * 32), kSetupThreads, 0, s>>>(m, n, rp, ci, av, err_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&code, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    *err_host = code == 0 ? RGDBEK_OK : code == 2 ? RGDBEK_ERR_BAD_CSR : RGDBEK_ERR_NONFINITE;
    return cudaSuccess;
}

cudaError_t build_csc(long long m, long long n, long long nnz, const long long *rp, const int *ci,
                      const double *av, long long *cp, int *ri, double *cv, long long *key_a,
                      long long *key_b, int *row_of, long long *cursor, long long *blk_sums,
                      cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(long long), s)) != cudaSuccess) return e;
    if (nnz > 0) {
        row_of_kernel<<<setup_grid(m * 32), kSetupThreads, 0, s>>>(m, rp, row_of);
        histogram_kernel<<<setup_grid(nnz), kSetupThreads, 0, s>>>(nnz, ci, cursor);
    }
    // column pointers = exclusive scan of the counts (counts live in cursor,
    // copied to key_b as the scan input because cursor is rewritten)
    const long long chunk = 1024;
    const int nblk = (int)((n + chunk - 1) / chunk);
    if ((e = cudaMemcpyAsync(key_b, cursor, (size_t)n * sizeof(long long),
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    scan_reduce_kernel<<<nblk, kSetupThreads, 0, s>>>(n, chunk, key_b, blk_sums);
    scan_blocks_kernel<<<1, 1024, 0, s>>>(nblk, blk_sums);
    scan_apply_kernel<<<nblk, kSetupThreads, 0, s>>>(n, chunk, key_b, blk_sums, cp, cursor);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nnz > 0) {
        scatter_kernel<<<setup_grid(nnz), kSetupThreads, 0, s>>>(nnz, ci, cursor, key_a);
        sort_columns_kernel<<<setup_grid(n * 32), kSetupThreads, 0, s>>>(n, cp, key_a, key_b);
        gather_csc_kernel<<<setup_grid(nnz), kSetupThreads, 0, s>>>(nnz, key_b, row_of, av, ri, cv);
    }
    return cudaGetLastError();
}

cudaError_t line_norms2(long long nlines, const long long *ptr, const double *val, double *out,
                        cudaStream_t s) {
    line_norms_kernel<<<setup_grid(nlines * 32), kSetupThreads, 0, s>>>(nlines, ptr, val, out);
    return cudaGetLastError();
}

}  // namespace rgd
