// Block selection without any device allocation: rgdbek_sample_noalloc.
//
// Some callers cannot allocate device memory when they need a block drawn:
// an application whose memory pool has already reserved the GPU's memory (a
// cudaMalloc would fail or fragment it), a latency-critical loop in which
// the implicit device synchronisation of cudaMalloc / cudaFree is not
// acceptable, or a plugin whose host forbids allocation after start-up.  For
// them this entry point runs the same sampling kernel as rgdbek_sample, but
// its scratch memory (quantised prefix sums, draw marks, positions, per-CTA
// partials and the control block) lives in one file-scope device array of
// fixed size, created when the library is loaded.
//
// Host code never uses the array's name as an address: the address is
// fetched once per device with cudaGetSymbolAddress, with that device
// current, and passed to the kernels.
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "rgdbek_internal.h"

namespace rgd {
namespace {

constexpr long long kNoAllocMaxLen = RGDBEK_NOALLOC_MAX_LEN;
constexpr int kMaxDevices = 64;

// scratch layout (each part 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffQ = 0;
constexpr size_t kOffFlag = kOffQ + align256(sizeof(unsigned long long) * kNoAllocMaxLen);
constexpr size_t kOffPos = kOffFlag + align256(sizeof(unsigned char) * kNoAllocMaxLen);
constexpr size_t kOffPd = kOffPos + align256(sizeof(int) * kNoAllocMaxLen);
constexpr size_t kOffPi = kOffPd + align256(sizeof(double) * D_NSLOTS * kMaxGrid);
constexpr size_t kOffCtrl = kOffPi + align256(sizeof(long long) * I_NSLOTS * kMaxGrid);
constexpr size_t kScratchBytes = kOffCtrl + align256(sizeof(Ctrl));

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_sample_scratch[kScratchBytes];

// copies the block size out of the control block: the count, -1 for a
// negative or non-finite weight, -2 if the kernel gave up a device wait
__global__ void noalloc_count_kernel(const Ctrl *c, int64_t *count) {
    const int st = c->status;
    *count = st == RGDBEK_OK ? (int64_t)c->sample_count : (int64_t)-2;
}

struct DeviceSetup {
    unsigned char *scratch = nullptr;  // device address of g_sample_scratch
    int grid = 0;
    bool done = false;                 // set only once the set-up has succeeded
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the scratch address and the
// cooperative grid of the sampling kernel.  A failed set-up is not recorded:
// the next call on the device tries again.
int device_setup(DeviceSetup **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RGDBEK_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return RGDBEK_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.done) {
        void *p = nullptr;
        int sms = 0;
        const int fit = sample_blocks_per_sm(kSolveMaxThreads);
        if (cudaGetSymbolAddress(&p, g_sample_scratch) != cudaSuccess || p == nullptr ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            fit < 1) {
            cudaGetLastError();  // clear the recorded error: the caller's next call must not see it
            return RGDBEK_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char *>(p);
        const long long g = (long long)fit * sms;
        d.grid = (int)(g > kMaxGrid ? kMaxGrid : g);
        d.done = true;
    }
    *out = &d;
    return RGDBEK_OK;
}

}  // namespace
}  // namespace rgd

using namespace rgd;

extern "C" int rgdbek_sample_noalloc(const double *eps, int64_t len, int64_t s, uint64_t seed,
                                     uint64_t sysid, int64_t k, int phase, int32_t *idx,
                                     int64_t *count, void *stream) {
    if (!eps || !idx || !count || s < 0 || k < 0 || (phase != 0 && phase != 1))
        return RGDBEK_ERR_INVALID_ARG;
    if (len < 1 || len > kNoAllocMaxLen) return RGDBEK_ERR_INVALID_ARG;
    if (s > (long long)RGDBEK_MAX_DRAWS_PER_ENTRY * len) return RGDBEK_ERR_INVALID_ARG;
    DeviceSetup *d = nullptr;
    const int st = device_setup(&d);
    if (st != RGDBEK_OK) return st;

    Params P{};
    P.Q = reinterpret_cast<unsigned long long *>(d->scratch + kOffQ);
    P.flag = d->scratch + kOffFlag;
    P.rowpos = reinterpret_cast<int *>(d->scratch + kOffPos);
    P.pd = reinterpret_cast<double *>(d->scratch + kOffPd);
    P.pi = reinterpret_cast<long long *>(d->scratch + kOffPi);
    P.ctrl = reinterpret_cast<Ctrl *>(d->scratch + kOffCtrl);
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // the control block (barrier counter, status) must start from its reset
    // state; the kernel itself clears the marks and overwrites the rest
    cudaError_t e = launch_reset_ctrl(P.ctrl, cs);
    if (e == cudaSuccess)
        e = launch_sample(P, d->grid, kSolveMaxThreads, eps, (long long)len, (long long)s, seed,
                          sysid, (unsigned long long)k, (unsigned long long)phase, idx, false, 0.0,
                          cs);
    if (e == cudaSuccess) {
        noalloc_count_kernel<<<1, 1, 0, cs>>>(P.ctrl, count);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? RGDBEK_OK : RGDBEK_ERR_CUDA;
}
