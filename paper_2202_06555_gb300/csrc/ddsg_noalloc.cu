// ddsg_noalloc.cu -- hdmr_eval_noalloc: interpolant evaluation that allocates
// no device memory.
//
// hdmr_eval needs scratch space for the encoded queries and takes it from a
// workspace the handle grows with cudaMalloc. Some callers cannot allow that:
// code that owns all device memory through its own pool or runs under a fixed
// memory cap (a cudaMalloc behind its back fails or fragments the pool), and
// code that must not trigger allocation once it is serving (latency-critical
// loops, allocator callbacks). This entry point takes the scratch from one
// fixed-size array in static device memory instead. Its size is stated below;
// every GPU that loads this library keeps it reserved until the process exits.
//
// The array is shared by all calls on a device and keeps the previous call's
// contents; each call overwrites every word it reads (the encoded coordinates
// and the per-query flags of its n queries), so nothing has to be cleared.
// Two calls whose kernels overlap on the GPU (e.g. on two streams) race on it:
// serialize them.
//
// Set-up: the first call on a device (a call with n = 0 does only this) looks
// up the array's device address there. Under lazy module loading (CUDA's
// default) that lookup is also what loads the array's module on the device, so
// the 16 MiB are committed then: a caller under a hard memory cap makes that
// first call while it sets up, before its cap or any stream capture begins.
// The cached address is that of the device's current context; after a
// cudaDeviceReset every handle's tables are gone too, so no handle created
// before the reset may be used again, with this entry point or any other.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ddsg_internal.h"

using namespace ddsg;

namespace {

// 2^21 words of 8 bytes = 16 MiB: n*d encoded coordinates plus n int32 flags.
constexpr size_t kNoAllocWords = (size_t)1 << 21;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch per device

// Device address of the scratch array on the current device (looked up once
// per device; in host code the symbol itself is only a host-side stand-in).
int scratch_address(int dev, uint64_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(DDSG_ERR_ARG, "hdmr_eval_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(DDSG_ERR_CUDA, "hdmr_eval_noalloc: cudaGetSymbolAddress failed for the static scratch array");
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<uint64_t *>(g_scratch_addr[dev]);
    return DDSG_OK;
}

}  // namespace

extern "C" int64_t hdmr_eval_noalloc_capacity(int d) {
    if (d < 1) return 0;
    // n*d words for the coordinates and ceil(n/2) words for the flags
    return (int64_t)((2 * kNoAllocWords) / (2 * (size_t)d + 1));
}

extern "C" int hdmr_eval_noalloc(hdmr_t *h, int64_t n, const double *x_dev, double *y_dev,
                                 int precision, int form, ddsg_stream_t stream) {
    if (n < 0) return set_error(DDSG_ERR_ARG, "hdmr_eval_noalloc: n < 0");
    HandleView v;
    int rc = handle_eval_view(h, precision, form, &v);
    if (rc) return rc;
    if (n > 0 && (!x_dev || !y_dev)) return set_error(DDSG_ERR_ARG, "hdmr_eval_noalloc: NULL x or y");
    if (n > hdmr_eval_noalloc_capacity(v.d))
        return set_error(DDSG_ERR_ARG,
                         "hdmr_eval_noalloc: batch too large for the 16 MiB static scratch "
                         "(n must be <= hdmr_eval_noalloc_capacity(d)); split the batch");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(DDSG_ERR_CUDA, "hdmr_eval_noalloc: no current device");
    if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess)
        return set_error(DDSG_ERR_CUDA, "hdmr_eval_noalloc: cannot select the handle's device");
    uint64_t *X = nullptr;
    rc = scratch_address(v.device, &X);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!rc && n > 0) {
        cudaError_t e;
        {
            HandleProfScope ps(h, DDSG_K_ENCODE, st);
            e = launch_encode_queries(n, v.d, x_dev, v.lo, v.span, X, v.stats, st);
        }
        if (e == cudaSuccess) {
            EvalArgs a;
            a.t = v.tables;
            a.d = v.d;
            a.m = v.m;
            a.n = n;
            a.X = X;
            a.y = y_dev;
            a.hash = nullptr;
            a.count = nullptr;
            a.form = form;
            a.precision = precision;
            a.cfg = v.cfg;
            a.err = reinterpret_cast<unsigned long long *>(v.stats + 2);   // bounded waits that gave up
            a.withhold_from = v.withhold_from;
            HandleProfScope ps(h, DDSG_K_EVAL, st);
            e = launch_eval(a, st);
        }
        if (e != cudaSuccess) rc = set_error(DDSG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (prev != v.device) cudaSetDevice(prev);
    return rc;
}
