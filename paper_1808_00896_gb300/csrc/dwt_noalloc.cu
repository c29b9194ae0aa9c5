// dwt_noalloc.cu -- soft_dwt_forward_noalloc: the forward DWT step for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- for
// example a plug-in inside a host application or framework that owns the
// whole device memory pool and forbids allocations outside it, or a
// fixed-budget real-time pipeline that allocates only at start-up and must not
// pay cudaMalloc's implicit device synchronisation later.  Such a caller cannot
// create a plan (soft_plan_create allocates the S workspace, the tables and a
// cuFFT plan), so this entry point takes no plan.
//
// Its working tables (quadrature weights, beta tables, log-factorials, the
// cluster work list and the coefficient run offsets) live in one file-scope
// static __device__ array of fixed size, which every GPU that loads the
// library keeps until the process exits.  The tables are rebuilt by kernels on
// the caller's stream at every call, so nothing from an earlier call is relied
// on; concurrent calls that overlap on the GPU share the array and race.
//
// The kernels it runs have no device-side failure mode: the FP64 DWT kernel
// has no waits and no internal consistency checks (unlike the tensor-core
// kernels, which record timeouts in a plan's error word), so there is no
// error word here; argument, set-up and launch errors are returned.
#include "soft.h"
#include "soft_internal.cuh"

#include <cstdio>
#include <mutex>

namespace softgb {
namespace {

// Largest bandwidth whose tables fit the static array.
constexpr int kNoAllocMaxB = 256;

// Byte layout of the array for bandwidth B (each part 256-byte aligned).
struct NoAllocLayout {
    size_t w, lw, cosb, lcos, lsin, lfact, clusters, runoff, total;
};

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ constexpr NoAllocLayout noalloc_layout(int B) {
    NoAllocLayout L{};
    const size_t n = 2 * (size_t)B;
    size_t o = 0;
    L.w = o;        o = align256(o + n * sizeof(double));
    L.lw = o;       o = align256(o + n * sizeof(double));
    L.cosb = o;     o = align256(o + n * sizeof(double));
    L.lcos = o;     o = align256(o + n * sizeof(double));
    L.lsin = o;     o = align256(o + n * sizeof(double));
    L.lfact = o;    o = align256(o + (n + 1) * sizeof(double));
    L.clusters = o; o = align256(o + (size_t)B * (B + 1) / 2 * sizeof(int2));
    L.runoff = o;   o = align256(o + (size_t)(2 * B - 1) * (2 * B - 1) * sizeof(int64_t));
    L.total = o;
    return L;
}

constexpr size_t kNoAllocBytes = noalloc_layout(kNoAllocMaxB).total;  // about 2.3 MiB (2,377,472 bytes)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Start of the l-run of (m, m') in the coefficient array (layout of soft.h):
// rows m hold B^2 - m^2 entries; within row m (mu = |m|) the run of m' has
// length B - max(mu, |m'|).
__device__ int64_t run_start_dev(int B, int m, int mp) {
    auto sum_sq = [](int64_t x) { return x * (x + 1) * (2 * x + 1) / 6; };
    const int64_t BB = (int64_t)B * B;
    const int64_t sq = m <= 0 ? sum_sq(B - 1) - sum_sq(-m) : sum_sq(B - 1) + sum_sq(m - 1);
    const int64_t row = (int64_t)(m + B - 1) * BB - sq;
    const int64_t mu = m < 0 ? -m : m;
    int64_t in;
    if (mp <= -mu) {
        const int64_t K = B + mp - 1;
        in = K * (K + 1) / 2;
    } else {
        const int64_t K1 = B - mu - 1;
        in = K1 * (K1 + 1) / 2;
        if (mp <= mu + 1) in += (mp + mu) * (B - mu);
        else in += (2 * mu + 1) * (B - mu) + (mp - mu - 1) * (2 * B - mu - mp) / 2;
    }
    return row + in;
}

// Cluster work list (representatives m >= m' >= 0, m ascending, so the longest
// runs come first) and the run-offset table, written into the static array.
__global__ void noalloc_layout_kernel(int B, int2 *clusters, int64_t *runoff) {
    const int ncl = B * (B + 1) / 2;
    const int R = 2 * B - 1;
    const int stride = gridDim.x * blockDim.x;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncl; c += stride) {
        int m = (int)((sqrt(8.0 * c + 1.0) - 1.0) * 0.5);
        while (m * (m + 1) / 2 > c) --m;
        while ((m + 1) * (m + 2) / 2 <= c) ++m;
        clusters[c] = make_int2(m, c - m * (m + 1) / 2);
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * R; e += stride) {
        const int m = e / R - (B - 1), mp = e % R - (B - 1);
        runoff[e] = run_start_dev(B, m, mp);
    }
}

// Device address of the static array, looked up once per device.  Only a
// successful lookup is kept: a failed one (say, made inside a stream capture)
// is retried by the next call.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu[kMaxDevices];

cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu[dev]);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();  // the lookup's error is not sticky: clear it for the caller
            return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

soft_status fail(const char *where, cudaError_t e) {
    set_last_error_message(where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SOFT_ERR_OUT_OF_MEMORY : SOFT_ERR_CUDA;
}

}  // namespace
}  // namespace softgb

using namespace softgb;

extern "C" soft_status soft_dwt_forward_noalloc(int B, const double *S, double *coef, void *stream) {
    if (B < 1 || !S || !coef || S == reinterpret_cast<const double *>(coef) ||
        (reinterpret_cast<uintptr_t>(S) & 15u) || (reinterpret_cast<uintptr_t>(coef) & 15u))
        return SOFT_ERR_INVALID_ARG;
    if (B > kNoAllocMaxB) {
        char msg[96];
        std::snprintf(msg, sizeof msg, "B=%d exceeds the static scratch limit B<=%d", B, kNoAllocMaxB);
        set_last_error_message("soft_dwt_forward_noalloc", msg);
        return SOFT_ERR_UNSUPPORTED;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail("soft_dwt_forward_noalloc: cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error_message("soft_dwt_forward_noalloc", "device ordinal beyond the supported 64");
        return SOFT_ERR_UNSUPPORTED;
    }
    // Set-up, once per device, with that device current: the device address of the array.
    unsigned char *base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return fail("soft_dwt_forward_noalloc: cudaGetSymbolAddress", e);

    const NoAllocLayout L = noalloc_layout(B);
    Tables tb;
    tb.B = B;
    tb.ncl = B * (B + 1) / 2;
    double *w = reinterpret_cast<double *>(base + L.w);
    double *lw = reinterpret_cast<double *>(base + L.lw);
    double *cosb = reinterpret_cast<double *>(base + L.cosb);
    double *lcos = reinterpret_cast<double *>(base + L.lcos);
    double *lsin = reinterpret_cast<double *>(base + L.lsin);
    double *lfact = reinterpret_cast<double *>(base + L.lfact);
    int2 *clusters = reinterpret_cast<int2 *>(base + L.clusters);
    int64_t *runoff = reinterpret_cast<int64_t *>(base + L.runoff);
    tb.w = w; tb.lw = lw; tb.cosb = cosb; tb.lcos = lcos; tb.lsin = lsin; tb.lfact = lfact;
    tb.clusters = clusters; tb.runoff = runoff; tb.err = nullptr;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = launch_tables(B, w, cosb, lcos, lsin, lfact, s);
    if (e == cudaSuccess) e = launch_log_weights(B, w, lw, s);
    if (e == cudaSuccess) {
        noalloc_layout_kernel<<<64, 256, 0, s>>>(B, clusters, runoff);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_dwt_forward_fp64(tb, reinterpret_cast<const double2 *>(S), reinterpret_cast<double2 *>(coef), s);
    return e == cudaSuccess ? SOFT_OK : fail("soft_dwt_forward_noalloc: kernel launch", e);
}
