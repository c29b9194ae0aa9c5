// soft_api.cu -- plans and the C ABI declared in include/soft.h.
//
// A plan owns, on one device: the quadrature and beta tables (computed by a
// kernel), the cluster work list, the coefficient run-offset table, the S
// workspace ((2B)^3 complex doubles) and the slice-FFT tables (the library's
// own FFT for power-of-two 2B, else a batched 2-D cuFFT plan over the 2B beta
// slices).  The transforms are the two steps of Sec. 2.4: a 2-D FFT per
// beta slice and the DWT per order pair (forward), or the iDWT per order pair
// and a 2-D FFT per slice (inverse).
#include "soft.h"
#include "soft_internal.cuh"

#include <cufft.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <new>
#include <vector>

using namespace softgb;

namespace {

constexpr uint64_t kPlanMagic = 0x534f46545f504c4eULL;  // "SOFT_PLN"
std::atomic<unsigned long long> g_launches{0};
std::atomic<long long> g_live_allocs{0};  // device allocations the library holds (soft_live_allocations)
thread_local unsigned long long t_launches = 0;  // this thread's share, to size graph captures

}  // namespace

void softgb::count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}

unsigned long long soft_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

long long soft_live_allocations(void) { return g_live_allocs.load(std::memory_order_relaxed); }

struct soft_plan_s {
    uint64_t magic;
    int B, dtype, device;
    double *w, *cosb, *lcos, *lsin, *lfact;
    int2 *clusters;
    int ncl;
    std::vector<int2> h_clusters;  // host copy of the cluster work list
    int64_t *runoff;
    double2 *S;
    int *err;
    cufftHandle fft;
    bool fft_made;
    double *lw;  // log w_B(j)
    double *seedtab, *rectab;  // per-cluster seeds and recurrence coefficients, built at creation
    int *fwd_order, *inv_order;  // FP64 and FP64-TC plans: the DWT and iDWT dispatch orders (Tables)
    float4 *dftw;              // FP64-TC plans with power-of-two 2B: double-float FFT twiddles (else null)
    int *dfexp;                // and its row (real-grid inverse: column) scales (n^2 ints)
    FftTw64 *tw64;             // FP64 / FP64-TC plans with power-of-two 2B: FP64 FFT twiddles (FP64 plans'
                               // slice FFT, both plans' real-grid FFT; else null: cuFFT Z2Z)
    int *colexp;               // FP64-TC plans: per-(m, m') exponents of S for the DWT's column scales
    int wexp;                  // 2^wexp > max_j w_B(j)
    // Mixed-precision plans: FP32 grid staging and S in layout [m][m'][j], FP32 cuFFT plans.
    float2 *g32, *S32;
    cufftHandle fft32f, fft32i;
    bool fft32f_made, fft32i_made;
    double2 *stage_grid, *stage_coef;  // for the host-buffer entry points, allocated on first use
    // Host-buffer entry points with the library's own slice FFT: a copy stream and
    // events that pipeline the grid's host copies with the FFTs, slice chunk by
    // slice chunk (created on first use).
    static constexpr int kHostChunks = 8;
    cudaStream_t copy_stream;
    bool copy_made;
    cudaEvent_t hev[kHostChunks + 1];
    double2 *corr_coef;                // correlation coefficients, allocated on first use
    // Sharded transforms (allocated on first use): the device copies of a
    // cluster subset (plan cluster indices) and of an order-pair column list,
    // and the host map (m, m') -> plan cluster index.
    int *dsub;
    int2 *dcols;
    std::vector<int> h_cluster_pos;
    double *amax_v;                    // arg-max partial results (argmax_parts() each)
    int64_t *amax_i;

    // Per-phase timing (soft_plan_enable_timing): 3 events per timed call.
    static constexpr int kMaxRec = 4096;
    bool timing;
    int fwd_variant, inv_variant;  // tile-shape variants chosen by soft_plan_set_variant
    // Allocation-failure injection for tests: device allocations this plan may
    // still make (-1 = no limit), from SOFT_TEST_ALLOC_BUDGET at creation.
    long long alloc_budget;
    int nrec;
    int rec_kind[kMaxRec];             // 0 = forward, 1 = inverse
    std::vector<cudaEvent_t> events;   // 3 * kMaxRec, created on first use
    double ms[4];
    int64_t counts[4];

    Tables tables() const {
        Tables t;
        t.B = B; t.ncl = ncl; t.w = w; t.lw = lw; t.cosb = cosb; t.lcos = lcos; t.lsin = lsin; t.lfact = lfact;
        t.clusters = clusters; t.runoff = runoff; t.err = err;
        t.fwd_variant = fwd_variant; t.inv_variant = inv_variant;
        t.seedtab = seedtab; t.rectab = rectab; t.fwd_order = fwd_order; t.inv_order = inv_order;
        t.wexp = wexp; t.colexp = colexp;
        return t;
    }
};

namespace {

// Keeps the caller's current device unchanged across a call.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

thread_local char g_last_error[256] = "";

void set_error(const char *where, const char *what) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, what);
}

soft_status fail_cuda(const char *where, cudaError_t e) {
    set_error(where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SOFT_ERR_OUT_OF_MEMORY : SOFT_ERR_CUDA;
}

soft_status fail_cufft(const char *where, cufftResult r) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "cufftResult %d", (int)r);
    set_error(where, buf);
    return SOFT_ERR_CUDA;
}

bool valid(const soft_plan_s *p) { return p != nullptr && p->magic == kPlanMagic; }

// Every device allocation of the library goes through dev_alloc / dev_free,
// which keep the count soft_live_allocations() reports.  An allocation made
// for plan p fails as out of memory once p's test budget is used up.
cudaError_t dev_alloc(soft_plan_s *p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (p && p->alloc_budget >= 0) {
        if (p->alloc_budget == 0) return cudaErrorMemoryAllocation;
        --p->alloc_budget;
    }
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1, std::memory_order_relaxed);
    else *ptr = nullptr;
    return e;
}

template <class T>
cudaError_t dev_alloc(soft_plan_s *p, T **ptr, size_t bytes) {
    void *v = nullptr;
    const cudaError_t e = dev_alloc(p, &v, bytes);
    *ptr = static_cast<T *>(v);
    return e;
}

template <class T>
void dev_free(T *&ptr) {
    if (ptr) {
        cudaFree(const_cast<void *>(static_cast<const void *>(ptr)));
        g_live_allocs.fetch_sub(1, std::memory_order_relaxed);
        ptr = nullptr;
    }
}

// SOFT_TEST_ALLOC_BUDGET=N (a test hook, off when unset): a plan created
// while it is set may make N device allocations in all; the next fails as
// out of memory.  Read once per soft_plan_create.
long long alloc_budget_from_env() {
    const char *v = std::getenv("SOFT_TEST_ALLOC_BUDGET");
    if (!v || !*v) return -1;
    char *end = nullptr;
    const long long n = std::strtoll(v, &end, 10);
    return (end && *end == '\0' && n >= 0) ? n : -1;
}

}  // namespace

namespace softgb {
void set_last_error_message(const char *where, const char *what) { set_error(where, what); }
}  // namespace softgb

namespace {
bool aligned16(const void *ptr) { return ptr != nullptr && (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }
soft_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SOFT_OK;
    set_error("CUDA", cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return SOFT_ERR_OUT_OF_MEMORY;
    return SOFT_ERR_CUDA;
}

int64_t sum_sq(int64_t x) { return x * (x + 1) * (2 * x + 1) / 6; }  // 1^2 + ... + x^2

// Start of the run of (m, m') in the coefficient array (layout in soft.h), closed form.
// Row m holds B^2 - m^2 entries; within row m (mu = |m|) the run of m' has length
// B - max(mu, |m'|).
int64_t run_start(int B, int m, int mp) {
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
        if (mp <= mu + 1) {
            in += (mp + mu) * (B - mu);
        } else {
            const int64_t c = mp - mu - 1;
            in += (2 * mu + 1) * (B - mu) + c * (2 * B - mu - mp) / 2;
        }
    }
    return row + in;
}

// Plans whose S is FP64 in layout [j][m][m'] with Z2Z FFTs (plain FP64 and FP64 on tensor cores).
bool fp64_layout(int dtype) { return dtype == SOFT_FP64 || dtype == SOFT_FP64_TC; }

cudaError_t launch_dwt_forward_plan(const soft_plan_s *p, const double2 *S, double2 *coef, cudaStream_t s,
                                    int flags) {
    return p->dtype == SOFT_FP64_TC ? launch_dwt_forward_tc(p->tables(), S, coef, s, flags)
                                    : launch_dwt_forward_fp64(p->tables(), S, coef, s, flags);
}

cudaError_t launch_dwt_inverse_plan(const soft_plan_s *p, const double2 *coef, double2 *S, cudaStream_t s,
                                    int flags) {
    return p->dtype == SOFT_FP64_TC ? launch_dwt_inverse_tc(p->tables(), coef, S, s, flags)
                                    : launch_dwt_inverse_fp64(p->tables(), coef, S, s, flags);
}

soft_status check_plan_args(const soft_plan_s *p, const void *a, const void *b) {
    if (!valid(p)) return SOFT_ERR_INVALID_ARG;
    if (!aligned16(a) || !aligned16(b) || a == b) return SOFT_ERR_INVALID_ARG;
    return SOFT_OK;
}

size_t grid_elems(int B) { return (size_t)(2 * B) * (2 * B) * (2 * B); }

// Adds the pending timing records to the sums (waits for their events).
void fold_timing(soft_plan_s *p) {
    for (int r = 0; r < p->nrec; ++r) {
        cudaEvent_t *e = &p->events[3 * r];
        float a = 0.f, b = 0.f;
        if (cudaEventSynchronize(e[2]) != cudaSuccess) continue;
        cudaEventElapsedTime(&a, e[0], e[1]);
        cudaEventElapsedTime(&b, e[1], e[2]);
        const int k = p->rec_kind[r] == 0 ? 0 : 2;
        p->ms[k] += a; p->ms[k + 1] += b;
        p->counts[k] += 1; p->counts[k + 1] += 1;
    }
    p->nrec = 0;
}

// Returns the 3 events of a new timing record, or nullptr when timing is off.
cudaEvent_t *timing_slot(soft_plan_s *p, int kind) {
    if (!p->timing) return nullptr;
    if (p->events.empty()) {
        p->events.resize(3 * soft_plan_s::kMaxRec);
        for (auto &e : p->events)
            if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    }
    if (p->nrec == soft_plan_s::kMaxRec) fold_timing(p);
    cudaEvent_t *e = &p->events[3 * p->nrec];
    if (!e[0] || !e[1] || !e[2]) return nullptr;
    p->rec_kind[p->nrec++] = kind;
    return e;
}

void free_plan(soft_plan_s *p) {
    if (!p) return;
    for (auto &e : p->events)
        if (e) cudaEventDestroy(e);
    for (auto &e : p->hev)
        if (e) cudaEventDestroy(e);
    if (p->copy_made) cudaStreamDestroy(p->copy_stream);
    if (p->fft_made) cufftDestroy(p->fft);
    if (p->fft32f_made) cufftDestroy(p->fft32f);
    if (p->fft32i_made) cufftDestroy(p->fft32i);
    dev_free(p->lw); dev_free(p->g32); dev_free(p->S32);
    dev_free(p->seedtab); dev_free(p->rectab); dev_free(p->fwd_order); dev_free(p->inv_order);
    dev_free(p->dftw); dev_free(p->dfexp); dev_free(p->tw64); dev_free(p->colexp);
    dev_free(p->w); dev_free(p->cosb); dev_free(p->lcos); dev_free(p->lsin); dev_free(p->lfact);
    dev_free(p->clusters); dev_free(p->runoff); dev_free(p->S); dev_free(p->err);
    dev_free(p->stage_grid); dev_free(p->stage_coef);
    dev_free(p->corr_coef); dev_free(p->amax_v); dev_free(p->amax_i);
    dev_free(p->dsub); dev_free(p->dcols);
    p->magic = 0;
    delete p;
}

// Mixed plans, the steps around the DWT: grid (FP64) -> S32 [m][m'][j] ...
soft_status mixed_grid_to_S(soft_plan_s *p, const double *grid, cudaStream_t s) {
    cudaError_t e = launch_f64_to_f32(reinterpret_cast<const double2 *>(grid), p->g32, (int64_t)grid_elems(p->B), s);
    if (e != cudaSuccess) return fail_cuda("grid conversion kernel launch", e);
    cufftResult r = cufftSetStream(p->fft32f, s);
    if (r != CUFFT_SUCCESS) return fail_cufft("cufftSetStream", r);
    // S(m,m';j) with exp(+i...) = cuFFT INVERSE, in place per contiguous slice,
    // then transposed from [j][m][m'] to [m][m'][j].
    r = cufftExecC2C(p->fft32f, reinterpret_cast<cufftComplex *>(p->g32), reinterpret_cast<cufftComplex *>(p->g32),
                     CUFFT_INVERSE);
    if (r != CUFFT_SUCCESS) return fail_cufft("cufftExecC2C (forward slices)", r);
    const int n = 2 * p->B;
    e = launch_transpose32(p->g32, p->S32, n, (int64_t)n * n, s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("transpose kernel launch", e);
}

// ... and S32 -> grid (FP64): transpose, FFT with exp(-i...), conversion.
soft_status mixed_S_to_grid(soft_plan_s *p, double *grid, cudaStream_t s) {
    const int n = 2 * p->B;
    cudaError_t e = launch_transpose32(p->S32, p->g32, n * n, (int64_t)n, s);
    if (e != cudaSuccess) return fail_cuda("transpose kernel launch", e);
    cufftResult r = cufftSetStream(p->fft32f, s);
    if (r != CUFFT_SUCCESS) return fail_cufft("cufftSetStream", r);
    r = cufftExecC2C(p->fft32f, reinterpret_cast<cufftComplex *>(p->g32), reinterpret_cast<cufftComplex *>(p->g32),
                     CUFFT_FORWARD);
    if (r != CUFFT_SUCCESS) return fail_cufft("cufftExecC2C (inverse slices)", r);
    e = launch_f32_to_f64(p->g32, reinterpret_cast<double2 *>(grid), (int64_t)grid_elems(p->B), s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("grid conversion kernel launch", e);
}

soft_status run_forward_mixed(soft_plan_s *p, const double *grid, double *coef, cudaStream_t s, int flags) {
    cudaEvent_t *ev = timing_slot(p, 0);
    if (ev) cudaEventRecord(ev[0], s);
    soft_status st = mixed_grid_to_S(p, grid, s);
    if (st != SOFT_OK) return st;
    if (ev) cudaEventRecord(ev[1], s);
    cudaError_t e = launch_dwt_forward_mixed(p->dtype, p->tables(), p->lw, p->S32, coef, s, flags);
    if (e != cudaSuccess) return fail_cuda("mixed DWT kernel launch", e);
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

soft_status run_inverse_mixed(soft_plan_s *p, const double *coef, double *grid, cudaStream_t s, int flags) {
    cudaEvent_t *ev = timing_slot(p, 1);
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_zero_nyquist32(p->B, p->S32, s);
    if (e != cudaSuccess) return fail_cuda("S clearing kernel launch", e);
    e = launch_dwt_inverse_mixed(p->dtype, p->tables(), coef, p->S32, s, flags);
    if (e != cudaSuccess) return fail_cuda("mixed iDWT kernel launch", e);
    if (ev) cudaEventRecord(ev[1], s);
    soft_status st = mixed_S_to_grid(p, grid, s);
    if (st != SOFT_OK) return st;
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

// The 2-D DFTs of the beta slices in the FP64 layouts, in -> out
// ([j][i][k] <-> [j][m][m']), exp(sign i ...), unnormalised: the library's
// double-float (FP64-TC plans) or FP64 (FP64 plans) FFT for power-of-two 2B,
// cuFFT Z2Z otherwise.  For sign < 0 `in` is the plan's S and may be
// overwritten.  Slices j0 .. j0 + nsl - 1 only (`in` and `out` point at slice
// 0); a partial range needs the library's own FFT (own_slice_fft()).
bool own_slice_fft(const soft_plan_s *p) { return p->dftw || p->tw64; }

soft_status slice_fft(soft_plan_s *p, const double2 *in, double2 *out, int sign, cudaStream_t s, int j0 = 0,
                      int nsl = -1) {
    const int n = 2 * p->B;
    if (nsl < 0) nsl = n;
    const size_t off = (size_t)j0 * n * n;
    if (p->dftw) {
        cudaError_t e = launch_df_fft2(p->B, in + off, out + off, reinterpret_cast<float4 *>(p->S) + off, p->dftw, sign,
                                       p->dfexp + (size_t)j0 * n, s, nsl);
        return e == cudaSuccess ? SOFT_OK : fail_cuda("double-float FFT launch", e);
    }
    if (p->tw64) {
        cudaError_t e = launch_fft64_2d(p->B, in + off, out + off, p->tw64, sign, s, nsl);
        return e == cudaSuccess ? SOFT_OK : fail_cuda("FP64 FFT launch", e);
    }
    if (j0 != 0 || nsl != n) return SOFT_ERR_INVALID_ARG;
    cufftResult r = cufftSetStream(p->fft, s);
    if (r != CUFFT_SUCCESS) return fail_cufft("cufftSetStream", r);
    // cuFFT's INVERSE direction is exp(+i ...), its FORWARD direction exp(-i ...)
    r = cufftExecZ2Z(p->fft, reinterpret_cast<cufftDoubleComplex *>(const_cast<double2 *>(in)),
                     reinterpret_cast<cufftDoubleComplex *>(out), sign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD);
    return r == CUFFT_SUCCESS ? SOFT_OK : fail_cufft(sign > 0 ? "cufftExecZ2Z (forward slices)"
                                                              : "cufftExecZ2Z (inverse slices)", r);
}

soft_status ensure_copy_stream(soft_plan_s *p) {
    if (!p->copy_made) {
        const cudaError_t e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail_cuda("copy stream", e);
        p->copy_made = true;
    }
    for (auto &ev : p->hev) {
        if (ev) continue;
        const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { ev = nullptr; return fail_cuda("copy events", e); }
    }
    return SOFT_OK;
}

// Slice chunk c of K: slices [c n / K, (c + 1) n / K).
int chunk_begin(int n, int K, int c) { return (int)((int64_t)c * n / K); }

// Number of slice chunks of the host pipeline: chunks of at least 8 MiB for
// the FP64 FFT and 32 MiB for the double-float FFT (whose columns pass takes
// up to 32 columns per block, so smaller chunks leave SMs idle), at most
// kHostChunks.  Smaller chunks measured slower: each one costs launches and
// event round trips.
int host_chunks(const soft_plan_s *p) {
    const int n = 2 * p->B;
    const double bytes = 16.0 * (double)n * n * n;
    const double per = (p->dftw ? 32.0 : 8.0) * 1024 * 1024;
    return std::max(1, std::min(std::min(soft_plan_s::kHostChunks, n), (int)(bytes / per)));
}

// Forward FFT stage fed from host memory: chunk c of the grid is copied to
// the device buffer `grid` on the plan's copy stream, and its slices'
// FFTs run on `s` as soon as that copy lands, while the next chunk copies.
soft_status forward_fft_from_host(soft_plan_s *p, const double *grid_host, double2 *grid, cudaStream_t s) {
    const int n = 2 * p->B, K = host_chunks(p);
    const size_t slice = (size_t)n * n;
    cudaStream_t cs = p->copy_stream;
    // the copies overwrite `grid`: they wait for the work already queued on s
    cudaError_t e = cudaEventRecord(p->hev[K], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, p->hev[K], 0);
    if (e != cudaSuccess) return fail_cuda("copy stream ordering", e);
    for (int c = 0; c < K; ++c) {
        const int j0 = chunk_begin(n, K, c), j1 = chunk_begin(n, K, c + 1);
        e = cudaMemcpyAsync(grid + j0 * slice, reinterpret_cast<const double2 *>(grid_host) + j0 * slice,
                            sizeof(double2) * slice * (j1 - j0), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(p->hev[c], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->hev[c], 0);
        if (e != cudaSuccess) return fail_cuda("grid chunk copy", e);
        soft_status st = slice_fft(p, grid, p->S, +1, s, j0, j1 - j0);
        if (st != SOFT_OK) return st;
    }
    return SOFT_OK;
}

// Inverse FFT stage drained to host memory: the FFTs of chunk c's slices
// run on `s` into the device buffer `grid`, and the chunk is copied to the
// host on the copy stream while the next chunk's FFTs run; `s` then waits
// for the last copy.
soft_status inverse_fft_to_host(soft_plan_s *p, double2 *grid, double *grid_host, cudaStream_t s) {
    const int n = 2 * p->B, K = host_chunks(p);
    const size_t slice = (size_t)n * n;
    cudaStream_t cs = p->copy_stream;
    for (int c = 0; c < K; ++c) {
        const int j0 = chunk_begin(n, K, c), j1 = chunk_begin(n, K, c + 1);
        soft_status st = slice_fft(p, p->S, grid, -1, s, j0, j1 - j0);
        if (st != SOFT_OK) return st;
        cudaError_t e = cudaEventRecord(p->hev[c], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, p->hev[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(reinterpret_cast<double2 *>(grid_host) + j0 * slice, grid + j0 * slice,
                                sizeof(double2) * slice * (j1 - j0), cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return fail_cuda("grid chunk copy", e);
    }
    cudaError_t e = cudaEventRecord(p->hev[K], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->hev[K], 0);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("copy stream ordering", e);
}

// flags: kApplyW | kApplyV for the forward transform, 0 for the adjoint of the inverse.
// grid_host: when set, `grid` is a device staging buffer that the FFT stage
// fills from this host copy of the grid, chunk by chunk.
soft_status run_forward(soft_plan_s *p, const double *grid, double *coef, cudaStream_t s,
                        int flags = kApplyW | kApplyV, const double *grid_host = nullptr) {
    if (!fp64_layout(p->dtype)) return run_forward_mixed(p, grid, coef, s, flags);
    cudaEvent_t *ev = timing_slot(p, 0);
    if (ev) cudaEventRecord(ev[0], s);
    // S(m,m';j) = sum_{i,k} f exp(+i(m alpha_i + m' gamma_k)), unnormalised.
    soft_status st =
        grid_host ? forward_fft_from_host(p, grid_host, reinterpret_cast<double2 *>(const_cast<double *>(grid)), s)
                  : slice_fft(p, reinterpret_cast<const double2 *>(grid), p->S, +1, s);
    if (st != SOFT_OK) return st;
    if (ev) cudaEventRecord(ev[1], s);
    cudaError_t e = launch_dwt_forward_plan(p, p->S, reinterpret_cast<double2 *>(coef), s, flags);
    if (e != cudaSuccess) return fail_cuda("DWT kernel launch", e);
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

// flags: 0 for the inverse transform, kApplyV | kApplyW for the adjoint of the forward.
// grid_host: when set, the FFT stage also copies `grid` (a device staging
// buffer) to this host buffer, chunk by chunk.
soft_status run_inverse(soft_plan_s *p, const double *coef, double *grid, cudaStream_t s, int flags = 0,
                        double *grid_host = nullptr) {
    if (!fp64_layout(p->dtype)) return run_inverse_mixed(p, coef, grid, s, flags);
    cudaEvent_t *ev = timing_slot(p, 1);
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_zero_nyquist(p->B, p->S, s);
    if (e != cudaSuccess) return fail_cuda("S clearing kernel launch", e);
    e = launch_dwt_inverse_plan(p, reinterpret_cast<const double2 *>(coef), p->S, s, flags);
    if (e != cudaSuccess) return fail_cuda("iDWT kernel launch", e);
    if (ev) cudaEventRecord(ev[1], s);
    // f = sum_{m,m'} S exp(-i(m alpha_i + m' gamma_k)), unnormalised.
    soft_status st = grid_host ? inverse_fft_to_host(p, reinterpret_cast<double2 *>(grid), grid_host, s)
                               : slice_fft(p, p->S, reinterpret_cast<double2 *>(grid), -1, s);
    if (st != SOFT_OK) return st;
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

soft_status ensure_staging(soft_plan_s *p) {
    if (!p->stage_grid) {
        const cudaError_t e = dev_alloc(p, &p->stage_grid, sizeof(double2) * grid_elems(p->B));
        if (e != cudaSuccess) return fail_cuda("host-call grid staging buffer", e);
    }
    if (!p->stage_coef) {
        const cudaError_t e = dev_alloc(p, &p->stage_coef, sizeof(double2) * (size_t)soft_num_coeffs(p->B));
        if (e != cudaSuccess) return fail_cuda("host-call coefficient staging buffer", e);
    }
    return SOFT_OK;
}

// ---------------------------------------------------------------------------
// Batches: a list of transforms (any mix of bandwidths and modes, one plan per
// entry) captured once into a CUDA graph and replayed on the caller's stream.
// The FP64 transforms of a batch, of any bandwidths, share one persistent
// DWT (forward) or iDWT (inverse, correlation) launch over all their
// (transform, cluster) items, heaviest first; mixed-precision transforms of
// one (mode, B) share one tensor-core launch per group of up to 8; FP64-TC
// transforms run their per-plan kernels inside the same graph.
// ---------------------------------------------------------------------------
enum BatchKind { kBatchInverse = 0, kBatchForward = 1, kBatchCorrelate = 2 };

struct BatchGraph {
    int kind = 0;
    std::vector<soft_plan_s *> plans;
    std::vector<const void *> key;  // every pointer argument, in order
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;  // kernel launches recorded in the graph
    BatchXform *d_xf = nullptr;
    int2 *d_items = nullptr;
    int *d_counter = nullptr;
    ~BatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        dev_free(d_xf); dev_free(d_items); dev_free(d_counter);
    }
};

std::mutex g_batch_mu;
std::list<BatchGraph *> g_batches;  // most recently used first
constexpr size_t kMaxCachedBatches = 16;

void purge_batches_of(const soft_plan_s *p) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find((*it)->plans.begin(), (*it)->plans.end(), p) != (*it)->plans.end()) {
            delete *it;
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}

// Records the batch's work on stream cs (which is being captured).
soft_status record_batch(BatchGraph *bg, int n, const void *const *a, const void *const *b, const void *const *c,
                         const void *const *d, int64_t *best_index, double *best_value, cudaStream_t cs) {
    std::vector<int> pers, rest;
    int maxB = 1;
    for (int i = 0; i < n; ++i) {
        soft_plan_s *p = bg->plans[i];
        if (p->dtype == SOFT_FP64) {
            pers.push_back(i);
            maxB = std::max(maxB, p->B);
        } else {
            rest.push_back(i);
        }
    }
    cudaError_t e = cudaSuccess;
    if (!pers.empty() && bg->kind == kBatchForward) {
        // every FP64 transform's slice FFTs into its plan's S, then one persistent
        // DWT launch over all their (transform, cluster) items
        e = cudaMemsetAsync(bg->d_counter, 0, sizeof(int), cs);
        if (e != cudaSuccess) return fail_cuda("batched forward DWT", e);
        int nitems = 0;
        for (int i : pers) {
            soft_plan_s *p = bg->plans[i];
            soft_status st = slice_fft(p, static_cast<const double2 *>(a[i]), p->S, +1, cs);
            if (st != SOFT_OK) return st;
            nitems += p->ncl;
        }
        e = launch_dwt_fp64_persistent(bg->d_xf, bg->d_items, nitems, bg->d_counter, maxB, cs);
        if (e != cudaSuccess) return fail_cuda("batched forward DWT", e);
    } else if (!pers.empty()) {
        e = cudaMemsetAsync(bg->d_counter, 0, sizeof(int), cs);
        for (int i : pers) {
            soft_plan_s *p = bg->plans[i];
            if (e == cudaSuccess && bg->kind == kBatchCorrelate)
                e = launch_corr_coeffs(p->B, static_cast<const double2 *>(a[i]), static_cast<const double2 *>(b[i]),
                                       p->runoff, p->corr_coef, cs);
            if (e == cudaSuccess) e = launch_zero_nyquist(p->B, p->S, cs);
        }
        if (e == cudaSuccess) {
            int nitems = 0;
            for (int i : pers) nitems += bg->plans[i]->ncl;
            e = launch_idwt_fp64_persistent(bg->d_xf, bg->d_items, nitems, bg->d_counter, maxB, cs);
        }
        if (e != cudaSuccess) return fail_cuda("batched inverse DWT", e);
        for (int i : pers) {
            soft_plan_s *p = bg->plans[i];
            double *grid = bg->kind == kBatchCorrelate ? static_cast<double *>(const_cast<void *>(c[i]))
                                                       : static_cast<double *>(const_cast<void *>(b[i]));
            soft_status st = slice_fft(p, p->S, reinterpret_cast<double2 *>(grid), -1, cs);
            if (st != SOFT_OK) return st;
            if (bg->kind == kBatchCorrelate) {
                e = launch_argmax_real(reinterpret_cast<const double2 *>(grid), (int64_t)grid_elems(p->B), p->amax_v,
                                       p->amax_i, best_index + i, best_value + i, cs);
                if (e != cudaSuccess) return fail_cuda("batched arg-max", e);
            }
        }
    }
    // Mixed-precision transforms of one (mode, B): groups of 8, 4, 2, 1 share one
    // DWT launch, so each Wigner-d tile feeds 16 x group tensor-core columns.
    std::vector<int> single;
    if (bg->kind != kBatchCorrelate) {
        std::vector<bool> taken(n, false);
        for (int i : rest) {
            soft_plan_s *p = bg->plans[i];
            if (fp64_layout(p->dtype) || taken[i]) continue;
            std::vector<int> grp;
            for (int j : rest)
                if (!taken[j] && bg->plans[j]->dtype == p->dtype && bg->plans[j]->B == p->B) grp.push_back(j);
            for (size_t g0 = 0; g0 < grp.size();) {
                const size_t left = grp.size() - g0;
                const int nb = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
                const float2 *Sv[kMaxMixedBatch];
                float2 *Sw[kMaxMixedBatch];
                double *cw[kMaxMixedBatch];
                const double *cr[kMaxMixedBatch];
                for (int t = 0; t < nb; ++t) {
                    const int idx = grp[g0 + t];
                    soft_plan_s *q = bg->plans[idx];
                    taken[idx] = true;
                    Sv[t] = q->S32;
                    Sw[t] = q->S32;
                    cw[t] = static_cast<double *>(const_cast<void *>(b[idx]));
                    cr[t] = static_cast<const double *>(a[idx]);
                    soft_status st = SOFT_OK;
                    if (bg->kind == kBatchForward) {
                        st = mixed_grid_to_S(q, static_cast<const double *>(a[idx]), cs);
                    } else {
                        cudaError_t e0 = launch_zero_nyquist32(q->B, q->S32, cs);
                        if (e0 != cudaSuccess) st = fail_cuda("S clearing kernel launch", e0);
                    }
                    if (st != SOFT_OK) return st;
                }
                const Tables tb = p->tables();
                e = bg->kind == kBatchForward
                        ? launch_dwt_forward_mixed_batch(p->dtype, tb, nb, Sv, cw, cs)
                        : launch_dwt_inverse_mixed_batch(p->dtype, tb, nb, cr, Sw, cs);
                if (e != cudaSuccess) return fail_cuda("batched mixed DWT", e);
                if (bg->kind == kBatchInverse)
                    for (int t = 0; t < nb; ++t) {
                        const int idx = grp[g0 + t];
                        soft_status st =
                            mixed_S_to_grid(bg->plans[idx], static_cast<double *>(const_cast<void *>(b[idx])), cs);
                        if (st != SOFT_OK) return st;
                    }
                g0 += nb;
            }
        }
        for (int i : rest)
            if (!taken[i]) single.push_back(i);
    } else {
        single = rest;
    }
    for (int i : single) {
        soft_plan_s *p = bg->plans[i];
        soft_status st = SOFT_OK;
        if (bg->kind == kBatchForward) {
            st = run_forward(p, static_cast<const double *>(a[i]), static_cast<double *>(const_cast<void *>(b[i])), cs);
        } else if (bg->kind == kBatchInverse) {
            st = run_inverse(p, static_cast<const double *>(a[i]), static_cast<double *>(const_cast<void *>(b[i])), cs);
        } else {
            double *grid = static_cast<double *>(const_cast<void *>(c[i]));
            e = launch_corr_coeffs(p->B, static_cast<const double2 *>(a[i]), static_cast<const double2 *>(b[i]),
                                   p->runoff, p->corr_coef, cs);
            if (e != cudaSuccess) return fail_cuda("batched correlation coefficients", e);
            st = run_inverse(p, reinterpret_cast<const double *>(p->corr_coef), grid, cs);
            if (st == SOFT_OK) {
                e = launch_argmax_real(reinterpret_cast<const double2 *>(grid), (int64_t)grid_elems(p->B), p->amax_v,
                                       p->amax_i, best_index + i, best_value + i, cs);
                if (e != cudaSuccess) return fail_cuda("batched arg-max", e);
            }
        }
        if (st != SOFT_OK) return st;
    }
    (void)d;
    return SOFT_OK;
}

// Validates a batch, finds or builds its graph, and launches it on `stream`.
soft_status run_batch(int kind, int n, const soft_plan *plans, const void *const *a, const void *const *b,
                      const void *const *c, int64_t *best_index, double *best_value, void *stream) {
    if (n < 1 || !plans || !a || !b || (kind == kBatchCorrelate && (!c || !best_index || !best_value)))
        return SOFT_ERR_INVALID_ARG;
    std::vector<const void *> key;
    std::vector<soft_plan_s *> ps(n);
    int device = -1;
    for (int i = 0; i < n; ++i) {
        soft_plan_s *p = plans[i];
        if (!valid(p)) return SOFT_ERR_INVALID_ARG;
        if (device < 0) device = p->device;
        if (p->device != device) return SOFT_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ps[j] == p) return SOFT_ERR_INVALID_ARG;  // each entry needs its own plan workspace
        ps[i] = p;
        if (!aligned16(a[i]) || !aligned16(b[i]) || (c && !aligned16(c[i]))) return SOFT_ERR_INVALID_ARG;
        key.push_back(p); key.push_back(a[i]); key.push_back(b[i]); key.push_back(c ? c[i] : nullptr);
    }
    key.push_back(best_index); key.push_back(best_value);
    DeviceGuard g(device);
    cudaStream_t user = static_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchGraph *bg = nullptr;
    for (auto it = g_batches.begin(); it != g_batches.end(); ++it)
        if ((*it)->kind == kind && (*it)->key == key) {
            bg = *it;
            g_batches.erase(it);
            g_batches.push_front(bg);
            break;
        }
    if (!bg) {
        bg = new (std::nothrow) BatchGraph();
        if (!bg) return SOFT_ERR_OUT_OF_MEMORY;
        bg->kind = kind;
        bg->plans = ps;
        bg->key = key;
        // Workspaces and the persistent kernel's tables, allocated before capture.
        std::vector<BatchXform> xf(n);
        std::vector<std::pair<int64_t, int2>> items;
        for (int i = 0; i < n; ++i) {
            soft_plan_s *p = ps[i];
            if (kind == kBatchCorrelate && !p->corr_coef) {
                cudaError_t e = dev_alloc(p, &p->corr_coef, sizeof(double2) * (size_t)soft_num_coeffs(p->B));
                if (e != cudaSuccess) { delete bg; return fail_cuda("correlation workspace", e); }
            }
            xf[i].tb = p->tables();
            xf[i].coef = kind == kBatchCorrelate ? reinterpret_cast<const double *>(p->corr_coef)
                                                 : static_cast<const double *>(a[i]);
            xf[i].S = p->S;
            xf[i].Sin = p->S;
            xf[i].coef_out = kind == kBatchForward ? static_cast<double *>(const_cast<void *>(b[i])) : nullptr;
            xf[i].flags = kind == kBatchForward ? (kApplyW | kApplyV) : 0;
            if (p->dtype == SOFT_FP64)
                for (int cidx = 0; cidx < p->ncl; ++cidx) {
                    const int2 cl = p->h_clusters[cidx];
                    const int np = (cl.x == 0 && cl.y == 0) ? 1 : (cl.y == 0 || cl.x == cl.y) ? 4 : 8;
                    // FP64 work of the item, 2B samples x (B - m) degrees x: the iDWT's real
                    // columns + 2 of recurrence; the DWT's 16 columns whatever the partner
                    // count (its folded half-warps still occupy the FP64 pipe), 8 partners first
                    const int64_t deg = (int64_t)(p->B - cl.x) * (2 * p->B);
                    items.push_back({kind == kBatchForward ? deg * 18 + np : deg * (np == 8 ? 18 : 10),
                                     make_int2(i, cidx)});
                }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, int2> &x, const std::pair<int64_t, int2> &y) { return x.first > y.first; });
        std::vector<int2> hitems(items.size());
        for (size_t t = 0; t < items.size(); ++t) hitems[t] = items[t].second;
        cudaError_t e = dev_alloc(ps[0], &bg->d_xf, sizeof(BatchXform) * n);
        if (e == cudaSuccess) e = dev_alloc(ps[0], &bg->d_items, sizeof(int2) * std::max<size_t>(1, hitems.size()));
        if (e == cudaSuccess) e = dev_alloc(ps[0], &bg->d_counter, sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(bg->d_xf, xf.data(), sizeof(BatchXform) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !hitems.empty())
            e = cudaMemcpy(bg->d_items, hitems.data(), sizeof(int2) * hitems.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { delete bg; return fail_cuda("batch set-up", e); }

        // Capture on a private stream (per-phase timing is not recorded inside graphs).
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete bg; return fail_cuda("batch capture stream", e); }
        std::vector<bool> timing(n);
        for (int i = 0; i < n; ++i) { timing[i] = ps[i]->timing; ps[i]->timing = false; }
        cudaGraph_t graph = nullptr;
        const unsigned long long t0 = t_launches;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        soft_status st = e == cudaSuccess ? record_batch(bg, n, a, b, c, nullptr, best_index, best_value, cs)
                                          : fail_cuda("cudaStreamBeginCapture", e);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        // recorded, not run: the launch count takes them at each replay instead
        bg->launches = t_launches - t0;
        g_launches.fetch_sub(bg->launches, std::memory_order_relaxed);
        for (int i = 0; i < n; ++i) ps[i]->timing = timing[i];
        if (st == SOFT_OK && e2 != cudaSuccess) st = fail_cuda("cudaStreamEndCapture", e2);
        if (st == SOFT_OK) {
            e = cudaGraphInstantiate(&bg->exec, graph, 0);
            if (e != cudaSuccess) st = fail_cuda("cudaGraphInstantiate", e);
        }
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (st != SOFT_OK) { delete bg; return st; }
        g_batches.push_front(bg);
        while (g_batches.size() > kMaxCachedBatches) {
            delete g_batches.back();
            g_batches.pop_back();
        }
    }
    cudaError_t e = cudaGraphLaunch(bg->exec, user);
    if (e != cudaSuccess) return fail_cuda("cudaGraphLaunch", e);
    g_launches.fetch_add(bg->launches, std::memory_order_relaxed);
    return SOFT_OK;
}

// ---------------------------------------------------------------------------
// Sharded transforms: cluster subsets and S column lists.
// ---------------------------------------------------------------------------
int partner_count(int m, int mp) { return (m == 0 && mp == 0) ? 1 : (mp == 0 || m == mp) ? 4 : 8; }

// Work of a cluster for the shard balance: the DWT's per-degree cost (16
// columns, 8 partners first at equal degree count), as the dispatch orders.
int64_t cluster_work(int B, int m, int mp) { return (int64_t)(B - m) * 16 + partner_count(m, mp); }

// Plan cluster indices of the listed representatives, into the plan's device
// subset list (allocated on first use), on stream s.
soft_status upload_subset(soft_plan_s *p, const int *reps, int count, cudaStream_t s) {
    if (count < 0 || count > p->ncl || (count > 0 && !reps)) return SOFT_ERR_INVALID_ARG;
    if (p->h_cluster_pos.empty()) {
        p->h_cluster_pos.assign((size_t)p->B * (p->B + 1) / 2, -1);
        for (int c = 0; c < p->ncl; ++c) {
            const int2 r = p->h_clusters[c];
            p->h_cluster_pos[(size_t)r.x * (r.x + 1) / 2 + r.y] = c;
        }
    }
    if (!p->dsub) {
        const cudaError_t e = dev_alloc(p, &p->dsub, sizeof(int) * (size_t)p->ncl);
        if (e != cudaSuccess) return fail_cuda("cluster subset list", e);
    }
    std::vector<int> idx((size_t)count);
    for (int i = 0; i < count; ++i) {
        const int m = reps[2 * i], mp = reps[2 * i + 1];
        if (mp < 0 || mp > m || m >= p->B) return SOFT_ERR_INVALID_ARG;
        idx[i] = p->h_cluster_pos[(size_t)m * (m + 1) / 2 + mp];
    }
    if (count == 0) return SOFT_OK;
    // pageable source: the copy is staged before cudaMemcpyAsync returns, so the
    // temporary may go; stream order keeps earlier kernels' reads of the list first
    const cudaError_t e = cudaMemcpyAsync(p->dsub, idx.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("cluster subset copy", e);
}

soft_status upload_columns(soft_plan_s *p, const int *pairs, int npairs, cudaStream_t s) {
    const int R = 2 * p->B - 1;
    if (npairs < 0 || npairs > R * R || (npairs > 0 && !pairs)) return SOFT_ERR_INVALID_ARG;
    for (int i = 0; i < npairs; ++i)
        if (std::abs(pairs[2 * i]) >= p->B || std::abs(pairs[2 * i + 1]) >= p->B) return SOFT_ERR_INVALID_ARG;
    if (!p->dcols) {
        const cudaError_t e = dev_alloc(p, &p->dcols, sizeof(int2) * (size_t)R * R);
        if (e != cudaSuccess) return fail_cuda("column list", e);
    }
    if (npairs == 0) return SOFT_OK;
    const cudaError_t e = cudaMemcpyAsync(p->dcols, pairs, sizeof(int2) * (size_t)npairs, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("column list copy", e);
}

}  // namespace

extern "C" {

int soft_max_bandwidth(void) { return kMaxB; }

int64_t soft_num_coeffs(int B) {
    if (B < 1) return -1;
    return (int64_t)B * (4LL * B * B - 1) / 3;
}

int64_t soft_coef_index(int B, int l, int m, int mp) {
    if (B < 1) return -1;
    const int am = m < 0 ? -m : m, amp = mp < 0 ? -mp : mp;
    const int l0 = am > amp ? am : amp;
    if (l < l0 || l >= B) return -1;
    return run_start(B, m, mp) + (l - l0);
}

const char *soft_last_error(void) { return g_last_error; }

const char *soft_status_string(int status) {
    switch (status) {
        case SOFT_OK: return "SOFT_OK";
        case SOFT_ERR_INVALID_ARG: return "SOFT_ERR_INVALID_ARG";
        case SOFT_ERR_OUT_OF_MEMORY: return "SOFT_ERR_OUT_OF_MEMORY";
        case SOFT_ERR_CUDA: return "SOFT_ERR_CUDA";
        case SOFT_ERR_UNSUPPORTED: return "SOFT_ERR_UNSUPPORTED";
        case SOFT_ERR_TIMEOUT: return "SOFT_ERR_TIMEOUT";
        case SOFT_ERR_DEVICE: return "SOFT_ERR_DEVICE";
        default: return "SOFT_ERR_UNKNOWN";
    }
}

soft_status soft_plan_create(soft_plan *out, int B, int dtype) {
    if (!out) return SOFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1) return SOFT_ERR_INVALID_ARG;
    if (B > kMaxB) return SOFT_ERR_UNSUPPORTED;
    if (dtype != SOFT_FP64 && dtype != SOFT_MIXED_BF16X3 && dtype != SOFT_MIXED_TF32 && dtype != SOFT_FP64_TC)
        return SOFT_ERR_INVALID_ARG;
    soft_plan_s *p = new (std::nothrow) soft_plan_s();
    if (!p) return SOFT_ERR_OUT_OF_MEMORY;
    p->magic = kPlanMagic;
    p->B = B;
    p->dtype = dtype;
    p->alloc_budget = alloc_budget_from_env();
    if (cudaGetDevice(&p->device) != cudaSuccess) { free_plan(p); return SOFT_ERR_CUDA; }

    const int n = 2 * B;
    const int R = 2 * B - 1;
    // Cluster work list, heaviest first: work ~ (B - m) * number of partners.
    std::vector<int2> cl;
    cl.reserve((size_t)B * (B + 1) / 2);
    for (int m = 0; m < B; ++m)
        for (int mp = 0; mp <= m; ++mp) cl.push_back(make_int2(m, mp));
    auto weight = [B](const int2 &c) {
        const int np = (c.x == 0 && c.y == 0) ? 1 : (c.y == 0 || c.x == c.y) ? 4 : 8;
        return (int64_t)(B - c.x) * np;
    };
    std::stable_sort(cl.begin(), cl.end(), [&](const int2 &a, const int2 &b) { return weight(a) > weight(b); });
    p->ncl = (int)cl.size();
    p->h_clusters = cl;
    std::vector<int64_t> ro((size_t)R * R);
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) ro[runoff_index(B, m, mp)] = run_start(B, m, mp);

    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = dev_alloc(p, ptr, bytes);
    };
    alloc((void **)&p->w, sizeof(double) * n);
    alloc((void **)&p->cosb, sizeof(double) * n);
    alloc((void **)&p->lcos, sizeof(double) * n);
    alloc((void **)&p->lsin, sizeof(double) * n);
    alloc((void **)&p->lfact, sizeof(double) * (n + 1));
    alloc((void **)&p->clusters, sizeof(int2) * cl.size());
    alloc((void **)&p->runoff, sizeof(int64_t) * ro.size());
    alloc((void **)&p->err, sizeof(int));
    alloc((void **)&p->amax_v, sizeof(double) * argmax_parts());
    alloc((void **)&p->amax_i, sizeof(int64_t) * argmax_parts());
    alloc((void **)&p->lw, sizeof(double) * n);
    alloc((void **)&p->seedtab, sizeof(double) * (size_t)n * cl.size());
    alloc((void **)&p->rectab, sizeof(double) * 3 * (size_t)B * cl.size());
    // Mixed plans keep the shared order: their forward tile spans every degree
    // of a cluster up to B = 128, so their cost hardly depends on the degree count.
    if (fp64_layout(dtype)) alloc((void **)&p->fwd_order, sizeof(int) * cl.size());
    if (fp64_layout(dtype)) alloc((void **)&p->inv_order, sizeof(int) * cl.size());
    if (dtype == SOFT_FP64_TC) alloc((void **)&p->colexp, sizeof(int) * 2 * (size_t)n * n);
    if (dtype == SOFT_FP64_TC && df_fft_supported(B)) {
        alloc((void **)&p->dftw, sizeof(float4) * (size_t)(n / 2));
        alloc((void **)&p->dfexp, sizeof(int) * (size_t)n * n);
    }
    // FP64 twiddles: the FP64 plans' slice FFT, and the real-grid FFT of FP64 and FP64-TC plans
    if (fp64_layout(dtype) && fft64_supported(B)) alloc((void **)&p->tw64, sizeof(FftTw64) * fft64_twiddle_count(B));
    if (fp64_layout(dtype)) {
        alloc((void **)&p->S, sizeof(double2) * grid_elems(B));
    } else {
        alloc((void **)&p->g32, sizeof(float2) * grid_elems(B));
        alloc((void **)&p->S32, sizeof(float2) * grid_elems(B));
    }
    if (e != cudaSuccess) { free_plan(p); return fail_cuda("plan workspace", e); }

    e = cudaMemcpy(p->clusters, cl.data(), sizeof(int2) * cl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->fwd_order && p->inv_order) {
        // Longest first by each kernel's time per cluster.  The FP64 forward DWT
        // spends the same time per degree on 4 partners as on 8 (its idle
        // half-warps would still occupy the FP64 pipe, and it folds them away),
        // and the FP64-TC kernels always compute 16 columns: order by degree
        // count, 8 partners first at equal count.  The FP64 iDWT walks 16 real
        // columns for 8 partners and 8 otherwise, plus 2 FMAs of recurrence per
        // degree.
        auto partners = [](const int2 &c) { return (c.x == 0 && c.y == 0) ? 1 : (c.y == 0 || c.x == c.y) ? 4 : 8; };
        auto longest_first = [&](auto cost) {
            std::vector<int> ord(cl.size());
            for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost(cl[a]) > cost(cl[b]); });
            return ord;
        };
        const std::vector<int> fo = longest_first([&](const int2 &c) {
            return (int64_t)(B - c.x) * 16 + partners(c);
        });
        const std::vector<int> io = dtype == SOFT_FP64 ? longest_first([&](const int2 &c) {
            return (int64_t)(B - c.x) * (partners(c) == 8 ? 18 : 10);
        }) : fo;
        e = cudaMemcpy(p->fwd_order, fo.data(), sizeof(int) * fo.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->inv_order, io.data(), sizeof(int) * io.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(p->runoff, ro.data(), sizeof(int64_t) * ro.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, sizeof(int));
    if (e == cudaSuccess) e = launch_tables(B, p->w, p->cosb, p->lcos, p->lsin, p->lfact, 0);
    if (e == cudaSuccess) e = launch_log_weights(B, p->w, p->lw, 0);
    if (e == cudaSuccess) e = launch_cluster_tables(p->tables(), p->seedtab, p->rectab, 0);
    if (e == cudaSuccess && p->dftw) e = launch_df_twiddles(B, p->dftw, 0);
    if (e == cudaSuccess && p->tw64) e = launch_fft64_twiddles(B, p->tw64, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { free_plan(p); return cuda_status(e); }
    {
        // weight scale: the power of two just above the largest quadrature weight
        std::vector<double> hw((size_t)n);
        e = cudaMemcpy(hw.data(), p->w, sizeof(double) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { free_plan(p); return cuda_status(e); }
        double wmax = 0.0;
        for (double v : hw) wmax = std::max(wmax, std::fabs(v));
        int ex = 0;
        std::frexp(wmax, &ex);  // wmax = f 2^ex, f in [0.5, 1)
        p->wexp = wmax > 0.0 ? ex : 0;
    }

    long long dims[2] = {n, n};
    const long long slice = (long long)n * n;
    size_t work = 0;
    cufftResult r;
    if (p->dftw || p->tw64) {
        // Power-of-two 2B in the FP64 layouts: the library's own FFTs need no cuFFT plan.
    } else if (fp64_layout(dtype)) {
        // One batched 2-D Z2Z plan over the 2B contiguous beta slices, S in layout [j][m][m'].
        if (cufftCreate(&p->fft) != CUFFT_SUCCESS) { free_plan(p); return SOFT_ERR_CUDA; }
        p->fft_made = true;
        r = cufftMakePlanMany64(p->fft, 2, dims, nullptr, 1, slice, nullptr, 1, slice, CUFFT_Z2Z, n, &work);
        if (r != CUFFT_SUCCESS) { free_plan(p); return fail_cufft("cufftMakePlanMany64 (Z2Z)", r); }
    } else {
        // One FP32 C2C plan over the 2B contiguous slices, run in place on the
        // staging buffer in both directions; a tiled transpose moves S between
        // the FFT layout [j][m][m'] and the DWT layout [m][m'][j].
        if (cufftCreate(&p->fft32f) != CUFFT_SUCCESS) { free_plan(p); return SOFT_ERR_CUDA; }
        p->fft32f_made = true;
        r = cufftMakePlanMany64(p->fft32f, 2, dims, nullptr, 1, slice, nullptr, 1, slice, CUFFT_C2C, n, &work);
        if (r != CUFFT_SUCCESS) { free_plan(p); return fail_cufft("cufftMakePlanMany64 (C2C)", r); }
    }
    *out = p;
    return SOFT_OK;
}

soft_status soft_destroy(soft_plan p) {
    if (!p) return SOFT_OK;
    if (!valid(p)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    purge_batches_of(p);
    free_plan(p);
    return SOFT_OK;
}

int soft_plan_bandwidth(soft_plan p) { return valid(p) ? p->B : -1; }

soft_status soft_plan_sync(soft_plan p) {
    if (!valid(p)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    e = cudaMemcpy(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (h != 0) {
        cudaMemset(p->err, 0, sizeof(int));
        return h == 2 ? SOFT_ERR_TIMEOUT : SOFT_ERR_DEVICE;
    }
    return SOFT_OK;
}

soft_status soft_forward(soft_plan p, const double *grid, double *coef, void *stream) {
    soft_status st = check_plan_args(p, grid, coef);
    if (st != SOFT_OK) return st;
    DeviceGuard g(p->device);
    return run_forward(p, grid, coef, static_cast<cudaStream_t>(stream));
}

soft_status soft_inverse(soft_plan p, const double *coef, double *grid, void *stream) {
    soft_status st = check_plan_args(p, coef, grid);
    if (st != SOFT_OK) return st;
    DeviceGuard g(p->device);
    return run_inverse(p, coef, grid, static_cast<cudaStream_t>(stream));
}

// Real grids (FP64 and FP64-TC plans with power-of-two 2B): the slice FFTs
// (FP64 for FP64 plans, double-float for FP64-TC plans from B = 2 on, as
// their complex-grid FFTs) run on the m' >= 0 half of the spectrum (real-row
// DFTs of half length; every contracted partner has m' >= 0) and the DWT /
// iDWT contract only one partner of each conjugate pair (kRealSym).
soft_status soft_forward_real(soft_plan p, const double *grid, double *coef, void *stream) {
    soft_status st = check_plan_args(p, grid, coef);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype) || !p->tw64) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t *ev = timing_slot(p, 0);
    if (ev) cudaEventRecord(ev[0], s);
    // the m' >= 0 half the DWT reads
    cudaError_t e = p->dftw && df_real_fft_supported(p->B)
                        ? launch_df_fft2_r2c(p->B, grid, p->S, p->dftw, +1, p->dfexp, s)
                        : launch_fft64_2d_r2c(p->B, grid, p->S, p->tw64, +1, s);
    if (e != cudaSuccess) return fail_cuda("real-grid FFT launch", e);
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_dwt_forward_plan(p, p->S, reinterpret_cast<double2 *>(coef), s, kApplyW | kApplyV | kRealSym);
    if (e != cudaSuccess) return fail_cuda("DWT kernel launch", e);
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

soft_status soft_inverse_real(soft_plan p, const double *coef, double *grid, void *stream) {
    soft_status st = check_plan_args(p, coef, grid);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype) || !p->tw64) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t *ev = timing_slot(p, 1);
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_zero_nyquist(p->B, p->S, s);
    if (e != cudaSuccess) return fail_cuda("S clearing kernel launch", e);
    e = launch_dwt_inverse_plan(p, reinterpret_cast<const double2 *>(coef), p->S, s, kRealSym);
    if (e != cudaSuccess) return fail_cuda("iDWT kernel launch", e);
    if (ev) cudaEventRecord(ev[1], s);
    e = p->dftw && df_real_fft_supported(p->B) ? launch_df_fft2_c2r(p->B, p->S, grid, p->dftw, -1, p->dfexp, s)
                                               : launch_fft64_2d_c2r(p->B, p->S, grid, p->tw64, -1, s);
    if (e != cudaSuccess) return fail_cuda("real-grid FFT launch", e);
    if (ev) cudaEventRecord(ev[2], s);
    return SOFT_OK;
}

soft_status soft_forward_adjoint(soft_plan p, const double *coef, double *grid, void *stream) {
    soft_status st = check_plan_args(p, coef, grid);
    if (st != SOFT_OK) return st;
    DeviceGuard g(p->device);
    return run_inverse(p, coef, grid, static_cast<cudaStream_t>(stream), kApplyV | kApplyW);
}

soft_status soft_inverse_adjoint(soft_plan p, const double *grid, double *coef, void *stream) {
    soft_status st = check_plan_args(p, grid, coef);
    if (st != SOFT_OK) return st;
    DeviceGuard g(p->device);
    return run_forward(p, grid, coef, static_cast<cudaStream_t>(stream), 0);
}

soft_status soft_batched_inverse(int n, const soft_plan *plans, const double *const *coefs, double *const *grids,
                                 void *stream) {
    return run_batch(kBatchInverse, n, plans, reinterpret_cast<const void *const *>(coefs),
                     reinterpret_cast<const void *const *>(grids), nullptr, nullptr, nullptr, stream);
}

soft_status soft_batched_forward(int n, const soft_plan *plans, const double *const *grids, double *const *coefs,
                                 void *stream) {
    return run_batch(kBatchForward, n, plans, reinterpret_cast<const void *const *>(grids),
                     reinterpret_cast<const void *const *>(coefs), nullptr, nullptr, nullptr, stream);
}

soft_status soft_batched_correlate(int n, const soft_plan *plans, const double *const *f_sh,
                                   const double *const *g_sh, double *const *grids, int64_t *best_index,
                                   double *best_value, void *stream) {
    return run_batch(kBatchCorrelate, n, plans, reinterpret_cast<const void *const *>(f_sh),
                     reinterpret_cast<const void *const *>(g_sh), reinterpret_cast<const void *const *>(grids),
                     best_index, best_value, stream);
}

soft_status soft_correlation_coeffs(soft_plan p, const double *f_sh, const double *g_sh, double *coef, void *stream) {
    if (!valid(p) || !aligned16(f_sh) || !aligned16(g_sh) || !aligned16(coef)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    return cuda_status(launch_corr_coeffs(p->B, reinterpret_cast<const double2 *>(f_sh),
                                          reinterpret_cast<const double2 *>(g_sh), p->runoff,
                                          reinterpret_cast<double2 *>(coef), static_cast<cudaStream_t>(stream)));
}

soft_status soft_correlate(soft_plan p, const double *f_sh, const double *g_sh, double *grid, int64_t *best_index,
                           double *best_value, void *stream) {
    if (!valid(p) || !aligned16(f_sh) || !aligned16(g_sh) || !aligned16(grid)) return SOFT_ERR_INVALID_ARG;
    if ((best_index == nullptr) != (best_value == nullptr)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!p->corr_coef) {
        cudaError_t e = dev_alloc(p, &p->corr_coef, sizeof(double2) * (size_t)soft_num_coeffs(p->B));
        if (e != cudaSuccess) return fail_cuda("correlation workspace", e);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_corr_coeffs(p->B, reinterpret_cast<const double2 *>(f_sh),
                                       reinterpret_cast<const double2 *>(g_sh), p->runoff, p->corr_coef, s);
    if (e != cudaSuccess) return fail_cuda("correlation coefficient kernel launch", e);
    soft_status st = run_inverse(p, reinterpret_cast<const double *>(p->corr_coef), grid, s);
    if (st != SOFT_OK || !best_index) return st;
    e = launch_argmax_real(reinterpret_cast<const double2 *>(grid), (int64_t)grid_elems(p->B), p->amax_v, p->amax_i,
                           best_index, best_value, s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("arg-max kernel launch", e);
}

soft_status soft_argmax_real(const double *data, int64_t count, int64_t *index_out, double *value_out,
                             double *scratch, void *stream) {
    if (!aligned16(data) || count < 1 || !index_out || !value_out || !aligned16(scratch)) return SOFT_ERR_INVALID_ARG;
    double *sv = scratch;
    int64_t *si = reinterpret_cast<int64_t *>(scratch + argmax_parts());
    return cuda_status(launch_argmax_real(reinterpret_cast<const double2 *>(data), count, sv, si, index_out,
                                          value_out, static_cast<cudaStream_t>(stream)));
}

int soft_argmax_scratch_doubles(void) { return 2 * argmax_parts(); }

soft_status soft_dwt_forward(soft_plan p, const double *S, double *coef, void *stream) {
    soft_status st = check_plan_args(p, S, coef);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype)) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    return cuda_status(launch_dwt_forward_plan(p, reinterpret_cast<const double2 *>(S),
                                               reinterpret_cast<double2 *>(coef), static_cast<cudaStream_t>(stream),
                                               kApplyW | kApplyV));
}

soft_status soft_dwt_inverse(soft_plan p, const double *coef, double *S, void *stream) {
    soft_status st = check_plan_args(p, coef, S);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype)) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_zero_nyquist(p->B, reinterpret_cast<double2 *>(S), s);
    if (e == cudaSuccess)
        e = launch_dwt_inverse_plan(p, reinterpret_cast<const double2 *>(coef), reinterpret_cast<double2 *>(S), s, 0);
    return cuda_status(e);
}

// With the library's own slice FFT (FP64 and FP64-TC plans, power-of-two 2B)
// the grid's host copy is pipelined with the FFTs in slice chunks on the
// plan's copy stream; otherwise the copy, the transform and the copy back run
// in sequence on `stream`.  Both synchronise `stream` (and the copy stream)
// before returning, also after an error, so no copy into the caller's host
// buffers is left in flight.
soft_status finish_host_call(soft_plan_s *p, cudaStream_t s, soft_status st) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (p->copy_made) {
        const cudaError_t e2 = cudaStreamSynchronize(p->copy_stream);
        if (e == cudaSuccess) e = e2;
    }
    if (st != SOFT_OK) return st;
    return cuda_status(e);
}

soft_status soft_forward_host(soft_plan p, const double *grid_host, double *coef_host, void *stream) {
    if (!valid(p) || !grid_host || !coef_host) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    soft_status st = ensure_staging(p);
    if (st != SOFT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool pipelined = fp64_layout(p->dtype) && own_slice_fft(p);
    if (pipelined) {
        st = ensure_copy_stream(p);
        if (st != SOFT_OK) return st;
        st = run_forward(p, reinterpret_cast<const double *>(p->stage_grid), reinterpret_cast<double *>(p->stage_coef),
                         s, kApplyW | kApplyV, grid_host);
    } else {
        cudaError_t e = cudaMemcpyAsync(p->stage_grid, grid_host, sizeof(double2) * grid_elems(p->B),
                                        cudaMemcpyHostToDevice, s);
        st = e == cudaSuccess ? run_forward(p, reinterpret_cast<const double *>(p->stage_grid),
                                            reinterpret_cast<double *>(p->stage_coef), s)
                              : fail_cuda("grid copy", e);
    }
    if (st == SOFT_OK) {
        const cudaError_t e = cudaMemcpyAsync(coef_host, p->stage_coef, sizeof(double2) * (size_t)soft_num_coeffs(p->B),
                                              cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = fail_cuda("coefficient copy", e);
    }
    return finish_host_call(p, s, st);
}

soft_status soft_inverse_host(soft_plan p, const double *coef_host, double *grid_host, void *stream) {
    if (!valid(p) || !coef_host || !grid_host) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    soft_status st = ensure_staging(p);
    if (st != SOFT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool pipelined = fp64_layout(p->dtype) && own_slice_fft(p);
    if (pipelined) st = ensure_copy_stream(p);
    if (st != SOFT_OK) return st;
    cudaError_t e = cudaMemcpyAsync(p->stage_coef, coef_host, sizeof(double2) * (size_t)soft_num_coeffs(p->B),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return finish_host_call(p, s, fail_cuda("coefficient copy", e));
    st = run_inverse(p, reinterpret_cast<const double *>(p->stage_coef), reinterpret_cast<double *>(p->stage_grid), s,
                     0, pipelined ? grid_host : nullptr);
    if (st == SOFT_OK && !pipelined) {
        e = cudaMemcpyAsync(grid_host, p->stage_grid, sizeof(double2) * grid_elems(p->B), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = fail_cuda("grid copy", e);
    }
    return finish_host_call(p, s, st);
}

soft_status soft_selftest_bounded_wait(soft_plan p, int polls, void *stream) {
    if (!valid(p) || polls < 1 || polls > (1 << 20)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    return cuda_status(launch_bounded_wait_selftest((uint32_t)polls, p->err, static_cast<cudaStream_t>(stream)));
}

int soft_plan_num_variants(soft_plan p, int kernel) {
    if (!valid(p) || (kernel != 0 && kernel != 1)) return -1;
    if (p->dtype == SOFT_FP64) return kernel == 0 ? dwt_forward_fp64_variants(p->B) : dwt_inverse_fp64_variants(p->B);
    if (p->dtype == SOFT_FP64_TC) return 1;
    return kernel == 0 ? 2 : 1;
}

soft_status soft_plan_set_variant(soft_plan p, int kernel, int variant) {
    const int nv = soft_plan_num_variants(p, kernel);
    if (nv < 0 || variant < 0 || variant >= nv) return SOFT_ERR_INVALID_ARG;
    if (kernel == 0) p->fwd_variant = variant;
    else p->inv_variant = variant;
    return SOFT_OK;
}

soft_status soft_plan_enable_timing(soft_plan p, int on) {
    if (!valid(p)) return SOFT_ERR_INVALID_ARG;
    p->timing = on != 0;
    return SOFT_OK;
}

soft_status soft_plan_read_timing(soft_plan p, double *ms_out, int64_t *counts_out) {
    if (!valid(p)) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    fold_timing(p);
    for (int k = 0; k < 4; ++k) {
        if (ms_out) ms_out[k] = p->ms[k];
        if (counts_out) counts_out[k] = p->counts[k];
        p->ms[k] = 0.0;
        p->counts[k] = 0;
    }
    return SOFT_OK;
}

soft_status soft_cluster_shard(int B, int nranks, int rank, int *reps_out, int *count_out) {
    if (B < 1 || B > kMaxB || nranks < 1 || rank < 0 || rank >= nranks || !reps_out || !count_out)
        return SOFT_ERR_INVALID_ARG;
    std::vector<int2> cl;
    for (int m = 0; m < B; ++m)
        for (int mp = 0; mp <= m; ++mp) cl.push_back(make_int2(m, mp));
    std::stable_sort(cl.begin(), cl.end(), [B](const int2 &a, const int2 &b) {
        return cluster_work(B, a.x, a.y) > cluster_work(B, b.x, b.y);
    });
    std::vector<int64_t> load((size_t)nranks, 0);
    int cnt = 0;
    for (const int2 &c : cl) {
        const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());  // lowest rank on ties
        load[r] += cluster_work(B, c.x, c.y);
        if (r == rank) {
            reps_out[2 * cnt] = c.x;
            reps_out[2 * cnt + 1] = c.y;
            ++cnt;
        }
    }
    *count_out = cnt;
    return SOFT_OK;
}

int soft_cluster_columns(int count, const int *reps, int *pairs_out) {
    if (count < 0 || (count > 0 && (!reps || !pairs_out))) return -1;
    int q = 0;
    for (int i = 0; i < count; ++i) {
        const int m = reps[2 * i], mp = reps[2 * i + 1];
        if (mp < 0 || mp > m) return -1;
        const Partners P = make_partners(m, mp);
        for (int k = 0; k < P.np; ++k) {
            pairs_out[2 * q] = P.m[k];
            pairs_out[2 * q + 1] = P.mp[k];
            ++q;
        }
    }
    return q;
}

soft_status soft_dwt_forward_clusters(soft_plan p, const double *S, double *coef, const int *reps, int count,
                                      void *stream) {
    soft_status st = check_plan_args(p, S, coef);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype)) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = upload_subset(p, reps, count, s);
    if (st != SOFT_OK || count == 0) return st;
    Tables tb = p->tables();
    tb.ncl = count;
    tb.fwd_order = p->dsub;
    tb.inv_order = p->dsub;
    const cudaError_t e =
        p->dtype == SOFT_FP64_TC
            ? launch_dwt_forward_tc(tb, reinterpret_cast<const double2 *>(S), reinterpret_cast<double2 *>(coef), s)
            : launch_dwt_forward_fp64(tb, reinterpret_cast<const double2 *>(S), reinterpret_cast<double2 *>(coef), s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("cluster DWT launch", e);
}

soft_status soft_dwt_inverse_clusters(soft_plan p, const double *coef, double *S, const int *reps, int count,
                                      void *stream) {
    soft_status st = check_plan_args(p, coef, S);
    if (st != SOFT_OK) return st;
    if (!fp64_layout(p->dtype)) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = upload_subset(p, reps, count, s);
    if (st != SOFT_OK) return st;
    cudaError_t e0 = launch_zero_nyquist(p->B, reinterpret_cast<double2 *>(S), s);  // the -B rows and columns
    if (e0 != cudaSuccess || count == 0) return e0 == cudaSuccess ? SOFT_OK : fail_cuda("S clearing launch", e0);
    Tables tb = p->tables();
    tb.ncl = count;
    tb.fwd_order = p->dsub;
    tb.inv_order = p->dsub;
    const cudaError_t e =
        p->dtype == SOFT_FP64_TC
            ? launch_dwt_inverse_tc(tb, reinterpret_cast<const double2 *>(coef), reinterpret_cast<double2 *>(S), s)
            : launch_dwt_inverse_fp64(tb, reinterpret_cast<const double2 *>(coef), reinterpret_cast<double2 *>(S), s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("cluster iDWT launch", e);
}

soft_status soft_gather_columns(soft_plan p, const double *S, int j0, int nslices, const int *pairs, int npairs,
                                double *out, void *stream) {
    soft_status st = check_plan_args(p, S, out);
    if (st != SOFT_OK) return st;
    const int n = 2 * p->B;
    if (j0 < 0 || nslices < 0 || j0 + nslices > n) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = upload_columns(p, pairs, npairs, s);
    if (st != SOFT_OK) return st;
    const cudaError_t e = launch_gather_columns(reinterpret_cast<const double2 *>(S), p->B, j0, nslices, p->dcols,
                                                npairs, reinterpret_cast<double2 *>(out), s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("column gather launch", e);
}

soft_status soft_scatter_columns(soft_plan p, const double *in, int j0, int nslices, const int *pairs, int npairs,
                                 double *S, void *stream) {
    soft_status st = check_plan_args(p, in, S);
    if (st != SOFT_OK) return st;
    const int n = 2 * p->B;
    if (j0 < 0 || nslices < 0 || j0 + nslices > n) return SOFT_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = upload_columns(p, pairs, npairs, s);
    if (st != SOFT_OK) return st;
    const cudaError_t e = launch_scatter_columns(reinterpret_cast<const double2 *>(in), p->B, j0, nslices, p->dcols,
                                                 npairs, reinterpret_cast<double2 *>(S), s);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("column scatter launch", e);
}

soft_status soft_slice_fft(soft_plan p, const double *in, double *out, int sign, int j0, int nslices, void *stream) {
    if (!valid(p) || !aligned16(in) || !aligned16(out) || (sign != 1 && sign != -1)) return SOFT_ERR_INVALID_ARG;
    const int n = 2 * p->B;
    if (j0 < 0 || nslices < 1 || j0 + nslices > n) return SOFT_ERR_INVALID_ARG;
    if (!fp64_layout(p->dtype) || !own_slice_fft(p)) return SOFT_ERR_UNSUPPORTED;
    DeviceGuard g(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double2 *i2 = reinterpret_cast<const double2 *>(in);
    double2 *o2 = reinterpret_cast<double2 *>(out);
    const size_t off = (size_t)j0 * n * n;
    const cudaError_t e =
        p->dftw ? launch_df_fft2(p->B, i2, o2, reinterpret_cast<float4 *>(p->S) + off, p->dftw, sign,
                                 p->dfexp + (size_t)j0 * n, s, nslices)
                : launch_fft64_2d(p->B, i2, o2, p->tw64, sign, s, nslices);
    return e == cudaSuccess ? SOFT_OK : fail_cuda("slice FFT launch", e);
}

}  // extern "C"
