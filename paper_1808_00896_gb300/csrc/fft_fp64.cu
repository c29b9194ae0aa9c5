// fft_fp64.cu -- batched 2-D FFT of the beta slices in FP64, for the FP64
// plans (SOFT_FP64) with power-of-two n = 2B (other n keep cuFFT Z2Z).
//
// Step 1 of Sec. 2.4 (and its inverse): for every beta sample j the 2-D DFT
//   S(m, m'; j) = sum_{i,k} f(alpha_i, beta_j, gamma_k) exp(s i (m alpha_i + m' gamma_k)),
// unnormalised, s = +1 for the forward transform and -1 for the inverse, on
// the n x n slice.
//
// On GB300 the FP64 pipe retires 2 FMA per clock per SM and every other
// instruction class is far wider, so the cost of an FP64 FFT is its count of
// FP64 operations.  The butterflies therefore use the FMA factorisation of
// Goedecker (SIAM J. Sci. Comput. 18, 1997): with the twiddle written as
// w = mu (1 + i tau), |tau| <= 1, the pair a +- w b costs 6 FMAs instead of a
// complex product and two complex sums (8 operations).  The first two radix-2
// stages, whose twiddles are 1 and +-i, are fused into the load as one
// twiddle-free radix-4 step (16 additions per 4 points).  A length-n DFT thus
// takes 4 + 3 (log2 n - 2) FP64 operations per point.
//
// Two passes:
//   rows:    length-n DFT along the contiguous index of every row (n^2 rows);
//   columns: length-n DFT along the middle index for every (slice, column),
//            in place.
// Each DFT is an in-place radix-2 decimation-in-time transform in shared
// memory over bit-reversed input, its stages taken in pairs (radix 4) with a
// last radix-2 stage when log2 n is odd.
#include "soft_internal.cuh"

#include <algorithm>

namespace softgb {
namespace {

// a <- a + w b, b <- a - w b for w in factored form (FftTw64):
//   swap = 0: w = m (1 + i tau), m1 = m2 = m;
//   swap = 1: w = i m (1 + i tau), m1 = -m, m2 = m;
// z = (1 + i tau) b, then a + w b = (a.re + m1 p, a.im + m2 q) with
// (p, q) = (z.re, z.im), or (z.im, z.re) when swap.
__device__ __forceinline__ void bfly(double2 &a, double2 &b, const FftTw64 &w) {
    const double zr = fma(-w.tau, b.y, b.x), zi = fma(w.tau, b.x, b.y);
    const double p = w.swap ? zi : zr, q = w.swap ? zr : zi;
    const double ar = a.x, ai = a.y;
    a = make_double2(fma(w.m1, p, ar), fma(w.m2, q, ai));
    b = make_double2(fma(-w.m1, p, ar), fma(-w.m2, q, ai));
}

// The first two radix-2 stages of the decimation in time on
// x0..x3 = x[t], x[t + n/2], x[t + n/4], x[t + 3n/4] (the contents of
// bit-reversed positions 4 rev(t) + 0..3): twiddles 1, 1 and exp(+- i pi/2).
__device__ __forceinline__ void first_radix4(const double2 x0, const double2 x1, const double2 x2, const double2 x3,
                                             bool conj, double2 *dst) {
    const double2 a0 = make_double2(x0.x + x1.x, x0.y + x1.y), a1 = make_double2(x0.x - x1.x, x0.y - x1.y);
    const double2 a2 = make_double2(x2.x + x3.x, x2.y + x3.y), a3 = make_double2(x2.x - x3.x, x2.y - x3.y);
    dst[0] = make_double2(a0.x + a2.x, a0.y + a2.y);
    dst[2] = make_double2(a0.x - a2.x, a0.y - a2.y);
    const double2 u = make_double2(a1.x - a3.y, a1.y + a3.x);  // a1 + i a3
    const double2 v = make_double2(a1.x + a3.y, a1.y - a3.x);  // a1 - i a3
    dst[1] = conj ? v : u;
    dst[3] = conj ? u : v;
}

// Bit reversal of t within `bits` bits (0 for bits == 0).
__device__ __forceinline__ int bitrev_n(int t, int bits) {
    return bits ? (int)(__brev((unsigned)t) >> (32 - bits)) : 0;
}

// Stages from sub-DFT half-size h = 2^lh on, for `cnt` DFTs of length n held
// at s + r ld (r < cnt), by all threads of the block: radix-4 passes (stages
// of sizes 2h and 4h), then one radix-2 stage when one is left.  tw[t] is the
// factored exp(+- 2 pi i t / n), t < n/2.
__device__ void stages(double2 *s, int cnt, int ld, int n, int logn, int h, int lh, const FftTw64 *tw) {
    for (; 4 * h <= n; h *= 4, lh += 2) {
        const int nq = cnt * (n >> 2);
        __syncthreads();
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int row = q >> (logn - 2), qq = q & ((n >> 2) - 1);
            const int k = qq & (h - 1), g = qq >> lh;
            double2 *p = s + row * ld + g * 4 * h + k;
            double2 x0 = p[0], x1 = p[h], x2 = p[2 * h], x3 = p[3 * h];
            const FftTw64 w1 = tw[k << (logn - 1 - lh)];  // exp(+- 2 pi i k / (2h))
            bfly(x0, x1, w1);
            bfly(x2, x3, w1);
            bfly(x0, x2, tw[k << (logn - 2 - lh)]);        // exp(+- 2 pi i k / (4h))
            bfly(x1, x3, tw[(k + h) << (logn - 2 - lh)]);  // exp(+- 2 pi i (k + h) / (4h))
            p[0] = x0;
            p[h] = x1;
            p[2 * h] = x2;
            p[3 * h] = x3;
        }
    }
    if (2 * h == n) {  // one radix-2 stage of size n is left
        const int nb = cnt * h;
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int row = b >> lh, k = b & (h - 1);
            double2 *p = s + row * ld + k;
            double2 x0 = p[0], x1 = p[h];
            bfly(x0, x1, tw[k]);
            p[0] = x0;
            p[h] = x1;
        }
    }
    __syncthreads();
}

constexpr int kThreads = 256;
constexpr int kTile = 1024;  // elements per block and pass (at least one row or column)

__device__ void load_twiddles(FftTw64 *tw, const FftTw64 *__restrict__ twg, int n) {
    for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) tw[t] = twg[t];
}

// Element e of the input: complex, or real (REAL_IN, imaginary part 0).
template <bool REAL_IN>
__device__ __forceinline__ double2 load_in(const void *in, int64_t e) {
    if constexpr (REAL_IN) return make_double2(static_cast<const double *>(in)[e], 0.0);
    else return static_cast<const double2 *>(in)[e];
}

// Rows pass: nrows rows of n contiguous elements, `rpb` rows per block,
// in -> out (the same memory is allowed: a block reads its rows before it
// writes them).  `in` holds double2, or doubles when REAL_IN.
template <bool REAL_IN>
__global__ void __launch_bounds__(kThreads) fft64_rows_kernel(const void *in, double2 *out, int64_t nrows, int n,
                                                               int logn, int rpb, const FftTw64 *__restrict__ twg,
                                                               int conj) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FftTw64 *tw = reinterpret_cast<FftTw64 *>(smraw);                              // [n/2]
    double2 *s = reinterpret_cast<double2 *>(smraw + sizeof(FftTw64) * (n >> 1));  // [rpb][n]
    load_twiddles(tw, twg, n);
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int rows = (int)std::min<int64_t>(rpb, nrows - r0);
    if (logn >= 2) {
        const int n4 = n >> 2;
        for (int q = threadIdx.x; q < rows * n4; q += blockDim.x) {
            const int rl = q / n4, t = q - rl * n4;
            const int64_t x = (r0 + rl) * n + t;
            first_radix4(load_in<REAL_IN>(in, x), load_in<REAL_IN>(in, x + (n >> 1)), load_in<REAL_IN>(in, x + n4),
                         load_in<REAL_IN>(in, x + 3 * n4), conj != 0, s + rl * n + 4 * bitrev_n(t, logn - 2));
        }
        stages(s, rows, n, n, logn, 4, 2, tw);
    } else {
        for (int e = threadIdx.x; e < rows * n; e += blockDim.x) s[e] = load_in<REAL_IN>(in, r0 * n + e);  // n = 2
        stages(s, rows, n, n, logn, 1, 0, tw);
    }
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) out[r0 * n + e] = s[e];
}

// Columns pass: for every slice and column, the length-n DFT along the middle
// index (stride n), `kb` adjacent columns per block, in place, or (REAL_OUT)
// only the real parts written to `rout` (same layout, doubles).  Only the
// first `ncols` columns of each slice are transformed (n for complex data, B
// for the m' >= 0 half of a real grid's transform).  Shared memory holds
// column c at s + c (n + 1) (the pad spreads the columns over the banks).
template <bool REAL_OUT>
__global__ void __launch_bounds__(kThreads) fft64_cols_kernel(double2 *data, double *rout, int n, int logn, int kb,
                                                               const FftTw64 *__restrict__ twg, int conj, int ncols) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FftTw64 *tw = reinterpret_cast<FftTw64 *>(smraw);
    double2 *s = reinterpret_cast<double2 *>(smraw + sizeof(FftTw64) * (n >> 1));
    load_twiddles(tw, twg, n);
    const int ld = n + 1;
    const int tiles = ncols / kb;
    const int64_t js = blockIdx.x / tiles;
    const int k0 = (blockIdx.x % tiles) * kb;
    double2 *base = data + js * n * n + k0;
    if (logn >= 2) {
        const int n4 = n >> 2;
        for (int q = threadIdx.x; q < kb * n4; q += blockDim.x) {
            const int t = q / kb, c = q - t * kb;
            const double2 *x = base + (int64_t)t * n + c;
            first_radix4(x[(int64_t)0], x[(int64_t)(n >> 1) * n], x[(int64_t)n4 * n], x[(int64_t)3 * n4 * n],
                         conj != 0, s + c * ld + 4 * bitrev_n(t, logn - 2));
        }
        stages(s, kb, ld, n, logn, 4, 2, tw);
    } else {
        for (int e = threadIdx.x; e < kb * n; e += blockDim.x) {
            const int i = e / kb, c = e - i * kb;
            s[c * ld + i] = base[(int64_t)i * n + c];
        }
        stages(s, kb, ld, n, logn, 1, 0, tw);
    }
    for (int e = threadIdx.x; e < kb * n; e += blockDim.x) {
        const int i = e / kb, c = e - i * kb;
        if constexpr (REAL_OUT) rout[js * n * n + k0 + (int64_t)i * n + c] = s[c * ld + i].x;
        else base[(int64_t)i * n + c] = s[c * ld + i];
    }
}

// ---------------------------------------------------------------------------
// Real grids.  A real row x[0..n) has X[n-k] = conj X[k], so only X[0..N),
// N = n/2, is formed, from one N-point complex DFT of the packed samples
// z[t] = x[2t] + i x[2t+1]:
//   E[k] = (Z[k] + conj Z[N-k]) / 2,  O[k] = (Z[k] - conj Z[N-k]) / (2i)  (indices mod N),
//   X[k] = E[k] + w^k O[k],  w = exp(s 2 pi i / n):
// E and O are the DFTs of the even and odd samples (real sequences, so their
// DFTs are conjugate-symmetric), recombined as in one decimation-in-time step.
// The inverse runs it backwards: for a Hermitian row (X[n-k] = conj X[k], the
// Nyquist term X[N] zero as in the plan's S) the real samples come from one
// N-point DFT of
//   Z[k] = (X[k] + conj X[N-k]) + i v^k (X[k] - conj X[N-k]),  v = exp(s 2 pi i / n),
// as x[2t] = Re z[t], x[2t+1] = Im z[t] (the sum over k split into k < N and
// k + N, with X[k + N] = conj X[N - k] and v^N = -1).
// ---------------------------------------------------------------------------

// w b for w in the factored form of bfly().
__device__ __forceinline__ double2 twmul(const FftTw64 &w, const double2 b) {
    const double zr = fma(-w.tau, b.y, b.x), zi = fma(w.tau, b.x, b.y);
    const double p = w.swap ? zi : zr, q = w.swap ? zr : zi;
    return make_double2(w.m1 * p, w.m2 * q);
}

// The tables of a real-row kernel: the n-point twiddles w^k (k < N) and the
// N-point ones exp(s 2 pi i t / N) = w^(2t) (t < N/2).
__device__ void load_real_twiddles(FftTw64 *tw, FftTw64 *twN, const FftTw64 *__restrict__ twg, int N) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twg[t];
    for (int t = threadIdx.x; t < (N >> 1); t += blockDim.x) twN[t] = twg[2 * t];
}

// The N-point DFT (N = 2^logN) of `rows` rows held in natural order at
// zin + r N (global or shared memory), into s + r N in natural order.
__device__ __forceinline__ void half_dft(const double2 *zin, double2 *s, int rows, int N, int logN, const FftTw64 *twN,
                                         bool conj) {
    if (logN >= 2) {
        const int N4 = N >> 2;
        for (int q = threadIdx.x; q < rows * N4; q += blockDim.x) {
            const int rl = q / N4, t = q - rl * N4;
            const double2 *z = zin + (int64_t)rl * N + t;
            first_radix4(z[0], z[N >> 1], z[N4], z[3 * N4], conj, s + rl * N + 4 * bitrev_n(t, logN - 2));
        }
        stages(s, rows, N, N, logN, 4, 2, twN);
    } else {  // N = 1 or 2: bit-reversed order is the natural one
        for (int e = threadIdx.x; e < rows * N; e += blockDim.x) s[e] = zin[e];
        stages(s, rows, N, N, logN, 1, 0, twN);
    }
}

// Rows pass of a real grid: nrows real rows of n samples (`in`) -> X[0..N) of
// each row at out + row n (columns N..n-1 of `out` are not written).
__global__ void __launch_bounds__(kThreads) fft64_rows_r2c_kernel(const double *in, double2 *out, int64_t nrows, int n,
                                                                   int logN, int rpb, const FftTw64 *__restrict__ twg,
                                                                   int conj) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = n >> 1;
    FftTw64 *tw = reinterpret_cast<FftTw64 *>(smraw);  // [N]
    FftTw64 *twN = tw + N;                              // [max(1, N/2)]
    double2 *s = reinterpret_cast<double2 *>(twN + max(1, N >> 1));  // [rpb][N]
    load_real_twiddles(tw, twN, twg, N);
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int rows = (int)std::min<int64_t>(rpb, nrows - r0);
    __syncthreads();
    half_dft(reinterpret_cast<const double2 *>(in) + r0 * N, s, rows, N, logN, twN, conj != 0);
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e / N, k = e - rl * N;
        const double2 a = s[rl * N + k], b = s[rl * N + ((N - k) & (N - 1))];
        const double2 E = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        const double2 O = make_double2(0.5 * (a.y + b.y), 0.5 * (b.x - a.x));
        const double2 wO = twmul(tw[k], O);
        out[(r0 + rl) * n + k] = make_double2(E.x + wO.x, E.y + wO.y);
    }
}

// Rows pass back to a real grid: X[0..N) of each row at in + row n (X[N] = 0)
// -> nrows real rows of n samples in `out`.
__global__ void __launch_bounds__(kThreads) fft64_rows_c2r_kernel(const double2 *in, double *out, int64_t nrows, int n,
                                                                   int logN, int rpb, const FftTw64 *__restrict__ twg,
                                                                   int conj) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = n >> 1;
    FftTw64 *tw = reinterpret_cast<FftTw64 *>(smraw);
    FftTw64 *twN = tw + N;
    double2 *xs = reinterpret_cast<double2 *>(twN + max(1, N >> 1));  // [rpb][N]: X, then the DFT
    double2 *zs = xs + (size_t)rpb * N;                                // [rpb][N]: Z
    load_real_twiddles(tw, twN, twg, N);
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int rows = (int)std::min<int64_t>(rpb, nrows - r0);
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e / N, k = e - rl * N;
        xs[e] = in[(r0 + rl) * n + k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e / N, k = e - rl * N;
        const double2 a = xs[e];
        const double2 b = k ? xs[rl * N + N - k] : make_double2(0.0, 0.0);  // X[N - k]; X[N] = 0
        const double2 A = make_double2(a.x + b.x, a.y - b.y);                 // X[k] + conj X[N-k]
        const double2 C = twmul(tw[k], make_double2(a.x - b.x, a.y + b.y));   // v^k (X[k] - conj X[N-k])
        zs[e] = make_double2(A.x - C.y, A.y + C.x);                           // A + i C
    }
    __syncthreads();
    half_dft(zs, xs, rows, N, logN, twN, conj != 0);
    double2 *o = reinterpret_cast<double2 *>(out) + r0 * N;  // (x[2t], x[2t+1]) = (Re z[t], Im z[t])
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) o[e] = xs[e];
}

// tw[t] for t < n/2: exp(sign 2 pi i t / n) in the factored form of bfly().
__global__ void twiddle64_kernel(int n, int sign, FftTw64 *tw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n / 2) return;
    const double a = 2.0 * t / n;
    const double c = cospi(a), s = sign * sinpi(a);
    FftTw64 w;
    w.pad = 0;
    if (fabs(c) >= fabs(s)) {  // w = c (1 + i s/c)
        w.swap = 0;
        w.tau = s / c;
        w.m1 = c;
        w.m2 = c;
    } else {  // w = i s (1 - i c/s)
        w.swap = 1;
        w.tau = -c / s;
        w.m1 = -s;
        w.m2 = s;
    }
    tw[t] = w;
}

int ilog2_pow2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

// The two passes: rows `in` -> `mid` (complex; `in` complex, or real when
// REAL_IN), then columns in place on `mid`, or (REAL_OUT) from `mid` to the
// real parts in `rout`.  All pointers at the first of `nslices` slices.
template <bool REAL_IN, bool REAL_OUT>
cudaError_t fft64_passes(int B, const void *in, double2 *mid, double *rout, const FftTw64 *tw, int sign,
                         cudaStream_t s, int nslices) {
    const int n = 2 * B, logn = ilog2_pow2(n);
    if (logn < 1 || nslices < 1 || nslices > n) return cudaErrorInvalidValue;
    const FftTw64 *t = sign < 0 ? tw + n / 2 : tw;
    const int conj = sign < 0 ? 1 : 0;
    const int64_t nrows = (int64_t)nslices * n;
    const int rpb = std::max(1, kTile / n);
    const size_t twb = sizeof(FftTw64) * (size_t)(n / 2);
    const size_t rbytes = twb + sizeof(double2) * (size_t)rpb * n;
    cudaError_t e = cudaFuncSetAttribute(fft64_rows_kernel<REAL_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rbytes);
    if (e != cudaSuccess) return e;
    fft64_rows_kernel<REAL_IN><<<(unsigned)((nrows + rpb - 1) / rpb), kThreads, rbytes, s>>>(in, mid, nrows, n, logn,
                                                                                             rpb, t, conj);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int kb = std::min(n, std::max(2, kTile / n));
    const size_t cbytes = twb + sizeof(double2) * (size_t)kb * (n + 1);
    e = cudaFuncSetAttribute(fft64_cols_kernel<REAL_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cbytes);
    if (e != cudaSuccess) return e;
    fft64_cols_kernel<REAL_OUT><<<(unsigned)((int64_t)nslices * (n / kb)), kThreads, cbytes, s>>>(mid, rout, n, logn,
                                                                                                 kb, t, conj, n);
    count_launch();
    return cudaGetLastError();
}

// The half-spectrum passes of a real grid (all 2B slices): r2c rows `in` ->
// `S` columns 0..B-1, then those columns in place; or (c2r) those columns of
// `S` in place, then rows to the real `out`.
cudaError_t fft64_real_passes(int B, bool r2c, const double *in, double2 *S, double *out, const FftTw64 *tw, int sign,
                              cudaStream_t s) {
    const int n = 2 * B, logn = ilog2_pow2(n), N = B;
    if (logn < 1) return cudaErrorInvalidValue;
    const FftTw64 *t = sign < 0 ? tw + n / 2 : tw;
    const int conj = sign < 0 ? 1 : 0;
    const int64_t nrows = (int64_t)n * n;
    const int rpb = std::max(1, kTile / N);
    const size_t twb = sizeof(FftTw64) * ((size_t)N + std::max(1, N / 2));
    const int kb = std::min(N, std::max(2, kTile / n));
    const size_t cbytes = sizeof(FftTw64) * (size_t)(n / 2) + sizeof(double2) * (size_t)kb * (n + 1);
    cudaError_t e = cudaFuncSetAttribute(fft64_cols_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cbytes);
    if (e != cudaSuccess) return e;
    const unsigned cgrid = (unsigned)((int64_t)n * (N / kb));
    if (r2c) {
        const size_t rbytes = twb + sizeof(double2) * (size_t)rpb * N;
        e = cudaFuncSetAttribute(fft64_rows_r2c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rbytes);
        if (e != cudaSuccess) return e;
        fft64_rows_r2c_kernel<<<(unsigned)((nrows + rpb - 1) / rpb), kThreads, rbytes, s>>>(in, S, nrows, n, logn - 1,
                                                                                           rpb, t, conj);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        fft64_cols_kernel<false><<<cgrid, kThreads, cbytes, s>>>(S, nullptr, n, logn, kb, t, conj, N);
        count_launch();
        return cudaGetLastError();
    }
    fft64_cols_kernel<false><<<cgrid, kThreads, cbytes, s>>>(S, nullptr, n, logn, kb, t, conj, N);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t rbytes = twb + 2 * sizeof(double2) * (size_t)rpb * N;
    e = cudaFuncSetAttribute(fft64_rows_c2r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rbytes);
    if (e != cudaSuccess) return e;
    fft64_rows_c2r_kernel<<<(unsigned)((nrows + rpb - 1) / rpb), kThreads, rbytes, s>>>(S, out, nrows, n, logn - 1,
                                                                                       rpb, t, conj);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool fft64_supported(int B) {
    const int n = 2 * B;
    return n >= 2 && n <= 2 * kMaxB && ilog2_pow2(n) >= 0;
}

size_t fft64_twiddle_count(int B) { return (size_t)2 * (size_t)B; }

cudaError_t launch_fft64_twiddles(int B, FftTw64 *tw, cudaStream_t s) {
    const int n = 2 * B, half = n / 2;
    twiddle64_kernel<<<(half + 127) / 128, 128, 0, s>>>(n, +1, tw);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    twiddle64_kernel<<<(half + 127) / 128, 128, 0, s>>>(n, -1, tw + half);
    count_launch();
    return cudaGetLastError();
}

// 2-D DFT of `nslices` consecutive n x n slices (n = 2B): `in` (layout
// [j][i][k]) -> `out` ([j][m][m']), exp(sign i ...), unnormalised; `out` may
// be `in`.  Both point at the first slice of the range.
cudaError_t launch_fft64_2d(int B, const double2 *in, double2 *out, const FftTw64 *tw, int sign, cudaStream_t s,
                            int nslices) {
    return fft64_passes<false, false>(B, in, out, nullptr, tw, sign, s, nslices);
}

// The same for a real grid `in` ((2B)^3 doubles) into the complex `out`.
cudaError_t launch_fft64_2d_from_real(int B, const double *in, double2 *out, const FftTw64 *tw, int sign,
                                      cudaStream_t s) {
    return fft64_passes<true, false>(B, in, out, nullptr, tw, sign, s, 2 * B);
}

// The same for a complex `in` whose result is real (Hermitian input, up to
// rounding): `in` is overwritten (the rows pass runs in place) and the real
// parts of the result go to `out` ((2B)^3 doubles).
cudaError_t launch_fft64_2d_to_real(int B, double2 *in, double *out, const FftTw64 *tw, int sign, cudaStream_t s) {
    return fft64_passes<false, true>(B, in, in, out, tw, sign, s, 2 * B);
}

// Real grid `in` -> the m' = 0..B-1 half of S (columns B..2B-1 of every slice
// are left as they are): real-row DFTs, then the B columns.
cudaError_t launch_fft64_2d_r2c(int B, const double *in, double2 *S, const FftTw64 *tw, int sign, cudaStream_t s) {
    return fft64_real_passes(B, true, in, S, nullptr, tw, sign, s);
}

// The m' = 0..B-1 half of a Hermitian S (S(-m,-m') = conj S(m,m'), the
// m' = -B column zero) -> the real grid `out`; S's columns 0..B-1 are
// overwritten.
cudaError_t launch_fft64_2d_c2r(int B, double2 *S, double *out, const FftTw64 *tw, int sign, cudaStream_t s) {
    return fft64_real_passes(B, false, nullptr, S, out, tw, sign, s);
}

}  // namespace softgb
