// fft_df.cu -- batched 2-D FFT of the beta slices in double-float arithmetic
// on the FP32 pipe, for the FP64-accurate tensor-core mode (SOFT_FP64_TC).
//
// Step 1 of Sec. 2.4 (and its inverse): for every beta sample j the 2-D DFT
//   S(m, m'; j) = sum_{i,k} f(alpha_i, beta_j, gamma_k) exp(s i (m alpha_i + m' gamma_k)),
// unnormalised, s = +1 for the forward transform and -1 for the inverse, on
// the n x n slice, n = 2B.  The GB300's FP32 pipe is ~58x wider than its FP64
// pipe, so the butterflies run on unevaluated pairs of floats ("double-float",
// hi + lo with |lo| <= ulp(hi)/2, ~48 significant bits) built from the
// error-free sum of Knuth (two-sum) and the FMA-based error-free product;
// every row is scaled by the power of two of its largest magnitude (so the
// pairs stay inside the FP32 exponent range for any data) and split from FP64;
// results are recombined into FP64 and scaled back.  Power-of-two n only (the
// plan falls back to cuFFT otherwise).
//
// Two passes, no extra memory:
//   rows:    length-n DFT along the contiguous index of every row (n^2 rows),
//            FP64 in, double-float out;
//   columns: length-n DFT along the middle index for every (slice, column),
//            in place on the double-float data, FP64 out.
// Each DFT is an in-place radix-2 decimation-in-time transform in shared
// memory: bit-reversed load, log2(n) butterfly stages, natural-order store.
// Real grids take the half-spectrum form of the same passes (below): half-
// length row DFTs of packed sample pairs, and the columns m' = 0..B-1 only.
#include "soft_internal.cuh"
#include "tcgen05.cuh"

#include <algorithm>

namespace softgb {
namespace {

struct dfloat {
    float hi, lo;
};

// s + e = a + b exactly (Knuth's two-sum, no ordering assumption).
__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// a + b with the error of the leading sum recovered; the trailing parts are
// added plainly.  The error is ~2^-47 of |a| + |b|, which is the norm-wise
// bound a DFT needs (a butterfly's output error relative to its inputs).
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }

struct dcomplex {
    dfloat re, im;
};

__device__ __forceinline__ dcomplex load_df(const float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 store_df(const dcomplex v) { return make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }

// FP64 -> double-float: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact in FP64).
__device__ __forceinline__ dfloat split_f64(double x) {
    const float hi = tc::f64_to_f32_rn(x);
    return {hi, tc::f64_to_f32_rn(x - tc::f32_to_f64(hi))};
}

__device__ __forceinline__ double join_f64(dfloat v) { return tc::f32_to_f64(v.hi) + tc::f32_to_f64(v.lo); }

// v 2^k by an exponent-field add (v normal or 0; results below the normal
// range flush to signed 0).
__device__ __forceinline__ double scale2(double v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0 || e == 0x7FF || k == 0) return e == 0 ? 0.0 * v : v;
    const int e2 = e + k;
    if (e2 <= 0) return __longlong_as_double((long long)(b & (1ull << 63)));
    if (e2 >= 0x7FF) return __longlong_as_double((long long)((b & (1ull << 63)) | (0x7FFull << 52)));
    return __longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((unsigned long long)e2 << 52)));
}

// 2^k as a float for the power-of-two scalings of the double-float values
// (0 below the FP32 normal range, where the scaled values are negligible).
__device__ __forceinline__ float pow2f(int k) { return k < -126 ? 0.f : __int_as_float((min(k, 127) + 127) << 23); }

// Row scales: every row of the first pass is scaled by the power of two of
// its own largest magnitude, s_r = (its largest biased exponent) - 1023, so
// the double-float values stay inside the FP32 exponent range whatever the
// data's scale; the column pass brings the rows of a slice to their common
// largest scale by exact power-of-two products before its DFTs, and scales
// the results back.  All-zero rows get kZeroRow.
constexpr int kZeroRow = -100000;

// a b + sg c d in double-float: the two leading products with their exact
// errors (FMA), their error-free sum, and the cross terms folded in by FMAs
// (lo * lo terms, <= 2^-48 relative, dropped).
__device__ __forceinline__ dfloat df_dot2(dfloat a, dfloat b, dfloat c, dfloat d, float sg) {
    const float p1 = a.hi * b.hi, p2 = sg * (c.hi * d.hi);
    const float e1 = fmaf(a.hi, b.hi, -p1), e2 = sg * fmaf(c.hi, d.hi, -sg * p2);
    const dfloat s = two_sum(p1, p2);
    float t = s.lo + (e1 + e2);
    t = fmaf(a.hi, b.lo, t);
    t = fmaf(a.lo, b.hi, t);
    t = fmaf(sg * c.hi, d.lo, t);
    t = fmaf(sg * c.lo, d.hi, t);
    return fast_two_sum(s.hi, t);
}

// w * x (w conjugated when conj).
__device__ __forceinline__ dcomplex cmul(dcomplex w, dcomplex x, bool conj) {
    if (conj) w.im = df_neg(w.im);
    return {df_dot2(w.re, x.re, w.im, x.im, -1.f), df_dot2(w.re, x.im, w.im, x.re, 1.f)};
}

__device__ __forceinline__ dcomplex cadd(dcomplex a, dcomplex b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dcomplex csub(dcomplex a, dcomplex b) {
    return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))};
}
// x * (+i) when pos, x * (-i) otherwise.
__device__ __forceinline__ dcomplex mul_i(dcomplex x, bool pos) {
    return pos ? dcomplex{df_neg(x.im), x.re} : dcomplex{x.im, df_neg(x.re)};
}

__device__ __forceinline__ int bitrev(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// The log2(n) butterfly stages of `cnt` independent length-n DFTs stored
// contiguously in s (each bit-reversed on entry), by all threads of the block:
// pairs of radix-2 decimation-in-time stages fused into one radix-4 pass over
// shared memory (sizes 2h and 4h), plus a last radix-2 stage when log2(n) is
// odd.  tw[t] = exp(+2 pi i t / n), t < n/2; conj selects the - sign.
__device__ void dft_stages(float4 *s, int cnt, int n, int logn, const float4 *tw, bool conj) {
    int h = 1, lh = 0;  // first sub-stage has size 2h
    for (; 4 * h <= n; h *= 4, lh += 2) {
        const int nq = cnt * (n >> 2);
        __syncthreads();
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int row = q >> (logn - 2), qq = q & ((n >> 2) - 1);
            const int k = qq & (h - 1), g = qq >> lh;
            const int i0 = row * n + g * 4 * h + k;
            const dcomplex w1 = load_df(tw[k << (logn - 1 - lh)]);  // exp(+- 2 pi i k / (2h))
            const dcomplex w2 = load_df(tw[k << (logn - 2 - lh)]);  // exp(+- 2 pi i k / (4h))
            const dcomplex x0 = load_df(s[i0]), x1 = load_df(s[i0 + h]);
            const dcomplex x2 = load_df(s[i0 + 2 * h]), x3 = load_df(s[i0 + 3 * h]);
            const dcomplex t1 = cmul(w1, x1, conj), t3 = cmul(w1, x3, conj);
            const dcomplex a0 = cadd(x0, t1), a1 = csub(x0, t1), a2 = cadd(x2, t3), a3 = csub(x2, t3);
            const dcomplex u2 = cmul(w2, a2, conj);
            const dcomplex u3 = mul_i(cmul(w2, a3, conj), !conj);  // exp(+- 2 pi i (k + h) / (4h)) = w2 (+-i)
            s[i0] = store_df(cadd(a0, u2));
            s[i0 + 2 * h] = store_df(csub(a0, u2));
            s[i0 + h] = store_df(cadd(a1, u3));
            s[i0 + 3 * h] = store_df(csub(a1, u3));
        }
    }
    if (2 * h == n) {  // odd log2(n): one radix-2 stage of size n
        const int nb = cnt * (n >> 1);
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int row = b >> (logn - 1), k = b & (h - 1);
            const int i = row * n + k, j = i + h;
            const dcomplex t = cmul(load_df(tw[k]), load_df(s[j]), conj);
            const dcomplex a = load_df(s[i]);
            s[i] = store_df(cadd(a, t));
            s[j] = store_df(csub(a, t));
        }
    }
    __syncthreads();
}

constexpr int kFftThreads = 256;

// Rows pass: nrows rows of n (contiguous), FP64 in, double-float out,
// possibly to the same memory (each block reads its rows before writing
// them); every row scaled by its own power of two, recorded in rexp.  `rpb`
// rows per block.
__global__ void __launch_bounds__(kFftThreads) fft_rows_kernel(const double2 *in, float4 *out, int64_t nrows, int n,
                                                                int logn, int rpb, const float4 *__restrict__ twg,
                                                                int conj, int *__restrict__ rexp) {
    extern __shared__ __align__(16) float4 sm[];
    float4 *tw = sm;              // [n/2]
    float4 *s = sm + (n >> 1);    // [rpb][n]
    for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) tw[t] = twg[t];
    __shared__ int rmax[256];  // largest biased exponent of each row; rpb <= 256
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    for (int t = threadIdx.x; t < rpb; t += blockDim.x) rmax[t] = 0;
    // each thread holds at most kPer of the block's rpb * n <= 1024 elements
    constexpr int kPer = 4;
    double2 v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) v[u] = make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * kFftThreads;
        if (e < rpb * n && r0 + (e >> logn) < nrows) {
            v[u] = in[(r0 + (e >> logn)) * n + (e & (n - 1))];
            const int ex = (int)max(((unsigned long long)__double_as_longlong(v[u].x) >> 52) & 0x7FF,
                                    ((unsigned long long)__double_as_longlong(v[u].y) >> 52) & 0x7FF);
            if (ex) atomicMax(&rmax[e >> logn], ex);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * kFftThreads;
        if (e < rpb * n) {
            const int rl = e >> logn, sh = rmax[rl] ? 1023 - rmax[rl] : 0;
            const dfloat re = split_f64(scale2(v[u].x, sh)), im = split_f64(scale2(v[u].y, sh));
            s[rl * n + bitrev(e & (n - 1), logn)] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
    for (int t = threadIdx.x; t < rpb; t += blockDim.x)
        if (r0 + t < nrows) rexp[r0 + t] = rmax[t] ? rmax[t] - 1023 : kZeroRow;
    dft_stages(s, rpb, n, logn, tw, conj != 0);
    for (int e = threadIdx.x; e < rpb * n; e += blockDim.x) {
        const int64_t r = r0 + (e >> logn);
        if (r < nrows) out[r * n + (e & (n - 1))] = s[e];
    }
}

// Columns pass: for every slice and each of its first `ncols` columns (n,
// or B for the m' >= 0 half of a real grid's spectrum), the length-n DFT
// along the middle index (stride n), `kb` adjacent columns per block;
// double-float in, FP64 (double2) out, possibly to the same memory (each
// block reads its whole tile before writing it).
__global__ void __launch_bounds__(kFftThreads) fft_cols_kernel(const float4 *in, double2 *out, int n, int logn, int kb,
                                                                int ncols, const float4 *__restrict__ twg, int conj,
                                                                const int *__restrict__ rexp) {
    extern __shared__ __align__(16) float4 sm[];
    float4 *tw = sm;              // [n/2]
    float4 *s = sm + (n >> 1);    // [kb][n], column-major: column c at s + c n
    for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) tw[t] = twg[t];
    const int tiles = ncols / kb;
    const int64_t js = blockIdx.x / tiles;
    const int k0 = (blockIdx.x % tiles) * kb;
    const int64_t base = js * n * n + k0;
    // the slice's common scale: the largest of its rows' scales
    __shared__ int smax;
    __shared__ int sexp[2 * kMaxB];
    if (threadIdx.x == 0) smax = kZeroRow;
    __syncthreads();
    int lm = kZeroRow;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int x = rexp[js * n + i];
        sexp[i] = x;
        lm = max(lm, x);
    }
    atomicMax(&smax, lm);
    __syncthreads();
    const int sref = smax;
    for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
        const int i = e / kb, c = e % kb;
        const float f = pow2f(sexp[i] - sref);
        const float4 x = in[base + (int64_t)i * n + c];
        s[c * n + bitrev(i, logn)] = make_float4(x.x * f, x.y * f, x.z * f, x.w * f);
    }
    dft_stages(s, kb, n, logn, tw, conj != 0);
    const int sh = sref == kZeroRow ? 0 : sref;
    for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
        const int i = e / kb, c = e % kb;
        const dcomplex v = load_df(s[c * n + i]);
        out[base + (int64_t)i * n + c] = make_double2(scale2(join_f64(v.re), sh), scale2(join_f64(v.im), sh));
    }
}

// ---------------------------------------------------------------------------
// Real grids.  A real row x[0..n) has X[n-k] = conj X[k], so only X[0..N),
// N = n/2, is formed, from one N-point DFT of the packed samples
// z[t] = x[2t] + i x[2t+1]:
//   X[k] = E[k] + w^k O[k],  w = exp(s 2 pi i / n),
//   E[k] = (Z[k] + conj Z[N-k]) / 2,  O[k] = (Z[k] - conj Z[N-k]) / (2i)  (indices of Z mod N),
// E and O being the DFTs of the even and odd samples.  Backwards, for a
// Hermitian row whose Nyquist term X[N] is zero (as in the plan's S), the
// samples come from one N-point DFT of
//   Z[k] = (X[k] + conj X[N-k]) + i v^k (X[k] - conj X[N-k]),  v = exp(s 2 pi i / n),
// as x[2t] = Re z[t], x[2t+1] = Im z[t] (the sum over k split into k < N and
// k + N, with X[k + N] = conj X[N - k] and v^N = -1).
// The forward runs the rows (r2c, every row scaled by its own power of two as
// in fft_rows_kernel), then fft_cols_kernel on the columns m' = 0..N-1.  The
// inverse runs those columns first (FP64 in, every column scaled by its own
// power of two), then the rows (c2r), which bring a slice's columns to their
// common scale before the packing.
// ---------------------------------------------------------------------------

// Biased exponent of the larger part of v (0 for zeros and subnormals).
__device__ __forceinline__ int biased_exponent2(double2 v) {
    return (int)max(((unsigned long long)__double_as_longlong(v.x) >> 52) & 0x7FF,
                    ((unsigned long long)__double_as_longlong(v.y) >> 52) & 0x7FF);
}

__device__ __forceinline__ dfloat df_half(dfloat a) { return {0.5f * a.hi, 0.5f * a.lo}; }
__device__ __forceinline__ dcomplex dc_scale(dcomplex a, float f) {
    return {{a.re.hi * f, a.re.lo * f}, {a.im.hi * f, a.im.lo * f}};
}

// The real-row kernels' twiddles: tw[k] = w^k (k < N), twN[t] = w^(2t) =
// exp(+2 pi i t / N) (t < N/2), from the n-point table.
__device__ void load_real_twiddles_df(float4 *tw, float4 *twN, const float4 *__restrict__ twg, int N) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twg[t];
    for (int t = threadIdx.x; t < (N >> 1); t += blockDim.x) twN[t] = twg[2 * t];
}

// Rows pass of a real grid: nrows real rows of n samples (`in`, FP64) ->
// X[0..N) of each row, double-float, at out + row n (columns N..n-1 are not
// written); every row scaled by its own power of two, recorded in rexp as in
// fft_rows_kernel.  `rpb` rows per block (rpb <= 256).
__global__ void __launch_bounds__(kFftThreads) fft_rows_r2c_kernel(const double *in, float4 *out, int64_t nrows, int n,
                                                                    int logN, int rpb, const float4 *__restrict__ twg,
                                                                    int conj, int *__restrict__ rexp) {
    extern __shared__ __align__(16) float4 sm[];
    const int N = n >> 1;
    float4 *tw = sm;                // [N]
    float4 *twN = sm + N;           // [N/2]
    float4 *s = twN + (N >> 1);     // [rpb][N]
    load_real_twiddles_df(tw, twN, twg, N);
    __shared__ int rmax[256];  // largest biased exponent of each row
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int rows = (int)min((int64_t)rpb, nrows - r0);
    for (int t = threadIdx.x; t < rows; t += blockDim.x) rmax[t] = 0;
    __syncthreads();
    // the packed pairs, still FP64, into their bit-reversed slots (a double2
    // fills a float4 slot), and the row maxima
    const double2 *zin = reinterpret_cast<const double2 *>(in) + r0 * N;
    double2 *sd = reinterpret_cast<double2 *>(s);
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const double2 z = zin[e];
        const int ex = biased_exponent2(z);
        if (ex) atomicMax(&rmax[e >> logN], ex);
        sd[(e >> logN) * N + bitrev(e & (N - 1), logN)] = z;
    }
    __syncthreads();
    // scaled and split in place, each slot by the thread that filled it
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e >> logN, i = rl * N + bitrev(e & (N - 1), logN);
        const int sh = rmax[rl] ? 1023 - rmax[rl] : 0;
        const double2 z = sd[i];
        const dfloat re = split_f64(scale2(z.x, sh)), im = split_f64(scale2(z.y, sh));
        s[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    for (int t = threadIdx.x; t < rows; t += blockDim.x) rexp[r0 + t] = rmax[t] ? rmax[t] - 1023 : kZeroRow;
    dft_stages(s, rows, N, logN, twN, conj != 0);
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e >> logN, k = e & (N - 1);
        const dcomplex a = load_df(s[rl * N + k]), b = load_df(s[rl * N + ((N - k) & (N - 1))]);
        const dcomplex E = {df_half(df_add(a.re, b.re)), df_half(df_add(a.im, df_neg(b.im)))};
        const dcomplex O = {df_half(df_add(a.im, b.im)), df_half(df_add(b.re, df_neg(a.re)))};
        out[(r0 + rl) * n + k] = store_df(cadd(E, cmul(load_df(tw[k]), O, conj != 0)));
    }
}

// Columns pass of the inverse on the m' >= 0 half of a Hermitian spectrum:
// for every slice, the length-n DFT along the middle index of columns
// 0..ncols-1, `kb` (<= 64) adjacent columns per block; FP64 in, double-float
// out, possibly to the same memory (each block reads its whole tile before
// writing it).  Every column is scaled by the power of two of its own largest
// magnitude, recorded in cexp[slice ncols + column] (kZeroRow when all zero).
__global__ void __launch_bounds__(kFftThreads) fft_cols_f64_kernel(const double2 *in, float4 *out, int n, int logn,
                                                                    int kb, int ncols, const float4 *__restrict__ twg,
                                                                    int conj, int *__restrict__ cexp) {
    extern __shared__ __align__(16) float4 sm[];
    float4 *tw = sm;              // [n/2]
    float4 *s = sm + (n >> 1);    // [kb][n], column c at s + c n
    for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) tw[t] = twg[t];
    __shared__ int cmax[64];
    const int tiles = ncols / kb;
    const int64_t js = blockIdx.x / tiles;
    const int k0 = (blockIdx.x % tiles) * kb;
    const int64_t base = js * n * n + k0;
    for (int t = threadIdx.x; t < kb; t += blockDim.x) cmax[t] = 0;
    __syncthreads();
    double2 *sd = reinterpret_cast<double2 *>(s);
    for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
        const int i = e / kb, c = e % kb;
        const double2 v = in[base + (int64_t)i * n + c];
        const int ex = biased_exponent2(v);
        if (ex) atomicMax(&cmax[c], ex);
        sd[c * n + bitrev(i, logn)] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
        const int i = e / kb, c = e % kb, idx = c * n + bitrev(i, logn);
        const int sh = cmax[c] ? 1023 - cmax[c] : 0;
        const double2 v = sd[idx];
        const dfloat re = split_f64(scale2(v.x, sh)), im = split_f64(scale2(v.y, sh));
        s[idx] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    for (int t = threadIdx.x; t < kb; t += blockDim.x) cexp[js * ncols + k0 + t] = cmax[t] ? cmax[t] - 1023 : kZeroRow;
    dft_stages(s, kb, n, logn, tw, conj != 0);
    for (int e = threadIdx.x; e < n * kb; e += blockDim.x) {
        const int i = e / kb, c = e % kb;
        out[base + (int64_t)i * n + c] = s[c * n + i];
    }
}

// Rows pass back to a real grid: X[0..N) of each row at in + row n
// (double-float, column k of slice j scaled by 2^-cexp[j N + k]; X[N] = 0) ->
// nrows real rows of n samples in `out` (FP64).  `rpb` divides n, so a
// block's rows lie in one slice, whose columns are brought to their largest
// scale by exact power-of-two products.
__global__ void __launch_bounds__(kFftThreads) fft_rows_c2r_kernel(const float4 *in, double *out, int64_t nrows, int n,
                                                                    int logN, int rpb, const float4 *__restrict__ twg,
                                                                    int conj, const int *__restrict__ cexp) {
    extern __shared__ __align__(16) float4 sm[];
    const int N = n >> 1;
    float4 *tw = sm;                // [N]
    float4 *twN = sm + N;           // [N/2]
    float4 *s = twN + (N >> 1);     // [rpb][N]
    load_real_twiddles_df(tw, twN, twg, N);
    __shared__ float fs[kMaxB];     // per column: 2^(cexp - the slice's largest)
    __shared__ int smax;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t js = r0 / n;
    const int rows = (int)min((int64_t)rpb, nrows - r0);
    if (threadIdx.x == 0) smax = kZeroRow;
    __syncthreads();
    int lm = kZeroRow;
    for (int k = threadIdx.x; k < N; k += blockDim.x) lm = max(lm, cexp[js * N + k]);
    atomicMax(&smax, lm);
    __syncthreads();
    const int sref = smax;
    for (int k = threadIdx.x; k < N; k += blockDim.x) fs[k] = pow2f(cexp[js * N + k] - sref);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const int rl = e >> logN, k = e & (N - 1);
        const float4 *row = in + (r0 + rl) * n;
        const dcomplex a = dc_scale(load_df(row[k]), fs[k]);
        const dcomplex b = k ? dc_scale(load_df(row[N - k]), fs[N - k]) : dcomplex{{0.f, 0.f}, {0.f, 0.f}};
        const dcomplex A = {df_add(a.re, b.re), df_add(a.im, df_neg(b.im))};  // X[k] + conj X[N-k]
        const dcomplex D = {df_add(a.re, df_neg(b.re)), df_add(a.im, b.im)};  // X[k] - conj X[N-k]
        const dcomplex C = cmul(load_df(tw[k]), D, conj != 0);
        s[rl * N + bitrev(k, logN)] = store_df(cadd(A, mul_i(C, true)));  // A + i C
    }
    dft_stages(s, rows, N, logN, twN, conj != 0);
    const int sh = sref == kZeroRow ? 0 : sref;
    double2 *o = reinterpret_cast<double2 *>(out) + r0 * N;  // (x[2t], x[2t+1]) = (Re z[t], Im z[t])
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
        const dcomplex z = load_df(s[e]);
        o[e] = make_double2(scale2(join_f64(z.re), sh), scale2(join_f64(z.im), sh));
    }
}

// tw[t] = exp(+2 pi i t / n) in double-float, t < n/2.
__global__ void twiddle_kernel(int n, float4 *tw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n / 2) {
        const double a = 2.0 * t / n;
        const dfloat c = split_f64(cospi(a)), s = split_f64(sinpi(a));
        tw[t] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
}

int ilog2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

}  // namespace

bool df_fft_supported(int B) {
    const int n = 2 * B;
    return n >= 2 && n <= 2 * kMaxB && ilog2_exact(n) >= 0;
}

cudaError_t launch_df_twiddles(int B, float4 *tw, cudaStream_t s) {
    const int n = 2 * B;
    twiddle_kernel<<<(n / 2 + 127) / 128, 128, 0, s>>>(n, tw);
    count_launch();
    return cudaGetLastError();
}

// 2-D DFT of `nslices` consecutive n x n slices (n = 2B): `in` (FP64, layout
// [j][i][k]) -> `out` (FP64, [j][m][m']), exp(sign i ...), unnormalised.
// `work` is a double-float buffer of nslices n^2 float4 (16 bytes each); it
// may be `in` or `out`.  `rexp` is nslices n ints of scratch (the row
// scales).  All four point at the first slice of the range.
cudaError_t launch_df_fft2(int B, const double2 *in, double2 *out, float4 *work, const float4 *tw, int sign,
                           int *rexp, cudaStream_t s, int nslices) {
    const int n = 2 * B, logn = ilog2_exact(n);
    if (logn < 1 || nslices < 1 || nslices > n) return cudaErrorInvalidValue;
    const int conj = sign < 0 ? 1 : 0;
    const int64_t nrows = (int64_t)nslices * n;
    const int rpb = std::max(1, 512 / n);
    const size_t rbytes = sizeof(float4) * ((size_t)n / 2 + (size_t)rpb * n);
    cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rbytes);
    if (e != cudaSuccess) return e;
    fft_rows_kernel<<<(unsigned)((nrows + rpb - 1) / rpb), kFftThreads, rbytes, s>>>(in, work, nrows, n, logn, rpb,
                                                                                     tw, conj, rexp);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int kb = std::min(n, std::max(4, 4096 / n));
    const size_t cbytes = sizeof(float4) * ((size_t)n / 2 + (size_t)kb * n);
    e = cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cbytes);
    if (e != cudaSuccess) return e;
    fft_cols_kernel<<<(unsigned)((int64_t)nslices * (n / kb)), kFftThreads, cbytes, s>>>(work, out, n, logn, kb, n,
                                                                                          tw, conj, rexp);
    count_launch();
    return cudaGetLastError();
}

bool df_real_fft_supported(int B) { return B >= 2 && df_fft_supported(B); }

// Real grid `in` ((2B)^3 doubles, layout [j][i][k]) -> the m' = 0..B-1 half
// of S ([j][m][m'], columns B..2B-1 of every slice left as they are),
// exp(sign i ...): real-row DFTs into S's memory as double-float, then the B
// columns back to FP64 in place.  `rexp`: n^2 ints of scratch.
cudaError_t launch_df_fft2_r2c(int B, const double *in, double2 *S, const float4 *tw, int sign, int *rexp,
                               cudaStream_t s) {
    if (!df_real_fft_supported(B)) return cudaErrorInvalidValue;
    const int n = 2 * B, N = B, logn = ilog2_exact(n);
    const int conj = sign < 0 ? 1 : 0;
    const int64_t nrows = (int64_t)n * n;
    float4 *work = reinterpret_cast<float4 *>(S);
    const int rpb = std::min(256, std::max(1, 1024 / N));  // 1024 values, one radix-4 step per thread and stage
    const size_t rbytes = sizeof(float4) * ((size_t)N + (size_t)(N / 2) + (size_t)rpb * N);
    cudaError_t e = cudaFuncSetAttribute(fft_rows_r2c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rbytes);
    if (e != cudaSuccess) return e;
    fft_rows_r2c_kernel<<<(unsigned)((nrows + rpb - 1) / rpb), kFftThreads, rbytes, s>>>(in, work, nrows, n, logn - 1,
                                                                                         rpb, tw, conj, rexp);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int kb = std::min(N, std::max(4, 4096 / n));
    const size_t cbytes = sizeof(float4) * ((size_t)n / 2 + (size_t)kb * n);
    e = cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cbytes);
    if (e != cudaSuccess) return e;
    fft_cols_kernel<<<(unsigned)((int64_t)n * (N / kb)), kFftThreads, cbytes, s>>>(work, S, n, logn, kb, N, tw, conj,
                                                                                   rexp);
    count_launch();
    return cudaGetLastError();
}

// The m' = 0..B-1 half of a Hermitian S (S(-m,-m') = conj S(m,m'), the
// m' = -B column zero) -> the real grid `out`, exp(sign i ...): the B columns
// in place into double-float, then the rows to FP64 real samples.  S's
// columns 0..B-1 are overwritten.  `cexp`: 2B^2 ints of scratch.
cudaError_t launch_df_fft2_c2r(int B, double2 *S, double *out, const float4 *tw, int sign, int *cexp,
                               cudaStream_t s) {
    if (!df_real_fft_supported(B)) return cudaErrorInvalidValue;
    const int n = 2 * B, N = B, logn = ilog2_exact(n);
    const int conj = sign < 0 ? 1 : 0;
    const int64_t nrows = (int64_t)n * n;
    float4 *work = reinterpret_cast<float4 *>(S);
    const int kb = std::min(N, std::max(4, 4096 / n));
    if (kb > 64) return cudaErrorInvalidValue;
    const size_t cbytes = sizeof(float4) * ((size_t)n / 2 + (size_t)kb * n);
    cudaError_t e = cudaFuncSetAttribute(fft_cols_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cbytes);
    if (e != cudaSuccess) return e;
    fft_cols_f64_kernel<<<(unsigned)((int64_t)n * (N / kb)), kFftThreads, cbytes, s>>>(S, work, n, logn, kb, N, tw,
                                                                                       conj, cexp);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rpb = std::min(n, std::max(1, 1024 / N));  // a power of two dividing n
    const size_t rbytes = sizeof(float4) * ((size_t)N + (size_t)(N / 2) + (size_t)rpb * N);
    e = cudaFuncSetAttribute(fft_rows_c2r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rbytes);
    if (e != cudaSuccess) return e;
    fft_rows_c2r_kernel<<<(unsigned)(nrows / rpb), kFftThreads, rbytes, s>>>(work, out, nrows, n, logn - 1, rpb, tw,
                                                                             conj, cexp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace softgb
