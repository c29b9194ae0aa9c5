// dwt_fp64tc.cu -- FP64-accurate DWT / iDWT with the contraction on the
// tcgen05 tensor cores (mode SOFT_FP64_TC).
//
// Same mathematics as dwt_fp64.cu (Sec. 2.4: f = V_B T_B W_B S per order pair,
// S = T_B^T f), the same FP64 Wigner-d recurrence (Eq. (Wigner_d_recurrence),
// rescaled, from the plan's per-cluster tables) and FP64 S (the 2-D FFTs of
// this mode are in fft_df.cu).  Only the contraction moves, from 16 FP64 FMAs
// per Wigner-d entry to the tensor cores, by the error-free splitting idea of
// Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//
//   * every operand entry is read as a fixed-point number against a
//     power-of-two scale and cut into kDig = 7 balanced base-128 digits
//     (|q| <= 64), each an exact BF16:  v 2^alpha ~= sum_i q_i 2^(-6-7i),
//     error <= 2^-49 of the scale;
//   * digit products are integers of magnitude <= 2^12, so an FP32 TMEM
//     accumulator summing all digit pairs (i, k) of one level i + k over a
//     contraction of K <= 1024 terms stays exact for levels 0..3
//     ((level + 1) 2^22 <= 2^24); levels 4..6 carry a relative weight
//     <= 2^-28, where FP32 rounding is immaterial, and pairs of level >= 7
//     (weight <= 2^-49) are dropped;
//   * per K step, the MMA of A digit i runs against B digits 0..6-i stacked as
//     the N = 16 (7 - i) rows of one operand and accumulates into TMEM columns
//     16 i .. 16 i + N - 1, so level k of output column c always lands in
//     column 16 k + c: 7 MMAs per K step, 112 accumulator columns;
//   * the epilogue recombines the levels -- the four exact leading ones in
//     64-bit integers, so that no FP32 rounding touches them -- and builds the
//     FP64 result by integer operations with the scales folded into its
//     exponent.
//
// Scales.  The rescaled recurrence yields e(t) = d(l0+t)/sig_t.  With
// sig_t = 2^E_t mu_t, mu_t in [1, 2), e(t) 2^E_t = d/mu_t is in [-1, 1]
// because |d| <= 1.  The forward also carries w_B(j) (folded into the seeds),
// bounded by 2^-ew (ew fixed per plan).  Data columns (S in the forward, the
// sign-, V- and mu-folded coefficients in the inverse) are scaled by 2^-F_c,
// F_c the exponent just above the column's largest magnitude over the
// contraction (for S from one coalesced pass, colexp_kernel, before the DWT).
//
// The forward contracts K = 2B <= 1024 beta samples and the inverse K = L <= B
// degrees, both within the exactness bound for B <= 512.
#include "soft.h"
#include "soft_internal.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

namespace softgb {
namespace {

constexpr int kDig = 7;              // digits per operand entry (and levels kept)
constexpr int kCols = 16;            // 8 partners x (re, im)
constexpr int kNB = kDig * kCols;    // 112 B-operand rows: digit k of column c at row 16 k + c
constexpr uint32_t kTmemCols = 512;  // the forward's 4 tile accumulators of 112 (128) columns
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ int mod_n(int a, int n) { return a < 0 ? a + n : a; }

// FP32 bit pattern of f - 64 for a 7-bit field f <= 255 (BF16 in the upper
// half): 0x4B400000 | f is the float 1.5 2^23 + f, so one bitwise OR (which
// merges with the field's mask) and one FP32 add.
__device__ __forceinline__ uint32_t field_digit_bits(uint32_t f) {
    return __float_as_uint(__uint_as_float(0x4B400000u | f) - 12582976.0f);
}

// Balanced base-128 digits of N = floor(v 2^(alpha + 48) + 1/2) for
// |v 2^alpha| <= 1: N = sum_i q_i 128^(6 - i), so v 2^alpha ~= sum_i q_i
// 2^(-6-7i) to within 2^-49, |q_i| <= 64.  Returned as FP32 bit patterns
// (BF16 in the upper halves).  Integer operations only; magnitudes below 2^-49
// of the scale give 0.
//
// With K7 = sum_i 64 128^i, P = N + K7 >= 0 has the ordinary base-128 digits
// q_i + 64 (the leading one up to 128, the others in [0, 127]): the balanced
// digits with the lower six in [-64, 63] are unique, so the seven digits are
// independent bit fields of P instead of a carry chain.  P comes from
// T = floor(v 2^(alpha + 49)) (an arithmetic shift of the signed significand)
// as P = (T + 1 + 2 K7) >> 1, so the digit fields are read from
// Q = T + 1 + 2 K7 one bit higher up.
constexpr long long kDigitOffset = 64ll * ((1ll << 49) - 1) / 127;  // K7

__device__ __forceinline__ void digits7(double v, int alpha, uint32_t (&q)[kDig]) {
    const long long b = __double_as_longlong(v);
    const int e = (int)(((unsigned long long)b >> 52) & 0x7FF);
    // |v| 2^(alpha + 49) = significand >> s, s >= 3 within the bound; zero (and
    // subnormal) inputs shift everything out
    const int s = min(1026 - alpha - e, 63);
    const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const long long T = (b < 0 ? -M : M) >> s;
    const unsigned long long Q = (unsigned long long)(T + (2 * kDigitOffset + 1));  // < 2^51
    const uint32_t lo = (uint32_t)Q, hi = (uint32_t)(Q >> 22);  // digit i at bit 1 + 7 (6 - i) of Q
    q[6] = field_digit_bits((lo >> 1) & 127);
    q[5] = field_digit_bits((lo >> 8) & 127);
    q[4] = field_digit_bits((lo >> 15) & 127);
    q[3] = field_digit_bits(hi & 127);
    q[2] = field_digit_bits((hi >> 7) & 127);
    q[1] = field_digit_bits((hi >> 14) & 127);
    q[0] = field_digit_bits(hi >> 21);
}

// Unbiased exponent of a positive normal double.
__device__ __forceinline__ int exponent_of(double v) {
    return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF) - 1023;
}

// Magnitude bits of |v| (orders like |v| for finite values).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// Column exponent F with |x| < 2^F for every |x| <= the double whose magnitude bits are mb.
__device__ __forceinline__ int column_exponent(unsigned long long mb) {
    return mb == 0 ? 0 : (int)(mb >> 52) - 1023 + 1;
}

// v 2^k by an exponent-field add (v normal or 0; results below the normal range flush to 0).
__device__ __forceinline__ double ldexp_bits(double v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0 || e == 0x7FF) return v;
    const int e2 = e + k;
    if (e2 <= 0) return __longlong_as_double((long long)(b & (1ull << 63)));
    if (e2 >= 0x7FF) return __longlong_as_double((long long)((b & (1ull << 63)) | (0x7FFull << 52)));
    return __longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((unsigned long long)e2 << 52)));
}

// FP32 pattern of an exact integer |v| <= 2^24 -> int (integer operations).
__device__ __forceinline__ int exact_f32_int(uint32_t b) {
    const int e = (int)((b >> 23) & 0xFF);
    const uint32_t m2 = ((b & 0x7FFFFFu) | 0x800000u) << 1;
    const int v = (int)(m2 >> min(151 - e, 31));
    return (b >> 31) ? -v : v;
}

// X 2^k as a double for |X| < 2^63 (integer operations; low bits beyond 53
// truncated, results below the normal range flush to 0).
__device__ __forceinline__ double int64_ldexp(long long X, int k) {
    if (X == 0) return 0.0;
    const unsigned long long s = (unsigned long long)X & (1ull << 63);
    const unsigned long long a = X < 0 ? 0ull - (unsigned long long)X : (unsigned long long)X;
    const int lz = __clzll((long long)a);
    const int e = 1023 + 63 - lz + k;  // biased exponent of the leading bit
    if (e <= 0) return __longlong_as_double((long long)s);
    const unsigned long long mant = (lz >= 11 ? a << (lz - 11) : a >> (11 - lz)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(s | ((unsigned long long)e << 52) | mant));
}

// Epilogue for one warp's 32 TMEM lanes: the 16 outputs of this lane's row,
//   out_c = 2^(F_c - 12) T_c,  T = L0 + 2^-7 L1 + 2^-14 L2 + 2^-21 L3 + 2^-28 R',
// R' = L4 + 2^-7 L5 + 2^-14 L6 in FP32 (weight <= 2^-28: its rounding is
// immaterial).  Levels 0..3 are exact integers and are combined exactly in
// 64-bit integers, X = 2^39 T:
//   X = (((L0 128 + L1) 128 + L2) 128 + L3) 2^18 + round(2^11 R'),
// so most of the result's bits -- which sit in levels 1..3 whenever entries
// are small against their scales -- never pass through FP32 rounding.  No
// FP64 arithmetic.  Warp-collective (tcgen05.ld).
__device__ __forceinline__ void epilogue_levels(uint32_t tbase, const int *colexp, double (&out)[kCols]) {
    uint32_t d[16];
    float rp[16];
    tc::tmem_ld16(tbase + kCols * 6, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) rp[c] = __uint_as_float(d[c]);
#pragma unroll 1
    for (int k = 5; k >= 4; --k) {
        tc::tmem_ld16(tbase + kCols * k, d);
#pragma unroll
        for (int c = 0; c < 16; ++c) rp[c] = fmaf(rp[c], 0x1p-7f, __uint_as_float(d[c]));
    }
    int y[16];
    tc::tmem_ld16(tbase, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) y[c] = exact_f32_int(d[c]);
    tc::tmem_ld16(tbase + kCols, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) y[c] = y[c] * 128 + exact_f32_int(d[c]);  // <= 2^30
    long long X[16];
    tc::tmem_ld16(tbase + 2 * kCols, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) X[c] = (long long)y[c] * 128 + exact_f32_int(d[c]);
    tc::tmem_ld16(tbase + 3 * kCols, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        X[c] = X[c] * 128 + exact_f32_int(d[c]);
        X[c] = X[c] * (1ll << 18) + __float2ll_rn(rp[c] * 0x1p11f);
        out[c] = int64_ldexp(X[c], colexp[c] - 12 - 39);
    }
}

// Store the digits of 4 consecutive K entries (k0 a multiple of 4) of operand
// row `row` into the 7 digit planes: 8 bytes per plane at plane0 + i * plane
// (+ the row and K-group offsets of the no-swizzle K-major layout).
__device__ __forceinline__ void put_digits4(unsigned char *plane0, int plane, int lbo, int row, int k0,
                                            const double (&v)[4], const int (&alpha)[4]) {
    uint32_t d[4][kDig];
#pragma unroll
    for (int u = 0; u < 4; ++u) digits7(v[u], alpha[u], d[u]);
    unsigned char *dst = plane0 + (k0 / 8) * lbo + 16 * row + 2 * (k0 % 8);
#pragma unroll
    for (int i = 0; i < kDig; ++i) {
        uint2 w;
        w.x = __byte_perm(d[0][i], d[1][i], 0x7632);
        w.y = __byte_perm(d[2][i], d[3][i], 0x7632);
        *reinterpret_cast<uint2 *>(dst + i * plane) = w;
    }
}

// One K chunk of MMAs (issued by one thread): for each K step of 16, A digit
// i (plane i) against B digits 0..6-i into TMEM columns 16 i ..; committed to mbar.
template <int M>
__device__ __forceinline__ void issue_levels(uint32_t tmem, const unsigned char *A, int a_plane, uint32_t a_lbo,
                                             const unsigned char *Bop, uint32_t b_lbo, bool first, int ksteps,
                                             uint64_t *mbar) {
    tc::fence_after_sync();
    // Descriptors advance by adding (byte offset >> 4) to their 14-bit start
    // address field: every offset is a multiple of 16 bytes, and shared-memory
    // addresses stay below 2^18 bytes, so the field never carries.
    const uint64_t ad0 = tc::smem_desc(tc::smem_u32(A), a_lbo, 128), bd0 = tc::smem_desc(tc::smem_u32(Bop), b_lbo, 128);
    for (int s = 0; s < ksteps; ++s) {
        const uint64_t bd = bd0 + (uint64_t)((s * 2 * b_lbo) >> 4);
        const uint64_t as = ad0 + (uint64_t)((s * 2 * (int)a_lbo) >> 4);
#pragma unroll
        for (int i = 0; i < kDig; ++i) {
            constexpr uint32_t kIdesc0 = tc::instr_desc(1, M, kCols * kDig);
            const uint32_t idesc = kIdesc0 - ((uint32_t)(kCols * i) >> 3 << 17);  // N = 16 (7 - i)
            const uint64_t ad = as + (uint64_t)((i * a_plane) >> 4);
            tc::mma_bf16(tmem + kCols * i, ad, bd, idesc, (first && s == 0 && i == 0) ? 0u : 1u);
        }
    }
    tc::mma_commit(mbar);
}

// ---------------------------------------------------------------------------
// Both kernels split the CTA into warp-specialised roles; the forward's are
// below (the inverse runs eight producer and eight converter warps over two
// sample tiles, laid out at its kernel):
//   producers  (128 threads, warps 0-3) run the FP64 recurrence -- two FMAs
//              per Wigner-d entry and nothing else -- and write the raw FP64
//              values into a staging ring of kStages groups, kGroup rows
//              (forward) or degrees (inverse) per group;
//   converters (256 threads, warps 4-11) cut staged values and the data
//              operand into digits (4 values per thread and task) and run the
//              epilogue (warps 4-7, one per TMEM lane quarter).  Two converter
//              warps per scheduler hide the latency of the integer digit chains;
//   issuer     (lane 0 of warp 12) issues each chunk's MMAs once the
//              converters signal the operands ready.  A tcgen05.mma of these
//              shapes occupies its issuing thread for ~45 cycles, so issuing
//              from a converter would stall that whole group; from its own
//              warp the issue overlaps the converters' next B operand.
// So the FP64 pipe (producers) and the integer pipes (converters) work in
// parallel instead of in one warp's instruction stream.  Hand-off through
// mbarriers (full: one arrival per producer warp, empty: one per converter
// warp, each after a __syncwarp that orders the warp's staging accesses
// before its lane 0's release; ready: one converter arrival per chunk, mma:
// the tcgen05 commit); every wait is bounded and its verdict warp-uniform.
// A ring of two 16-row groups hands off half as often as four 8-row ones
// for the same staging bytes: each hand-off costs the single producer warp
// of a scheduler FP64-pipe time that no other warp fills.  Converters, which
// synchronise among themselves once per chunk to agree that the operands are
// complete, take that barrier as an AND reduction of their wait verdicts so
// that a timeout makes the whole group leave together; producers and the
// issuer synchronise with nobody but the mbarriers and leave individually.
// ---------------------------------------------------------------------------
constexpr int kProd = 128;    // producer threads (warps 0-3)
constexpr int kConv = 256;    // converter threads (warps 4-11)
constexpr int kIssuer = kProd + kConv;  // lane 0 of warp 12 issues the MMAs
constexpr int kSetup = kIssuer + 32;    // warp 13 prepares the next cluster's tables
constexpr int kThreadsFwd = kSetup + 32;  // 448 threads (the forward)
constexpr int kBarConv = 1;   // named barrier of the converters

constexpr int kStages = 2;    // staging ring depth (groups)
constexpr int kGroup = 16;    // rows (forward) or degrees (inverse) per staged group

struct PipeBars {
    uint64_t full[kStages], empty[kStages], ready, mma;
    uint64_t data[2];  // TMA copies of the data operand into B buffer 0 / 1 (forward)
};

__device__ __forceinline__ void init_pipe(PipeBars &pb) {
#pragma unroll
    for (int b = 0; b < kStages; ++b) {
        tc::mbar_init(&pb.full[b], kProd / 32);
        tc::mbar_init(&pb.empty[b], kConv / 32);
    }
    tc::mbar_init(&pb.ready, 1);
    tc::mbar_init(&pb.mma, 1);
    tc::mbar_init(&pb.data[0], 1);
    tc::mbar_init(&pb.data[1], 1);
}

// Issuer: wait until the converters have written the operands of the next chunk.
__device__ __forceinline__ bool issuer_acquire(PipeBars &pb, uint32_t &rph) {
    const bool done = tc::mbar_wait(&pb.ready, rph, kWaitPolls);
    rph ^= 1u;
    return done;
}

// Producer: wait until staging buffer gi % kStages is free (its previous group
// consumed).  Producers take no named barrier anywhere, so each warp decides
// alone: one that gives up stops arriving, and the converters' own bounded
// waits end.  Warp-collective; the verdict is the same on every lane.
__device__ __forceinline__ bool producer_acquire(PipeBars &pb, uint32_t gi) {
    return __all_sync(0xffffffffu, tc::mbar_wait(&pb.empty[gi % kStages], ((gi / kStages) & 1) ^ 1u, kWaitPolls));
}

// Converter: wait until staging buffer gi % kStages holds group gi.  Each
// converter warp decides alone here (no barrier per group): a warp that gives
// up skips the rest of its chunk, and the AND-reducing barrier that closes
// every chunk (chunk_done) gives the whole group that verdict.  Warp-collective.
__device__ __forceinline__ bool converter_acquire(PipeBars &pb, uint32_t gi) {
    return __all_sync(0xffffffffu, tc::mbar_wait(&pb.full[gi % kStages], (gi / kStages) & 1, kWaitPolls));
}

// Producer / converter warp: its staging writes / reads of group gi are done.
__device__ __forceinline__ void release_full(PipeBars &pb, uint32_t gi) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&pb.full[gi % kStages]);
}
__device__ __forceinline__ void release_empty(PipeBars &pb, uint32_t gi) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&pb.empty[gi % kStages]);
}

// Converter: all converters have written the chunk's operands (or one gave up).
__device__ __forceinline__ bool chunk_done(bool ok) { return tc::group_and(kBarConv, kConv, ok); }

// Converter: wait for the chunk MMAs committed last.
// `ok` joins this thread's own verdict so far into the group's.
__device__ __forceinline__ bool converter_wait_mma(PipeBars &pb, uint32_t &mph, bool ok = true) {
    const bool done = tc::mbar_wait(&pb.mma, mph, kWaitPolls);
    mph ^= 1u;
    return tc::group_and(kBarConv, kConv, done && ok);
}

// ---------------------------------------------------------------------------
// Forward DWT, persistent.  One CTA per SM walks the clusters
// fwd_order[blockIdx.x + k gridDim.x], k = 0, 1, ... (longest first, dealt out
// round robin); tiles of TM = 64 degrees (M), K chunks of KC = 128 beta
// samples, one producer per sample.  The tiles of a cluster are taken in
// passes of up to four, whose accumulators stay in TMEM (columns 128 t + 0..111
// for the pass's tile t), and each pass runs chunk by chunk: for chunk c the
// producers carry their samples' recurrence through all the pass's tiles, and
// the converters cut the chunk's data operand once for all of them.  The
// producers keep the recurrence state of their samples at the end of a pass
// in registers for the next (only clusters of more than 256 degrees have a
// second pass).  The roles run on across cluster boundaries, and a fourth one
// prepares each cluster's tables ahead of use:
//   set-up     (warp 13) fills slot k & 1 with cluster k's partner table,
//              column scales, recurrence coefficients and digit exponents as
//              soon as cluster k-2 has released it, so the prologue of a
//              cluster overlaps the previous cluster's work;
// and the TMEM allocation, barrier set-up and launch happen once per SM
// instead of once per cluster.  Slot hand-off by mbarriers: slot_full (the
// set-up warp's 32 arrivals), slot_empty (every producer after its last
// group of the cluster, every converter after the cluster's last epilogue).
// Converter schedule per step (pass, chunk, tile): at the chunk's first tile,
// its data operand into B buffer (chunk step) % 2 (TMA copies issued one chunk
// ahead, cut into digits in place); wait for the previous step's MMAs (then the
// epilogue when they closed a tile, possibly of the previous cluster); A digits
// of the staged groups; MMAs of the step.
//   dynamic smem: A planes [7] | B operand [2] | staging [kStages][kGroup rows][KC] |
//                 slot [2] { rA, rAc [B doubles], alpha [B ints] }
// ---------------------------------------------------------------------------

struct SlotHdr {
    ClusterSmem cs;
    int colexp[kCols];
};

// Doubles per table slot of the persistent forward: rA, rAc, then B ints.
__host__ __device__ constexpr size_t fwd_slot_doubles(int B) { return 2 * (size_t)B + ((size_t)B + 1) / 2; }

__global__ void __launch_bounds__(kThreadsFwd, 1) dwt_forward_tc_kernel(Tables tb, const __grid_constant__ CUtensorMap tmS,
                                                                        double *__restrict__ coef, int flags) {
    constexpr int KC = kProd, TM = 64, G = kGroup, MAXC = 2 * kMaxB / KC;
    constexpr int A_LBO = TM * 16 + 16, A_PLANE = (KC / 8) * A_LBO;
    constexpr int B_LBO = kNB * 16 + 16, B_BYTES = (KC / 8) * B_LBO;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SlotHdr hdr[2];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) PipeBars pb;
    __shared__ __align__(8) uint64_t slot_full[2], slot_empty[2];
    const int B = tb.B, n = 2 * B, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunks = (n + KC - 1) / KC;
    const int wshift = (flags & kApplyW) ? -tb.wexp : 0;  // 2^wshift max_j w_B(j) < 1 for the weighted seeds

    unsigned char *A = smem;
    unsigned char *X = smem + kDig * A_PLANE;  // [2][B_BYTES]
    double *stage = reinterpret_cast<double *>(X + 2 * B_BYTES);  // [kStages][G][KC]
    double *slotd = stage + kStages * G * KC;
    const size_t SLOT = fwd_slot_doubles(B);
    auto slot_rA = [&](int s) { return slotd + s * SLOT; };
    auto slot_rAc = [&](int s) { return slotd + s * SLOT + B; };
    auto slot_alpha = [&](int s) { return reinterpret_cast<int *>(slotd + s * SLOT + 2 * B); };
    // The k-th cluster of this CTA (false past the end of the list).
    auto cluster_of = [&](int k, int &cidx, int &m, int &mp) {
        const int idx = blockIdx.x + k * gridDim.x;
        if (idx >= tb.ncl) return false;
        cidx = tb.fwd_order ? tb.fwd_order[idx] : idx;
        const int2 rep = tb.clusters[cidx];
        m = rep.x;
        mp = rep.y;
        return true;
    };

    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
    if (tid == 0) {
        init_pipe(pb);
        for (int s2 = 0; s2 < 2; ++s2) {
            tc::mbar_init(&slot_full[s2], 32);
            tc::mbar_init(&slot_empty[s2], kProd + kConv);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp == kSetup / 32) {
        // ---- set-up: the tables of cluster k into slot k & 1 ----
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1;
            if (k >= 2) {  // slot s last held cluster k - 2
                const bool done = tc::mbar_wait(&slot_empty[s], ((k >> 1) - 1) & 1, kWaitPolls);
                ok = __all_sync(0xffffffffu, done);
                if (!ok) break;
            }
            SlotHdr &h = hdr[s];
            if (lane == 0) fill_cluster(tb, m, mp, h.cs);
            const int L = B - m;
            const double *src = tb.rectab + (size_t)cidx * B * 3;
            double *rA = slot_rA(s), *rAc = slot_rAc(s);
            int *alpha = slot_alpha(s);
            for (int t = lane; t < L; t += 32) {
                rA[t] = src[3 * t];
                rAc[t] = src[3 * t + 1];
                alpha[t] = exponent_of(src[3 * t + 2]) + wshift;  // digit exponent of row t: sig_t's, with the weight scale
            }
            __syncwarp();
            if (lane < kCols) {
                // column scales of S_p (re and im), from the per-(m, m') exponents written by
                // colexp_kernel before this launch (the mirror does not change a maximum)
                const int p = lane >> 1, np = h.cs.np;
                const bool real = (flags & kRealSym) && np > 1;
                int e = 0;
                if (p < np && !(real && (p & 1)))
                    e = tb.colexp[((int64_t)mod_n(h.cs.pm[p], n) * n + mod_n(h.cs.pmp[p], n)) * 2 + (lane & 1)];
                h.colexp[lane] = e == 0 ? 0 : e - 1023 + 1;
            }
            tc::mbar_arrive(&slot_full[s]);
        }
    } else if (tid < kProd) {
        // ---- producers: sample j = c KC + t of every chunk c, rows in groups of G ----
        const int t = tid;
        uint32_t gi = 0;
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1, l0 = m;
            ok = tc::mbar_wait(&slot_full[s], (k >> 1) & 1, kWaitPolls);
            if (!ok) break;
            const double *rA = slot_rA(s), *rAc = slot_rAc(s);
            const int ntile = (B - l0 + TM - 1) / TM, npass = (ntile + 3) / 4;
            double dcs[MAXC], dps[MAXC];  // each chunk's recurrence state at the end of a pass
            for (int pp = 0; pp < npass && ok; ++pp) {
                const int t0 = 4 * pp, nt = min(4, ntile - t0);
#pragma unroll
                for (int c = 0; c < MAXC; ++c) {
                    if (c >= nchunks || !ok) break;
                    const int j = c * KC + t;
                    const bool col = j < n;
                    const double x = col ? tb.cosb[j] : 0.0;
                    double dc = 0.0, dp = 0.0;
                    if (pp == 0) {
                        if (col) {
                            const double sd = tb.seedtab[(size_t)cidx * n + j];
                            dc = (flags & kApplyW) ? sd * tb.w[j] : sd;
                        }
                    } else {
                        dc = dcs[c];
                        dp = dps[c];
                    }
#pragma unroll 1
                    for (int tt = 0; tt < nt && ok; ++tt) {
                        const int lb = l0 + TM * (t0 + tt), rows = min(TM, B - lb);
                        const int ngroups = (rows + G - 1) / G;  // groups past the cluster's last degree are skipped
#pragma unroll 1
                        for (int g = 0; g < ngroups; ++g, ++gi) {  // rolled: the chunk loop around it is unrolled
                            ok = producer_acquire(pb, gi);
                            if (!ok) break;
                            double *st = stage + (gi % kStages) * G * KC + t;
                            const int nv = min(G, rows - g * G);  // warp-uniform
                            const int q0 = lb + g * G - l0;
                            if (!col) {
                                for (int rr = 0; rr < nv; ++rr) st[rr * KC] = 0.0;
                            } else if (nv == G) {
                                // a whole group: straight-line code, no predicated FP64 work, in
                                // halves of 8 rows.  A half's coefficients are loaded before its
                                // first staging store (a store could alias them, so later loads
                                // would wait for it), and the first FMA of a row, which does not
                                // depend on the recurrence, runs two rows ahead of the second, so
                                // that the dependent chain finds the FP64 pipe busy rather than
                                // idle while it waits.
#pragma unroll
                                for (int hh = 0; hh < G; hh += 8) {
                                    double ca[8], cb[8];
#pragma unroll
                                    for (int rr = 0; rr < 8; ++rr) {
                                        ca[rr] = rA[q0 + hh + rr];
                                        cb[rr] = rAc[q0 + hh + rr];
                                    }
                                    double u0 = fma(ca[0], x, -cb[0]), u1 = fma(ca[1], x, -cb[1]);
#pragma unroll
                                    for (int rr = 0; rr < 8; ++rr) {
                                        st[(hh + rr) * KC] = dc;
                                        const double nx = fma(u0, dc, -dp);
                                        u0 = u1;
                                        if (rr + 2 < 8) u1 = fma(ca[rr + 2], x, -cb[rr + 2]);
                                        dp = dc;
                                        dc = nx;
                                    }
                                }
                            } else {
#pragma unroll 1
                                for (int rr = 0; rr < nv; ++rr) {
                                    st[rr * KC] = dc;
                                    const double nx = fma(fma(rA[q0 + rr], x, -rAc[q0 + rr]), dc, -dp);
                                    dp = dc;
                                    dc = nx;
                                }
                            }
                            // staged rows nv..G-1 are never read: the converters take rows < `rows` only
                            release_full(pb, gi);
                        }
                    }
                    dcs[c] = dc;
                    dps[c] = dp;
                }
            }
            if (ok) tc::mbar_arrive(&slot_empty[s]);  // this producer is done with the slot's tables
        }
    } else if (tid >= kProd && tid < kIssuer) {
        // ---- converters ----
        const int t = tid - kProd;
        const int wq = warp & 3;  // TMEM lane quarter of this warp
        uint32_t gi = 0, mph = 0, bc = 0;  // bc: chunk steps (B buffer bc & 1)
        bool pending = false;     // MMAs committed and not yet waited for
        // the tile those MMAs close (prows > 0), for the deferred epilogue: its first degree,
        // rows, accumulator (128 ptile), cluster slot, first degree of the cluster and index
        int plb = 0, prows = 0, ptile = 0, pslot = 0, pl0 = 0, pcidx = 0;
        bool plast = false;       // ... and whether that tile is its cluster's last
        auto epilogue = [&]() {
            // Degree plb + 16 w + i sits in TMEM lane 32 w + i (i < 16), w = lane quarter (warps 4-7).
            tc::fence_after_sync();
            if (t < 128) {
                const SlotHdr &h = hdr[pslot];
                const int np = h.cs.np;
                const bool real = (flags & kRealSym) && np > 1;
                const int r = 16 * wq + lane;
                const int l = plb + r, q = l - pl0;
                double v16[kCols];
                epilogue_levels(tmem + ((uint32_t)(wq * 32) << 16) + 128 * ptile, h.colexp, v16);
                if (lane < 16 && r < prows) {
                    // V_l sig_t 2^-alpha_t
                    const double V = (flags & kApplyV) ? (2.0 * l + 1.0) / (8.0 * M_PI * B) : 1.0;
                    const double v = ldexp_bits(V * tb.rectab[((size_t)pcidx * B + q) * 3 + 2], -slot_alpha(pslot)[q]);
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        if (p >= np) break;
                        if (real && (p & 1)) continue;  // written from its pair below
                        const double vs = ((h.cs.sign[p] < 0.0) != (h.cs.lpar[p] && (l & 1))) ? -v : v;
                        const double2 f = make_double2(vs * v16[2 * p], vs * v16[2 * p + 1]);
                        *reinterpret_cast<double2 *>(coef + 2 * (h.cs.off[p] + q)) = f;
                        if (real) {  // partner p + 1 = (-m, -m'): (-1)^(m-m') conj f
                            const bool odd = (h.cs.pm[p] - h.cs.pmp[p]) & 1;
                            *reinterpret_cast<double2 *>(coef + 2 * (h.cs.off[p + 1] + q)) =
                                odd ? make_double2(-f.x, f.y) : make_double2(f.x, -f.y);
                        }
                    }
                }
            }
            tc::fence_before_sync();
        };
        // B operand task of this thread: partner bp (re and im), beta samples
        // bk0..bk0+3 of a chunk.  The partners' S columns reach the chunk's B buffer
        // by TMA one (tile, chunk) step ahead, as boxes of BJ samples x (re, im) (box
        // row r of partner p at byte p PS + 16 r, PS = 16 BJ rounded up to the 128-byte
        // alignment of a TMA destination; a mirrored partner's box is the reversed
        // sample range), and are cut into digits in place.  The partner boxes share
        // their bank alignment, so a thread reads its four rows starting at row
        // bp mod 4: the 8 lanes of a sample quad then spread over 4 row residues.
        const int bp = lane & 7, bk0 = 4 * (4 * (warp - 4) + (lane >> 3)), brot = bp & 3;
        const int BJ = min(KC, n), PS = (16 * BJ + 127) & ~127;
        auto b_used = [&](const SlotHdr &h, int p) {
            return p < h.cs.np && !((flags & kRealSym) && h.cs.np > 1 && (p & 1));
        };
        // thread 0: the copies of chunk c of the cluster in h into B buffer `buf`
        auto issue_b = [&](const SlotHdr &h, int c, int buf) {
            uint32_t bytes = 0;
#pragma unroll 1
            for (int p = 0; p < 8; ++p)
                if (b_used(h, p)) bytes += 16u * BJ;
            tc::mbar_arrive_expect_tx(&pb.data[buf], bytes);
#pragma unroll 1
            for (int p = 0; p < 8; ++p)
                if (b_used(h, p))
                    tc::tma_load_4d(X + buf * B_BYTES + p * PS, &tmS, 0, mod_n(h.cs.pmp[p], n),
                                    mod_n(h.cs.pm[p], n), h.cs.mir[p] ? n - c * KC - BJ : c * KC, &pb.data[buf]);
        };
        // this thread's raw values of chunk c from B buffer Xb: w[u] = sample bk0 + ((u + brot) & 3)
        auto read_raw = [&](const SlotHdr &h, int c, const unsigned char *Xb, double2 (&w)[4]) {
            const int kvalid = min(KC, n - c * KC);
            const bool mir = h.cs.mir[bp], used = b_used(h, bp);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = bk0 + ((u + brot) & 3);
                const int r = mir ? BJ - 1 - k : k;
                w[u] = used && k < kvalid ? *reinterpret_cast<const double2 *>(Xb + bp * PS + 16 * r)
                                          : make_double2(0.0, 0.0);
            }
        };
        uint32_t dph = 0;     // bit b: parity of pb.data[b]'s next completion
        int inflight = -1;    // B buffer whose copies are issued and not yet seen complete
        double2 wn[4];        // raw values of this step
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1, l0 = m;
            {
                const bool done = tc::mbar_wait(&slot_full[s], (k >> 1) & 1, kWaitPolls);
                ok = tc::group_and(kBarConv, kConv, done);
                if (!ok) break;
            }
            const SlotHdr &h = hdr[s];
            const int *alpha = slot_alpha(s);
            const int ntile = (B - l0 + TM - 1) / TM, npass = (ntile + 3) / 4;
            for (int pp = 0; pp < npass && ok; ++pp) {
                const int t0 = 4 * pp, nt = min(4, ntile - t0);
                for (int c = 0; c < nchunks && ok; ++c, ++bc) {
                    const int kvalid = min(KC, n - c * KC);
                    const int ksteps = (kvalid + 15) / 16;
                    const int kfill = ksteps * 16;
                    const int buf = bc & 1;
                    unsigned char *Xc = X + buf * B_BYTES;
                    for (int tt = 0; tt < nt && ok; ++tt) {
                        const int lb = l0 + TM * (t0 + tt), rows = min(TM, B - lb);
                        if (tt == 0) {
                            // the chunk's data operand, once for all the pass's tiles
                            if (inflight != buf) {  // the cluster's first chunk: copy now (the buffer's MMAs are done)
                                if (t == 0) issue_b(h, c, buf);
                                inflight = buf;
                            }
                            const bool done = tc::mbar_wait(&pb.data[buf], (dph >> buf) & 1, kWaitPolls);
                            if (done) {
                                dph ^= 1u << buf;
                                inflight = -1;
                            }
                            read_raw(h, c, Xc, wn);
                            ok = tc::group_and(kBarConv, kConv, done);  // every raw value read before any digit lands
                            if (!ok) break;
                            if (bk0 < kfill) {
                                double vr[4], vi[4];
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const int q = (k - brot) & 3;
                                    const double2 x = q == 0 ? wn[0] : q == 1 ? wn[1] : q == 2 ? wn[2] : wn[3];
                                    vr[k] = x.x;
                                    vi[k] = x.y;
                                }
                                const int ar = -h.colexp[2 * bp], ai = -h.colexp[2 * bp + 1];
                                const int alr[4] = {ar, ar, ar, ar}, ali[4] = {ai, ai, ai, ai};
                                put_digits4(Xc, 16 * kCols, B_LBO, 2 * bp, bk0, vr, alr);
                                put_digits4(Xc, 16 * kCols, B_LBO, 2 * bp + 1, bk0, vi, ali);
                            }
                        }
                        if (pending) {
                            ok = converter_wait_mma(pb, mph);
                            pending = false;
                            if (!ok) break;
                            if (prows > 0) epilogue();
                            if (plast) tc::mbar_arrive(&slot_empty[pslot]);  // the previous cluster is finished
                        }
                        // the previous chunk's MMAs (the other B buffer's) are done: the next chunk's
                        // copies (the next of this pass, else the first of the next pass)
                        if (tt == 0 && !(c == nchunks - 1 && pp + 1 >= npass)) {
                            if (t == 0) issue_b(h, c + 1 == nchunks ? 0 : c + 1, buf ^ 1);
                            inflight = buf ^ 1;
                        }
                        // A operand: staged rows G g + t / 32 and G g + t / 32 + 8, samples
                        // 4 (t % 32) .. + 3; the groups past the cluster's last degree are
                        // neither staged nor read
                        const int rr = t >> 5, k4 = 4 * (t & 31);
                        const int ngroups = (rows + G - 1) / G;
                        for (int g = 0; g < ngroups; ++g, ++gi) {
                            ok = converter_acquire(pb, gi);
                            if (!ok) break;
#pragma unroll
                            for (int hh = 0; hh < G; hh += 8) {
                                const int r = g * G + hh + rr;
                                if (r < rows && k4 < kfill) {
                                    const double2 *src = reinterpret_cast<const double2 *>(
                                        stage + (gi % kStages) * G * KC + (hh + rr) * KC + k4);
                                    const double2 w0 = src[0], w1 = src[1];
                                    const double v[4] = {w0.x, w0.y, w1.x, w1.y};
                                    const int a = alpha[lb + r - l0];
                                    const int al[4] = {a, a, a, a};
                                    put_digits4(A, A_PLANE, A_LBO, r, k4, v, al);
                                }
                            }
                            release_empty(pb, gi);
                        }
                        tc::fence_proxy_async();
                        ok = chunk_done(ok);
                        if (!ok) break;
                        if (t == 0) tc::mbar_arrive(&pb.ready);
                        pending = true;
                        plb = lb;
                        prows = c == nchunks - 1 ? rows : 0;
                        ptile = tt;
                        plast = c == nchunks - 1 && pp + 1 >= npass && tt + 1 >= nt;
                        pslot = s;
                        pl0 = l0;
                        pcidx = cidx;
                    }
                }
            }
        }
        if (pending) {
            // the last tile's MMAs (or, after a timeout, MMAs still in flight)
            const bool done = converter_wait_mma(pb, mph);
            if (ok && done && prows > 0) epilogue();
            ok = ok && done;
        }
        // after a timeout: copies still in flight land before the CTA leaves
        if (inflight >= 0) tc::mbar_wait(&pb.data[inflight], (dph >> inflight) & 1, kWaitPolls);
    } else if (tid == kIssuer) {
        // ---- issuer: the MMAs of every step, in the converters' order, into the
        // accumulator of the step's tile ----
        uint32_t rph = 0, bc = 0;
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int ntile = (B - m + TM - 1) / TM, npass = (ntile + 3) / 4;
            for (int pp = 0; pp < npass && ok; ++pp) {
                const int nt = min(4, ntile - 4 * pp);
                for (int c = 0; c < nchunks && ok; ++c, ++bc) {
                    const int ksteps = (min(KC, n - c * KC) + 15) / 16;
                    for (int tt = 0; tt < nt && ok; ++tt) {
                        ok = issuer_acquire(pb, rph);
                        if (!ok) break;
                        issue_levels<TM>(tmem + 128 * tt, A, A_PLANE, A_LBO, X + (bc & 1) * B_BYTES, B_LBO, c == 0,
                                         ksteps, &pb.mma);
                    }
                }
            }
        }
    }
    if (!ok && tb.err) atomicExch(tb.err, 2);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Inverse DWT, persistent as the forward: one CTA per SM walks the clusters
// inv_order[blockIdx.x + k gridDim.x].  M = the beta samples = the TMEM lanes,
// so the A operand (the Wigner-d digits) lives in tensor memory; the shared
// memory that the forward spends on digit planes holds staging rings instead.
// Two tiles of 128 beta samples are in flight (tile slot tau = 0, 1; samples
// jb0 + 128 tau + 0..127 of a pair of tiles), K chunks of 32 degrees:
//   producers  (warps 0-7; warp w takes tile slot w / 4, two warps per
//              scheduler) run the FP64 recurrence of one sample per thread and
//              stage 16 degrees (one MMA K step) per group in their tile's ring
//              slot [128][18] (16 used; the pad spreads the rows over the banks);
//   converters (warps 8-15; warp 8 + 4 tau + q takes tile slot tau and TMEM
//              lane quarter q) read their own lanes' staged values, cut them
//              into digits and store them with tcgen05.st, two degrees per
//              32-bit column; they run their tile's epilogue, and warps 12-15
//              build the B operand (shared by both tiles: one cluster);
//   issuer     (lane 0 of warp 16) and set-up warp (warp 17) as in the forward.
// TMEM: tile tau's accumulators in columns 128 tau + 0..111, its A buffer in
// columns kAcolInv + tau kAbufCols + 16 i + k / 2 (digit i, chunk-relative
// degree k).  Per step (one chunk of both tiles): converters wait for their
// tile's previous MMAs (mdone[tau]) and run a closed tile's epilogue; all
// converters meet (so the other tile's MMAs and the B buffers are done too)
// and signal `ready`; they write the next step's B operand and then this
// step's A digits (afull[tau]).  The issuer waits for ready and afull[0],
// issues tile 0's MMAs (committed to mdone[0]), then waits for afull[1] and
// issues tile 1's.  Both tiles of a pair share each chunk's B operand; a
// pair's second tile wholly past the last sample is skipped by every role, and
// the idle lanes of a partly filled tile run on zeros and are not stored.
// The set-up warp fills slot k & 1 with cluster k's partner table, recurrence
// coefficients, digit exponents, the factors V_l mu_t of its coefficients and
// the column scales of those products (the largest magnitude of each of the 16
// data columns over the degrees).  Every wait bounded.
//   dynamic smem: B operand [2] | rings [2][kRingInv][128][kRowInv] |
//                 slot [2] { rA, rAc, rG [B doubles], alpha [B ints] }
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t inv_slot_doubles(int B) { return 3 * (size_t)B + ((size_t)B + 1) / 2; }
constexpr int kKCInv = 32;                         // degrees per K chunk of the inverse
constexpr uint32_t kAbufCols = kDig * kKCInv / 2;  // 112 TMEM columns per A buffer
constexpr uint32_t kAcolInv = 256;                 // first TMEM column of the A buffers
constexpr uint32_t kTmemColsInv = 512;             // >= kAcolInv + 2 kAbufCols
constexpr int kRingInv = 3;                        // staging ring depth per tile (groups of 16 degrees)
constexpr int kRowInv = 18;                        // doubles per sample row of a ring slot (16 used)
constexpr int kProdInv = 256;                      // producer threads (warps 0-7)
constexpr int kConvInv = 256;                      // converter threads (warps 8-15)
constexpr int kIssuerInv = kProdInv + kConvInv;    // lane 0 of warp 16
constexpr int kSetupInv = kIssuerInv + 32;         // warp 17
constexpr int kThreadsInv = kSetupInv + 32;        // 576 threads

struct InvBars {
    uint64_t full[2][kRingInv], empty[2][kRingInv], afull[2], mdone[2], ready;
};

// One K chunk of MMAs with A in tensor memory (issued by one thread): for each
// K step of 16 degrees, A digit i (TMEM columns acol + 16 i + 8 s ..) against
// B digits 0..6-i into accumulator columns dcol + 16 i ..; completion
// committed to mbar.
__device__ __forceinline__ void issue_levels_ta(uint32_t tmem, uint32_t dcol, uint32_t acol, const unsigned char *Bop,
                                                uint32_t b_lbo, bool first, int ksteps, uint64_t *mbar) {
    tc::fence_after_sync();
    const uint64_t bd0 = tc::smem_desc(tc::smem_u32(Bop), b_lbo, 128);
    for (int s = 0; s < ksteps; ++s) {
        const uint64_t bd = bd0 + (uint64_t)((s * 2 * b_lbo) >> 4);
#pragma unroll
        for (int i = 0; i < kDig; ++i) {
            constexpr uint32_t kIdesc0 = tc::instr_desc(1, 128, kCols * kDig);
            const uint32_t idesc = kIdesc0 - ((uint32_t)(kCols * i) >> 3 << 17);  // N = 16 (7 - i)
            tc::mma_bf16_ta(tmem + dcol + kCols * i, tmem + acol + 16 * i + 8 * s, bd, idesc,
                            (first && s == 0 && i == 0) ? 0u : 1u);
        }
    }
    tc::mma_commit(mbar);
}

__global__ void __launch_bounds__(kThreadsInv, 1) dwt_inverse_tc_kernel(Tables tb, const double *__restrict__ coef,
                                                                        double2 *__restrict__ S, int flags) {
    constexpr int TM = 128, KC = kKCInv;
    constexpr int B_LBO = kNB * 16 + 16, B_BYTES = (KC / 8) * B_LBO;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SlotHdr hdr[2];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) InvBars ib;
    __shared__ __align__(8) uint64_t slot_full[2], slot_empty[2];
    const int B = tb.B, n = 2 * B, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = (n + 2 * TM - 1) / (2 * TM);  // pairs of sample tiles per cluster

    unsigned char *X = smem;  // [2][B_BYTES]
    double *ring = reinterpret_cast<double *>(X + 2 * B_BYTES);  // [2][kRingInv][TM][kRowInv]
    double *slotd = ring + 2 * kRingInv * TM * kRowInv;
    const size_t SLOT = inv_slot_doubles(B);
    auto slot_rA = [&](int s) { return slotd + s * SLOT; };
    auto slot_rAc = [&](int s) { return slotd + s * SLOT + B; };
    auto slot_rG = [&](int s) { return slotd + s * SLOT + 2 * B; };
    auto slot_alpha = [&](int s) { return reinterpret_cast<int *>(slotd + s * SLOT + 3 * B); };
    auto ring_row = [&](int tau, int r, int row) {
        return ring + (((size_t)tau * kRingInv + r) * TM + row) * kRowInv;
    };
    auto cluster_of = [&](int k, int &cidx, int &m, int &mp) {
        const int idx = blockIdx.x + k * gridDim.x;
        if (idx >= tb.ncl) return false;
        cidx = tb.inv_order ? tb.inv_order[idx] : idx;
        const int2 rep = tb.clusters[cidx];
        m = rep.x;
        mp = rep.y;
        return true;
    };

    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemColsInv);
    if (tid == 0) {
        for (int tau = 0; tau < 2; ++tau) {
            for (int r = 0; r < kRingInv; ++r) {
                tc::mbar_init(&ib.full[tau][r], 4);   // the tile's 4 producer warps
                tc::mbar_init(&ib.empty[tau][r], 4);  // the tile's 4 converter warps
            }
            tc::mbar_init(&ib.afull[tau], 4);
            tc::mbar_init(&ib.mdone[tau], 1);
        }
        tc::mbar_init(&ib.ready, 1);
        for (int s2 = 0; s2 < 2; ++s2) {
            tc::mbar_init(&slot_full[s2], 32);
            tc::mbar_init(&slot_empty[s2], kProdInv + kConvInv);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp == kSetupInv / 32) {
        // ---- set-up: the tables of cluster k into slot k & 1 ----
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1;
            if (k >= 2) {  // slot s last held cluster k - 2
                const bool done = tc::mbar_wait(&slot_empty[s], ((k >> 1) - 1) & 1, kWaitPolls);
                ok = __all_sync(0xffffffffu, done);
                if (!ok) break;
            }
            SlotHdr &h = hdr[s];
            if (lane == 0) fill_cluster(tb, m, mp, h.cs);
            const int l0 = m, L = B - m;
            const double *src = tb.rectab + (size_t)cidx * B * 3;
            double *rA = slot_rA(s), *rAc = slot_rAc(s), *rG = slot_rG(s);
            int *alpha = slot_alpha(s);
            for (int t = lane; t < L; t += 32) {
                rA[t] = src[3 * t];
                rAc[t] = src[3 * t + 1];
                const double sg = src[3 * t + 2];
                const int a = exponent_of(sg);
                alpha[t] = a;
                const double v = (flags & kApplyV) ? (2.0 * (l0 + t) + 1.0) / (8.0 * M_PI * B) : 1.0;
                rG[t] = v * ldexp_bits(sg, -a);  // V_l mu_t
            }
            __syncwarp();
            // column maxima of F[t][2p (+1)] = sign_p(l) V_l mu_t f(l, m_p, m'_p): lane
            // (p, quarter) takes partner p = lane & 7 at degrees t = quarter, quarter + 4, ...
            {
                const int p = lane & 7, np = h.cs.np;
                const bool real = (flags & kRealSym) && np > 1;
                unsigned long long m0 = 0, m1 = 0;
                if (p < np && !(real && (p & 1)))
                    for (int t = lane >> 3; t < L; t += 4) {
                        const double2 c = *reinterpret_cast<const double2 *>(coef + 2 * (h.cs.off[p] + t));
                        m0 = max(m0, abs_bits(rG[t] * c.x));
                        m1 = max(m1, abs_bits(rG[t] * c.y));
                    }
#pragma unroll
                for (int off = 8; off < 32; off <<= 1) {
                    m0 = max(m0, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)m0, off));
                    m1 = max(m1, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)m1, off));
                }
                if (lane < 8) {
                    h.colexp[2 * lane] = column_exponent(m0);
                    h.colexp[2 * lane + 1] = column_exponent(m1);
                }
            }
            tc::mbar_arrive(&slot_full[s]);
        }
    } else if (tid < kProdInv) {
        // ---- producers: sample jb0 + 128 tau + tp walks the degrees ----
        // Group counts and degree counts are warp-uniform (an idle lane's values
        // are zero because its recurrence starts from zero).
        const int tau = warp >> 2, tp = tid & 127;
        uint32_t gi = 0;
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1, L = B - m;
            ok = __all_sync(0xffffffffu, tc::mbar_wait(&slot_full[s], (k >> 1) & 1, kWaitPolls));
            if (!ok) break;
            const double *rA = slot_rA(s), *rAc = slot_rAc(s);
            const int nch = (L + KC - 1) / KC;  // K chunks of a tile
            for (int jp = 0; jp < npairs && ok; ++jp) {
                if (2 * TM * jp + TM * tau >= n) continue;  // the pair's second tile lies past the last sample
                const int j = 2 * TM * jp + TM * tau + tp;
                double x = 0.0, dc = 0.0, dp = 0.0;
                if (j < n) { x = tb.cosb[j]; dc = tb.seedtab[(size_t)cidx * n + j]; }
                for (int c = 0; c < nch && ok; ++c) {
                    const int cnt = min(KC, L - c * KC);
                    const int ng = (cnt + 15) / 16;  // groups of 16 degrees up to the padded K
                    for (int g = 0; g < ng; ++g, ++gi) {
                        const int r = gi % kRingInv;
                        ok = __all_sync(0xffffffffu,
                                        tc::mbar_wait(&ib.empty[tau][r], ((gi / kRingInv) & 1) ^ 1u, kWaitPolls));
                        if (!ok) break;
                        double2 *st = reinterpret_cast<double2 *>(ring_row(tau, r, tp));
#pragma unroll
                        for (int hh = 0; hh < 16; hh += 8) {  // halves of 8 degrees
                            double v[8];
                            const int nv = max(0, min(8, cnt - 16 * g - hh));  // degrees of this half
                            const int q0 = c * KC + 16 * g + hh;
                            if (nv == 8) {
                                // a whole half: straight-line code, no predicated FP64 work; the
                                // first FMA of a row runs two rows ahead of the dependent second
                                double ca[8], cb[8];
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    ca[u] = rA[q0 + u];
                                    cb[u] = rAc[q0 + u];
                                }
                                double u0 = fma(ca[0], x, -cb[0]), u1 = fma(ca[1], x, -cb[1]);
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    v[u] = dc;
                                    const double nx = fma(u0, dc, -dp);
                                    u0 = u1;
                                    if (u + 2 < 8) u1 = fma(ca[u + 2], x, -cb[u + 2]);
                                    dp = dc;
                                    dc = nx;
                                }
                            } else {  // the tile's last, partial half, or padding
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    v[u] = 0.0;
                                    if (u < nv) {
                                        v[u] = dc;
                                        const double nx = fma(fma(rA[q0 + u], x, -rAc[q0 + u]), dc, -dp);
                                        dp = dc;
                                        dc = nx;
                                    }
                                }
                            }
#pragma unroll
                            for (int h = 0; h < 4; ++h) st[hh / 2 + h] = make_double2(v[2 * h], v[2 * h + 1]);
                        }
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&ib.full[tau][r]);
                    }
                }
            }
            if (ok) tc::mbar_arrive(&slot_empty[s]);  // this producer is done with the slot's tables
        }
    } else if (tid < kIssuerInv) {
        // ---- converters: A digits into TMEM, the epilogue, the B operand ----
        const int t = tid - kProdInv;             // 0..255
        const int tau = (warp - 8) >> 2, wq = warp & 3;
        const int tl = wq * 32 + lane;            // this thread's TMEM lane = sample within the tile
        const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
        uint32_t mph = 0, cc = 0, gi = 0;
        bool pending = false;
        // the tile pair whose last MMAs are pending (pjb >= 0: its first sample) for the
        // deferred epilogue, its cluster's slot, and whether it is that cluster's last pair
        int pjb = -1, pslot = 0;
        bool plast = false;
        auto epilogue = [&]() {
            // Sample pjb + 128 tau + tl sits in TMEM lane tl of tile tau's accumulators.
            tc::fence_after_sync();
            const SlotHdr &h = hdr[pslot];
            const int np = h.cs.np;
            const bool real = (flags & kRealSym) && np > 1;
            const int jt = pjb + TM * tau + tl;
            double v16[kCols];
            epilogue_levels(tlane + 128 * tau, h.colexp, v16);
            if (jt < n) {
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    if (p >= np) break;
                    if (real && (p & 1)) continue;  // written from its pair below
                    const int jj = h.cs.mir[p] ? n - 1 - jt : jt;
                    double re = v16[2 * p], im = v16[2 * p + 1];
                    if (flags & kApplyW) {
                        const double wj = tb.w[jj];
                        re *= wj;
                        im *= wj;
                    }
                    S[((int64_t)jj * n + mod_n(h.cs.pm[p], n)) * n + mod_n(h.cs.pmp[p], n)] = make_double2(re, im);
                    if (real)  // partner p + 1 = (-m, -m'): the conjugate, at the same beta sample
                        S[((int64_t)jj * n + mod_n(h.cs.pm[p + 1], n)) * n + mod_n(h.cs.pmp[p + 1], n)] =
                            make_double2(re, -im);
                }
            }
            tc::fence_before_sync();
        };
        // B operand task of warps 12-15 (bt = 0..127): column q2 (partner bp = q2 / 2, re
        // or im), degrees bk0 .. + 3 of a chunk, written one step ahead of its MMAs
        const int bt = t - 128, q2 = bt & 15, bp = q2 >> 1, bk0 = 4 * ((bt & 127) >> 4);
        const bool btask = t >= 128;
        auto put_b = [&](const SlotHdr &h, const double *rG, int lb, int l0, unsigned char *Xb) {
            if (!btask) return;
            const int cnt = min(KC, B - lb), kfill = (cnt + 15) / 16 * 16;
            if (bk0 >= kfill) return;
            const bool used = bp < h.cs.np && !((flags & kRealSym) && h.cs.np > 1 && (bp & 1));
            // F = sign_p(l) V_l mu_t f(l, m_p, m'_p), formed here in FP64
            double v[4];
            int al[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                al[u] = -h.colexp[q2];
                const int kk = bk0 + u;
                v[u] = 0.0;
                if (used && kk < cnt) {
                    const int q = lb + kk - l0, l = lb + kk;
                    const bool neg = (h.cs.sign[bp] < 0.0) != (h.cs.lpar[bp] && (l & 1));
                    v[u] = (neg ? -rG[q] : rG[q]) * coef[2 * (h.cs.off[bp] + q) + (q2 & 1)];
                }
            }
            put_digits4(Xb, 16 * kCols, B_LBO, q2, bk0, v, al);
            tc::fence_proxy_async();
        };
        bool b_ready = false;  // the current step's B operand is written
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            const int s = k & 1, l0 = m;
            {
                const bool done = tc::mbar_wait(&slot_full[s], (k >> 1) & 1, kWaitPolls);
                ok = tc::group_and(kBarConv, kConvInv, done);
                if (!ok) break;
            }
            const SlotHdr &h = hdr[s];
            const double *rG = slot_rG(s);
            const int *ralpha = slot_alpha(s);
            for (int jp = 0; jp < npairs && ok; ++jp) {
                const bool live = 2 * TM * jp + TM * tau < n;  // else this tile slot idles for the pair
                for (int lb = l0, c = 0; lb < B && ok; lb += KC, ++c, ++cc) {
                    const int cnt = min(KC, B - lb);
                    const int ng = (cnt + 15) / 16;
                    bool wok = true;
                    if (pending) {  // this tile's previous MMAs; the epilogue if they closed a tile pair
                        wok = tc::mbar_wait(&ib.mdone[tau], mph, kWaitPolls);
                        mph ^= 1u;
                        pending = false;
                        if (wok && pjb >= 0) epilogue();
                    }
                    if (!b_ready) put_b(h, rG, lb, l0, X + (cc & 1) * B_BYTES);  // the cluster's first step
                    // both tiles' previous MMAs and epilogues and this step's B operand are done
                    ok = tc::group_and(kBarConv, kConvInv, ok && wok);
                    if (!ok) break;
                    if (t == 0) tc::mbar_arrive(&ib.ready);
                    // the next step's B operand (the other buffer, free now): the next degree
                    // chunk, else the first of the next tile pair
                    b_ready = lb + KC < B || jp + 1 < npairs;
                    if (b_ready) put_b(h, rG, lb + KC < B ? lb + KC : l0, l0, X + ((cc + 1) & 1) * B_BYTES);
                    // this tile's A digits (its buffer is free: its previous MMAs are done)
                    bool aok = true;
                    if (live) {
                        const uint32_t acol = tlane + kAcolInv + tau * kAbufCols;
                        for (int g = 0; g < ng && aok; ++g) {
                            const uint32_t gg = gi + g, r = gg % kRingInv;
                            aok = __all_sync(0xffffffffu, tc::mbar_wait(&ib.full[tau][r], (gg / kRingInv) & 1, kWaitPolls));
                            if (!aok) break;
                            const double2 *src = reinterpret_cast<const double2 *>(ring_row(tau, r, tl));
                            double v[16];
#pragma unroll
                            for (int h2 = 0; h2 < 8; ++h2) {
                                const double2 w2 = src[h2];
                                v[2 * h2] = w2.x;
                                v[2 * h2 + 1] = w2.y;
                            }
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(&ib.empty[tau][r]);
#pragma unroll
                            for (int hh = 0; hh < 16; hh += 8) {
                                uint32_t pk[kDig][4];
#pragma unroll
                                for (int c2 = 0; c2 < 4; ++c2) {
                                    const int q = lb - l0 + 16 * g + hh + 2 * c2;  // degree - l0
                                    uint32_t d0[kDig], d1[kDig];
                                    digits7(v[hh + 2 * c2], q < B - l0 ? ralpha[q] : 0, d0);
                                    digits7(v[hh + 2 * c2 + 1], q + 1 < B - l0 ? ralpha[q + 1] : 0, d1);
#pragma unroll
                                    for (int i = 0; i < kDig; ++i) pk[i][c2] = __byte_perm(d0[i], d1[i], 0x7632);
                                }
#pragma unroll
                                for (int i = 0; i < kDig; ++i)
                                    tc::tmem_st4(acol + 16 * i + 8 * g + hh / 2, pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
                            }
                        }
                        gi += ng;
                        tc::tmem_wait_st();
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&ib.afull[tau]);
                    }
                    ok = ok && aok;
                    pending = live;
                    pjb = lb + KC >= B ? 2 * TM * jp : -1;
                    // the cluster's last step: its slot is released after this step's epilogue
                    if (plast) tc::mbar_arrive(&slot_empty[pslot]);
                    plast = lb + KC >= B && jp + 1 >= npairs;
                    pslot = s;
                }
            }
        }
        if (pending) {
            const bool done = tc::mbar_wait(&ib.mdone[tau], mph, kWaitPolls);
            if (ok && done && pjb >= 0) epilogue();
            ok = ok && done;
        }
    } else if (tid == kIssuerInv) {
        // ---- issuer: per step, tile 0's MMAs once ready and its A digits are done, then tile 1's ----
        uint32_t rph = 0, cc = 0, aph = 0;  // aph bit tau: parity of afull[tau]'s next completion
        for (int k = 0; ok; ++k) {
            int cidx, m, mp;
            if (!cluster_of(k, cidx, m, mp)) break;
            for (int jp = 0; jp < npairs && ok; ++jp)
                for (int lb = m, c = 0; lb < B && ok; lb += KC, ++c, ++cc) {
                    ok = tc::mbar_wait(&ib.ready, rph, kWaitPolls);
                    rph ^= 1u;
                    const int ksteps = (min(KC, B - lb) + 15) / 16;
                    for (int tau = 0; tau < 2 && ok; ++tau) {
                        if (2 * TM * jp + TM * tau >= n) continue;  // an idle tile slot
                        ok = tc::mbar_wait(&ib.afull[tau], (aph >> tau) & 1, kWaitPolls);
                        aph ^= 1u << tau;
                        if (!ok) break;
                        issue_levels_ta(tmem, 128 * tau, kAcolInv + tau * kAbufCols, X + (cc & 1) * B_BYTES, B_LBO,
                                        c == 0, ksteps, &ib.mdone[tau]);
                    }
                }
        }
    }
    if (!ok && tb.err) atomicExch(tb.err, 2);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemColsInv);
}

// colexp[(m n + m') 2 + h] = the largest biased FP64 exponent of the real
// (h = 0) or imaginary (h = 1) part of S[j][m][m'] over j: one thread per
// (m, m'), loads coalesced across threads, one pass over S.
__global__ void __launch_bounds__(256) colexp_kernel(const double2 *__restrict__ S, int n, int *__restrict__ colexp) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
        int e0 = 0, e1 = 0;
#pragma unroll 8
        for (int j = 0; j < n; ++j) {
            const double2 v = S[j * nn + q];
            e0 = max(e0, (int)((abs_bits(v.x) >> 52) & 0x7FF));
            e1 = max(e1, (int)((abs_bits(v.y) >> 52) & 0x7FF));
        }
        colexp[2 * q] = e0;
        colexp[2 * q + 1] = e1;
    }
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

}  // namespace

cudaError_t launch_dwt_forward_tc(const Tables &tb, const double2 *S, double2 *coef, cudaStream_t s, int flags) {
    if (!tb.seedtab || !tb.rectab || !tb.colexp) return cudaErrorInvalidValue;
    {
        const int64_t nn = 4LL * tb.B * tb.B;
        colexp_kernel<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 152 * 16), 256, 0, s>>>(S, 2 * tb.B, tb.colexp);
        count_launch();
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    constexpr int KC = kProd, A_PLANE = (KC / 8) * (64 * 16 + 16), B_BYTES = (KC / 8) * (kNB * 16 + 16);
    const int B = tb.B;
    const uint64_t n = 2 * (uint64_t)B;
    // S as a 4-D FP64 tensor (re/im, m', m, j), boxes of (2, 1, 1, min(128, 2B)): one
    // partner column over a chunk of beta samples per copy (rows of 16 bytes)
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    if (reinterpret_cast<uintptr_t>(S) % 16 != 0) return cudaErrorMisalignedAddress;
    CUtensorMap tmS;
    const cuuint64_t dims[4] = {2, n, n, n};
    const cuuint64_t strides[3] = {16, 16 * n, 16 * n * n};
    const cuuint32_t box[4] = {2, 1, 1, (cuuint32_t)std::min<uint64_t>(KC, n)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (encode(&tmS, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<double2 *>(S), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t bytes = (size_t)kDig * A_PLANE + 2 * (size_t)B_BYTES +
                         sizeof(double) * (kStages * kGroup * (size_t)KC + 2 * fwd_slot_doubles(B));
    cudaError_t e =
        cudaFuncSetAttribute(dwt_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // persistent: one CTA per SM (the shared memory allows no second one)
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(tb.ncl, sms));
    dwt_forward_tc_kernel<<<grid, kThreadsFwd, bytes, s>>>(tb, tmS, reinterpret_cast<double *>(coef), flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dwt_inverse_tc(const Tables &tb, const double2 *coef, double2 *S, cudaStream_t s, int flags) {
    if (!tb.seedtab || !tb.rectab) return cudaErrorInvalidValue;
    constexpr int B_BYTES = (kKCInv / 8) * (kNB * 16 + 16);
    const int B = tb.B;
    const size_t bytes =
        2 * (size_t)B_BYTES + sizeof(double) * (2 * (size_t)kRingInv * 128 * kRowInv + 2 * inv_slot_doubles(B));
    cudaError_t e =
        cudaFuncSetAttribute(dwt_inverse_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;  // persistent: one CTA per SM (its 512 TMEM columns)
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(tb.ncl, sms));
    dwt_inverse_tc_kernel<<<grid, kThreadsInv, bytes, s>>>(tb, reinterpret_cast<const double *>(coef), S, flags);
    count_launch();
    return cudaGetLastError();
}

}  // namespace softgb
