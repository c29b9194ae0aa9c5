// dwt_mixed.cu -- mixed-precision DWT / iDWT on the tcgen05 tensor cores.
//
// Same mathematics as dwt_fp64.cu (Sec. 2.4: f = V_B T_B W_B S per order
// pair, S = T_B^T f), with the contraction moved to the tensor cores:
//   * the Wigner-d block T is generated on the fly by the FP64 three-term
//     recurrence of Eq. (Wigner_d_recurrence) from log-domain seeds, one
//     column block per symmetry cluster (Sec. 3), exactly as in the FP64 path;
//   * each FP64 entry is narrowed with integer bit operations (the FP64 pipe
//     stays free for the recurrence) and stored in shared memory as the
//     tensor-core A operand, either split into BF16 hi + lo (mode BF16X3:
//     three MMAs hi*hi + hi*lo + lo*hi per K step, ~2^-16 relative products)
//     or as TF32 (one MMA per K step, ~2^-11);
//   * the cluster's partners (8 x re/im = the N = 16 columns) are the B operand;
//   * tcgen05.mma accumulates each K chunk in FP32 in TMEM (M = 64 or 128
//     rows, N = 16 per transform); the chunk partials are combined across
//     chunks by compensated (TwoSum) FP32 sums kept in TMEM; the forward's
//     epilogue adds hi + lo and applies V_l and the partner signs in FP64, the
//     inverse's rounds hi + lo once to its FP32 S.
// Forward: M = degrees l (tiles of 128), K = beta samples (chunks of 128);
// the recurrence state of every beta sample is carried across degree tiles in
// shared memory.  Inverse: M = beta samples (tiles of 128), K = degrees
// (chunks of 128); each thread owns one beta sample and walks l.
// The quadrature weight w_B(j) is folded into the forward's seeds (the
// recurrence is linear in d), so the forward reads S unscaled.
//
// S here is the mixed plan's FP32 workspace in layout [m mod 2B][m' mod 2B][j]
// (beta fastest), written and read by cuFFT C2C with strided layouts, so that
// the per-partner loads and stores of 128 beta samples are contiguous.
#include "soft.h"
#include "soft_internal.cuh"
#include "tcgen05.cuh"

#include <algorithm>

namespace softgb {
namespace {

// Inverse: M = 128 beta samples (one warpgroup = the 128 TMEM lanes), K chunks of
// 64 degrees.  Forward: M = 64 degrees (tcgen05 M = 64 puts row 16w + i in TMEM
// lane 32w + i), K chunks of NT beta samples, one per thread.  Both keep the A
// operand at 256 bytes per recurrence chain so that more chains fit per SM.
constexpr int kNT = 128;       // inverse: threads per CTA
constexpr int kTile = 128;     // inverse: M rows per tile
constexpr int kChunk = 64;     // inverse: K degrees staged per round
constexpr int kFwdTile = 64;   // forward: M rows (degrees) per tile
constexpr int kNCols = 16;     // N: 8 partners x (re, im)
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ int mod_n(int a, int n) { return a < 0 ? a + n : a; }

// Shared operand buffers for one K chunk of an M x KC tile with NC = 16 NB
// columns (8 partners x (re, im) for each of NB transforms).
template <int MODE, int M = kTile, int KC = kChunk, int NC = kNCols>
struct Operands {
    static constexpr int EB = MODE == SOFT_MIXED_TF32 ? 4 : 2;        // bytes per element
    static constexpr int KPC = 16 / EB;                              // K elements per 16 bytes
    // A: K-direction stride between core matrices, padded by 16 bytes so that the
    // 8-column groups written by one warp fall in different shared-memory banks.
    static constexpr int A_LBO = M * 16 + 16;
    static constexpr int A_BYTES = (KC / KPC) * A_LBO;                // one A plane
    static constexpr int B_LBO = NC * 16 + 16;                       // same padding for B
    static constexpr int B_BYTES = (KC / KPC) * B_LBO;               // one B plane
    static constexpr int PLANES = MODE == SOFT_MIXED_TF32 ? 1 : 2;   // (hi, lo) for BF16X3
    static constexpr int BYTES = PLANES * (A_BYTES + B_BYTES);
};

// TMEM columns for an N-column FP32 accumulator (power of two, >= 32).
template <int NC>
constexpr uint32_t tmem_cols() {
    static_assert(NC <= 512, "TMEM holds 512 columns");
    return NC <= 32 ? 32u : NC <= 64 ? 64u : NC <= 128 ? 128u : NC <= 256 ? 256u : 512u;
}

// Store one value into plane(s) of an operand tile at (r, k).
template <int MODE>
__device__ __forceinline__ void put(unsigned char *plane0, int plane_bytes, int rows, int r, int k, float v) {
    if (MODE == SOFT_MIXED_TF32) {
        *reinterpret_cast<float *>(plane0 + tc::kmajor_offset(r, k, rows, 4)) = tc::round_tf32(v);
    } else {
        uint16_t hi, lo;
        tc::split_bf16(v, hi, lo);
        const uint32_t o = tc::kmajor_offset(r, k, rows, 2);
        *reinterpret_cast<uint16_t *>(plane0 + o) = hi;
        *reinterpret_cast<uint16_t *>(plane0 + plane_bytes + o) = lo;
    }
}

// Store 16 bytes of consecutive K elements (8 BF16 or 4 TF32) of row r,
// starting at k0 (a multiple of the per-16-byte count), into the A plane(s).
template <int MODE>
__device__ __forceinline__ void put_vec(unsigned char *plane0, int plane_bytes, int lbo, int r, int k0,
                                        const float (&v)[16 / Operands<MODE>::EB]) {
    const uint32_t o = (uint32_t)((k0 / Operands<MODE>::KPC) * lbo + (r / 8) * 128 + (r % 8) * 16);
    if (MODE == SOFT_MIXED_TF32) {
        uint4 w;
        w.x = __float_as_uint(tc::round_tf32(v[0]));
        w.y = __float_as_uint(tc::round_tf32(v[1]));
        w.z = __float_as_uint(tc::round_tf32(v[2]));
        w.w = __float_as_uint(tc::round_tf32(v[3]));
        *reinterpret_cast<uint4 *>(plane0 + o) = w;
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint16_t h0, l0, h1, l1;
            tc::split_bf16(v[2 * u], h0, l0);
            tc::split_bf16(v[2 * u + 1], h1, l1);
            h[u] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            l[u] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        }
        *reinterpret_cast<uint4 *>(plane0 + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(plane0 + plane_bytes + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Store 8 consecutive K elements (k0 a multiple of 8) of B-operand row r.
template <int MODE>
__device__ __forceinline__ void put_b8(unsigned char *plane0, int plane_bytes, int lbo, int r, int k0,
                                       const float (&v)[8]) {
    if constexpr (MODE == SOFT_MIXED_TF32) {
        const float a[4] = {v[0], v[1], v[2], v[3]}, b[4] = {v[4], v[5], v[6], v[7]};
        put_vec<MODE>(plane0, plane_bytes, lbo, r, k0, a);
        put_vec<MODE>(plane0, plane_bytes, lbo, r, k0 + 4, b);
    } else {
        put_vec<MODE>(plane0, plane_bytes, lbo, r, k0, v);
    }
}

// K elements per MMA (32 bytes of K).
template <int MODE>
constexpr int kstep_elems() { return 32 / Operands<MODE>::EB; }

// Issue the MMAs of one K chunk (thread 0 only) and commit them to mbar.
template <int MODE, int M, int KC, int NC>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, const unsigned char *A, const unsigned char *Bop,
                                            bool first, int ksteps, uint64_t *mbar) {
    using O = Operands<MODE, M, KC, NC>;
    tc::fence_after_sync();
    const uint32_t abase = tc::smem_u32(A), bbase = tc::smem_u32(Bop);
    constexpr uint32_t LBO_A = O::A_LBO, LBO_B = O::B_LBO, SBO = 128;
    if (MODE == SOFT_MIXED_TF32) {
        constexpr uint32_t idesc = tc::instr_desc(2, M, NC);
        for (int s = 0; s < ksteps; ++s) {
            const uint64_t ad = tc::smem_desc(abase + s * 2 * LBO_A, LBO_A, SBO);
            const uint64_t bd = tc::smem_desc(bbase + s * 2 * LBO_B, LBO_B, SBO);
            tc::mma_tf32(tmem, ad, bd, idesc, (first && s == 0) ? 0u : 1u);
        }
    } else {
        constexpr uint32_t idesc = tc::instr_desc(1, M, NC);
        const uint32_t alo = abase + O::A_BYTES, blo = bbase + O::B_BYTES;
        for (int s = 0; s < ksteps; ++s) {
            const uint32_t ao = s * 2 * LBO_A, bo = s * 2 * LBO_B;
            tc::mma_bf16(tmem, tc::smem_desc(abase + ao, LBO_A, SBO), tc::smem_desc(bbase + bo, LBO_B, SBO), idesc,
                         (first && s == 0) ? 0u : 1u);
            tc::mma_bf16(tmem, tc::smem_desc(abase + ao, LBO_A, SBO), tc::smem_desc(blo + bo, LBO_B, SBO), idesc, 1u);
            tc::mma_bf16(tmem, tc::smem_desc(alo + ao, LBO_A, SBO), tc::smem_desc(bbase + bo, LBO_B, SBO), idesc, 1u);
        }
    }
    tc::mma_commit(mbar);
}

// Seed for the mixed modes: the FP64 log-seed y = log2(seed) is split into
// k = floor(y) and f = y - k; 2^f comes from the FP32 special-function unit
// and k goes straight into the FP64 exponent field.  Relative error ~3e-7 --
// far below the ~1e-5 of the split-BF16 products -- at ~7 FP64 operations
// instead of a full FP64 exp, with the FP64 exponent range kept (values
// below ~1e-308 flush to 0, as in the FP64 path).
__device__ __forceinline__ double seed_rep_mixed(int m, int mp, double lognorm, double lc, double ls) {
    double lg = lognorm;
    if (m + mp > 0) lg = fma((double)(m + mp), lc, lg);
    if (m - mp > 0) lg = fma((double)(m - mp), ls, lg);
    const double y = lg * 1.4426950408889634074;  // log2(e)
    const double kf = floor(y);
    const int k = (int)kf;
    const float p = exp2f((float)(y - kf));       // [1, 2]
    const unsigned long long b = (unsigned long long)__double_as_longlong(tc::f32_to_f64(p));
    const int e = (int)((b >> 52) & 0x7FF) + k;   // biased exponent of the product
    if (e <= 0) return 0.0;
    return __longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((unsigned long long)e << 52)));
}

// The transforms of one launch: same bandwidth (shared tables), own data.
struct MixedBatch {
    Tables tb;
    const float2 *S[kMaxMixedBatch];  // FP32 S workspaces, layout [m][m'][j]
    double *coef[kMaxMixedBatch];     // interleaved complex coefficients
};

// ---------------------------------------------------------------------------
// Compensated sums over K chunks (FP32 partials, error-free TwoSum
// accumulation), in TMEM beside the accumulator.  For a CTA with NC = 16 NB
// accumulator columns the TMEM layout is
//   [0, NC)       the accumulator of the current K chunk (FP32, fresh each chunk)
//   [NC, 2 NC)    running sum hi,   [2 NC, 3 NC) running sum lo
// so hi + lo holds the sum over the finished chunks of the FP32 chunk partials
// to ~2^-48 of their magnitude.  drain_chunk() is called by warps 0..3 (each
// reads its own TMEM lane quarter) after the chunk's MMA has completed.
// Batches of NB >= 4 transforms drain once per group of kDrainGroup chunks
// (the group accumulating in FP32, 512 beta samples or 256 degrees), since a
// drain costs NB times a single transform's and the sums' 2 x 16 NB TMEM
// columns would halve the CTAs per SM; a tile of one group keeps its FP32
// accumulator and needs no sums (and no TMEM for them).
template <int NB>
constexpr int drain_group() { return NB >= 4 ? 4 : 1; }
// ---------------------------------------------------------------------------
template <int NB>
__device__ __forceinline__ void drain_chunk(uint32_t tmem_row, bool first) {
    constexpr int NC = 16 * NB;
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        uint32_t x[16], hi[16], lo[16];
        tc::tmem_ld16(tmem_row + 16 * b, x);
        if (first) {
#pragma unroll
            for (int c = 0; c < 16; ++c) { hi[c] = x[c]; lo[c] = 0u; }
        } else {
            tc::tmem_ld16(tmem_row + NC + 16 * b, hi);
            tc::tmem_ld16(tmem_row + 2 * NC + 16 * b, lo);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float h = __uint_as_float(hi[c]), l = __uint_as_float(lo[c]);
                tc::comp_add(h, l, __uint_as_float(x[c]));
                hi[c] = __float_as_uint(h);
                lo[c] = __float_as_uint(l);
            }
        }
        tc::tmem_st16(tmem_row + NC + 16 * b, hi);
        tc::tmem_st16(tmem_row + 2 * NC + 16 * b, lo);
    }
}

// ---------------------------------------------------------------------------
// Forward DWT (mixed).  One CTA per cluster, KC producer threads = KC beta
// samples per K chunk (one recurrence chain per thread), M tiles of 64
// degrees, N = 16 NB columns: the T tile produced once serves the NB
// transforms of the batch.  Each chunk's MMA starts a fresh FP32
// accumulator; once it completes, its partial is added into the compensated
// TMEM sums (drain_chunk) before the operands are refilled, and after a
// tile's last chunk the epilogue applies V_l and the partner signs in FP64.
// (A second operand stage, to overlap the next chunk's recurrence with the
// MMA, halves the CTAs per SM and measured slower.)
//   dynamic smem: operands (A planes, then B planes) | dprev[2B] | dcur[2B] |
//                 rA,rAc,rV [B each]; the table-building scratch (Bc, sig)
//   lives in the operand area, not yet in use then.
// ---------------------------------------------------------------------------
template <int MODE, int KC, int NB, bool LD>
__global__ void __launch_bounds__(LD ? 2 * KC : KC, 1) dwt_forward_mixed_kernel(MixedBatch mb, int flags) {
    // KC producer threads (one beta sample each per chunk); with LD, a second
    // group of KC threads loads the B operand while the producers run the recurrence.
    constexpr int NT = LD ? 2 * KC : KC;
    constexpr int TM = kFwdTile, NC = 16 * NB;
    using O = Operands<MODE, TM, KC, NC>;
    constexpr int G = drain_group<NB>();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ ClusterSmem cs;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    const Tables &tb = mb.tb;
    const int B = tb.B, n = 2 * B, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool comp = (n + KC - 1) / KC > G;  // more than one drain group per tile: compensated sums in TMEM
    const uint32_t tcols = comp ? tmem_cols<3 * NC>() : tmem_cols<NC>();
    const int cidx = tb.fwd_order ? tb.fwd_order[blockIdx.x] : (int)blockIdx.x;
    const int2 rep = tb.clusters[cidx];
    const int m = rep.x, mp = rep.y, l0 = m, L = B - l0;

    double *dprev = reinterpret_cast<double *>(smem + O::BYTES);
    double *dcur = dprev + n;
    double *rA = dcur + n, *rAc = rA + B, *rV = rAc + B;
    double *rBc = reinterpret_cast<double *>(smem), *rSig = rBc + B;  // scratch inside the operand area

    load_cluster(tb, m, mp, cs);
    for (int t = tid; t < L; t += NT) rV[t] = (flags & kApplyV) ? (2.0 * (l0 + t) + 1.0) / (8.0 * M_PI * B) : 1.0;
    cluster_recurrence<NT>(tb, cidx, l0, L, m, mp, rA, rAc, rBc, rSig, rV);
    {
        const double lognorm = seed_lognorm(tb, m, mp);
        for (int j = tid; j < n; j += NT) {
            // w_B(j) d(l0,m,m';beta_j): from the plan's seed table, or exp2f of the log-seed
            if (tb.seedtab) {
                const double sd = tb.seedtab[(size_t)cidx * n + j];
                dcur[j] = (flags & kApplyW) ? sd * tb.w[j] : sd;
            } else {
                dcur[j] = seed_rep_mixed(m, mp, (flags & kApplyW) ? lognorm + tb.lw[j] : lognorm, tb.lcos[j],
                                         tb.lsin[j]);
            }
            dprev[j] = 0.0;
        }
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, tcols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's TMEM lane quarter
    const int np = cs.np;
    const int nchunks = (n + KC - 1) / KC;
    const int total = ((L + TM - 1) / TM) * nchunks;  // (tile, chunk) steps
    uint32_t phase = 0;
    bool ok = true;

    // Step `it` waits for chunk it-1's MMA, folds its partial into the sums
    // (and finishes that tile if it was its last chunk), then refills the
    // operands with chunk it and issues its MMA.
    for (int it = 0; it <= total; ++it) {
        const bool issue = it < total;
        const int tile = it / nchunks, c = it % nchunks;
        const int lb = l0 + tile * TM, rows = issue ? min(TM, B - lb) : 0;
        unsigned char *A = smem;
        unsigned char *X = A + O::PLANES * O::A_BYTES;
        const int kvalid = min(KC, n - c * KC);
        const int ksteps = (kvalid + kstep_elems<MODE>() - 1) / kstep_elems<MODE>();
        const int kfill = ksteps * kstep_elems<MODE>();
        if (it > 0) {
            // chunk it-1's MMA: wait for it, then fold its partial into the sums
            const bool done = tc::mbar_wait(&mbar, phase, kWaitPolls);
            phase ^= 1u;
            ok = __syncthreads_and(done);  // CTA-wide verdict keeps every barrier uniform
            if (!ok) break;
            tc::fence_after_sync();
            const int pt = (it - 1) / nchunks, pc = (it - 1) % nchunks;
            if (warp < 4) {
                if (comp && (pc % G == G - 1 || pc == nchunks - 1)) drain_chunk<NB>(trow, pc < G);
                if (pc == nchunks - 1) {
                    // Epilogue of tile pt: degree l = plb + 16 w + i sits in TMEM lane 32 w + i
                    // (i < 16); (hi + lo) V_l sig_l and the partner sign in FP64 (lo = 0 and hi
                    // the accumulator itself when the tile is one drain group).
                    const int plb = l0 + pt * TM, prow = min(TM, B - plb);
                    const int r = 16 * warp + lane;
                    const int l = plb + r, q = l - l0;
                    const bool live = lane < 16 && r < prow;
#pragma unroll 1
                    for (int b = 0; b < NB; ++b) {
                        uint32_t hi[16], lo[16];
                        if (comp) {
                            tc::tmem_ld16(trow + NC + 16 * b, hi);
                            tc::tmem_ld16(trow + 2 * NC + 16 * b, lo);
                        } else {
                            tc::tmem_ld16(trow + 16 * b, hi);
#pragma unroll
                            for (int c2 = 0; c2 < 16; ++c2) lo[c2] = 0u;
                        }
                        if (live) {
                            const double v = rV[q];
#pragma unroll
                            for (int p = 0; p < 8; ++p) {
                                if (p >= np) break;
                                const double vs = ((cs.sign[p] < 0.0) != (cs.lpar[p] && (l & 1))) ? -v : v;
                                double2 out;
                                out.x = vs * (tc::f32_to_f64(__uint_as_float(hi[2 * p])) +
                                              tc::f32_to_f64(__uint_as_float(lo[2 * p])));
                                out.y = vs * (tc::f32_to_f64(__uint_as_float(hi[2 * p + 1])) +
                                              tc::f32_to_f64(__uint_as_float(lo[2 * p + 1])));
                                *reinterpret_cast<double2 *>(mb.coef[b] + 2 * (cs.off[p] + q)) = out;
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
        }
        if (issue) {
            // A: column tid = beta sample j, rows = degrees lb..lb+rows-1.  Rows past
            // `rows` are left as they are: they only reach TMEM lanes that are never read.
            unsigned char *acol = A + (tid / O::KPC) * O::A_LBO + (tid % O::KPC) * O::EB;
            const int j = c * KC + tid;
            if (tid >= KC) {
                // loader threads: no column of A
            } else if (tid < kvalid) {
                const double x = tb.cosb[j];
                double dc = dcur[j], dp = dprev[j];
                for (int r = 0; r < rows; ++r) {
                    const float v = tc::f64_to_f32_trunc(dc);
                    if (MODE == SOFT_MIXED_TF32) {
                        *reinterpret_cast<float *>(acol + 16 * r) = tc::round_tf32(v);
                    } else {
                        uint16_t hi, lo;
                        tc::split_bf16(v, hi, lo);
                        *reinterpret_cast<uint16_t *>(acol + 16 * r) = hi;
                        *reinterpret_cast<uint16_t *>(acol + O::A_BYTES + 16 * r) = lo;
                    }
                    const int q = lb + r - l0;
                    const double nx = fma(fma(rA[q], x, -rAc[q]), dc, -dp);
                    dp = dc;
                    dc = nx;
                }
                dcur[j] = dc;
                dprev[j] = dp;
            } else if (tid < kfill) {
                for (int r = 0; r < TM; ++r) {
                    if (MODE == SOFT_MIXED_TF32) {
                        *reinterpret_cast<float *>(acol + 16 * r) = 0.f;
                    } else {
                        *reinterpret_cast<uint16_t *>(acol + 16 * r) = 0;
                        *reinterpret_cast<uint16_t *>(acol + O::A_BYTES + 16 * r) = 0;
                    }
                }
            }
            // B: X chunk, row 16 b + 2p (+1) = re (im) of partner p of transform b, k = beta sample;
            // each thread moves 8 consecutive samples (two 16-byte loads per 4, one 16-byte store per row).
            for (int e = LD ? tid - KC : tid; e >= 0 && e < 8 * NB * (KC / 8); e += LD ? KC : NT) {
                const int bp = e / (KC / 8), k0 = 8 * (e % (KC / 8));
                const int b = bp >> 3, p = bp & 7;
                if (k0 >= kfill) continue;
                float re[8], im[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) { re[u] = 0.f; im[u] = 0.f; }
                if (p < np) {
                    const float2 *run = mb.S[b] + ((int64_t)mod_n(cs.pm[p], n) * n + mod_n(cs.pmp[p], n)) * n;
                    const int j0 = c * KC + k0;
                    if (k0 + 8 <= kvalid) {
                        // samples j0..j0+7, or n-8-j0..n-1-j0 read in reverse for mirrored partners
                        const float4 *q = reinterpret_cast<const float4 *>(run + (cs.mir[p] ? n - 8 - j0 : j0));
                        float2 w[8];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float4 t = q[h];
                            w[2 * h] = make_float2(t.x, t.y);
                            w[2 * h + 1] = make_float2(t.z, t.w);
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float2 t = cs.mir[p] ? w[7 - u] : w[u];
                            re[u] = t.x;
                            im[u] = t.y;
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (k0 + u < kvalid) {
                                const int jj = j0 + u;
                                const float2 t = run[cs.mir[p] ? n - 1 - jj : jj];
                                re[u] = t.x;
                                im[u] = t.y;
                            }
                    }
                }
                put_b8<MODE>(X, O::B_BYTES, O::B_LBO, 16 * b + 2 * p, k0, re);
                put_b8<MODE>(X, O::B_BYTES, O::B_LBO, 16 * b + 2 * p + 1, k0, im);
            }
            tc::fence_proxy_async();
        }
        __syncthreads();  // operands of chunk it complete; the accumulator is free for it
        if (issue && tid == 0) {
            tc::fence_after_sync();
            issue_chunk<MODE, TM, KC, NC>(tmem, A, X, c % G == 0, ksteps, &mbar);  // a group starts fresh
        }
    }
    if (!ok && tid == 0 && tb.err) atomicExch(tb.err, 2);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tcols);
}

// ---------------------------------------------------------------------------
// Inverse DWT (mixed).  One CTA per cluster, looping over tiles of 128 beta
// samples; K = degrees in chunks of 64; N = 16 NB columns (the sign-folded
// coefficients of the NB transforms), so each generated T tile serves the batch.
// Each chunk's MMA starts a fresh FP32 accumulator, and its partial is folded
// into the compensated TMEM sums (drain_chunk) before the next chunk: the sum
// over l is FP32 within a chunk of 64 degrees and compensated across chunks.
//   dynamic smem: operands | rA,rAc,rBc,rSig [B each]
// ---------------------------------------------------------------------------
template <int MODE, int NB, bool LD>
__global__ void __launch_bounds__(LD ? 2 * kNT : kNT, 1) dwt_inverse_mixed_kernel(MixedBatch mb, int flags) {
    // kNT producer threads (one beta sample each); with LD, kNT more threads load the B operand.
    constexpr int NT = LD ? 2 * kNT : kNT;
    constexpr int NC = 16 * NB;
    using O = Operands<MODE, kTile, kChunk, NC>;
    constexpr int G = drain_group<NB>();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ ClusterSmem cs;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    const Tables &tb = mb.tb;
    const int B = tb.B, n = 2 * B, tid = threadIdx.x, warp = tid >> 5;
    const int cidx = tb.inv_order ? tb.inv_order[blockIdx.x] : (int)blockIdx.x;
    const int2 rep = tb.clusters[cidx];
    const int m = rep.x, mp = rep.y, l0 = m, L = B - l0;
    const bool comp = (L + kChunk - 1) / kChunk > G;  // more than one drain group: compensated sums in TMEM
    const uint32_t tcols = comp ? tmem_cols<3 * NC>() : tmem_cols<NC>();

    unsigned char *A = smem;
    unsigned char *F = smem + O::PLANES * O::A_BYTES;
    double *rA = reinterpret_cast<double *>(smem + O::BYTES), *rAc = rA + B, *rBc = rAc + B, *rSig = rBc + B;
    float *fsc = reinterpret_cast<float *>(rSig + B);  // [B] sig_l (V_l) in FP32, the B operand's scale

    load_cluster(tb, m, mp, cs);
    cluster_recurrence<NT>(tb, cidx, l0, L, m, mp, rA, rAc, rBc, rSig, nullptr);
    for (int t = tid; t < L; t += NT)
        fsc[t] = tc::f64_to_f32_rn(rSig[t] * ((flags & kApplyV) ? (2.0 * (l0 + t) + 1.0) / (8.0 * M_PI * B) : 1.0));
    if (warp == 0) tc::tmem_alloc(&tmem_slot, tcols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's TMEM lane quarter
    const int np = cs.np;
    const double lognorm = seed_lognorm(tb, m, mp);
    uint32_t phase = 0;
    bool ok = true;

    for (int jb = 0; jb < n && ok; jb += kTile) {
        const int j = jb + tid;
        const bool active = tid < kNT && j < n;
        double x = 0.0, dc = 0.0, dp = 0.0;
        if (active) {
            x = tb.cosb[j];
            dc = tb.seedtab ? tb.seedtab[(size_t)cidx * n + j] : seed_rep_mixed(m, mp, lognorm, tb.lcos[j], tb.lsin[j]);
        }
        for (int lb = l0, c = 0; lb < B && ok; lb += kChunk, ++c) {
            const int cnt = min(kChunk, B - lb);
            const int ksteps = (cnt + kstep_elems<MODE>() - 1) / kstep_elems<MODE>();
            const int kfill = ksteps * kstep_elems<MODE>();
            // A: row tid = beta sample j, K = degrees lb..lb+cnt-1 (zero up to kfill);
            // 16-byte vector stores.  Rows of inactive samples are never read back.
            constexpr int VEC = 16 / O::EB;
            if (active) {
                for (int k0 = 0; k0 < kfill; k0 += VEC) {
                    float v[VEC];
#pragma unroll
                    for (int u = 0; u < VEC; ++u) {
                        v[u] = 0.f;
                        if (k0 + u < cnt) {
                            v[u] = tc::f64_to_f32_trunc(dc);
                            const int q = lb + k0 + u - l0;
                            const double nx = fma(fma(rA[q], x, -rAc[q]), dc, -dp);
                            dp = dc;
                            dc = nx;
                        }
                    }
                    put_vec<MODE>(A, O::A_BYTES, O::A_LBO, tid, k0, v);
                }
            }
            // B: F chunk, row 16 b + 2p (+1) = sign- and sig-folded re (im) of partner p of
            // transform b at degrees lb + k0 .. lb + k0 + 7 (8 per thread, 16-byte stores).
            for (int e = LD ? tid - kNT : tid; e >= 0 && e < 8 * NB * (kChunk / 8); e += LD ? kNT : NT) {
                const int bp = e / (kChunk / 8), k0 = 8 * (e % (kChunk / 8));
                const int b = bp >> 3, p = bp & 7;
                if (k0 >= kfill) continue;
                float re[8], im[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) { re[u] = 0.f; im[u] = 0.f; }
                if (p < np) {
                    const double2 *run = reinterpret_cast<const double2 *>(mb.coef[b]) + cs.off[p] + (lb - l0);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = k0 + u;
                        if (k < cnt) {
                            const int l = lb + k;
                            const double2 cv = run[k];
                            const bool neg = (cs.sign[p] < 0.0) != (cs.lpar[p] && (l & 1));
                            const float v = neg ? -fsc[l - l0] : fsc[l - l0];  // FP32 scale: no FP64 work here
                            re[u] = v * tc::f64_to_f32_rn(cv.x);
                            im[u] = v * tc::f64_to_f32_rn(cv.y);
                        }
                    }
                }
                put_b8<MODE>(F, O::B_BYTES, O::B_LBO, 16 * b + 2 * p, k0, re);
                put_b8<MODE>(F, O::B_BYTES, O::B_LBO, 16 * b + 2 * p + 1, k0, im);
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0) issue_chunk<MODE, kTile, kChunk, NC>(tmem, A, F, c % G == 0, ksteps, &mbar);
            const bool done = tc::mbar_wait(&mbar, phase, kWaitPolls);
            phase ^= 1u;
            ok = __syncthreads_and(done);  // CTA-wide verdict keeps every barrier uniform
            if (!ok) break;
            tc::fence_after_sync();
            if (warp < 4 && comp && (c % G == G - 1 || lb + kChunk >= B)) drain_chunk<NB>(trow, c < G);
            tc::fence_before_sync();  // the next chunk's barrier orders the drain before its MMA
        }
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll 1
        for (int b = 0; b < NB && warp < 4; ++b) {
            uint32_t hi[16], lo[16];
            if (comp) {
                tc::tmem_ld16(trow + NC + 16 * b, hi);
                tc::tmem_ld16(trow + 2 * NC + 16 * b, lo);
            } else {  // one drain group: the FP32 accumulator itself
                tc::tmem_ld16(trow + 16 * b, hi);
#pragma unroll
                for (int c2 = 0; c2 < 16; ++c2) lo[c2] = 0u;
            }
            if (active) {
                float2 *Sb = const_cast<float2 *>(mb.S[b]);
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    if (p >= np) break;
                    const int jj = cs.mir[p] ? n - 1 - j : j;
                    // hi + lo rounded once to the FP32 of S (|lo| <= ulp(hi): the nearest
                    // float to the compensated sum), times w_B(j) for the adjoint's W; FP32
                    // only, so the epilogue takes nothing from the recurrence's FP64 pipe
                    const float wj = (flags & kApplyW) ? tc::f64_to_f32_rn(tb.w[jj]) : 1.0f;
                    const float re = __uint_as_float(hi[2 * p]) + __uint_as_float(lo[2 * p]);
                    const float im = __uint_as_float(hi[2 * p + 1]) + __uint_as_float(lo[2 * p + 1]);
                    Sb[((int64_t)mod_n(cs.pm[p], n) * n + mod_n(cs.pmp[p], n)) * n + jj] = make_float2(wj * re, wj * im);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok && tid == 0 && tb.err) atomicExch(tb.err, 2);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tcols);
}

// Self-test of the bounded wait used by the mixed kernels: one CTA polls an
// mbarrier that nothing arrives on, gives up after `polls` polls and records
// SOFT_ERR_TIMEOUT's code (2) in the error word, exactly as a DWT kernel would.
__global__ void bounded_wait_selftest_kernel(uint32_t polls, int *err) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    __syncthreads();
    const bool done = tc::mbar_wait(&mbar, 0u, polls);
    if (!__syncthreads_and(done) && threadIdx.x == 0 && err) atomicExch(err, 2);
}

// log w_B(j) for the forward's weighted seeds.
__global__ void log_weights_kernel(int n, const double *w, double *lw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) lw[t] = log(w[t]);
}

// Entries with m or m' = -B (index B) of the [m][m'][j] FP32 workspace.
__global__ void zero_nyquist32_kernel(int B, float2 *S) {
    const int n = 2 * B;
    const int64_t total = (int64_t)(2 * n - 1) * n;  // row mi = B (n*n entries) is handled as n rows of n
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int rowi = (int)(e / n), j = (int)(e % n);
        int64_t idx;
        if (rowi < n) idx = ((int64_t)B * n + rowi) * n + j;                    // mi = B, mk = rowi
        else { const int c = rowi - n; idx = ((int64_t)(c < B ? c : c + 1) * n + B) * n + j; }  // mk = B
        S[idx] = make_float2(0.f, 0.f);
    }
}

__global__ void f64_to_f32_kernel(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[i];
        out[i] = make_float2(tc::f64_to_f32_rn(v.x), tc::f64_to_f32_rn(v.y));
    }
}

__global__ void f32_to_f64_kernel(const float2 *__restrict__ in, double2 *__restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = in[i];
        out[i] = make_double2(tc::f32_to_f64(v.x), tc::f32_to_f64(v.y));
    }
}

// Y[q][j] = X[j][q] for a rows x cols complex64 matrix (rows = 2B beta
// samples, cols = (2B)^2 order pairs): 32 x 32 tiles through shared memory,
// coalesced on both sides.
__global__ void transpose32_kernel(const float2 *__restrict__ X, float2 *__restrict__ Y, int rows, int64_t cols) {
    __shared__ float2 tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy;
        const int64_t c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[dy][threadIdx.x] = X[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t c = c0 + dy;
        const int r = r0 + threadIdx.x;
        if (r < rows && c < cols) Y[c * rows + r] = tile[threadIdx.x][dy];
    }
}

int grid_for(int64_t count) { return (int)std::min<int64_t>((count + 255) / 256, 152 * 16); }

template <int MODE, int KC, int NB>
size_t mixed_forward_smem(int B) {
    static_assert(Operands<MODE, kFwdTile, KC, 16 * NB>::BYTES >= 2 * kMaxB * (int)sizeof(double), "scratch must fit");
    return (size_t)Operands<MODE, kFwdTile, KC, 16 * NB>::BYTES + sizeof(double) * (2 * (size_t)(2 * B) + 3 * (size_t)B);
}

template <int MODE, int NB>
size_t mixed_inverse_smem(int B) {
    return Operands<MODE, kTile, kChunk, 16 * NB>::BYTES + sizeof(double) * 4 * (size_t)B + sizeof(float) * (size_t)B;
}

// Dynamic shared memory large enough that no more CTAs share an SM than its
// 512 TMEM columns hold (a CTA that cannot allocate would wait in
// tcgen05.alloc, holding its SM slot): with K = 512 / tcols CTAs allowed,
// K + 1 of them must not fit the SM's 228 KB (1 KB of it reserved per CTA).
size_t tmem_limited_smem(size_t bytes, uint32_t tcols) {
    const size_t k = 512 / tcols;
    const size_t floor_bytes = 233472 / (k + 1) - 1000;
    return std::max(bytes, floor_bytes);
}

template <int MODE, int KC, int NB, bool LD>
cudaError_t run_forward_mixed(const MixedBatch &mb, cudaStream_t s, int flags) {
    const bool comp = (2 * mb.tb.B + KC - 1) / KC > drain_group<NB>();
    const size_t bytes = tmem_limited_smem(mixed_forward_smem<MODE, KC, NB>(mb.tb.B),
                                           comp ? tmem_cols<3 * 16 * NB>() : tmem_cols<16 * NB>());
    cudaError_t e = cudaFuncSetAttribute(dwt_forward_mixed_kernel<MODE, KC, NB, LD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    dwt_forward_mixed_kernel<MODE, KC, NB, LD><<<mb.tb.ncl, LD ? 2 * KC : KC, bytes, s>>>(mb, flags);
    count_launch();
    return cudaGetLastError();
}

template <int MODE, int NB, bool LD>
cudaError_t run_inverse_mixed(const MixedBatch &mb, cudaStream_t s, int flags) {
    const bool comp = (mb.tb.B + kChunk - 1) / kChunk > drain_group<NB>();  // the longest cluster's
    const size_t bytes = tmem_limited_smem(mixed_inverse_smem<MODE, NB>(mb.tb.B),
                                           comp ? tmem_cols<3 * 16 * NB>() : tmem_cols<16 * NB>());
    cudaError_t e = cudaFuncSetAttribute(dwt_inverse_mixed_kernel<MODE, NB, LD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    dwt_inverse_mixed_kernel<MODE, NB, LD><<<mb.tb.ncl, LD ? 2 * kNT : kNT, bytes, s>>>(mb, flags);
    count_launch();
    return cudaGetLastError();
}

// Forward shapes: one transform uses 128 beta samples per chunk up to 2B = 128
// and 256 beyond (two CTAs per SM at 2B = 1024); batches use 128 per chunk so
// that the N = 16 NB column operand stays small.
// Batches (NB >= 2) add a loader warpgroup: the B operand is NB times larger
// than for one transform, and its loads then overlap the recurrence.
template <int MODE>
cudaError_t forward_mixed_nb(const MixedBatch &mb, int nb, cudaStream_t s, int flags) {
    switch (nb) {
        case 1: {
            // variant 0: 128 samples per chunk up to 2B = 128, 256 beyond; variant 1: the other
            const bool k128 = (2 * mb.tb.B <= 128) != (mb.tb.fwd_variant == 1);
            return k128 ? run_forward_mixed<MODE, 128, 1, false>(mb, s, flags)
                        : run_forward_mixed<MODE, 256, 1, false>(mb, s, flags);
        }
        case 2: return run_forward_mixed<MODE, 128, 2, true>(mb, s, flags);
        case 4: return run_forward_mixed<MODE, 128, 4, true>(mb, s, flags);
        case 8: return run_forward_mixed<MODE, 128, 8, true>(mb, s, flags);
        default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t inverse_mixed_nb(const MixedBatch &mb, int nb, cudaStream_t s, int flags) {
    switch (nb) {
        case 1: return run_inverse_mixed<MODE, 1, false>(mb, s, flags);
        case 2: return run_inverse_mixed<MODE, 2, true>(mb, s, flags);
        case 4: return run_inverse_mixed<MODE, 4, true>(mb, s, flags);
        case 8: return run_inverse_mixed<MODE, 8, true>(mb, s, flags);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_log_weights(int B, const double *w, double *lw, cudaStream_t s) {
    const int n = 2 * B;
    log_weights_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, w, lw);
    count_launch();
    return cudaGetLastError();
}

// nb transforms of one bandwidth; nb in {1, 2, 4, 8} (a batch of other sizes
// is split by the caller).
cudaError_t launch_dwt_forward_mixed_batch(int mode, const Tables &tb, int nb, const float2 *const *S,
                                           double *const *coef, cudaStream_t s, int flags) {
    if (nb < 1 || nb > kMaxMixedBatch) return cudaErrorInvalidValue;
    MixedBatch mb{};
    mb.tb = tb;
    for (int b = 0; b < nb; ++b) { mb.S[b] = S[b]; mb.coef[b] = coef[b]; }
    return mode == SOFT_MIXED_TF32 ? forward_mixed_nb<SOFT_MIXED_TF32>(mb, nb, s, flags)
                                   : forward_mixed_nb<SOFT_MIXED_BF16X3>(mb, nb, s, flags);
}

cudaError_t launch_dwt_inverse_mixed_batch(int mode, const Tables &tb, int nb, const double *const *coef,
                                           float2 *const *S, cudaStream_t s, int flags) {
    if (nb < 1 || nb > kMaxMixedBatch) return cudaErrorInvalidValue;
    MixedBatch mb{};
    mb.tb = tb;
    for (int b = 0; b < nb; ++b) { mb.S[b] = S[b]; mb.coef[b] = const_cast<double *>(coef[b]); }
    return mode == SOFT_MIXED_TF32 ? inverse_mixed_nb<SOFT_MIXED_TF32>(mb, nb, s, flags)
                                   : inverse_mixed_nb<SOFT_MIXED_BF16X3>(mb, nb, s, flags);
}

cudaError_t launch_dwt_forward_mixed(int mode, const Tables &tb, const double *lw, const float2 *S, double *coef,
                                     cudaStream_t s, int flags) {
    (void)lw;  // tb.lw
    return launch_dwt_forward_mixed_batch(mode, tb, 1, &S, &coef, s, flags);
}

cudaError_t launch_dwt_inverse_mixed(int mode, const Tables &tb, const double *coef, float2 *S, cudaStream_t s,
                                     int flags) {
    return launch_dwt_inverse_mixed_batch(mode, tb, 1, &coef, &S, s, flags);
}

cudaError_t launch_bounded_wait_selftest(uint32_t polls, int *err, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(polls, err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_zero_nyquist32(int B, float2 *S, cudaStream_t s) {
    const int n = 2 * B;
    zero_nyquist32_kernel<<<grid_for((int64_t)(2 * n - 1) * n), 256, 0, s>>>(B, S);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_transpose32(const float2 *X, float2 *Y, int rows, int64_t cols, cudaStream_t s) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    transpose32_kernel<<<grid, dim3(32, 8), 0, s>>>(X, Y, rows, cols);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double2 *in, float2 *out, int64_t count, cudaStream_t s) {
    f64_to_f32_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float2 *in, double2 *out, int64_t count, cudaStream_t s) {
    f32_to_f64_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}

}  // namespace softgb
