// dwt_fp64.cu -- FP64 discrete Wigner transform (DWT) and its inverse (iDWT)
// on the GB300, plus the small table and S-clearing kernels.
//
// The DWT of orders (m,m') (Sec. 2.4, matrix form):
//   [f(l,m,m')]_l = V_B T_B W_B [S(m,m';j)]_j,   V = diag((2l+1)/(8 pi B)),
//   T = [d(l,m,m';beta_j)], W = diag(w_B(j)),     l = l0..B-1, j = 0..2B-1;
// the iDWT is [S(m,m';j)]_j = T_B^T [f(l,m,m')]_l.
//
// GB300 design.  One CTA per symmetry cluster (Sec. 3): the representative's
// column block T is generated ONCE, on the fly, by the three-term recurrence
// in FP64 (never stored in HBM) and serves the cluster's up to 8 partners,
// which become the 16 real right-hand sides of a skinny GEMM.  The path is
// bound by the FP64 pipe, so the kernels keep FP64 work to the contraction's
// 16 FMAs plus the recurrence's 3 operations per (l, j) entry; every table
// (weights, logs, recurrence coefficients) is computed once per CTA or plan.
#include "soft_internal.cuh"

#include <algorithm>

namespace softgb {

namespace {

__device__ __forceinline__ int mod_n(int a, int n) { return a < 0 ? a + n : a; }

// ---------------------------------------------------------------------------
// Plan tables: w_B(j) (Eq. (weights)), cos(beta_j), log cos(beta_j/2),
// log sin(beta_j/2) and log(k!).  Angles are formed as exact rationals of pi
// (sinpi/cospi) so that no rounded multiple of pi enters the arguments.
// ---------------------------------------------------------------------------
__global__ void tables_kernel(int B, double *w, double *cosb, double *lcos, double *lsin, double *lfact) {
    const int n = 2 * B;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const int64_t q = 2 * t + 1;  // beta_t = q pi / (4B)
        const int64_t per = 8LL * B;  // sin(r pi/(4B)) has period 8B in r
        double s = 0.0;
        for (int i = 0; i < B; ++i) {
            const int64_t r = ((2LL * i + 1) * q) % per;
            s += sinpi((double)r / (4.0 * B)) / (2.0 * i + 1.0);
        }
        w[t] = 2.0 * M_PI * sinpi((double)q / (4.0 * B)) / ((double)B * B) * s;
        cosb[t] = cospi((double)q / (4.0 * B));
        lcos[t] = log(cospi((double)q / (8.0 * B)));
        lsin[t] = log(sinpi((double)q / (8.0 * B)));
    }
    if (t <= n) lfact[t] = lgamma(t + 1.0);
}

// Zero the S entries of frequency -B (index B) in either order, which the
// iDWT never writes and the 2-D FFT of the inverse must see as 0.
__global__ void zero_nyquist_kernel(int B, double2 *S) {
    const int n = 2 * B;
    const int64_t total = (int64_t)n * (2 * n - 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / (2 * n - 1));
        const int r = (int)(e % (2 * n - 1));
        int64_t idx;
        if (r < n) idx = ((int64_t)j * n + B) * n + r;                      // m = -B row
        else { const int c = r - n; idx = ((int64_t)j * n + (c < B ? c : c + 1)) * n + B; }  // m' = -B col
        S[idx] = make_double2(0.0, 0.0);
    }
}

// ---------------------------------------------------------------------------
// Forward DWT.  NT threads, LT = NT/(16 TPI) degrees per tile, JPT beta samples
// per thread in the recurrence phase, TPI threads per output (each sums a
// contiguous 1/TPI of the beta range; the TPI partial sums are combined by shuffles).
//   dynamic smem: X[2B][16] (w_B(j') S_p(j'), partner p in columns 2p, 2p+1),
//                 T[LT][2B] (the current tile of T_B), rec[4][B] (A, Ac, Bc, V).
// Phase A: every thread advances the recurrence of its beta samples LT steps,
//          writing the tile of T.
// Phase B: thread (t, c) forms sum_j T[t][j] X[j][c] for output column c.
// ---------------------------------------------------------------------------
// One cluster of the forward DWT; every thread of the CTA calls it (the CTA
// kernel below and the persistent batch kernel).  smem as above, for this B.
template <int NT, int JPT, int TPI>
__device__ __forceinline__ void dwt_cluster(const Tables &tb, const double2 *__restrict__ S,
                                            double *__restrict__ coef, int flags, int cidx, int m, int mp,
                                            double *smem, ClusterSmem &cs) {
    constexpr int LT = NT / (16 * TPI);
    const int B = tb.B, n = 2 * B, tid = threadIdx.x;
    const int l0 = m, L = B - l0;

    double *X = smem;              // [n][16]
    double *T = X + (size_t)n * 16; // [LT][n]
    double *rA = T + (size_t)LT * n;
    double *rAc = rA + B;
    double *rBc = rAc + B;
    double *rV = rBc + B;
    double *rSig = rV + B;

    load_cluster(tb, m, mp, cs);
    for (int t = tid; t < L; t += NT) rV[t] = (flags & kApplyV) ? (2.0 * (l0 + t) + 1.0) / (8.0 * M_PI * B) : 1.0;
    cluster_recurrence<NT>(tb, cidx, l0, L, m, mp, rA, rAc, rBc, rSig, rV);
    const int np = cs.np;
    // Real input (kRealSym): f(l,-m,-m') = (-1)^(m-m') conj f(l,m,m'), and the
    // partners come in such conjugate pairs (2k, 2k+1), so only the even ones
    // are contracted (slot c holds partner c * pstep) and the odd ones are
    // written from them.
    const bool real = (flags & kRealSym) && np > 1;
    const int npc = real ? np / 2 : np, pstep = real ? 2 : 1;

    // X: S of every contracted partner, beta index mirrored where the
    // partner's column is d(.; pi - beta).  The weight w_B(j) is not applied
    // here: it enters T through the seeds below (T W, since the recurrence is
    // linear in d; w_B is symmetric under j -> 2B-1-j, so mirrored partners see
    // the same w).
    for (int e = tid; e < n * 8; e += NT) {
        const int j = e >> 3, c = e & 7;
        double2 v = make_double2(0.0, 0.0);
        if (c < npc) {
            const int p = c * pstep;
            const int src = cs.mir[p] ? n - 1 - j : j;
            v = S[((int64_t)src * n + mod_n(cs.pm[p], n)) * n + mod_n(cs.pmp[p], n)];
        }
        *reinterpret_cast<double2 *>(&X[j * 16 + 2 * c]) = v;
    }

    // Recurrence state of this thread's beta samples: seeds w_B(j) d(l0,m,m';beta_j).
    double x[JPT], dcur[JPT], dprev[JPT];
    {
        const double lognorm = seed_lognorm(tb, m, mp);
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            const int j = tid + k * NT;
            x[k] = 0.0; dcur[k] = 0.0; dprev[k] = 0.0;
            if (j < n) {
                x[k] = tb.cosb[j];
                dcur[k] = cluster_seed(tb, cidx, j, m, mp, lognorm, (flags & kApplyW) != 0);
            }
        }
    }
    __syncthreads();

    const int half = tid % TPI, ot = tid / TPI;  // phase-B output (degree in tile, column) and beta part
    static_assert(TPI == 1 || TPI == 2 || TPI == 4, "TPI");
    // The 16 lanes (x TPI) of a degree cover its 16 real output columns (8
    // partners x re/im).  With at most 4 contracted partners the upper 8
    // columns have no work, and for TPI <= 2 they would be half-warps that
    // still occupy the FP64 pipe, so there the lanes take 8 columns x 2 halves
    // of the beta range (combined by one more shuffle) instead.
    const bool fold = TPI <= 2 && npc <= 4;
    const int pt = ot >> 4, pc = fold ? (ot & 7) : (ot & 15);
    const int pp = pc >> 1;
    const int upper = fold ? (ot >> 3) & 1 : 0;  // second half of the beta range
    const int parts = fold ? 2 * TPI : TPI, part = half + TPI * upper;
    const int jlen = (n + parts - 1) / parts, jbeg = min(n, part * jlen);
    const int jcnt = min(jlen, n - jbeg);
    for (int lb = l0; lb < B; lb += LT) {
        const int nt = min(LT, B - lb);
        // Phase A
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            const int j = tid + k * NT;
            if (j < n) {
                for (int t = 0; t < nt; ++t) {
                    T[t * n + j] = dcur[k];
                    const int r = lb + t - l0;
                    const double nx = fma(fma(rA[r], x[k], -rAc[r]), dcur[k], -dprev[k]);
                    dprev[k] = dcur[k];
                    dcur[k] = nx;
                }
            }
        }
        __syncthreads();
        // Phase B
        const bool active = pt < nt && pp < npc;
        double acc = 0.0;
        if (active) {
            const double *Tr = T + pt * n + jbeg;
            const double *Xc = X + (size_t)jbeg * 16 + pc;
            // two chains: the FP64 pipe issues slowly enough that latency is hidden
            double a0 = 0.0, a1 = 0.0;
            int j = 0;
            for (; j + 2 <= jcnt; j += 2) {
                a0 = fma(Tr[j], Xc[j * 16], a0);
                a1 = fma(Tr[j + 1], Xc[(j + 1) * 16], a1);
            }
            if (j < jcnt) a0 = fma(Tr[j], Xc[j * 16], a0);
            acc = a0 + a1;
        }
        if (TPI >= 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (TPI >= 4) acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (fold) acc += __shfl_xor_sync(0xffffffffu, acc, 8 * TPI);  // the two beta halves (fold is CTA-uniform)
        if (active && half == 0 && upper == 0) {
            const int l = lb + pt, p = pp * pstep;
            const double v = rV[l - l0];
            const bool neg = (cs.sign[p] < 0.0) != (cs.lpar[p] && (l & 1));
            const double f = (neg ? -v : v) * acc;
            coef[2 * (cs.off[p] + (l - l0)) + (pc & 1)] = f;
            if (real) {  // partner p + 1 = (-m, -m') of partner p: (-1)^(m-m') conj f
                const bool flip = ((cs.pm[p] - cs.pmp[p]) & 1) != (pc & 1);
                coef[2 * (cs.off[p + 1] + (l - l0)) + (pc & 1)] = flip ? -f : f;
            }
        }
        __syncthreads();
    }
}

template <int NT, int JPT, int TPI>
__global__ void __launch_bounds__(NT, 1) dwt_forward_fp64_kernel(Tables tb, const double2 *__restrict__ S,
                                                               double *__restrict__ coef, int flags) {
    extern __shared__ __align__(16) double smem[];
    __shared__ ClusterSmem cs;
    const int cidx = tb.fwd_order ? tb.fwd_order[blockIdx.x] : (int)blockIdx.x;
    const int2 rep = tb.clusters[cidx];
    dwt_cluster<NT, JPT, TPI>(tb, S, coef, flags, cidx, rep.x, rep.y, smem, cs);
}

// ---------------------------------------------------------------------------
// Inverse DWT.  Every thread owns JPT beta samples, walks l = l0..B-1 with the
// recurrence in registers and accumulates NC real columns:
//   acc[c] += d(l; beta_j) * F[l][c],  F = sign-folded coefficients of the partners.
//   dynamic smem: F[B][16], rec[3][B].
// ---------------------------------------------------------------------------
template <int NT, int JPT, int NC>
__device__ __forceinline__ void idwt_walk(const double *F, const double *rA, const double *rAc, int L,
                                          double (&x)[JPT], double (&dcur)[JPT], double (&dprev)[JPT],
                                          double (&acc)[JPT][16]) {
    for (int t = 0; t < L; ++t) {
        const double *Fr = F + t * 16;
        const double A = rA[t], Ac = rAc[t];
#pragma unroll
        for (int c = 0; c < NC; c += 2) {
            const double2 f = *reinterpret_cast<const double2 *>(Fr + c);
#pragma unroll
            for (int k = 0; k < JPT; ++k) {
                acc[k][c] = fma(dcur[k], f.x, acc[k][c]);
                acc[k][c + 1] = fma(dcur[k], f.y, acc[k][c + 1]);
            }
        }
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            const double nx = fma(fma(A, x[k], -Ac), dcur[k], -dprev[k]);
            dprev[k] = dcur[k];
            dcur[k] = nx;
        }
    }
}

// Set-up of one cluster of an inverse DWT, by every thread of the CTA: the
// partner table, the rescaled recurrence coefficients and
//   F[t][2c (+1)] = sign_p(l) sig_t (V_l) f(l, m_p, m'_p)  (re, im),  l = l0 + t,
// the sign- and scale-folded coefficients of contracted partner p = c pstep.
// smem holds F[B][16] and the recurrence coefficients (4 x B doubles).  Real
// output (kRealSym): S(-m,-m';j) = conj S(m,m';j) for the conjugate partner
// pairs (2k, 2k+1); only the even partners are contracted (slot c holds
// partner c * pstep) and only their coefficients are read.  Ends with a barrier.
struct IdwtShape {
    int npc, pstep;
    bool real;
};

template <int NT>
__device__ __forceinline__ IdwtShape idwt_setup(const Tables &tb, const double *__restrict__ coef, int flags,
                                                int cidx, int m, int mp, double *smem, ClusterSmem &cs) {
    const int B = tb.B, tid = threadIdx.x;
    const int l0 = m, L = B - l0;
    double *F = smem;                  // [B][16]
    double *rA = F + (size_t)B * 16;
    double *rAc = rA + B;
    double *rBc = rAc + B;
    double *rSig = rBc + B;
    load_cluster(tb, m, mp, cs);
    cluster_recurrence<NT>(tb, cidx, l0, L, m, mp, rA, rAc, rBc, rSig, nullptr);
    const int np = cs.np;
    IdwtShape sh;
    sh.real = (flags & kRealSym) && np > 1;
    sh.npc = sh.real ? np / 2 : np;
    sh.pstep = sh.real ? 2 : 1;
    for (int e = tid; e < L * 8; e += NT) {
        const int t = e >> 3, c = e & 7;
        double2 v = make_double2(0.0, 0.0);
        if (c < sh.npc) {
            const int p = c * sh.pstep;
            const int l = l0 + t;
            double sg = (cs.lpar[p] && (l & 1)) ? -cs.sign[p] : cs.sign[p];
            sg *= rSig[t];
            if (flags & kApplyV) sg *= (2.0 * l + 1.0) / (8.0 * M_PI * B);
            const double2 cf = *reinterpret_cast<const double2 *>(coef + 2 * (cs.off[p] + t));
            v = make_double2(sg * cf.x, sg * cf.y);
        }
        *reinterpret_cast<double2 *>(&F[t * 16 + 2 * c]) = v;
    }
    __syncthreads();
    return sh;
}

// Stores beta sample j's contracted columns acc (times w_B(j') for the
// adjoint's W) into S: partner p at j' = j, or 2B-1-j for mirrored partners,
// and for real output also its conjugate partner.
__device__ __forceinline__ void idwt_store(const Tables &tb, double2 *__restrict__ S, int flags, const ClusterSmem &cs,
                                           const IdwtShape &sh, int j, const double (&acc)[16]) {
    const int n = 2 * tb.B;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (c < sh.npc) {
            const int p = c * sh.pstep;
            const int jj = cs.mir[p] ? n - 1 - j : j;
            const double wj = (flags & kApplyW) ? tb.w[jj] : 1.0;
            const double2 v = make_double2(wj * acc[2 * c], wj * acc[2 * c + 1]);
            S[((int64_t)jj * n + mod_n(cs.pm[p], n)) * n + mod_n(cs.pmp[p], n)] = v;
            if (sh.real)  // partner p + 1 = (-m, -m'): the conjugate, at the same beta sample
                S[((int64_t)jj * n + mod_n(cs.pm[p + 1], n)) * n + mod_n(cs.pmp[p + 1], n)] = make_double2(v.x, -v.y);
        }
    }
}

// One cluster of the inverse DWT; every thread of the CTA calls it.  smem holds
// F[B][16] and the recurrence coefficients (4 x B doubles).
template <int NT, int JPT>
__device__ __forceinline__ void idwt_cluster(const Tables &tb, const double *__restrict__ coef,
                                             double2 *__restrict__ S, int flags, int cidx, int m, int mp,
                                             double *smem, ClusterSmem &cs) {
    const int B = tb.B, n = 2 * B, tid = threadIdx.x;
    const int L = B - m;
    const IdwtShape sh = idwt_setup<NT>(tb, coef, flags, cidx, m, mp, smem, cs);
    const double *F = smem;
    const double *rA = F + (size_t)B * 16;
    const double *rAc = rA + B;

    double x[JPT], dcur[JPT], dprev[JPT];
    double acc[JPT][16];
    {
        const double lognorm = seed_lognorm(tb, m, mp);
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            const int j = tid + k * NT;
            x[k] = 0.0; dcur[k] = 0.0; dprev[k] = 0.0;
            if (j < n) {
                x[k] = tb.cosb[j];
                dcur[k] = cluster_seed(tb, cidx, j, m, mp, lognorm, false);
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[k][c] = 0.0;
        }
    }

    if (sh.npc > 4)      idwt_walk<NT, JPT, 16>(F, rA, rAc, L, x, dcur, dprev, acc);
    else if (sh.npc > 2) idwt_walk<NT, JPT, 8>(F, rA, rAc, L, x, dcur, dprev, acc);
    else                 idwt_walk<NT, JPT, 4>(F, rA, rAc, L, x, dcur, dprev, acc);

#pragma unroll
    for (int k = 0; k < JPT; ++k) {
        const int j = tid + k * NT;
        if (j < n) idwt_store(tb, S, flags, cs, sh, j, acc[k]);
    }
}

// ---------------------------------------------------------------------------
// Inverse DWT by Clenshaw's algorithm (a tile-shape variant of the FP64 iDWT;
// Sec. 2.4 names Clenshaw's algorithm as the O(B^4) way to run the DWT/iDWT
// along the three-term recurrence).  With d(l0+t) = sig_t e_t and e_{t+1} =
// a_t(x) e_t - e_{t-1}, a_t(x) = A'_t x - Ac'_t, e_{-1} = 0, the sum
//   S_c(j) = sum_t e_t(x_j) g_t(c),   g_t(c) = F[t][c] (sig_t folded in),
// runs backwards over the degrees with no Wigner-d value formed:
//   b_t = g_t + a_t(x_j) b_{t+1} - b_{t+2},  b_L = b_{L+1} = 0,  S_c(j) = e_0(x_j) b_0
// (summing by parts, the coefficient of every b_s, s >= 1, is the recurrence
// and vanishes).  Cost: one FMA for a_t per sample and degree, then an FMA and
// a subtraction per column -- 2 FP64 operations per column against the
// forward-recurrence iDWT's 1 FMA per column plus 2 shared ones, so with the
// 16 partner columns it does ~1.8x the FP64 work; each thread carries b_{t+1}
// and b_{t+2} of every column (32 doubles), so it takes one beta sample at a
// time and the CTA loops over the samples in blocks of NT.
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ void clenshaw_walk(const double *F, const double *rA, const double *rAc, int L, double x,
                                              double (&b1)[16]) {
    double b2[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) { b1[c] = 0.0; b2[c] = 0.0; }
    for (int t = L - 1; t >= 0; --t) {
        const double a = fma(rA[t], x, -rAc[t]);
        const double *Fr = F + t * 16;
#pragma unroll
        for (int c = 0; c < NC; c += 2) {
            const double2 g = *reinterpret_cast<const double2 *>(Fr + c);
            const double n0 = fma(a, b1[c], g.x - b2[c]);
            const double n1 = fma(a, b1[c + 1], g.y - b2[c + 1]);
            b2[c] = b1[c];
            b2[c + 1] = b1[c + 1];
            b1[c] = n0;
            b1[c + 1] = n1;
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) idwt_clenshaw_fp64_kernel(Tables tb, const double *__restrict__ coef,
                                                               double2 *__restrict__ S, int flags) {
    extern __shared__ __align__(16) double smem[];
    __shared__ ClusterSmem cs;
    const int B = tb.B, n = 2 * B;
    const int cidx = tb.inv_order ? tb.inv_order[blockIdx.x] : (int)blockIdx.x;
    const int2 rep = tb.clusters[cidx];
    const int m = rep.x, mp = rep.y, L = B - m;
    const IdwtShape sh = idwt_setup<NT>(tb, coef, flags, cidx, m, mp, smem, cs);
    const double *F = smem;
    const double *rA = F + (size_t)B * 16;
    const double *rAc = rA + B;
    const double lognorm = seed_lognorm(tb, m, mp);
    for (int j = threadIdx.x; j < n; j += NT) {
        const double x = tb.cosb[j];
        const double e0 = cluster_seed(tb, cidx, j, m, mp, lognorm, false);
        double b[16];
        if (sh.npc > 4)      clenshaw_walk<16>(F, rA, rAc, L, x, b);
        else if (sh.npc > 2) clenshaw_walk<8>(F, rA, rAc, L, x, b);
        else                 clenshaw_walk<4>(F, rA, rAc, L, x, b);
#pragma unroll
        for (int c = 0; c < 16; ++c) b[c] *= e0;
        idwt_store(tb, S, flags, cs, sh, j, b);
    }
}

template <int NT, int JPT>
__global__ void __launch_bounds__(NT, 1) dwt_inverse_fp64_kernel(Tables tb, const double *__restrict__ coef,
                                                               double2 *__restrict__ S, int flags) {
    extern __shared__ __align__(16) double smem[];
    __shared__ ClusterSmem cs;
    const int cidx = tb.inv_order ? tb.inv_order[blockIdx.x] : (int)blockIdx.x;
    const int2 rep = tb.clusters[cidx];
    idwt_cluster<NT, JPT>(tb, coef, S, flags, cidx, rep.x, rep.y, smem, cs);
}

// One CTA per cluster: the rescaled recurrence coefficients and the seeds of
// the cluster, written once per plan for every later DWT launch to load.
__global__ void __launch_bounds__(256) cluster_tables_kernel(Tables tb, double *__restrict__ seedtab,
                                                             double *__restrict__ rectab) {
    extern __shared__ __align__(16) double smem[];
    const int B = tb.B, n = 2 * B, c = blockIdx.x;
    const int2 rep = tb.clusters[c];
    const int m = rep.x, mp = rep.y, l0 = m, L = B - l0;
    double *rA = smem, *rAc = rA + B, *rBc = rAc + B, *rSig = rBc + B;
    scaled_recurrence_tables<256>(l0, L, m, mp, rA, rAc, rBc, rSig, nullptr);
    double *dst = rectab + (size_t)c * B * 3;
    for (int t = threadIdx.x; t < L; t += 256) {
        dst[3 * t] = rA[t];
        dst[3 * t + 1] = rAc[t];
        dst[3 * t + 2] = rSig[t];
    }
    const double lognorm = seed_lognorm(tb, m, mp);
    for (int j = threadIdx.x; j < n; j += 256)
        seedtab[(size_t)c * n + j] = seed_rep(m, mp, lognorm, tb.lcos[j], tb.lsin[j]);
}

// Persistent DWT / iDWT over a batch of FP64 transforms of any bandwidths:
// one CTA per SM slot pulls (transform, cluster) items, heaviest first, from an
// atomic counter until the list is exhausted.  No CTA waits on another.  The
// tile shape (NT threads x JPT beta samples, TPI threads per forward output)
// is the single-transform kernel's for the batch's largest bandwidth, so
// NT * JPT covers its 2B samples, and shared memory is sized for it.
template <int NT, int JPT>
__global__ void __launch_bounds__(NT) idwt_fp64_persistent_kernel(const BatchXform *__restrict__ xf,
                                                                  const int2 *__restrict__ items, int nitems,
                                                                  int *__restrict__ counter) {
    extern __shared__ __align__(16) double smem[];
    __shared__ ClusterSmem cs;
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= nitems) break;
        const int2 w = items[it];
        const BatchXform &X = xf[w.x];
        const int2 rep = X.tb.clusters[w.y];
        idwt_cluster<NT, JPT>(X.tb, X.coef, X.S, X.flags, w.y, rep.x, rep.y, smem, cs);
        __syncthreads();  // smem and `item` are reused by the next item
    }
}

template <int NT, int JPT, int TPI>
__global__ void __launch_bounds__(NT) dwt_fp64_persistent_kernel(const BatchXform *__restrict__ xf,
                                                                 const int2 *__restrict__ items, int nitems,
                                                                 int *__restrict__ counter) {
    extern __shared__ __align__(16) double smem[];
    __shared__ ClusterSmem cs;
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= nitems) break;
        const int2 w = items[it];
        const BatchXform &X = xf[w.x];
        const int2 rep = X.tb.clusters[w.y];
        dwt_cluster<NT, JPT, TPI>(X.tb, X.Sin, X.coef_out, X.flags, w.y, rep.x, rep.y, smem, cs);
        __syncthreads();
    }
}

template <int NT, int JPT, int TPI>
cudaError_t run_forward(const Tables &tb, const double2 *S, double *coef, cudaStream_t s, int flags) {
    const int B = tb.B, n = 2 * B;
    const size_t bytes = sizeof(double) * ((size_t)n * 16 + (size_t)(NT / (16 * TPI)) * n + 5 * (size_t)B);
    cudaError_t e = cudaFuncSetAttribute(dwt_forward_fp64_kernel<NT, JPT, TPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    dwt_forward_fp64_kernel<NT, JPT, TPI><<<tb.ncl, NT, bytes, s>>>(tb, S, coef, flags);
    count_launch();
    return cudaGetLastError();
}

template <int NT, int JPT>
cudaError_t run_inverse(const Tables &tb, const double *coef, double2 *S, cudaStream_t s, int flags) {
    const int B = tb.B;
    const size_t bytes = sizeof(double) * ((size_t)B * 16 + 4 * (size_t)B);
    cudaError_t e = cudaFuncSetAttribute(dwt_inverse_fp64_kernel<NT, JPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    dwt_inverse_fp64_kernel<NT, JPT><<<tb.ncl, NT, bytes, s>>>(tb, coef, S, flags);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tables(int B, double *w, double *cosb, double *lcos, double *lsin, double *lfact,
                          cudaStream_t s) {
    const int n = 2 * B;
    tables_kernel<<<(n + 1 + 127) / 128, 128, 0, s>>>(B, w, cosb, lcos, lsin, lfact);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cluster_tables(const Tables &tb, double *seedtab, double *rectab, cudaStream_t s) {
    Tables t = tb;
    t.seedtab = nullptr;
    t.rectab = nullptr;
    const size_t bytes = sizeof(double) * 4 * (size_t)tb.B;
    cluster_tables_kernel<<<tb.ncl, 256, bytes, s>>>(t, seedtab, rectab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_zero_nyquist(int B, double2 *S, cudaStream_t s) {
    const int n = 2 * B;
    const int64_t total = (int64_t)n * (2 * n - 1);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    zero_nyquist_kernel<<<blocks, 256, 0, s>>>(B, S);
    count_launch();
    return cudaGetLastError();
}

// Shape choice: the forward needs X (2B x 16) and a T tile (LT x 2B) in shared
// memory.  Up to 2B = 256, 256 threads with LT = 16 (68 KB, 3 CTAs per SM);
// beyond, LT = 8 with two threads per output, which keeps 256 threads per CTA
// (2B = 512: 104 KB, 2 CTAs per SM; 2B = 1024: 208 KB, 1 CTA of 8 warps).
// Tile-shape variants (NT, JPT, TPI) per bandwidth range; variant 0 is the
// default, the others are what the autotuner compares it against.
int dwt_forward_fp64_variants(int B) { return 2 * B <= 256 ? 3 : 2 * B <= 512 ? 3 : 2; }

cudaError_t launch_dwt_forward_fp64(const Tables &tb, const double2 *S, double2 *coef, cudaStream_t s, int flags) {
    const int n = 2 * tb.B;
    double *c = reinterpret_cast<double *>(coef);
    const int v = tb.fwd_variant;
    if (n <= 256) {
        if (v == 1) return run_forward<256, 1, 2>(tb, S, c, s, flags);
        if (v == 2) return run_forward<128, 2, 1>(tb, S, c, s, flags);
        return run_forward<256, 1, 1>(tb, S, c, s, flags);
    }
    if (n <= 512) {
        if (v == 1) return run_forward<256, 2, 1>(tb, S, c, s, flags);
        if (v == 2) return run_forward<512, 1, 4>(tb, S, c, s, flags);
        return run_forward<256, 2, 2>(tb, S, c, s, flags);
    }
    if (v == 1) return run_forward<512, 2, 4>(tb, S, c, s, flags);
    return run_forward<256, 4, 2>(tb, S, c, s, flags);
}

// Grid of a persistent kernel: every resident CTA slot of the device, at most one per item.
template <class K>
cudaError_t persistent_grid(K kernel, int nt, size_t bytes, int nitems, int *grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = std::max(1, std::min(nitems, std::max(1, per_sm) * sms));
    return cudaSuccess;
}

template <int NT, int JPT>
cudaError_t run_idwt_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                                cudaStream_t s) {
    const size_t bytes = sizeof(double) * ((size_t)maxB * 16 + 4 * (size_t)maxB);
    int grid = 0;
    cudaError_t e = persistent_grid(idwt_fp64_persistent_kernel<NT, JPT>, NT, bytes, nitems, &grid);
    if (e != cudaSuccess) return e;
    idwt_fp64_persistent_kernel<NT, JPT><<<grid, NT, bytes, s>>>(xf, items, nitems, counter);
    count_launch();
    return cudaGetLastError();
}

template <int NT, int JPT, int TPI>
cudaError_t run_dwt_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                               cudaStream_t s) {
    const int n = 2 * maxB;
    const size_t bytes = sizeof(double) * ((size_t)n * 16 + (size_t)(NT / (16 * TPI)) * n + 5 * (size_t)maxB);
    int grid = 0;
    cudaError_t e = persistent_grid(dwt_fp64_persistent_kernel<NT, JPT, TPI>, NT, bytes, nitems, &grid);
    if (e != cudaSuccess) return e;
    dwt_fp64_persistent_kernel<NT, JPT, TPI><<<grid, NT, bytes, s>>>(xf, items, nitems, counter);
    count_launch();
    return cudaGetLastError();
}

// Shapes for the batch's largest 2B: the single-transform iDWT's (up to 2B =
// 128 its two-samples-per-thread variant, which keeps small clusters from
// leaving most of a CTA idle).  The iDWT's sums do not depend on the shape.
cudaError_t launch_idwt_fp64_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                                        cudaStream_t s) {
    const int n = 2 * maxB;
    if (n <= 64) return run_idwt_persistent<32, 2>(xf, items, nitems, counter, maxB, s);
    if (n <= 128) return run_idwt_persistent<64, 2>(xf, items, nitems, counter, maxB, s);
    if (n <= 256) return run_idwt_persistent<256, 1>(xf, items, nitems, counter, maxB, s);
    if (n <= 512) return run_idwt_persistent<256, 2>(xf, items, nitems, counter, maxB, s);
    if (n <= 1024) return run_idwt_persistent<256, 4>(xf, items, nitems, counter, maxB, s);
    return cudaErrorInvalidValue;
}

// The single-transform DWT's default shape for the batch's largest 2B.
cudaError_t launch_dwt_fp64_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                                       cudaStream_t s) {
    const int n = 2 * maxB;
    if (n <= 256) return run_dwt_persistent<256, 1, 1>(xf, items, nitems, counter, maxB, s);
    if (n <= 512) return run_dwt_persistent<256, 2, 2>(xf, items, nitems, counter, maxB, s);
    if (n <= 1024) return run_dwt_persistent<256, 4, 2>(xf, items, nitems, counter, maxB, s);
    return cudaErrorInvalidValue;
}

// Tile-shape variants of the iDWT; the last one is Clenshaw's algorithm.
int dwt_inverse_fp64_variants(int B) { return (2 * B <= 256 ? 2 : 2 * B <= 512 ? 3 : 2) + 1; }

template <int NT>
cudaError_t run_inverse_clenshaw(const Tables &tb, const double *coef, double2 *S, cudaStream_t s, int flags) {
    const int B = tb.B;
    const size_t bytes = sizeof(double) * ((size_t)B * 16 + 4 * (size_t)B);
    cudaError_t e = cudaFuncSetAttribute(idwt_clenshaw_fp64_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    idwt_clenshaw_fp64_kernel<NT><<<tb.ncl, NT, bytes, s>>>(tb, coef, S, flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dwt_inverse_fp64(const Tables &tb, const double2 *coef, double2 *S, cudaStream_t s, int flags) {
    const int n = 2 * tb.B;
    const double *c = reinterpret_cast<const double *>(coef);
    const int v = tb.inv_variant;
    if (v == dwt_inverse_fp64_variants(tb.B) - 1)
        return n <= 64 ? run_inverse_clenshaw<64>(tb, c, S, s, flags) : n <= 128 ? run_inverse_clenshaw<128>(tb, c, S, s, flags)
                                                                          : run_inverse_clenshaw<256>(tb, c, S, s, flags);
    if (n <= 64) return v == 1 ? run_inverse<32, 2>(tb, c, S, s, flags) : run_inverse<64, 1>(tb, c, S, s, flags);
    if (n <= 128) return v == 1 ? run_inverse<64, 2>(tb, c, S, s, flags) : run_inverse<128, 1>(tb, c, S, s, flags);
    if (n <= 256) return v == 1 ? run_inverse<128, 2>(tb, c, S, s, flags) : run_inverse<256, 1>(tb, c, S, s, flags);
    if (n <= 512) {
        if (v == 1) return run_inverse<512, 1>(tb, c, S, s, flags);
        if (v == 2) return run_inverse<128, 4>(tb, c, S, s, flags);
        return run_inverse<256, 2>(tb, c, S, s, flags);
    }
    return v == 1 ? run_inverse<512, 2>(tb, c, S, s, flags) : run_inverse<256, 4>(tb, c, S, s, flags);
}

}  // namespace softgb
