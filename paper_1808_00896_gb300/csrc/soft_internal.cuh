// soft_internal.cuh -- device-side building blocks shared by the DWT kernels.
//
// Notation follows Sec. 2 of Lux, Wuelker, Chirikjian, "Parallelization of
// the FFT on SO(3)": bandwidth B, n = 2B samples per angle, beta_j =
// (2j+1)pi/(4B), Wigner-d d(l,m,m';beta), order pairs (m,m') with
// |m|,|m'| < B, degree l from l0 = max(|m|,|m'|) to B-1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace softgb {

constexpr int kMaxB = 512;
constexpr int kMaxMixedBatch = 8;  // transforms sharing one mixed-precision DWT launch

// Per-plan device tables (all FP64 unless stated).
// Called after every kernel launch of this library: the process-wide count
// that soft_launch_count() reports.
void count_launch();

struct Tables {
    int B;
    int ncl;                  // number of symmetry clusters, B(B+1)/2
    const double *w;          // [2B]  quadrature weights w_B(j), Eq. (weights)
    const double *lw;         // [2B]  log w_B(j) (the forward folds W into its seeds)
    const double *cosb;       // [2B]  cos(beta_j)
    const double *lcos;       // [2B]  log cos(beta_j / 2)
    const double *lsin;       // [2B]  log sin(beta_j / 2)
    const double *lfact;      // [2B+1] log(k!)
    const int2 *clusters;     // [ncl] representatives (m, m'), m >= m' >= 0, heaviest first
    const int64_t *runoff;    // [(2B-1)^2] start of the l-run of (m,m') in the coefficient array,
                              //   index (m + B - 1) * (2B - 1) + (m' + B - 1)
    int *err;                 // device error word (0 = fine)
    // Per-cluster tables built once per plan (null: computed on the fly in each CTA).
    const double *seedtab = nullptr;  // [ncl][2B]  d(l0,m,m';beta_j) of each cluster, unweighted
    const double *rectab = nullptr;   // [ncl][B][3] (A', Ac', sig) of the rescaled recurrence, l = l0 + t
    int wexp = 0;             // 2^wexp > max_j w_B(j) (the FP64-TC forward's weight scale)
    int *colexp = nullptr;    // FP64-TC plans: [2B][2B][2] largest biased FP64 exponent of |Re|, |Im| of
                              //   S(m, m'; .) over the beta samples, index (m mod 2B, m' mod 2B); written
                              //   before each forward DWT
    int fwd_variant = 0;      // tile-shape variant of the DWT kernel (0 = default)
    // [ncl] dispatch orders of the DWT and iDWT kernels (CTA b handles
    // cluster fwd_order[b] / inv_order[b]; null: cluster b), longest first by
    // each kernel's own cost per cluster.
    const int *fwd_order = nullptr;
    const int *inv_order = nullptr;
    int inv_variant = 0;      // tile-shape variant of the iDWT kernel
};

__host__ __device__ inline int64_t runoff_index(int B, int m, int mp) {
    return (int64_t)(m + B - 1) * (2 * B - 1) + (mp + B - 1);
}

// ---------------------------------------------------------------------------
// Symmetry clusters (Sec. 3, "Communication"): the order pairs whose Wigner-d
// columns follow from one representative (m, m'), m >= m' >= 0, by the seven
// relations of Eq. (Wigner_symmetries).  Partner p satisfies
//   d(l, m_p, m'_p; beta_j) = sign_p * (lpar_p ? (-1)^l : 1) * d(l, m, m'; beta_{j'}),
//   j' = mirror_p ? 2B-1-j : j            (beta -> pi - beta is j -> 2B-1-j).
// Clusters have 8 partners, or 4 when m' = 0 or m = m' (> 0), or 1 for (0,0).
// ---------------------------------------------------------------------------
struct Partners {
    int np;
    int m[8], mp[8];
    int mirror[8];
    int lpar[8];
    double sign[8];
};

__host__ __device__ inline double neg1pow(int k) { return (k & 1) ? -1.0 : 1.0; }

__host__ __device__ inline Partners make_partners(int m, int mp) {
    Partners P;
    int q = 0;
    auto add = [&](int a, int b, int mir, int lp, double s) {
        P.m[q] = a; P.mp[q] = b; P.mirror[q] = mir; P.lpar[q] = lp; P.sign[q] = s; ++q;
    };
    const double smm = neg1pow(m - mp);  // (-1)^(m-m')
    if (m == 0 && mp == 0) {
        add(0, 0, 0, 0, 1.0);
    } else if (mp == 0) {
        add(m, 0, 0, 0, 1.0);        // identity
        add(-m, 0, 0, 0, smm);       // d(l,-m,-m') = (-1)^(m-m') d(l,m,m')
        add(0, m, 0, 0, smm);        // d(l,m',m)   = (-1)^(m-m') d(l,m,m')
        add(0, -m, 0, 0, 1.0);       // d(l,-m',-m) = d(l,m,m')
    } else if (m == mp) {
        add(m, m, 0, 0, 1.0);
        add(-m, -m, 0, 0, 1.0);
        add(-m, m, 1, 1, neg1pow(m));  // d(l,-m,m';b) = (-1)^(l-m') d(l,m,m';pi-b)
        add(m, -m, 1, 1, neg1pow(m));  // d(l,m,-m';b) = (-1)^(l+m)  d(l,m,m';pi-b)
    } else {
        add(m, mp, 0, 0, 1.0);
        add(-m, -mp, 0, 0, smm);
        add(mp, m, 0, 0, smm);
        add(-mp, -m, 0, 0, 1.0);
        add(-m, mp, 1, 1, neg1pow(mp));  // (-1)^(l-m')
        add(m, -mp, 1, 1, neg1pow(m));   // (-1)^(l+m)
        add(-mp, m, 1, 1, neg1pow(mp));  // d(l,-m',m;b) = (-1)^(l-m') d(l,m,m';pi-b)
        add(mp, -m, 1, 1, neg1pow(m));   // d(l,m',-m;b) = (-1)^(l+m)  d(l,m,m';pi-b)
    }
    P.np = q;
    return P;
}

// ---------------------------------------------------------------------------
// Three-term recurrence, Eq. (Wigner_d_recurrence), for l >= 1:
//   d(l+1) = A_l (cos b - c_l) d(l) - Bc_l d(l-1)
//   A_l  = (l+1)(2l+1) / sqrt(((l+1)^2-m^2)((l+1)^2-m'^2)),   c_l = m m' / (l(l+1)),
//   Bc_l = (l+1) sqrt((l^2-m^2)(l^2-m'^2)) / (l sqrt(((l+1)^2-m^2)((l+1)^2-m'^2))).
// Stored as (A_l, A_l c_l, Bc_l) so that a step is fma(fma(A,x,-Ac), d, -Bc*dprev).
// The only cluster starting at l = 0 is (0,0), where d(1,0,0) = cos b: entry (1,0,0).
// At l = l0 > 0 the d(l0-1) coefficient vanishes, consistent with d(l0-1) := 0.
// ---------------------------------------------------------------------------
__device__ inline void recurrence_coeffs(int l, int m, int mp, double &A, double &Ac, double &Bc) {
    if (l == 0) { A = 1.0; Ac = 0.0; Bc = 0.0; return; }
    const double L1 = l + 1.0, ll = l, mm = m, nn = mp;
    const double den = sqrt((L1 * L1 - mm * mm) * (L1 * L1 - nn * nn));  // exact integer product
    const double a = L1 * (2.0 * ll + 1.0) / den;
    A = a;
    Ac = a * (mm * nn / (ll * (ll + 1.0)));
    Bc = L1 * sqrt((ll * ll - mm * mm) * (ll * ll - nn * nn)) / (ll * den);
}

// Rescaled recurrence.  With d(l0+t) = sig[t] e(t), sig[0] = sig[1] = 1 and
// sig[t+1] = Bc_{l0+t} sig[t-1], the recurrence above becomes
//   e(t+1) = (A'[t] x - Ac'[t]) e(t) - e(t-1),   A'[t] = A sig[t]/sig[t+1], Ac'[t] = Ac sig[t]/sig[t+1],
// i.e. two FP64 operations per step instead of three; the factor sig[t] is
// applied where d meets the data (V_l in the forward, the coefficients in the
// inverse).  Builds rA = A', rAc = Ac', rSig = sig for t < L in shared memory
// (rBc is scratch) and multiplies rV[t] by sig[t] if rV is given.  Called by
// all NT threads; ends with a barrier.
template <int NT>
__device__ inline void scaled_recurrence_tables(int l0, int L, int m, int mp, double *rA, double *rAc, double *rBc,
                                                double *rSig, double *rV) {
    const int tid = threadIdx.x;
    for (int t = tid; t < L; t += NT) {
        double a, ac, bc;
        recurrence_coeffs(l0 + t, m, mp, a, ac, bc);
        rA[t] = a; rAc[t] = ac; rBc[t] = bc;
    }
    __syncthreads();
    if (tid < 2) {  // the two parity chains of sig, one thread each
        double sg = 1.0;
        for (int t = tid; t < L; t += 2) {
            if (t >= 2) sg *= rBc[t - 1];
            rSig[t] = sg;
        }
    }
    __syncthreads();
    for (int t = tid; t < L; t += NT) {
        if (t + 1 < L) {
            const double r = rSig[t] / rSig[t + 1];
            rA[t] *= r;
            rAc[t] *= r;
        }
        if (rV) rV[t] *= rSig[t];
    }
    __syncthreads();
}

// Per-cluster recurrence tables in shared memory for cluster cidx: copied from
// the plan's precomputed table when there is one, computed otherwise.  Same
// contract as scaled_recurrence_tables (rBc is scratch; ends with a barrier).
template <int NT>
__device__ inline void cluster_recurrence(const Tables &tb, int cidx, int l0, int L, int m, int mp, double *rA,
                                          double *rAc, double *rBc, double *rSig, double *rV) {
    if (tb.rectab) {
        const double *src = tb.rectab + (size_t)cidx * tb.B * 3;
        for (int t = threadIdx.x; t < L; t += NT) {
            rA[t] = src[3 * t];
            rAc[t] = src[3 * t + 1];
            const double sg = src[3 * t + 2];
            rSig[t] = sg;
            if (rV) rV[t] *= sg;
        }
        __syncthreads();
    } else {
        scaled_recurrence_tables<NT>(l0, L, m, mp, rA, rAc, rBc, rSig, rV);
    }
}

// Seed d(l0, m, m'; beta_j), l0 = max(|m|,|m'|), for a representative m >= m' >= 0
// (the "+" case of the paper's first initial condition):
//   d(m, m, m') = sqrt((2m)! / ((m+m')!(m-m')!)) cos(b/2)^(m+m') sin(b/2)^(m-m'),
// evaluated as exp of its logarithm so that neither the factorials nor the
// powers leave the FP64 range; values below ~1e-308 flush to 0.
__device__ inline double seed_rep(int m, int mp, double lognorm, double lc, double ls) {
    double lg = lognorm;
    if (m + mp > 0) lg = fma((double)(m + mp), lc, lg);
    if (m - mp > 0) lg = fma((double)(m - mp), ls, lg);
    return exp(lg);
}

__device__ inline double seed_lognorm(const Tables &tb, int m, int mp) {
    return 0.5 * (tb.lfact[2 * m] - tb.lfact[m + mp] - tb.lfact[m - mp]);
}

// Seed of cluster cidx at beta_j, times w_B(j) when `weighted` (the forward's
// T W): from the plan's table, or exp of the log-domain seed.
__device__ inline double cluster_seed(const Tables &tb, int cidx, int j, int m, int mp, double lognorm, bool weighted) {
    if (tb.seedtab) {
        const double sd = tb.seedtab[(size_t)cidx * 2 * tb.B + j];
        return weighted ? sd * tb.w[j] : sd;
    }
    return seed_rep(m, mp, weighted ? lognorm + tb.lw[j] : lognorm, tb.lcos[j], tb.lsin[j]);
}

// Per-CTA cluster prologue: the partner table and the partners' run offsets,
// written by thread 0 into shared memory (the caller synchronises).
struct ClusterSmem {
    int np;
    int pm[8], pmp[8], mir[8], lpar[8];
    double sign[8];
    int64_t off[8];
};

// Fills cs for representative (m, m'); called by one thread.
__device__ inline void fill_cluster(const Tables &tb, int m, int mp, ClusterSmem &cs) {
    const Partners P = make_partners(m, mp);
    cs.np = P.np;
    for (int p = 0; p < 8; ++p) {
        const bool on = p < P.np;
        cs.pm[p] = on ? P.m[p] : 0;
        cs.pmp[p] = on ? P.mp[p] : 0;
        cs.mir[p] = on ? P.mirror[p] : 0;
        cs.lpar[p] = on ? P.lpar[p] : 0;
        cs.sign[p] = on ? P.sign[p] : 0.0;
        cs.off[p] = on ? tb.runoff[runoff_index(tb.B, P.m[p], P.mp[p])] : 0;
    }
}

__device__ inline void load_cluster(const Tables &tb, int m, int mp, ClusterSmem &cs) {
    if (threadIdx.x == 0) fill_cluster(tb, m, mp, cs);
}

// Scalings applied by the DWT kernels.  The transforms use
//   forward  f = V T W E x       (DWT with kApplyW | kApplyV)
//   inverse  x = E^H T^T f       (iDWT with no flag)
// and their adjoints, with the same kernels,
//   forward^H  = E^H W T^T V     (iDWT with kApplyV on the coefficients, kApplyW on S)
//   inverse^H  = T E             (DWT with no flag).
// kRealSym (FP64 kernels): the grid is real, so f(l,-m,-m') =
// (-1)^(m-m') conj f(l,m,m') and S(-m,-m';j) = conj S(m,m';j); of each
// conjugate pair of partners (2k, 2k+1) only 2k is contracted and 2k+1 is
// written from it (the forward writes its coefficients, the iDWT its S).
enum DwtFlags : int { kApplyW = 1, kApplyV = 2, kRealSym = 4 };

// One transform of a batch for the persistent FP64 DWT / iDWT kernels.
struct BatchXform {
    Tables tb;
    const double *coef;  // iDWT: interleaved complex coefficients (input)
    double2 *S;          // iDWT: the plan's S workspace, layout [j][m][m'] (output)
    const double2 *Sin;  // DWT: the plan's S after the forward FFT (input)
    double *coef_out;    // DWT: interleaved complex coefficients (output)
    int flags;
};
// Persistent launches over (transform, cluster) items of every bandwidth.
cudaError_t launch_idwt_fp64_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                                        cudaStream_t s);
cudaError_t launch_dwt_fp64_persistent(const BatchXform *xf, const int2 *items, int nitems, int *counter, int maxB,
                                       cudaStream_t s);

// Launchers (shard.cu): S columns of `ncols` order pairs (device list) over
// slices j0 .. j0 + nslices - 1, to / from a dense [nslices][ncols] buffer.
cudaError_t launch_gather_columns(const double2 *S, int B, int j0, int nslices, const int2 *cols, int ncols,
                                  double2 *out, cudaStream_t s);
cudaError_t launch_scatter_columns(const double2 *in, int B, int j0, int nslices, const int2 *cols, int ncols,
                                   double2 *S, cudaStream_t s);

// Launchers (correlate.cu).
cudaError_t launch_corr_coeffs(int B, const double2 *f, const double2 *g, const int64_t *runoff, double2 *coef,
                               cudaStream_t s);
cudaError_t launch_argmax_real(const double2 *data, int64_t count, double *scratch_v, int64_t *scratch_i,
                               int64_t *index_out, double *value_out, cudaStream_t s);
int argmax_parts();

// Records the detail returned by soft_last_error() on this host thread (soft_api.cu).
void set_last_error_message(const char *where, const char *what);

// Launchers (dwt_fp64.cu).
cudaError_t launch_dwt_forward_fp64(const Tables &tb, const double2 *S, double2 *coef, cudaStream_t s,
                                    int flags = kApplyW | kApplyV);
cudaError_t launch_dwt_inverse_fp64(const Tables &tb, const double2 *coef, double2 *S, cudaStream_t s,
                                    int flags = 0);
cudaError_t launch_zero_nyquist(int B, double2 *S, cudaStream_t s);
// Builds tb's per-cluster seed and recurrence tables into seedtab / rectab.
cudaError_t launch_cluster_tables(const Tables &tb, double *seedtab, double *rectab, cudaStream_t s);
int dwt_forward_fp64_variants(int B);
int dwt_inverse_fp64_variants(int B);
// Double-float 2-D FFT of `nslices` consecutive beta slices (fft_df.cu), for
// power-of-two 2B: `in` [j][i][k] FP64 -> `out` [j][m][m'] FP64, exp(sign i
// ...), unnormalised; `work` (nslices n^2 x 16 bytes) may alias `in` or `out`;
// `rexp`: nslices n ints of scratch; all at the range's first slice.
bool df_fft_supported(int B);
cudaError_t launch_df_twiddles(int B, float4 *tw, cudaStream_t s);
cudaError_t launch_df_fft2(int B, const double2 *in, double2 *out, float4 *work, const float4 *tw, int sign,
                           int *rexp, cudaStream_t s, int nslices);
// Its half-spectrum forms for real grids (B >= 2): real `in` -> columns
// m' = 0..B-1 of every slice of S (the rest untouched; S's memory is the
// double-float work buffer), and the Hermitian S's columns 0..B-1
// (overwritten) -> the real `out`.  `rexp` / `cexp`: n^2 / n B ints of scratch.
bool df_real_fft_supported(int B);
cudaError_t launch_df_fft2_r2c(int B, const double *in, double2 *S, const float4 *tw, int sign, int *rexp,
                               cudaStream_t s);
cudaError_t launch_df_fft2_c2r(int B, double2 *S, double *out, const float4 *tw, int sign, int *cexp,
                               cudaStream_t s);
// FP64 2-D FFT of `nslices` consecutive beta slices (fft_fp64.cu), for
// power-of-two 2B: same layouts and sign convention; `out` may be `in`; both
// at the range's first slice.  The twiddle table holds
// fft64_twiddle_count(B) entries (the + table, then the - table), each
// w = exp(i theta) factored as m (1 + i tau) (swap = 0; m1 = m2 = m) or
// i m (1 + i tau) (swap = 1; m1 = -m, m2 = m), |tau| <= 1.
struct FftTw64 {
    double tau, m1, m2;
    int swap, pad;
};
bool fft64_supported(int B);
size_t fft64_twiddle_count(int B);
cudaError_t launch_fft64_twiddles(int B, FftTw64 *tw, cudaStream_t s);
cudaError_t launch_fft64_2d(int B, const double2 *in, double2 *out, const FftTw64 *tw, int sign, cudaStream_t s,
                            int nslices);
// All 2B slices of a real grid `in` ((2B)^3 doubles) into the complex `out`.
cudaError_t launch_fft64_2d_from_real(int B, const double *in, double2 *out, const FftTw64 *tw, int sign,
                                      cudaStream_t s);
// All 2B slices of a complex `in` with a real result (Hermitian input): `in`
// is overwritten and the real parts go to `out` ((2B)^3 doubles).
cudaError_t launch_fft64_2d_to_real(int B, double2 *in, double *out, const FftTw64 *tw, int sign, cudaStream_t s);
// Half-spectrum forms for real grids: real `in` -> columns m' = 0..B-1 of
// every slice of S (the rest untouched), and the Hermitian S's columns
// 0..B-1 (overwritten) -> the real `out`.
cudaError_t launch_fft64_2d_r2c(int B, const double *in, double2 *S, const FftTw64 *tw, int sign, cudaStream_t s);
cudaError_t launch_fft64_2d_c2r(int B, double2 *S, double *out, const FftTw64 *tw, int sign, cudaStream_t s);
// FP64-accurate tensor-core DWT / iDWT (dwt_fp64tc.cu); same S layout and
// flags as the FP64 launchers; need the plan's per-cluster tables.
cudaError_t launch_dwt_forward_tc(const Tables &tb, const double2 *S, double2 *coef, cudaStream_t s,
                                  int flags = kApplyW | kApplyV);
cudaError_t launch_dwt_inverse_tc(const Tables &tb, const double2 *coef, double2 *S, cudaStream_t s,
                                  int flags = 0);
cudaError_t launch_tables(int B, double *w, double *cosb, double *lcos, double *lsin, double *lfact,
                          cudaStream_t s);

// Launchers (dwt_mixed.cu); mode is SOFT_MIXED_BF16X3 or SOFT_MIXED_TF32.
cudaError_t launch_log_weights(int B, const double *w, double *lw, cudaStream_t s);
cudaError_t launch_dwt_forward_mixed(int mode, const Tables &tb, const double *lw, const float2 *S, double *coef,
                                     cudaStream_t s, int flags = kApplyW | kApplyV);
cudaError_t launch_dwt_inverse_mixed(int mode, const Tables &tb, const double *coef, float2 *S, cudaStream_t s,
                                     int flags = 0);
// nb (1, 2, 4 or 8) transforms of one bandwidth in one launch: the generated
// Wigner-d tile feeds N = 16 nb tensor-core columns.
cudaError_t launch_dwt_forward_mixed_batch(int mode, const Tables &tb, int nb, const float2 *const *S,
                                           double *const *coef, cudaStream_t s, int flags = kApplyW | kApplyV);
cudaError_t launch_dwt_inverse_mixed_batch(int mode, const Tables &tb, int nb, const double *const *coef,
                                           float2 *const *S, cudaStream_t s, int flags = 0);
cudaError_t launch_zero_nyquist32(int B, float2 *S, cudaStream_t s);
cudaError_t launch_bounded_wait_selftest(uint32_t polls, int *err, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double2 *in, float2 *out, int64_t count, cudaStream_t s);
cudaError_t launch_transpose32(const float2 *X, float2 *Y, int rows, int64_t cols, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float2 *in, double2 *out, int64_t count, cudaStream_t s);

}  // namespace softgb
