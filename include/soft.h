/*
 * soft.h -- C ABI of the GB300 library for the fast Fourier transform on SO(3)
 * (the Kostelec-Rockmore FSOFT and its inverse, as reviewed and parallelised in
 * Lux, Wuelker, Chirikjian, "Parallelization of the FFT on SO(3)",
 * arXiv:1808.00896).
 *
 * Every entry point takes plain pointers and sizes; there are no C++ or torch
 * types in the signatures.  Errors are reported by return code only: nothing
 * aborts, throws or traps.  Unless an entry point says otherwise, all data
 * pointers are DEVICE pointers on the plan's device, owned by the caller,
 * 16-byte aligned, and must not overlap each other.  Inputs are never
 * modified.  Calls are asynchronous on the given stream (a cudaStream_t passed
 * as void*; NULL = the legacy default stream); the returned status covers
 * argument checks and launch errors, and a device-side error word is checked
 * by soft_plan_sync().
 *
 * Data layouts (the paper fixes the math, not the memory layout):
 *
 *   grid  -- (2B)^3 complex doubles (interleaved re, im), index [j][i][k]:
 *            grid[(j*2B + i)*2B + k] = f(alpha_i, beta_j, gamma_k) with the
 *            sampling angles of Eq. (quadrature): alpha_i = i*pi/B,
 *            beta_j = (2j+1)*pi/(4B), gamma_k = k*pi/B.  beta is slowest, so
 *            each beta slice is one contiguous 2B x 2B array.
 *
 *   coef  -- B(4B^2-1)/3 complex doubles, the Fourier coefficients f(l,m,m')
 *            of Eq. (fourier_representation).  For m = 1-B..B-1 (outer) and
 *            m' = 1-B..B-1 (inner) the run l = max(|m|,|m'|)..B-1 is
 *            contiguous; soft_coef_index() gives the offset of any entry.
 *
 *   S     -- (2B)^3 complex doubles, index [j][m mod 2B][m' mod 2B]: the
 *            separated sums S(m,m';j) of Sec. 2.4 (the output of the 2-D FFT
 *            of each beta slice); entries with m or m' = -B (index B) are 0.
 */
#ifndef SOFT_GB300_SOFT_H
#define SOFT_GB300_SOFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct soft_plan_s *soft_plan; /* opaque; created and owned by the library */

typedef enum {
    SOFT_OK = 0,
    SOFT_ERR_INVALID_ARG = 1,   /* bad B, NULL or misaligned pointer, bad dtype, stale plan */
    SOFT_ERR_OUT_OF_MEMORY = 2, /* device or pinned-host allocation failed */
    SOFT_ERR_CUDA = 3,          /* a CUDA runtime or cuFFT call failed */
    SOFT_ERR_UNSUPPORTED = 4,   /* B above soft_max_bandwidth(), or a mode not built */
    SOFT_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    SOFT_ERR_DEVICE = 6         /* a kernel flagged an internal inconsistency */
} soft_status;

typedef enum {
    SOFT_FP64 = 0,         /* every step in FP64 */
    SOFT_MIXED_BF16X3 = 1, /* contraction on tcgen05 tensor cores, split BF16 x3 (rel-L2 <= 5e-5) */
    SOFT_MIXED_TF32 = 2,   /* contraction on tcgen05 tensor cores, TF32 (rel-L2 <= 2e-3) */
    SOFT_FP64_TC = 3       /* FP64 recurrence and S; 2-D FFTs in double-float arithmetic (pairs of
                            * floats, ~48 bits; cuFFT Z2Z when 2B is not a power of two); contraction
                            * on tcgen05 tensor cores as exact fixed-point BF16 digit products (7
                            * base-128 digits per operand, FP32 TMEM sums exact for the leading
                            * levels); FP64 accuracy (rel-L2 <= 1e-10) */
} soft_dtype;

/* Largest bandwidth B the kernels accept. */
int soft_max_bandwidth(void);

/* Number of this library's kernels launched in the process so far, over all
 * plans and devices (monotonic).  The kernels of a batch's CUDA graph count
 * at each replay of the graph (not when it is captured).  Kernels that cuFFT
 * runs are not counted.  Thread-safe. */
unsigned long long soft_launch_count(void);

/* Number of device allocations the library holds right now, over all plans,
 * batch graphs and devices (each plan buffer, staging buffer and workspace
 * counts one).  Every failure path frees what it allocated, so the count
 * returns to its earlier value once the plans involved are destroyed.
 * Test support, not from the paper; with it goes a failure-injection hook:
 * when the environment variable SOFT_TEST_ALLOC_BUDGET=N is set at
 * soft_plan_create, that plan may make N device allocations in all (at
 * creation and later, e.g. the host-call staging buffers or the correlation
 * workspace) and the next one fails with SOFT_ERR_OUT_OF_MEMORY.  Unset, it
 * has no effect.  Thread-safe. */
long long soft_live_allocations(void);

/* Number of Fourier coefficients with l < B: B(4B^2-1)/3 (Sec. 2.4).
 * Returns -1 for B < 1. */
int64_t soft_num_coeffs(int B);

/* Offset of f(l,m,m') in the coefficient array for bandwidth B, or -1 when
 * not (max(|m|,|m'|) <= l < B). Host function, no device work. */
int64_t soft_coef_index(int B, int l, int m, int mp);

/* Human-readable name of a status code (static string, never NULL). */
const char *soft_status_string(int status);

/* Detail of the most recent failing call on this host thread (which CUDA or
 * cuFFT call failed and its error text); "" when none.  Valid until the next
 * library call on the same thread. */
const char *soft_last_error(void);

/* Create a plan for bandwidth B on the current CUDA device.  Allocates the
 * plan's device workspace ((2B)^3 complex doubles for S -- mixed plans: S and
 * a grid copy in complex floats instead --, 5B doubles of seeds and rescaled
 * recurrence coefficients per symmetry cluster, 2.7 GB at B = 512, and small
 * beta tables; SOFT_FP64_TC plans add 2 ints per order pair and (2B)^2 ints
 * of FFT scales),
 * builds the slice-FFT tables (FP64 and FP64-TC plans: the library's own FFT
 * when 2B is a power of two, else a cuFFT plan; mixed plans: FP32 cuFFT
 * plans) and computes the quadrature weights of Eq. (weights)
 * and the other beta tables on the device.  *out receives the handle, or NULL
 * on failure.  Returns SOFT_ERR_INVALID_ARG for B < 1 or out == NULL,
 * SOFT_ERR_UNSUPPORTED for B > soft_max_bandwidth() or an unbuilt dtype. */
soft_status soft_plan_create(soft_plan *out, int B, int dtype);

/* Release a plan and everything it owns.  NULL is accepted (no-op).
 * Synchronises the plan's device first. */
soft_status soft_destroy(soft_plan p);

/* Bandwidth of a plan, or -1 for NULL. */
int soft_plan_bandwidth(soft_plan p);

/* Wait for all work on the plan's device and read (and clear) the device
 * error word: SOFT_ERR_TIMEOUT if a tensor-core kernel's bounded wait gave up
 * since the last call (its results are then not to be used; the context stays
 * usable), SOFT_ERR_DEVICE if a kernel flagged another inconsistency. */
soft_status soft_plan_sync(soft_plan p);

/* Forward transform (FSOFT, Sec. 2.4): grid (device, (2B)^3 complex) ->
 * coef (device, B(4B^2-1)/3 complex), f(l,m,m') of Eq. (quadrature):
 *   2-D FFT of every beta slice (exp(+i...)) into the plan's S,
 *   then the DWT f = V_B T_B W_B S for every order pair (m,m').       */
soft_status soft_forward(soft_plan p, const double *grid, double *coef, void *stream);

/* Inverse transform (iFSOFT, Sec. 2.4): coef -> grid, the function values of
 * Eq. (fourier_representation) on the sampling grid:
 *   iDWT S = T_B^T f for every (m,m') into the plan's S, then 2-D FFT of
 *   every beta slice (exp(-i...)).                                      */
soft_status soft_inverse(soft_plan p, const double *coef, double *grid, void *stream);

/* Real grids (SOFT_FP64 and SOFT_FP64_TC plans with power-of-two 2B;
 * SOFT_ERR_UNSUPPORTED otherwise).  A real function has f(l,-m,-m') =
 * (-1)^(m-m') conj f(l,m,m') (from the symmetries of Eq. (Wigner_symmetries)),
 * and S(-m,-m';j) = conj S(m,m';j).  In each symmetry cluster the partners
 * come in such conjugate pairs, and these calls contract one partner of each
 * pair: half the DWT / iDWT contraction work.  Every contracted partner has
 * m' >= 0, so the slice FFTs (FP64 for SOFT_FP64 plans, double-float for
 * SOFT_FP64_TC plans with B >= 2, as their complex-grid FFTs) run on that
 * half of the spectrum: real-row DFTs of half length, and the column DFTs of
 * m' = 0..B-1 only.
 *   soft_forward_real: grid (device, (2B)^3 doubles, layout [j][i][k] as the
 *     complex grid) -> coef (device, B(4B^2-1)/3 complex), the same values as
 *     soft_forward of the grid with zero imaginary parts (the conjugate
 *     partners' coefficients are written from their pair exactly).
 *   soft_inverse_real: coef -> grid (device, (2B)^3 doubles), the real part
 *     of soft_inverse.  It reads only the coefficients of the contracted
 *     partners, so the others are taken to satisfy the symmetry whatever they
 *     hold; coefficients from soft_forward_real (or of any real function) do.
 * Both 16-byte aligned, as soft_forward / soft_inverse; asynchronous on
 * `stream`. */
soft_status soft_forward_real(soft_plan p, const double *grid, double *coef, void *stream);
soft_status soft_inverse_real(soft_plan p, const double *coef, double *grid, void *stream);

/* Adjoints, for gradients of objectives through the transforms.  Adjoint is
 * with respect to sum_k conj(a_k) b_k on both sides.  Writing the forward
 * transform as f = V_B T_B W_B E x (Sec. 2.4; E the per-slice 2-D DFT with
 * exp(+i...)) and the inverse as x = E^H T_B^T f:
 *   soft_forward_adjoint:  coef -> grid,  E^H W_B T_B^T V_B  (iDWT with V on
 *                          the coefficients and W on S, then the exp(-i) FFT)
 *   soft_inverse_adjoint:  grid -> coef,  T_B E  (the exp(+i) FFT, then the
 *                          DWT without V and W)
 * Same pointer rules and precision mode as the plan's forward/inverse. */
soft_status soft_forward_adjoint(soft_plan p, const double *coef, double *grid, void *stream);
soft_status soft_inverse_adjoint(soft_plan p, const double *grid, double *coef, void *stream);

/* Rotational correlation (fast rotational matching, which motivates the paper
 * in Sec. 1; the paper gives no formula, the identity below is checked by
 * brute force in the tests).  f_sh, g_sh: device, B^2 complex doubles each,
 * the spherical-harmonic coefficients of two functions on the sphere (index
 * l*l + m + l, l < B, orthonormal Y_lm with the Condon-Shortley phase).
 *   soft_correlation_coeffs: coef(l,m,m') = g_lm conj(f_lm'), the SO(3)
 *     Fourier coefficients of C(R) = int g(R^{-1} w) conj(f(w)) dw.
 *   soft_correlate: the same, then the inverse transform into grid (device,
 *     (2B)^3 complex): grid[j][i][k] = C(R_z(gamma_k) R_y(beta_j) R_z(alpha_i));
 *     if best_index / best_value (device int64 / double) are non-NULL, also
 *     the arg-max of Re C over the grid (linear index j*(2B)^2 + i*2B + k,
 *     lowest index on ties, NaN never wins).  The first call allocates the
 *     plan's coefficient workspace (B(4B^2-1)/3 complex doubles). */
soft_status soft_correlation_coeffs(soft_plan p, const double *f_sh, const double *g_sh, double *coef, void *stream);
soft_status soft_correlate(soft_plan p, const double *f_sh, const double *g_sh, double *grid, int64_t *best_index,
                           double *best_value, void *stream);

/* Batches: n transforms with n DISTINCT plans (any mix of bandwidths and
 * modes; each plan lends its workspace), one pointer per entry in host arrays
 * of device pointers.  The first call with a given (plans, pointers) captures
 * the whole batch into a CUDA graph on a private stream (instantiated once,
 * cached, most recent 16 kept; destroying a member plan drops it) and every
 * call replays it on `stream`.  The SOFT_FP64 transforms of a batch, of any
 * bandwidths, share one persistent DWT (forward) or iDWT (inverse,
 * correlation) launch that schedules all their (transform, symmetry cluster)
 * work items, heaviest first, through an atomic counter, in the tile shape of
 * the batch's largest B (iDWT results equal the per-plan calls' bit for bit;
 * DWT results equal them bit for bit when that shape is the plan's own, else
 * to rounding); mixed-precision transforms of one (mode, B) share one
 * tensor-core launch per group of up to 8; SOFT_FP64_TC entries run their
 * per-plan kernels inside the same graph.
 *   soft_batched_inverse:   coefs[i] -> grids[i]
 *   soft_batched_forward:   grids[i] -> coefs[i]
 *   soft_batched_correlate: (f_sh[i], g_sh[i]) -> grids[i] = C_i on the Euler
 *                           grid, best_index[i] / best_value[i] (device arrays
 *                           of n) = arg-max of Re C_i, as soft_correlate.
 * Make the first call outside any stream capture of the caller's. */
soft_status soft_batched_inverse(int n, const soft_plan *plans, const double *const *coefs, double *const *grids,
                                 void *stream);
soft_status soft_batched_forward(int n, const soft_plan *plans, const double *const *grids, double *const *coefs,
                                 void *stream);
soft_status soft_batched_correlate(int n, const soft_plan *plans, const double *const *f_sh,
                                   const double *const *g_sh, double *const *grids, int64_t *best_index,
                                   double *best_value, void *stream);

/* Arg-max of the real parts of count complex doubles (device), lowest index on
 * ties, NaN never wins: *index_out / *value_out (device).  scratch: device,
 * soft_argmax_scratch_doubles() doubles, 16-byte aligned. */
soft_status soft_argmax_real(const double *data, int64_t count, int64_t *index_out, double *value_out,
                             double *scratch, void *stream);
int soft_argmax_scratch_doubles(void);

/* The DWT step alone (Sec. 2.4, matrix form V_B T_B W_B): S (device, layout
 * above) -> coef.  S is read only.  SOFT_FP64 and SOFT_FP64_TC plans only
 * (SOFT_ERR_UNSUPPORTED for mixed plans, whose S is FP32 in another layout). */
soft_status soft_dwt_forward(soft_plan p, const double *S, double *coef, void *stream);

/* The iDWT step alone (Sec. 2.4, T_B^T): coef -> S (device, layout above,
 * every entry written, the -B rows/columns set to 0).  SOFT_FP64 and
 * SOFT_FP64_TC plans only. */
soft_status soft_dwt_inverse(soft_plan p, const double *coef, double *S, void *stream);

/* The DWT step alone, without a plan and without allocating any memory
 * (the paper has no counterpart: this is a deployment variant of
 * soft_dwt_forward).  For callers that cannot call cudaMalloc -- a plug-in
 * whose host application owns the whole device memory pool, or a fixed-budget
 * pipeline that allocates only at start-up and cannot take cudaMalloc's
 * implicit synchronisation later -- and so cannot create a plan.
 * S (device, layout above, read only) -> coef (device), bandwidth B on the
 * current device, asynchronous on `stream`; same result as soft_dwt_forward.
 * Its working tables live in a fixed 2.3 MiB static device array that every
 * GPU loading the library keeps until exit; they are rebuilt on `stream` at
 * every call.  Limits and rules:
 *   - B must be <= 256; larger B returns SOFT_ERR_UNSUPPORTED (detail in
 *     soft_last_error()).
 *   - The first call on a device looks up the array's device address (one-time
 *     set-up); make that first call before any stream capture.  A failed
 *     lookup returns SOFT_ERR_CUDA (detail in soft_last_error()) and is not
 *     kept: the next call tries again.
 *   - All calls share the array: calls whose GPU work overlaps (different
 *     streams, or devices sharing it) race and must be serialised by the caller.
 *   - The FP64 DWT kernel it runs has no device-side failure mode (no waits,
 *     no internal checks), so there is no device error word to read: the
 *     returned status covers arguments, set-up and launches.
 *   - No cudaMalloc, cudaFree or allocating library call is made. */
soft_status soft_dwt_forward_noalloc(int B, const double *S, double *coef, void *stream);

/* Sharding one transform over several GPUs (the beta <-> order-pair exchange:
 * the slice FFTs need every order pair of a few beta slices, the DWT every
 * beta slice of a few order pairs; Sec. 2.4's two steps, and Sec. 3's
 * partition of the DWTs by symmetry cluster).  Rank r of R owns the beta
 * slices [floor(r 2B / R), floor((r+1) 2B / R)) and the symmetry clusters
 * soft_cluster_shard() assigns it; one all-to-all between the two steps
 * moves the S columns (the caller's collective, e.g. NCCL through
 * torch.distributed).  The paper does not shard a single transform; its
 * parallelism is over clusters on one machine.
 *
 *   soft_cluster_shard: host function.  The representatives (m, m'),
 *     m >= m' >= 0, of the clusters rank `rank` of `nranks` owns, into
 *     reps_out[2i], reps_out[2i+1] (room for B(B+1)/2 pairs), their number
 *     into *count_out: the clusters by decreasing work ((B - m) degrees x
 *     (8 partners first)), each to the rank with the least work so far (ties
 *     to the lowest rank).  Every cluster goes to exactly one rank.
 *   soft_cluster_columns: host function.  The order pairs (m, m') of the
 *     given clusters' partners, in cluster order and each cluster's partner
 *     order, into pairs_out[2i], pairs_out[2i+1] (room for 8 count pairs);
 *     returns their number (the S columns those clusters read and write).
 *   soft_dwt_forward_clusters / soft_dwt_inverse_clusters: the DWT / iDWT of
 *     the listed clusters only (reps: host array of `count` representatives):
 *     the forward writes those clusters' coefficient runs and nothing else of
 *     coef; the inverse writes those clusters' S columns at every beta slice
 *     and sets the m = -B and m' = -B entries to 0 at every slice, and writes
 *     nothing else of S.  S in the full (2B)^3 layout.  SOFT_FP64 and
 *     SOFT_FP64_TC plans.  Results are those of soft_dwt_forward /
 *     soft_dwt_inverse for the same clusters, bit for bit.
 *   soft_gather_columns: out[js][c] = S[j0 + js][m_c][m'_c] for js < nslices
 *     and the `npairs` order pairs (host array pairs[2c], pairs[2c+1]);
 *     out: device, nslices x npairs complex doubles.
 *   soft_scatter_columns: the reverse, S[j0 + js][m_c][m'_c] = in[js][c].
 *   soft_slice_fft: the 2-D FFT of slices j0 .. j0 + nslices - 1 (sign +1:
 *     grid -> S with exp(+i...), the forward's; -1: S -> grid with exp(-i...),
 *     the inverse's; unnormalised), `in` and `out` pointing at slice j0 of
 *     their arrays (they may be arrays of just those slices).  SOFT_FP64 and
 *     SOFT_FP64_TC plans with power-of-two 2B.
 * All asynchronous on `stream`; pointer rules as soft_forward. */
soft_status soft_cluster_shard(int B, int nranks, int rank, int *reps_out, int *count_out);
int soft_cluster_columns(int count, const int *reps, int *pairs_out);
soft_status soft_dwt_forward_clusters(soft_plan p, const double *S, double *coef, const int *reps, int count,
                                      void *stream);
soft_status soft_dwt_inverse_clusters(soft_plan p, const double *coef, double *S, const int *reps, int count,
                                      void *stream);
soft_status soft_gather_columns(soft_plan p, const double *S, int j0, int nslices, const int *pairs, int npairs,
                                double *out, void *stream);
soft_status soft_scatter_columns(soft_plan p, const double *in, int j0, int nslices, const int *pairs, int npairs,
                                 double *S, void *stream);
soft_status soft_slice_fft(soft_plan p, const double *in, double *out, int sign, int j0, int nslices, void *stream);

/* Host-buffer forms: grid_host / coef_host are HOST pointers (pageable or
 * pinned).  The call copies the input to plan-owned device staging buffers
 * (allocated on first use), runs the transform on `stream`, copies the
 * result back and synchronises the stream before returning.  For SOFT_FP64
 * and SOFT_FP64_TC plans with power-of-two 2B the grid's copies overlap the
 * 2-D FFTs, in chunks of beta slices, on a second stream that the plan owns
 * (created on first use); the call then synchronises both streams before it
 * returns, also after an error, so no copy into the caller's buffers is left
 * in flight.  Results are identical to soft_forward / soft_inverse on the
 * same data.  Overlapping the copies needs pinned host memory. */
soft_status soft_forward_host(soft_plan p, const double *grid_host, double *coef_host, void *stream);
soft_status soft_inverse_host(soft_plan p, const double *coef_host, double *grid_host, void *stream);

/* Tile-shape variants, for autotuning (not from the paper).  kernel 0 is the
 * DWT, 1 the iDWT.  soft_plan_num_variants returns how many shapes exist for
 * the plan's bandwidth and mode (-1 for a bad plan or kernel); variant 0 is
 * the built-in default.  soft_plan_set_variant selects one for all later
 * calls on the plan (SOFT_ERR_INVALID_ARG if out of range).  Results do not
 * depend on the variant beyond rounding order. */
int soft_plan_num_variants(soft_plan p, int kernel);
soft_status soft_plan_set_variant(soft_plan p, int kernel, int variant);

/* Failure-detection self-test (not from the paper).  Every wait inside the
 * tensor-core kernels is a bounded poll of an mbarrier; when it runs out the
 * kernel stops its work, records a timeout in the plan's device error word and
 * returns, so the CUDA context stays usable and soft_plan_sync() reports
 * SOFT_ERR_TIMEOUT.  This entry point runs that same bounded wait on an
 * mbarrier that nothing arrives on, limited to `polls` polls (1..2^20), so the
 * path can be exercised without a real failure.  Asynchronous on `stream`. */
soft_status soft_selftest_bounded_wait(soft_plan p, int polls, void *stream);

/* Per-phase timing.  When enabled, every soft_forward / soft_inverse (and
 * soft_forward_real / soft_inverse_real) records
 * CUDA events (on the call's stream) around its 2-D FFT and its (i)DWT
 * kernel(s); soft_plan_read_timing() waits for them, adds up the elapsed
 * times since the last read and resets the sums.  ms_out[4] receives the
 * milliseconds spent in {forward FFT, DWT, iDWT (with the S clearing),
 * inverse FFT}; counts_out[4] the number of timed launches of each (either
 * pointer may be NULL).  Up to 4096 calls are held between two reads; a call
 * that finds 4096 pending first waits for them and folds them into the sums. */
soft_status soft_plan_enable_timing(soft_plan p, int on);
soft_status soft_plan_read_timing(soft_plan p, double *ms_out, int64_t *counts_out);

#ifdef __cplusplus
}
#endif

#endif /* SOFT_GB300_SOFT_H */
