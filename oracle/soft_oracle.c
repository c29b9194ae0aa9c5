/*
 * soft_oracle.c -- plain, slow FP64 CPU oracle for the fast Fourier transform
 * on SO(3) (Kostelec-Rockmore SOFT, as reviewed in Lux, Wuelker, Chirikjian,
 * "Parallelization of the FFT on SO(3)", arXiv:1808.00896, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library: every formula below is written out again from the paper.
 *
 * Conventions (all from Sec. 2 of the paper):
 *   grid[j][i][k] = f(alpha_i, beta_j, gamma_k), complex, interleaved re/im,
 *     alpha_i = i*pi/B, beta_j = (2j+1)*pi/(4B), gamma_k = k*pi/B  (Eq. quadrature)
 *   coefficient array: for m = 1-B..B-1 (outer), m' = 1-B..B-1 (inner), the
 *     run l = max(|m|,|m'|)..B-1 is contiguous.  (Layout is not in the paper;
 *     it is this library's choice and the oracle rebuilds it by plain counting.)
 *
 * Accumulation is straight FP64 in the order the formulas are written.
 *
 * Threads: when compiled with -fopenmp, the loops over independent order
 * pairs (m,m'), beta slices, sampled pairs and sampled grid points run on
 * oracle_set_threads() threads (1 by default).  Each pair, slice or point is
 * still computed by one thread in the order written above, so the results do
 * not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

static int g_threads = 1;

/* Threads for the parallel loops (clamped to >= 1; ignored without OpenMP). */
void oracle_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int oracle_get_threads(void) { return g_threads; }

/* 1 when the oracle was compiled with OpenMP (its loops then run on threads). */
int oracle_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sampling angles and quadrature weights, Eq. (quadrature) and Eq. (weights) */
/* ------------------------------------------------------------------------ */

double oracle_beta(int B, int j) { return (2.0 * j + 1.0) * OR_PI / (4.0 * B); }
double oracle_alpha(int B, int i) { return i * OR_PI / B; }

/* w_B(j) = (2 pi sin(beta_j) / B^2) * sum_{i<B} sin((2i+1) beta_j) / (2i+1) */
void oracle_weights(int B, double *w)
{
    for (int j = 0; j < 2 * B; ++j) {
        double bj = oracle_beta(B, j);
        double s = 0.0;
        for (int i = 0; i < B; ++i) s += sin((2.0 * i + 1.0) * bj) / (2.0 * i + 1.0);
        w[j] = 2.0 * OR_PI * sin(bj) / ((double)B * B) * s;
    }
}

/* ------------------------------------------------------------------------ */
/* Wigner-d, explicit Jacobi form (Sec. 2.2)                                 */
/* ------------------------------------------------------------------------ */

static double binom_d(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* Jacobi polynomial P_n^{(a,b)}(x) by its explicit finite sum
 * (Abramowitz-Stegun 22.3.1 form): sum_s C(n+a,n-s) C(n+b,s) ((x-1)/2)^s ((x+1)/2)^(n-s). */
double oracle_jacobi(int n, int a, int b, double x)
{
    double xm = 0.5 * (x - 1.0), xp = 0.5 * (x + 1.0), sum = 0.0;
    for (int s = 0; s <= n; ++s)
        sum += binom_d(n + a, n - s) * binom_d(n + b, s) * pow(xm, s) * pow(xp, n - s);
    return sum;
}

/* The explicit form as printed, usable where its exponents are non-negative,
 * i.e. m' >= |m|:
 *   d(l,m,m') = (-1)^(m+m') sqrt((l+m')!(l-m')! / ((l+m)!(l-m)!))
 *               sin(b/2)^(m'-m) cos(b/2)^(m+m') P_{l-m'}^{(m'-m, m+m')}(cos b)      */
static double wigner_d_explicit_region(int l, int m, int mp, double beta)
{
    double lf = 0.5 * (lgamma(l + mp + 1.0) + lgamma(l - mp + 1.0)
                       - lgamma(l + m + 1.0) - lgamma(l - m + 1.0));
    double sgn = ((m + mp) & 1) ? -1.0 : 1.0;
    return sgn * exp(lf) * pow(sin(0.5 * beta), mp - m) * pow(cos(0.5 * beta), m + mp)
           * oracle_jacobi(l - mp, mp - m, m + mp, cos(beta));
}

/* All (m,m') with |m|,|m'| <= l, reduced to the explicit region by the three
 * symmetries of Eq. (Wigner_symmetries) that keep beta fixed:
 *   d(l,m,m') = (-1)^(m-m') d(l,-m,-m') = (-1)^(m-m') d(l,m',m) = d(l,-m',-m).  */
double oracle_wigner_d_explicit(int l, int m, int mp, double beta)
{
    if (l < 0 || abs(m) > l || abs(mp) > l) return 0.0;
    int am = abs(m), amp = abs(mp);
    double par = ((m - mp) & 1) ? -1.0 : 1.0;
    if (amp >= am) {
        if (mp >= 0) return wigner_d_explicit_region(l, m, mp, beta);
        return par * wigner_d_explicit_region(l, -m, -mp, beta);
    }
    if (m >= 0) return par * wigner_d_explicit_region(l, mp, m, beta);
    return wigner_d_explicit_region(l, -mp, -m, beta);
}

/* ------------------------------------------------------------------------ */
/* Wigner-d by the three-term recurrence, Eq. (Wigner_d_recurrence), started */
/* from the paper's initial cases (the four seeds) at l0 = max(|m|,|m'|).    */
/* out[l - l0] = d(l,m,m';beta) for l = l0..B-1.                             */
/* ------------------------------------------------------------------------ */

/* The seed d(l0,m,m';beta), evaluated in the log domain so that the
 * factorials (overflowing past 170!) and the powers (underflowing) stay finite. */
double oracle_wigner_seed(int m, int mp, double beta)
{
    int am = abs(m), amp = abs(mp);
    double c = cos(0.5 * beta), s = sin(0.5 * beta);
    int mu, pc, ps, neg;
    double lognorm;
    if (am >= amp) {
        mu = am; /* l0 = |m|: d(mu, +-mu, m') */
        if (m >= 0) { pc = mu + mp; ps = mu - mp; neg = 0; }       /* cos^(m+m') (+sin)^(m-m') */
        else        { pc = mu - mp; ps = mu + mp; neg = ps & 1; }  /* cos^(m-m') (-sin)^(m+m') */
        lognorm = 0.5 * (lgamma(2.0 * mu + 1.0) - lgamma(mu + mp + 1.0) - lgamma(mu - mp + 1.0));
    } else {
        mu = amp; /* l0 = |m'|: d(mu, m, +-mu) */
        if (mp >= 0) { pc = mu + m; ps = mu - m; neg = ps & 1; }   /* cos^(m'+m) (-sin)^(m'-m) */
        else         { pc = mu - m; ps = mu + m; neg = 0; }        /* cos^(m'-m) (+sin)^(m'+m) */
        lognorm = 0.5 * (lgamma(2.0 * mu + 1.0) - lgamma(mu + m + 1.0) - lgamma(mu - m + 1.0));
    }
    if ((pc > 0 && c == 0.0) || (ps > 0 && s == 0.0)) return 0.0;
    double lg = lognorm;
    if (pc > 0) lg += pc * log(c);
    if (ps > 0) lg += ps * log(s);
    double v = exp(lg);
    return neg ? -v : v;
}

void oracle_wigner_d_column(int B, int m, int mp, double beta, double *out)
{
    int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
    if (l0 >= B) return;
    double x = cos(beta);
    double dprev = 0.0, dcur = oracle_wigner_seed(m, mp, beta);
    out[0] = dcur;
    for (int l = l0; l + 1 < B; ++l) {
        double next;
        if (l == 0) {
            /* only m = m' = 0 starts at l = 0; the recurrence is stated for
             * l >= 1, and d(1,0,0) = cos(beta) closes the gap. */
            next = x * dcur;
        } else {
            double L1 = l + 1.0, ll = l;
            double den = sqrt((L1 * L1 - (double)m * m) * (L1 * L1 - (double)mp * mp));
            double a = L1 * (2.0 * ll + 1.0) / den;
            double c = (double)m * mp / (ll * (ll + 1.0));
            double b = L1 * sqrt((ll * ll - (double)m * m) * (ll * ll - (double)mp * mp)) / (ll * den);
            next = a * (x - c) * dcur - b * dprev;
        }
        out[l + 1 - l0] = next;
        dprev = dcur;
        dcur = next;
    }
}

/* ------------------------------------------------------------------------ */
/* Coefficient layout (a library choice; counted out plainly here)            */
/* ------------------------------------------------------------------------ */

int64_t oracle_num_coeffs(int B) { return (int64_t)B * (4LL * B * B - 1) / 3; }

/* Start of the run of (m,m') in the coefficient array, by plain counting. */
static int64_t run_start(int B, int m, int mp)
{
    int64_t off = 0;
    for (int a = 1 - B; a <= B - 1; ++a)
        for (int b = 1 - B; b <= B - 1; ++b) {
            if (a == m && b == mp) return off;
            int l0 = abs(a) > abs(b) ? abs(a) : abs(b);
            off += B - l0;
        }
    return -1;
}

int64_t oracle_coef_index(int B, int l, int m, int mp)
{
    int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
    if (B < 1 || l < l0 || l >= B) return -1;
    return run_start(B, m, mp) + (l - l0);
}

/* ------------------------------------------------------------------------ */
/* 1-D and 2-D discrete Fourier transforms (own code, unnormalised)          */
/*   X[q] = sum_n x[n] exp(sign * 2 pi i q n / N)                            */
/* Radix-2 Cooley-Tukey for powers of two, the plain O(N^2) sum otherwise.   */
/* ------------------------------------------------------------------------ */

static void dft_plain(int n, double *x, int stride, int sign, double *tmp)
{
    for (int q = 0; q < n; ++q) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < n; ++t) {
            double ang = sign * 2.0 * OR_PI * (double)((int64_t)q * t % n) / n;
            double c = cos(ang), s = sin(ang);
            double xr = x[2 * (int64_t)t * stride], xi = x[2 * (int64_t)t * stride + 1];
            re += xr * c - xi * s;
            im += xr * s + xi * c;
        }
        tmp[2 * q] = re;
        tmp[2 * q + 1] = im;
    }
    for (int q = 0; q < n; ++q) {
        x[2 * (int64_t)q * stride] = tmp[2 * q];
        x[2 * (int64_t)q * stride + 1] = tmp[2 * q + 1];
    }
}

static void fft_radix2(int n, double *x, int stride, int sign, double *tmp)
{
    /* gather into tmp in bit-reversed order */
    int bits = 0;
    while ((1 << bits) < n) ++bits;
    for (int t = 0; t < n; ++t) {
        int r = 0;
        for (int b = 0; b < bits; ++b) r |= ((t >> b) & 1) << (bits - 1 - b);
        tmp[2 * r] = x[2 * (int64_t)t * stride];
        tmp[2 * r + 1] = x[2 * (int64_t)t * stride + 1];
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * OR_PI * k / len;
            double wr = cos(ang), wi = sin(ang);
            for (int s0 = 0; s0 < n; s0 += len) {
                double *u = tmp + 2 * (s0 + k), *v = tmp + 2 * (s0 + k + half);
                double vr = v[0] * wr - v[1] * wi, vi = v[0] * wi + v[1] * wr;
                v[0] = u[0] - vr; v[1] = u[1] - vi;
                u[0] += vr;       u[1] += vi;
            }
        }
    }
    for (int t = 0; t < n; ++t) {
        x[2 * (int64_t)t * stride] = tmp[2 * t];
        x[2 * (int64_t)t * stride + 1] = tmp[2 * t + 1];
    }
}

void oracle_dft1(int n, double *x, int stride, int sign)
{
    double *tmp = (double *)malloc(sizeof(double) * 2 * n);
    if ((n & (n - 1)) == 0) fft_radix2(n, x, stride, sign, tmp);
    else dft_plain(n, x, stride, sign, tmp);
    free(tmp);
}

/* In place on the contiguous n x n slices s = 0, stride, 2 stride, ... < nslices
 * (stride 1: every slice; larger strides only serve timing samples). */
static void dft2_slices_strided(int nslices, int n, double *data, int sign, int stride)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int s = 0; s < nslices; s += stride) {
        double *sl = data + 2 * (int64_t)s * n * n;
        for (int r = 0; r < n; ++r) oracle_dft1(n, sl + 2 * (int64_t)r * n, 1, sign); /* along k */
        for (int c = 0; c < n; ++c) oracle_dft1(n, sl + 2 * (int64_t)c, n, sign);     /* along i */
    }
}

/* In place on each of nslices contiguous n x n slices. */
void oracle_dft2_slices(int nslices, int n, double *data, int sign)
{
    dft2_slices_strided(nslices, n, data, sign, 1);
}

/* ------------------------------------------------------------------------ */
/* Sequential fast transforms, Sec. 2.4                                      */
/* ------------------------------------------------------------------------ */

static int mod_n(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* S(m,m';j) = sum_{i,k} f(alpha_i,beta_j,gamma_k) exp(+i(m alpha_i + m' gamma_k)),
 * i.e. an unnormalised 2-D DFT with the + sign on every beta slice. Stored
 * as S[j][m mod 2B][m' mod 2B]. */
static double *forward_separation(int B, const double *grid, int stride)
{
    int n = 2 * B;
    size_t cnt = (size_t)2 * n * n * n;
    double *S = (double *)malloc(sizeof(double) * cnt);
    if (!S) return NULL;
    memcpy(S, grid, sizeof(double) * cnt);
    dft2_slices_strided(n, n, S, +1, stride);
    return S;
}

/* Start of the run of every (m,m') in the coefficient array, in layout order
 * (index (m+B-1)(2B-1) + (m'+B-1)), counted out as the layout is defined. */
static int64_t *run_starts(int B)
{
    int R = 2 * B - 1;
    int64_t *o = (int64_t *)malloc(sizeof(int64_t) * (size_t)R * R);
    if (!o) return NULL;
    int64_t off = 0;
    size_t p = 0;
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) {
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            o[p++] = off;
            off += B - l0;
        }
    return o;
}

/* The DWT of orders (m,m'): f(l,m,m') = (2l+1)/(8 pi B) sum_j w_B(j) d(l,m,m';beta_j) S(m,m';j),
 * for l = l0..B-1, written to out (re, im pairs). dcol is scratch [2B][B]. */
static void dwt_pair(int B, int m, int mp, const double *S, const double *w, double *dcol, double *out)
{
    int n = 2 * B;
    int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
    int L = B - l0;
    for (int j = 0; j < n; ++j) oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol + (size_t)j * B);
    int mi = mod_n(m, n), mk = mod_n(mp, n);
    for (int t = 0; t < L; ++t) {
        int l = l0 + t;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n; ++j) {
            const double *s = S + 2 * (((size_t)j * n + mi) * n + mk);
            double f = w[j] * dcol[(size_t)j * B + t];
            re += f * s[0];
            im += f * s[1];
        }
        double v = (2.0 * l + 1.0) / (8.0 * OR_PI * B);
        out[2 * t] = v * re;
        out[2 * t + 1] = v * im;
    }
}

/* Forward SOFT: grid (2B)^3 complex -> coef (B(4B^2-1)/3 complex). Returns 0 on success.
 * stride > 1 is a TIMING SAMPLE, not a transform: only the slices j with
 * j mod stride = 0 and the rows m of order pairs with (m+B-1) mod stride =
 * stride/2 (the middle of each block of rows, so that the sampled rows'
 * lengths average like all rows') are computed, every pair (m,m') of a
 * sampled row in layout order, so the per-pair and per-slice work is about
 * 1/stride of the full run's while the memory access pattern stays that of
 * the full run.  A stride above 4B leaves only the fixed costs (the copy of
 * the grid, one slice).  The other coefficients are left as they are and the
 * computed ones read unprocessed slices. */
int oracle_forward_strided(int B, const double *grid, double *coef, int stride)
{
    if (B < 1 || stride < 1) return 1;
    int n = 2 * B, R = 2 * B - 1, npairs = R * R, err = 0;
    double *S = forward_separation(B, grid, stride);
    double *w = (double *)malloc(sizeof(double) * n);
    int64_t *offs = run_starts(B);
    if (!S || !w || !offs) { free(S); free(w); free(offs); return 2; }
    oracle_weights(B, w);
#pragma omp parallel num_threads(g_threads)
    {
        double *dcol = (double *)malloc(sizeof(double) * (size_t)n * B);
#pragma omp for schedule(dynamic, 4)
        for (int p = 0; p < npairs; ++p) {
            if ((p / R) % stride != stride / 2) continue;
            if (!dcol) {
#pragma omp atomic write
                err = 2;
                continue;
            }
            int m = p / R + 1 - B, mp = p % R + 1 - B;
            dwt_pair(B, m, mp, S, w, dcol, coef + 2 * offs[p]);
        }
        free(dcol);
    }
    free(S); free(w); free(offs);
    return err;
}

int oracle_forward(int B, const double *grid, double *coef) { return oracle_forward_strided(B, grid, coef, 1); }

/* Inverse SOFT: the iDWT S(j;m,m') = sum_l d(l,m,m';beta_j) f(l,m,m') (the
 * transposed matrix T_B^T), then f(alpha_i,beta_j,gamma_k) = sum_{m,m'} S
 * exp(-i(m alpha_i + m' gamma_k)), an unnormalised 2-D DFT with the - sign.
 * Frequencies +-B (index B) carry nothing.  stride > 1 is a TIMING SAMPLE as
 * in oracle_forward_strided (the same rows m and slices j; the grid is then
 * not the transform). */
int oracle_inverse_strided(int B, const double *coef, double *grid, int stride)
{
    if (B < 1 || stride < 1) return 1;
    int n = 2 * B, R = 2 * B - 1, npairs = R * R, err = 0;
    size_t cnt = (size_t)2 * n * n * n;
    int64_t *offs = run_starts(B);
    if (!offs) return 2;
    memset(grid, 0, sizeof(double) * cnt);
#pragma omp parallel num_threads(g_threads)
    {
        double *dcol = (double *)malloc(sizeof(double) * B);
#pragma omp for schedule(dynamic, 4)
        for (int p = 0; p < npairs; ++p) {
            if ((p / R) % stride != stride / 2) continue;
            if (!dcol) {
#pragma omp atomic write
                err = 2;
                continue;
            }
            int m = p / R + 1 - B, mp = p % R + 1 - B;
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            int L = B - l0;
            int mi = mod_n(m, n), mk = mod_n(mp, n);
            int64_t off = offs[p];
            for (int j = 0; j < n; ++j) {
                oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol);
                double re = 0.0, im = 0.0;
                for (int t = 0; t < L; ++t) {
                    re += dcol[t] * coef[2 * (off + t)];
                    im += dcol[t] * coef[2 * (off + t) + 1];
                }
                double *s = grid + 2 * (((size_t)j * n + mi) * n + mk);
                s[0] = re;
                s[1] = im;
            }
        }
        free(dcol);
    }
    free(offs);
    if (err) return err;
    dft2_slices_strided(n, n, grid, -1, stride);
    return 0;
}

int oracle_inverse(int B, const double *coef, double *grid) { return oracle_inverse_strided(B, coef, grid, 1); }

/* ------------------------------------------------------------------------ */
/* Direct O(B^6) transforms straight from Eq. (quadrature) and Eq.           */
/* (fourier_representation), with D from Eq. (Wigner_D) and d from the       */
/* explicit Jacobi form. For small B only.                                  */
/* ------------------------------------------------------------------------ */

int oracle_direct_forward(int B, const double *grid, double *coef)
{
    if (B < 1) return 1;
    int n = 2 * B;
    double *w = (double *)malloc(sizeof(double) * n);
    if (!w) return 2;
    oracle_weights(B, w);
    int64_t off = 0;
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) {
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            for (int l = l0; l < B; ++l) {
                double re = 0.0, im = 0.0;
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) {
                        double d = oracle_wigner_d_explicit(l, m, mp, oracle_beta(B, j));
                        for (int k = 0; k < n; ++k) {
                            /* conj(D) = exp(+i m alpha) d exp(+i m' gamma) */
                            double ang = m * oracle_alpha(B, i) + mp * oracle_alpha(B, k);
                            double cr = cos(ang) * d, ci = sin(ang) * d;
                            const double *f = grid + 2 * (((size_t)j * n + i) * n + k);
                            re += w[j] * (f[0] * cr - f[1] * ci);
                            im += w[j] * (f[0] * ci + f[1] * cr);
                        }
                    }
                double v = (2.0 * l + 1.0) / (8.0 * OR_PI * B);
                coef[2 * (off + l - l0)] = v * re;
                coef[2 * (off + l - l0) + 1] = v * im;
            }
            off += B - l0;
        }
    free(w);
    return 0;
}

int oracle_direct_inverse(int B, const double *coef, double *grid)
{
    if (B < 1) return 1;
    int n = 2 * B;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                double re = 0.0, im = 0.0;
                int64_t off = 0;
                for (int m = 1 - B; m <= B - 1; ++m)
                    for (int mp = 1 - B; mp <= B - 1; ++mp) {
                        int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
                        for (int l = l0; l < B; ++l) {
                            /* D = exp(-i m alpha) d exp(-i m' gamma) */
                            double d = oracle_wigner_d_explicit(l, m, mp, oracle_beta(B, j));
                            double ang = -(m * oracle_alpha(B, i) + mp * oracle_alpha(B, k));
                            double dr = cos(ang) * d, di = sin(ang) * d;
                            const double *c = coef + 2 * (off + l - l0);
                            re += c[0] * dr - c[1] * di;
                            im += c[0] * di + c[1] * dr;
                        }
                        off += B - l0;
                    }
                grid[2 * (((size_t)j * n + i) * n + k)] = re;
                grid[2 * (((size_t)j * n + i) * n + k) + 1] = im;
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sampled forms for large B: single (m,m') runs and single grid points.     */
/* ------------------------------------------------------------------------ */

/* Forward coefficients of the listed (m,m') pairs only. pairs = [m0,m'0,m1,m'1,...];
 * out receives the runs l = l0..B-1 of each pair back to back. S(m,m';j) is
 * the separated double sum, taken directly (first over k, then over i). */
int oracle_forward_pairs(int B, const double *grid, int npairs, const int *pairs, double *out)
{
    if (B < 1) return 1;
    int n = 2 * B, err = 0;
    double *w = (double *)malloc(sizeof(double) * n);
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (npairs > 0 ? npairs : 1));
    if (!w || !start) { free(w); free(start); return 2; }
    oracle_weights(B, w);
    int64_t o = 0;
    for (int p = 0; p < npairs; ++p) {
        int l0 = abs(pairs[2 * p]) > abs(pairs[2 * p + 1]) ? abs(pairs[2 * p]) : abs(pairs[2 * p + 1]);
        start[p] = o;
        if (l0 < B) o += B - l0;
    }
#pragma omp parallel num_threads(g_threads)
    {
        double *dcol = (double *)malloc(sizeof(double) * (size_t)n * B);
        double *Sj = (double *)malloc(sizeof(double) * 2 * n);
        double *ek = (double *)malloc(sizeof(double) * 2 * n);
        double *ei = (double *)malloc(sizeof(double) * 2 * n);
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < npairs; ++p) {
            if (!dcol || !Sj || !ek || !ei) {
#pragma omp atomic write
                err = 2;
                continue;
            }
            int m = pairs[2 * p], mp = pairs[2 * p + 1];
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            if (l0 >= B) continue;
            for (int t = 0; t < n; ++t) {
                ek[2 * t] = cos(mp * oracle_alpha(B, t)); ek[2 * t + 1] = sin(mp * oracle_alpha(B, t));
                ei[2 * t] = cos(m * oracle_alpha(B, t));  ei[2 * t + 1] = sin(m * oracle_alpha(B, t));
            }
            for (int j = 0; j < n; ++j) {
                double sr = 0.0, si = 0.0;
                for (int i = 0; i < n; ++i) {
                    double gr = 0.0, gi = 0.0;
                    const double *row = grid + 2 * (((size_t)j * n + i) * n);
                    for (int k = 0; k < n; ++k) {
                        gr += row[2 * k] * ek[2 * k] - row[2 * k + 1] * ek[2 * k + 1];
                        gi += row[2 * k] * ek[2 * k + 1] + row[2 * k + 1] * ek[2 * k];
                    }
                    sr += gr * ei[2 * i] - gi * ei[2 * i + 1];
                    si += gr * ei[2 * i + 1] + gi * ei[2 * i];
                }
                Sj[2 * j] = sr;
                Sj[2 * j + 1] = si;
            }
            for (int j = 0; j < n; ++j) oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol + (size_t)j * B);
            for (int t = 0; t < B - l0; ++t) {
                int l = l0 + t;
                double re = 0.0, im = 0.0;
                for (int j = 0; j < n; ++j) {
                    double f = w[j] * dcol[(size_t)j * B + t];
                    re += f * Sj[2 * j];
                    im += f * Sj[2 * j + 1];
                }
                double v = (2.0 * l + 1.0) / (8.0 * OR_PI * B);
                out[2 * (start[p] + t)] = v * re;
                out[2 * (start[p] + t) + 1] = v * im;
            }
        }
        free(dcol); free(Sj); free(ek); free(ei);
    }
    free(w); free(start);
    return err;
}

/* Inverse transform at single grid points: pts = [i0,j0,k0, i1,j1,k1, ...].
 * f(alpha_i,beta_j,gamma_k) = sum_{m,m'} exp(-i(m alpha_i + m' gamma_k)) sum_l d(l,m,m';beta_j) f(l,m,m'). */
int oracle_inverse_points(int B, const double *coef, int npts, const int *pts, double *out)
{
    if (B < 1) return 1;
    int err = 0;
#pragma omp parallel num_threads(g_threads)
    {
        double *dcol = (double *)malloc(sizeof(double) * B);
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < npts; ++p) {
            if (!dcol) {
#pragma omp atomic write
                err = 2;
                continue;
            }
            int i = pts[3 * p], j = pts[3 * p + 1], k = pts[3 * p + 2];
            double re = 0.0, im = 0.0;
            int64_t off = 0;
            for (int m = 1 - B; m <= B - 1; ++m)
                for (int mp = 1 - B; mp <= B - 1; ++mp) {
                    int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
                    int L = B - l0;
                    oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol);
                    double sr = 0.0, si = 0.0;
                    for (int t = 0; t < L; ++t) {
                        sr += dcol[t] * coef[2 * (off + t)];
                        si += dcol[t] * coef[2 * (off + t) + 1];
                    }
                    double ang = -(m * oracle_alpha(B, i) + mp * oracle_alpha(B, k));
                    double c = cos(ang), s = sin(ang);
                    re += sr * c - si * s;
                    im += sr * s + si * c;
                    off += L;
                }
            out[2 * p] = re;
            out[2 * p + 1] = im;
        }
        free(dcol);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* Adjoints (with respect to sum_k conj(a_k) b_k on both sides).             */
/* The forward transform is f = V T W E x (E: per-slice DFT with exp(+i)),    */
/* so its adjoint is E^H W T^T V: the inverse's steps with V applied to the  */
/* coefficients and W to S.  The inverse transform is E^H T^T, with adjoint  */
/* T E: the forward's steps without V and W.                                 */
/* ------------------------------------------------------------------------ */

int oracle_forward_adjoint(int B, const double *coef, double *grid)
{
    if (B < 1) return 1;
    int n = 2 * B;
    size_t cnt = (size_t)2 * n * n * n;
    double *dcol = (double *)malloc(sizeof(double) * B);
    double *w = (double *)malloc(sizeof(double) * n);
    if (!dcol || !w) { free(dcol); free(w); return 2; }
    oracle_weights(B, w);
    memset(grid, 0, sizeof(double) * cnt);
    int64_t off = 0;
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) {
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            int L = B - l0;
            int mi = mod_n(m, n), mk = mod_n(mp, n);
            for (int j = 0; j < n; ++j) {
                oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol);
                double re = 0.0, im = 0.0;
                for (int t = 0; t < L; ++t) {
                    double v = (2.0 * (l0 + t) + 1.0) / (8.0 * OR_PI * B);
                    re += dcol[t] * v * coef[2 * (off + t)];
                    im += dcol[t] * v * coef[2 * (off + t) + 1];
                }
                double *s = grid + 2 * (((size_t)j * n + mi) * n + mk);
                s[0] = w[j] * re;
                s[1] = w[j] * im;
            }
            off += L;
        }
    free(dcol); free(w);
    oracle_dft2_slices(n, n, grid, -1);
    return 0;
}

int oracle_inverse_adjoint(int B, const double *grid, double *coef)
{
    if (B < 1) return 1;
    int n = 2 * B;
    double *S = forward_separation(B, grid, 1);
    double *dcol = (double *)malloc(sizeof(double) * (size_t)n * B);
    if (!S || !dcol) { free(S); free(dcol); return 2; }
    int64_t off = 0;
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) {
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            int L = B - l0;
            int mi = mod_n(m, n), mk = mod_n(mp, n);
            for (int j = 0; j < n; ++j) oracle_wigner_d_column(B, m, mp, oracle_beta(B, j), dcol + (size_t)j * B);
            for (int t = 0; t < L; ++t) {
                double re = 0.0, im = 0.0;
                for (int j = 0; j < n; ++j) {
                    const double *s = S + 2 * (((size_t)j * n + mi) * n + mk);
                    re += dcol[(size_t)j * B + t] * s[0];
                    im += dcol[(size_t)j * B + t] * s[1];
                }
                coef[2 * (off + t)] = re;
                coef[2 * (off + t) + 1] = im;
            }
            off += L;
        }
    free(S); free(dcol);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Rotational correlation of two functions on the sphere (the fast            */
/* rotational matching application of Sec. 1).  With spherical-harmonic     */
/* coefficients f_lm, g_lm (index l*l + m + l, l < B), the correlation       */
/*   C(R) = int_{S^2} g(R^{-1} w) conj(f(w)) dw                              */
/* is the inverse transform of c(l,m,m') = g_lm conj(f_lm'), evaluated at    */
/* R = R_z(gamma) R_y(beta) R_z(alpha) on the sampling grid.                 */
/* ------------------------------------------------------------------------ */

int oracle_correlation_coeffs(int B, const double *f_sh, const double *g_sh, double *coef)
{
    if (B < 1) return 1;
    int64_t off = 0;
    for (int m = 1 - B; m <= B - 1; ++m)
        for (int mp = 1 - B; mp <= B - 1; ++mp) {
            int l0 = abs(m) > abs(mp) ? abs(m) : abs(mp);
            for (int l = l0; l < B; ++l) {
                const double *g = g_sh + 2 * ((int64_t)l * l + m + l);
                const double *f = f_sh + 2 * ((int64_t)l * l + mp + l);
                /* g * conj(f) */
                coef[2 * (off + l - l0)] = g[0] * f[0] + g[1] * f[1];
                coef[2 * (off + l - l0) + 1] = g[1] * f[0] - g[0] * f[1];
            }
            off += B - l0;
        }
    return 0;
}
