// correlate.cu -- rotational correlation of two spherical functions and the
// arg-max of its real part over the SO(3) sampling grid (the fast rotational
// matching application that motivates the paper, Sec. 1).
//
// For spherical-harmonic coefficients f_lm, g_lm (l < B, index l*l + m + l)
// the correlation C(R) = int_{S^2} g(R^{-1} w) conj(f(w)) dw has the SO(3)
// Fourier coefficients c(l,m,m') = g_lm conj(f_lm'), so the inverse transform
// of c gives C on the (2B)^3 Euler grid, R = R_z(gamma) R_y(beta) R_z(alpha).
#include "soft.h"
#include "soft_internal.cuh"

#include <algorithm>

namespace softgb {
namespace {

// One thread per (m, m') run: c(l,m,m') = g_{l m} conj(f_{l m'}) for l = l0..B-1.
__global__ void corr_coeffs_kernel(int B, const double2 *__restrict__ f, const double2 *__restrict__ g,
                                   const int64_t *__restrict__ runoff, double2 *__restrict__ coef) {
    const int R = 2 * B - 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * R; e += gridDim.x * blockDim.x) {
        const int m = e / R - (B - 1), mp = e % R - (B - 1);
        const int l0 = max(abs(m), abs(mp));
        int64_t o = runoff[e];
        for (int l = l0; l < B; ++l, ++o) {
            const double2 gv = g[l * l + m + l], fv = f[l * l + mp + l];
            coef[o] = make_double2(gv.x * fv.x + gv.y * fv.y, gv.y * fv.x - gv.x * fv.y);
        }
    }
}

struct ArgMax {
    double v;
    int64_t i;
};

// Larger value wins; on equal values the lower index (first occurrence).
// Entries with index < 0 (empty) or a NaN value never win.
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
    if (b.i < 0 || isnan(b.v)) return a;
    if (a.i < 0 || isnan(a.v)) return b;
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
    return a;
}

__device__ ArgMax block_argmax(ArgMax x) {
    __shared__ double sv[32];
    __shared__ long long si[32];
    for (int off = 16; off > 0; off >>= 1) {
        ArgMax y;
        y.v = __shfl_down_sync(0xffffffffu, x.v, off);
        y.i = __shfl_down_sync(0xffffffffu, (long long)x.i, off);
        x = better(x, y);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = x.v; si[warp] = x.i; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        x.v = lane < nw ? sv[lane] : -INFINITY;
        x.i = lane < nw ? si[lane] : -1;
        for (int off = 16; off > 0; off >>= 1) {
            ArgMax y;
            y.v = __shfl_down_sync(0xffffffffu, x.v, off);
            y.i = __shfl_down_sync(0xffffffffu, (long long)x.i, off);
            x = better(x, y);
        }
    }
    return x;  // valid in thread 0
}

// Pass 1: every block reduces a strided part of Re(data) to one candidate.
// NaN values never win (comparisons with NaN are false).
__global__ void argmax_pass1(const double2 *__restrict__ data, int64_t count, double *__restrict__ pv,
                             int64_t *__restrict__ pi) {
    ArgMax best{-INFINITY, -1};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        best = better(best, ArgMax{data[e].x, e});
    best = block_argmax(best);
    if (threadIdx.x == 0) { pv[blockIdx.x] = best.v; pi[blockIdx.x] = best.i; }
}

// Pass 2: one block over the candidates.
__global__ void argmax_pass2(const double *__restrict__ pv, const int64_t *__restrict__ pi, int nparts,
                             int64_t *__restrict__ index_out, double *__restrict__ value_out) {
    ArgMax best{-INFINITY, -1};
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) best = better(best, ArgMax{pv[t], pi[t]});
    best = block_argmax(best);
    if (threadIdx.x == 0) { *index_out = best.i; *value_out = best.v; }
}

}  // namespace

constexpr int kArgmaxParts = 152 * 4;

cudaError_t launch_corr_coeffs(int B, const double2 *f, const double2 *g, const int64_t *runoff, double2 *coef,
                               cudaStream_t s) {
    const int R = 2 * B - 1;
    const int blocks = std::min((R * R + 255) / 256, 152 * 8);
    corr_coeffs_kernel<<<blocks, 256, 0, s>>>(B, f, g, runoff, coef);
    count_launch();
    return cudaGetLastError();
}

// scratch_v / scratch_i: kArgmaxParts entries each.
cudaError_t launch_argmax_real(const double2 *data, int64_t count, double *scratch_v, int64_t *scratch_i,
                               int64_t *index_out, double *value_out, cudaStream_t s) {
    argmax_pass1<<<kArgmaxParts, 256, 0, s>>>(data, count, scratch_v, scratch_i);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    argmax_pass2<<<1, 512, 0, s>>>(scratch_v, scratch_i, kArgmaxParts, index_out, value_out);
    count_launch();
    return cudaGetLastError();
}

int argmax_parts() { return kArgmaxParts; }

}  // namespace softgb
