// shard.cu -- the exchange kernels of a transform sharded over several GPUs
// by beta slices (2-D FFT step) and by symmetry clusters (DWT step): the S
// columns of a list of order pairs, over a range of beta slices, packed into
// or unpacked from a dense buffer that the caller's all-to-all moves.
#include "soft_internal.cuh"

#include <algorithm>

namespace softgb {
namespace {

__device__ __forceinline__ int mod_n(int a, int n) { return a < 0 ? a + n : a; }

// out[js][c] = S[j0 + js][m_c mod n][m'_c mod n], js < nslices, c < ncols.
__global__ void gather_columns_kernel(const double2 *__restrict__ S, int n, int j0, int nslices,
                                      const int2 *__restrict__ cols, int ncols, double2 *__restrict__ out) {
    const int64_t total = (int64_t)nslices * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int js = (int)(e / ncols), c = (int)(e % ncols);
        const int2 mm = cols[c];
        out[e] = S[((int64_t)(j0 + js) * n + mod_n(mm.x, n)) * n + mod_n(mm.y, n)];
    }
}

// S[j0 + js][m_c mod n][m'_c mod n] = in[js][c].
__global__ void scatter_columns_kernel(const double2 *__restrict__ in, int n, int j0, int nslices,
                                       const int2 *__restrict__ cols, int ncols, double2 *__restrict__ S) {
    const int64_t total = (int64_t)nslices * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int js = (int)(e / ncols), c = (int)(e % ncols);
        const int2 mm = cols[c];
        S[((int64_t)(j0 + js) * n + mod_n(mm.x, n)) * n + mod_n(mm.y, n)] = in[e];
    }
}

int grid_for(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8)); }

}  // namespace

cudaError_t launch_gather_columns(const double2 *S, int B, int j0, int nslices, const int2 *cols, int ncols,
                                  double2 *out, cudaStream_t s) {
    const int64_t total = (int64_t)nslices * ncols;
    if (total == 0) return cudaSuccess;
    gather_columns_kernel<<<grid_for(total), 256, 0, s>>>(S, 2 * B, j0, nslices, cols, ncols, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter_columns(const double2 *in, int B, int j0, int nslices, const int2 *cols, int ncols,
                                   double2 *S, cudaStream_t s) {
    const int64_t total = (int64_t)nslices * ncols;
    if (total == 0) return cudaSuccess;
    scatter_columns_kernel<<<grid_for(total), 256, 0, s>>>(in, 2 * B, j0, nslices, cols, ncols, S);
    count_launch();
    return cudaGetLastError();
}

}  // namespace softgb
