// The data movements of Algorithm 3 (two-stage cyclic Sinkhorn for inputs with
// approximate cyclic symmetry), around the two solver calls:
//   Stage 1 input:  the first block row of the full cost, C_base[k] = C[0:m,
//                   k m:(k+1) m] (the blocks the fold of Eq. def_Kij uses), and
//                   the block averages alpha_i = (1/N) sum_k a_{k m + i}, beta
//                   likewise;
//   Stage 1:        ot_fold_cost(SOFTMIN) + ot_sinkhorn_reduced with the L2 row
//                   rule (App. F stops it at 1e-3);
//   Stage 2 input:  the N-fold concatenation of the Stage-1 column potential,
//                   g_{k m + j} = z_j, as the warm start of
//   Stage 2:        ot_sinkhorn_full on the original a, b, C.
#include "common.cuh"

namespace {

__global__ void __launch_bounds__(256) first_block_row_kernel(const float* __restrict__ C, int m, int N,
                                                              float* __restrict__ C_base) {
    const long long n = (long long)m * N;
    const long long total = (long long)N * m * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / ((long long)m * m));
        const long long r = e - (long long)k * m * m;
        const int i = (int)(r / m), j = (int)(r - (long long)i * m);
        C_base[e] = C[(long long)i * n + (long long)k * m + j];
    }
}

__global__ void __launch_bounds__(256) block_average_kernel(const float* __restrict__ v, int m, int N,
                                                            float* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += (double)v[(long long)k * m + i];
        out[i] = (float)(s / N);
    }
}

__global__ void __launch_bounds__(256) tile_kernel(const double* __restrict__ z, int m, int N, double* __restrict__ g) {
    const long long n = (long long)m * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        g[e] = z[e % m];
}

unsigned grid_1d(long long work) {
    long long b = (work + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

extern "C" int ot_first_block_row(int m, int N, const float* C, float* C_base, void* stream) {
    if (m <= 0 || N <= 0 || !C || !C_base) return OT_ERR_ARG;
    first_block_row_kernel<<<grid_1d((long long)N * m * m), 256, 0, (cudaStream_t)stream>>>(C, m, N, C_base);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

extern "C" int ot_block_average(int m, int N, const float* v, float* out, void* stream) {
    if (m <= 0 || N <= 0 || !v || !out) return OT_ERR_ARG;
    block_average_kernel<<<grid_1d(m), 256, 0, (cudaStream_t)stream>>>(v, m, N, out);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

extern "C" int ot_tile_potentials(int m, int N, const double* z, double* g, void* stream) {
    if (m <= 0 || N <= 0 || !z || !g) return OT_ERR_ARG;
    tile_kernel<<<grid_1d((long long)m * N), 256, 0, (cudaStream_t)stream>>>(z, m, N, g);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
