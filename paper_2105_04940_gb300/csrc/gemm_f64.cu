// gemm_f64.cu -- FP64 sampled product on CUDA cores (correctness mode; GB300's FP64 rate is low).
// out[M x N] (+)= A[M x K] * B[N x K]^T, both K-major.
#include "internal.h"

namespace bmm {

__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb, int64_t M,
                                                       int64_t N, int64_t k_host, const int64_t* __restrict__ k_dev,
                                                       double* __restrict__ out, int64_t ldo, int accumulate) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int64_t K = k_dev ? round_up(*k_dev, 64) : k_host;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e >> 4, kk = e & 15;
            const int64_t ka = k0 + kk;
            As[kk][r] = (m0 + r < M && ka < K) ? A[(m0 + r) * lda + ka] : 0.0;
            Bs[kk][r] = (n0 + r < N && ka < K) ? B[(n0 + r) * ldb + ka] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = m0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t c = n0 + tx + 16 * j;
            if (c < N) {
                double* o = out + r * ldo + c;
                *o = accumulate ? *o + acc[i][j] : acc[i][j];
            }
        }
    }
}

cudaError_t launch_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t N,
                            int64_t k_host, const int64_t* k_dev, double* out, int64_t ldo, int accumulate,
                            cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (ceil_div(M, 64) > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
    (count_launch(), gemm_f64_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, M, N, k_host, k_dev, out, ldo, accumulate));
    return cudaGetLastError();
}

}  // namespace bmm
