// gemm_f64.cu -- FP64 sampled product on CUDA cores (correctness mode; GB300's FP64 rate is low).
// out[M x N] (+)= A[M x K] * B[N x K]^T, both K-major.  64 x 64 output tiles; when they are fewer
// than the SMs and K is long (the paper's 26 x 28 products of depth up to 5e5), K is split over
// blockIdx.z: each split writes its partial tile to a workspace buffer and gemm_f64_reduce_kernel
// adds the splits in split order, so the result does not depend on scheduling.
#include "internal.h"

namespace bmm {

__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb, int64_t M,
                                                       int64_t N, int64_t k_host, const int64_t* __restrict__ k_dev,
                                                       double* __restrict__ out, int64_t ldo, int accumulate,
                                                       int64_t splits, double* __restrict__ part) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int64_t Kall = k_dev ? round_up(*k_dev, 64) : k_host;
    const int64_t chunk = round_up(ceil_div(Kall, splits), 16);
    const int64_t kb = (int64_t)blockIdx.z * chunk;
    const int64_t K = imin(Kall, kb + chunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = kb; k0 < K; k0 += 16) {
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
                if (splits > 1) {
                    part[((int64_t)blockIdx.z * M + r) * N + c] = acc[i][j];
                } else {
                    double* o = out + r * ldo + c;
                    *o = accumulate ? *o + acc[i][j] : acc[i][j];
                }
            }
        }
    }
}

__global__ void gemm_f64_reduce_kernel(const double* __restrict__ part, int64_t M, int64_t N, int64_t splits,
                                       double* __restrict__ out, int64_t ldo, int accumulate) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t r = e / N, c = e % N;
    double v = accumulate ? out[r * ldo + c] : 0.0;
    for (int64_t z = 0; z < splits; ++z) v += part[z * M * N + e];
    out[r * ldo + c] = v;
}

int64_t gemm_f64_splits(int64_t M, int64_t N, int64_t K) {
    const int64_t tiles = ceil_div(M, 64) * ceil_div(N, 64);
    if (tiles >= 76 || K < 4096) return 1;
    return imax(1, imin(imin(ceil_div(304, tiles), K / 2048), 65535));
}

int64_t gemm_f64_split_elems(int64_t M, int64_t N, int64_t K) {
    const int64_t s = gemm_f64_splits(M, N, K);
    return s > 1 ? s * M * N : 0;
}

cudaError_t launch_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t N,
                            int64_t k_host, const int64_t* k_dev, double* out, int64_t ldo, int accumulate,
                            cudaStream_t s, int64_t k_max, double* part, int64_t part_cap) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (ceil_div(M, 64) > 65535) return cudaErrorInvalidValue;
    int64_t splits = gemm_f64_splits(M, N, k_max > 0 ? k_max : k_host);
    if (splits > 1 && (part == nullptr || part_cap < splits * M * N)) splits = 1;
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64), (unsigned)splits);
    (count_launch(), gemm_f64_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, M, N, k_host, k_dev, out, ldo, accumulate,
                                                          splits, part));
    if (splits > 1)
        (count_launch(), gemm_f64_reduce_kernel<<<(unsigned)ceil_div(M * N, 256), 256, 0, s>>>(part, M, N, splits, out,
                                                                                                ldo, accumulate));
    return cudaGetLastError();
}

}  // namespace bmm
