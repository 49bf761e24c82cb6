// errors.cu -- error bars of the sampled product.
//
// Per listed entry (h, f) of CD: the variance of Lemma 3.1, eq. 3.7 (the sigma^2 of Thm 3.1),
// sum_k (1/c_k) [ sum_{i in k, p_i > 0} M_hi^2 N_if^2 / p_i - (sum_{i in k, p_i > 0} M_hi N_if)^2 ]
// for Alg. 2, or (1/c) [ sum_k ((M^k N_k)_hf)^2 / p_k - (sum_k (M^k N_k)_hf)^2 ] for c whole-block
// draws; and from the draws themselves the entry's value and the one-sample variance estimate
// sum_k c_k/(c_k - 1) sum_t (Z_t - Zbar_k)^2, Z_t = scale_t M_{h,i_t} N_{i_t,f} (blocks with c_k >= 2).
// For the whole matrix: E||MN - CD||_F^2 (Remark 2.2), eq. 3.10, and the bounds of Thm 3.3
// (eq. 3.11, 3.12), Thm 4.2 (eq. 4.3, 4.4) and Thm 4.4 (eq. 4.8, 4.9) with theta_1, theta_2 and
// beta read off the statistics.
//
// These are reports, not the hot path: one warp per entry (its lanes splitting the blocks or the
// draws) and one CTA for the whole-matrix sums, FP64 throughout.
#include <math.h>

#include "internal.h"

namespace bmm {

#define kNaN __longlong_as_double(0x7FF8000000000000LL)

__device__ __forceinline__ double mat_at(const MatView& A, int64_t r, int64_t c) {
    const int64_t o = A.row_major ? r * A.ld + c : c * A.ld + r;
    if (A.dtype == BMM_F64) return static_cast<const double*>(A.data)[o];
    if (A.dtype == BMM_F32) return (double)static_cast<const float*>(A.data)[o];
    return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(A.data)[o]);
}

__device__ __forceinline__ bool entry_of(const int64_t* entries, int64_t e, const MatView& M, const MatView& N,
                                         int64_t* h, int64_t* f) {
    *h = entries[2 * e];
    *f = entries[2 * e + 1];
    return *h >= 0 && *h < M.rows && *f >= 0 && *f < N.cols;
}

// ---------------------------------------------------------------- eq. 3.7 per entry
__global__ void __launch_bounds__(256) entry_variance_kernel(MatView M, MatView N, const int64_t* __restrict__ off,
                                                             int64_t K, int unit, const double* __restrict__ p,
                                                             const int64_t* __restrict__ ck, int64_t c,
                                                             const int64_t* __restrict__ entries, int64_t count,
                                                             double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= count) return;
    int64_t h, f;
    if (!entry_of(entries, e, M, N, &h, &f)) {
        if (lane == 0) out[e] = kNaN;  // an entry outside CD
        return;
    }
    double acc = 0.0, mean = 0.0;
    for (int64_t k = lane; k < K; k += 32) {
        // block ranges clamped to [0, n): a malformed offsets array cannot send a read outside M or N
        const int64_t a = imax(off[k], 0), b = imin(off[k + 1], M.cols);
        if (unit == BMM_UNIT_COLUMN) {
            double s = 0.0, dot = 0.0;
            for (int64_t i = a; i < b; ++i) {
                const double pi = p[i];
                if (pi > 0.0) {
                    const double t = mat_at(M, h, i) * mat_at(N, i, f);
                    s += t * t / pi;
                    dot += t;
                }
            }
            acc += (s - dot * dot) / (double)ck[k];
        } else {
            const double pk = p[k];
            if (pk > 0.0) {
                double d = 0.0;
                for (int64_t i = a; i < b; ++i) d += mat_at(M, h, i) * mat_at(N, i, f);
                acc += d * d / pk;
                mean += d;
            }
        }
    }
    acc = warp_sum(acc);
    mean = warp_sum(mean);
    if (lane == 0) out[e] = unit == BMM_UNIT_COLUMN ? acc : (acc - mean * mean) / (double)c;
}

cudaError_t launch_entry_variance(const MatView& M, const MatView& N, const int64_t* off, int64_t K, int unit,
                                  const double* p, const int64_t* ck, int64_t c, const int64_t* entries, int64_t count,
                                  double* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    (count_launch(), entry_variance_kernel<<<(unsigned)ceil_div(count * 32, 256), 256, 0, s>>>(
                         M, N, off, K, unit, p, ck, c, entries, count, out));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- draw offsets of Alg. 2
// start[k] = c_0 + ... + c_{k-1}, start[K] = the total, which must equal the number of draws.
__global__ void __launch_bounds__(1024) draw_starts_kernel(const int64_t* __restrict__ ck, int64_t K, int64_t draws,
                                                           int64_t* __restrict__ start, DevStatus* st) {
    __shared__ long long warp_tot[32];
    __shared__ long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < K; base += 1024) {
        const int64_t k = base + tid;
        const long long v = k < K ? (long long)ck[k] : 0;
        if (k < K && v < 1) set_status(st, BMM_ERR_SHAPE, (int)k);
        long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            long long w = warp_tot[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_tot[lane] = wi - w;
        }
        __syncthreads();
        const long long before = carry;
        if (k < K) start[k] = before + warp_tot[warp] + inc - v;
        __syncthreads();
        if (tid == 1023) carry = before + warp_tot[warp] + inc;
        __syncthreads();
    }
    if (tid == 0) {
        start[K] = carry;
        if (carry != draws) set_status(st, BMM_ERR_SHAPE, -1);
    }
}

// ---------------------------------------------------------------- one-sample estimate per entry
__global__ void __launch_bounds__(256) entry_estimate_kernel(MatView M, MatView N, const int64_t* __restrict__ off,
                                                             int64_t K, int unit, const int64_t* __restrict__ start,
                                                             const int32_t* __restrict__ idx,
                                                             const double* __restrict__ scale, int64_t draws,
                                                             const int64_t* __restrict__ entries, int64_t count,
                                                             double* __restrict__ cd_out, double* __restrict__ s2_out) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= count) return;
    int64_t h, f;
    if (!entry_of(entries, e, M, N, &h, &f)) {
        if (lane == 0) {
            cd_out[e] = kNaN;
            s2_out[e] = kNaN;
        }
        return;
    }
    if (unit == BMM_UNIT_COLUMN) {
        // lanes split the blocks; each block's draws twice (mean, then squared deviations)
        double cd = 0.0, s2 = 0.0;
        for (int64_t k = lane; k < K; k += 32) {
            const int64_t t0 = imax(start[k], 0), t1 = imin(start[k + 1], draws);
            double sz = 0.0;
            for (int64_t t = t0; t < t1; ++t) {
                const int64_t i = idx[t];
                sz += (uint64_t)i < (uint64_t)M.cols ? scale[t] * mat_at(M, h, i) * mat_at(N, i, f) : kNaN;
            }
            cd += sz;
            const int64_t n = t1 - t0;
            if (n >= 2) {
                const double zbar = sz / (double)n;
                double q = 0.0;
                for (int64_t t = t0; t < t1; ++t) {
                    const int64_t i = idx[t];
                    const double d =
                        ((uint64_t)i < (uint64_t)M.cols ? scale[t] * mat_at(M, h, i) * mat_at(N, i, f) : kNaN) - zbar;
                    q += d * d;
                }
                s2 += (double)n / (double)(n - 1) * q;
            }
        }
        cd = warp_sum(cd);
        s2 = warp_sum(s2);
        if (lane == 0) {
            cd_out[e] = cd;
            s2_out[e] = s2;
        }
    } else {
        // lanes split the draws; Z_t = scale_t (M^{k_t} N_{k_t})_hf
        double cd = 0.0;
        for (int64_t t = lane; t < draws; t += 32) {
            const int64_t k = idx[t];
            double d = kNaN;
            if ((uint64_t)k < (uint64_t)K) {
                d = 0.0;
                for (int64_t i = imax(off[k], 0); i < imin(off[k + 1], M.cols); ++i) d += mat_at(M, h, i) * mat_at(N, i, f);
            }
            cd += scale[t] * d;
        }
        cd = warp_sum(cd);
        double q = 0.0;
        if (draws >= 2) {
            const double zbar = cd / (double)draws;
            for (int64_t t = lane; t < draws; t += 32) {
                const int64_t k = idx[t];
                double d = kNaN;
                if ((uint64_t)k < (uint64_t)K) {
                    d = 0.0;
                    for (int64_t i = imax(off[k], 0); i < imin(off[k + 1], M.cols); ++i)
                        d += mat_at(M, h, i) * mat_at(N, i, f);
                }
                const double dz = scale[t] * d - zbar;
                q += dz * dz;
            }
            q = warp_sum(q) * ((double)draws / (double)(draws - 1));
        }
        if (lane == 0) {
            cd_out[e] = cd;
            s2_out[e] = q;
        }
    }
}

cudaError_t launch_entry_estimate(const MatView& M, const MatView& N, const int64_t* off, int64_t K, int unit,
                                  const int64_t* ck, const int32_t* idx, const double* scale, int64_t draws,
                                  const int64_t* entries, int64_t count, double* cd, double* s2, int64_t* start,
                                  DevStatus* st, cudaStream_t s) {
    if (unit == BMM_UNIT_COLUMN)
        (count_launch(), draw_starts_kernel<<<1, 1024, 0, s>>>(ck, K, draws, start, st));
    if (count <= 0) return cudaGetLastError();
    (count_launch(), entry_estimate_kernel<<<(unsigned)ceil_div(count * 32, 256), 256, 0, s>>>(
                         M, N, off, K, unit, start, idx, scale, draws, entries, count, cd, s2));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- whole-matrix report
__device__ double block_reduce(double v, int op, double* sm) {  // op 0 sum, 1 min, 2 max; 1024 threads
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = op == 0 ? v + w : (op == 1 ? fmin(v, w) : fmax(v, w));
    }
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    v = sm[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = op == 0 ? v + w : (op == 1 ? fmin(v, w) : fmax(v, w));
    }
    return v;
}

__global__ void __launch_bounds__(1024) error_report_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                            const double* __restrict__ p,
                                                            const int64_t* __restrict__ off, int64_t K, int64_t n,
                                                            const int64_t* __restrict__ ck,
                                                            const double* __restrict__ a,
                                                            const double* __restrict__ f,
                                                            const double* __restrict__ mf,
                                                            const double* __restrict__ nf,
                                                            const double* __restrict__ fhat, int64_t c, double delta,
                                                            double* __restrict__ out) {
    __shared__ double sm[32];
    const double inf = __longlong_as_double(0x7FF0000000000000LL);
    double e2 = 0.0, v310 = 0.0, ms = 0.0, ns = 0.0;
    double beta = 1.0, t1 = inf, t2 = -inf, h1 = inf, h2 = -inf;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const double ak = a[k];
        ms += mf[k];
        ns += nf[k];
        double q = 0.0;
        for (int64_t i = imax(off[k], 0); i < imin(off[k + 1], n); ++i) {  // clamped to [0, n)
            const double xy = x[i] * y[i];
            const double pi = p[i];
            if (pi > 0.0) q += xy / pi;
            if (ak > 0.0) {
                const double pstar = sqrt(xy) / ak;
                if (pstar > 0.0) beta = fmin(beta, pi / pstar);
            }
        }
        if (f != nullptr) {
            const double fk = f[k];
            e2 += (q - fk) / (double)ck[k];
            v310 += sqrt(fmax(ak * ak - fk, 0.0));
            if (ak > 0.0) {
                const double om = 1.0 - fk / (ak * ak);
                t1 = fmin(t1, om);
                t2 = fmax(t2, om);
                if (fhat != nullptr) {
                    const double th = fabs(1.0 - fhat[k] / (ak * ak));
                    h1 = fmin(h1, th);
                    h2 = fmax(h2, th);
                }
            }
        }
    }
    e2 = block_reduce(e2, 0, sm);
    v310 = block_reduce(v310, 0, sm);
    ms = block_reduce(ms, 0, sm);
    ns = block_reduce(ns, 0, sm);
    beta = block_reduce(beta, 1, sm);
    t1 = block_reduce(t1, 1, sm);
    t2 = block_reduce(t2, 2, sm);
    h1 = block_reduce(h1, 1, sm);
    h2 = block_reduce(h2, 2, sm);
    if (threadIdx.x != 0) return;
    const double nan = __longlong_as_double(0x7FF8000000000000LL);
    for (int j = 0; j < BMM_REPORT_LEN; ++j) out[j] = nan;
    const double cc = (double)c, prod = ms * ns;
    const double logt = sqrt(8.0 / beta * log(1.0 / delta));
    out[BMM_REPORT_BETA] = beta;
    out[BMM_REPORT_M_FRO2] = ms;
    out[BMM_REPORT_N_FRO2] = ns;
    if (f == nullptr) return;
    out[BMM_REPORT_EXPECTED_SQ_ERROR] = e2;
    out[BMM_REPORT_EQ310] = v310 * v310 / cc;
    out[BMM_REPORT_THETA1] = t1;
    out[BMM_REPORT_THETA2] = t2;
    const double phi = t1 > 0.0 ? sqrt(t2 - t1 * beta + t2 * t1 * beta) / sqrt(sqrt(t2 * t1)) : inf;
    out[BMM_REPORT_PHI] = phi;
    out[BMM_REPORT_EQ311] = phi * phi / (beta * cc) * prod;
    const double eta = t1 > 0.0 ? phi + sqrt(t2 / t1) * logt : inf;
    out[BMM_REPORT_ETA312] = eta;
    out[BMM_REPORT_EQ312] = eta * eta / (beta * cc) * prod;
    const double phihat = sqrt(1.0 - beta * (1.0 - t2));
    out[BMM_REPORT_PHIHAT] = phihat;
    out[BMM_REPORT_EQ43] = phihat * phihat / (beta * cc) * prod;
    const double eta44 = phihat + logt;
    out[BMM_REPORT_ETA44] = eta44;
    out[BMM_REPORT_EQ44] = eta44 * eta44 / (beta * cc) * prod;
    if (fhat == nullptr) return;
    out[BMM_REPORT_THETA1HAT] = h1;
    out[BMM_REPORT_THETA2HAT] = h2;
    const double phit = h1 > 0.0 ? sqrt(h2 - h1 * beta + t2 * h1 * beta) / sqrt(sqrt(h2 * h1)) : inf;
    out[BMM_REPORT_PHITILDE] = phit;
    out[BMM_REPORT_EQ48] = phit * phit / (beta * cc) * prod;
    const double eta49 = h1 > 0.0 ? phit + sqrt(h2 / h1) * logt : inf;
    out[BMM_REPORT_ETA49] = eta49;
    out[BMM_REPORT_EQ49] = eta49 * eta49 / (beta * cc) * prod;
}

cudaError_t launch_error_report(const double* x, const double* y, const double* p, const int64_t* off, int64_t K,
                                int64_t n, const int64_t* ck, const double* a, const double* f, const double* mf,
                                const double* nf, const double* fhat, int64_t c, double delta, double* out,
                                cudaStream_t s) {
    (count_launch(), error_report_kernel<<<1, 1024, 0, s>>>(x, y, p, off, K, n, ck, a, f, mf, nf, fhat, c, delta, out));
    return cudaGetLastError();
}

}  // namespace bmm
