// common.cuh -- device helpers shared by the kernels of the sm_103a library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

#include "../../include/bmm.h"

namespace bmm {

// ---------------------------------------------------------------- status word
// The first 256 bytes of the workspace: int32 status (first error wins), int32 detail.
struct DevStatus {
    int code;
    int detail;
};

__device__ __forceinline__ void set_status(DevStatus* st, int code, int detail = 0) {
    if (st != nullptr && atomicCAS(&st->code, 0, code) == 0) {
        atomicExch(&st->detail, detail);
    }
}

// ---------------------------------------------------------------- element loads
template <typename T> struct Elem;
template <> struct Elem<double> {
    static __device__ __forceinline__ double to_f64(double v) { return v; }
};
template <> struct Elem<float> {
    static __device__ __forceinline__ double to_f64(float v) { return (double)v; }
};
template <> struct Elem<__nv_bfloat16> {
    static __device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
};

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------- float-float sums
// A sum carried as hi + lo in FP32 with error-free transformations (TwoSum,
// and the exact FMA residual of a product).  The intrinsics keep the compiler
// from contracting or reassociating.  Callers fold the pair into FP64 every few
// dozen terms so the lo part never accumulates more than ~2^-48 relative error.
struct FF {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    // += a * b, exactly captured up to the FP32 rounding of lo
    __device__ __forceinline__ void add_prod(float a, float b) {
        float pr = __fmul_rn(a, b);
        float pe = __fmaf_rn(a, b, -pr);
        float t = __fadd_rn(hi, pr);
        float bp = __fsub_rn(t, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(pr, bp));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    // Fast2Sum: |hi| >= |lo| holds for the sums of squares and products accumulated here
    __device__ __forceinline__ void renorm() {
        const float s = __fadd_rn(hi, lo);
        lo = __fsub_rn(lo, __fsub_rn(s, hi));
        hi = s;
    }
    // += another float-float sum (TwoSum of the high parts, low parts added)
    __device__ __forceinline__ void add(const FF& o) {
        float t = __fadd_rn(hi, o.hi);
        float bp = __fsub_rn(t, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(o.hi, bp));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(e, o.lo));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Float-float product and square root (about 2^-44 relative; inputs and results normal FP32
// numbers): a b = a.hi b.hi (exact TwoProd) + the cross terms; sqrt(a) = s + (a - s^2) / (2 s) with
// s = sqrt(a.hi) and the residual a.hi - s^2 exact through an FMA.
__device__ __forceinline__ FF ff_mul(const FF& a, const FF& b) {
    const float ph = __fmul_rn(a.hi, b.hi);
    const float pl = __fadd_rn(__fmaf_rn(a.hi, b.hi, -ph), __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    FF r;
    r.hi = __fadd_rn(ph, pl);
    r.lo = __fsub_rn(pl, __fsub_rn(r.hi, ph));
    return r;
}
__device__ __forceinline__ FF ff_sqrt(const FF& a) {
    FF r;
    if (!(a.hi > 0.f)) { r.hi = 0.f; r.lo = 0.f; return r; }
    const float sh = __fsqrt_rn(a.hi);
    const float e = __fadd_rn(__fmaf_rn(-sh, sh, a.hi), a.lo);
    const float sl = __fmul_rn(e, __frcp_rn(__fmul_rn(2.f, sh)));
    r.hi = __fadd_rn(sh, sl);
    r.lo = __fsub_rn(sl, __fsub_rn(r.hi, sh));
    return r;
}

// Two independent float-float sums in paired FP32 registers: every operation is the one of FF
// applied to both halves with the sm_100+ two-wide FP32 instructions (one issue slot for two
// rounded operations), so each half is bit-identical to an FF that saw the same terms.
struct FF2 {
    float2 hi, lo;
    static __device__ __forceinline__ float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
    __device__ __forceinline__ void zero() { hi = make_float2(0.f, 0.f); lo = hi; }
    __device__ __forceinline__ void add_sq(float2 v) {
        const float2 pr = __fmul2_rn(v, v);
        const float2 pe = __ffma2_rn(v, v, neg(pr));
        const float2 t = __fadd2_rn(hi, pr);
        const float2 bp = __fadd2_rn(t, neg(hi));
        const float2 e = __fadd2_rn(__fadd2_rn(hi, neg(__fadd2_rn(t, neg(bp)))), __fadd2_rn(pr, neg(bp)));
        hi = t;
        lo = __fadd2_rn(lo, __fadd2_rn(e, pe));
    }
    // += v * v when the squares are exact in FP32 (v has at most 12 significant bits, e.g. BF16,
    // and v * v is a normal number): the TwoProd residual is zero and is left out
    __device__ __forceinline__ void add_sq_exact(float2 v) {
        const float2 pr = __fmul2_rn(v, v);
        const float2 t = __fadd2_rn(hi, pr);
        const float2 bp = __fadd2_rn(t, neg(hi));
        const float2 e = __fadd2_rn(__fadd2_rn(hi, neg(__fadd2_rn(t, neg(bp)))), __fadd2_rn(pr, neg(bp)));
        hi = t;
        lo = __fadd2_rn(lo, e);
    }
    __device__ __forceinline__ void renorm() {
        const float2 s = __fadd2_rn(hi, lo);
        lo = __fadd2_rn(lo, neg(__fadd2_rn(s, neg(hi))));
        hi = s;
    }
    __device__ __forceinline__ void add(const FF2& o) {
        const float2 t = __fadd2_rn(hi, o.hi);
        const float2 bp = __fadd2_rn(t, neg(hi));
        const float2 e = __fadd2_rn(__fadd2_rn(hi, neg(__fadd2_rn(t, neg(bp)))), __fadd2_rn(o.hi, neg(bp)));
        hi = t;
        lo = __fadd2_rn(lo, __fadd2_rn(e, o.lo));
    }
    __device__ __forceinline__ FF half(int i) const {
        FF r;
        r.hi = i ? hi.y : hi.x;
        r.lo = i ? lo.y : lo.x;
        return r;
    }
    // += a * b in each half (exact TwoProd residual)
    __device__ __forceinline__ void add_prod(float2 a, float2 b) {
        const float2 pr = __fmul2_rn(a, b);
        const float2 pe = __ffma2_rn(a, b, neg(pr));
        const float2 t = __fadd2_rn(hi, pr);
        const float2 bp = __fadd2_rn(t, neg(hi));
        const float2 e = __fadd2_rn(__fadd2_rn(hi, neg(__fadd2_rn(t, neg(bp)))), __fadd2_rn(pr, neg(bp)));
        hi = t;
        lo = __fadd2_rn(lo, __fadd2_rn(e, pe));
    }
    // the two halves added into one sum
    __device__ __forceinline__ FF both() const {
        FF r = half(0);
        r.add(half(1));
        r.renorm();
        return r;
    }
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
        uint32_t hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
        U4 n;
        n.x = hi1 ^ ctr.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ ctr.w ^ k1;
        n.w = lo0;
        ctr = n;
        k0 += W0;
        k1 += W1;
    }
    return ctr;
}

// 64-bit uniform of global draw t in stream sid: (x1 << 32) | x0.
__device__ __forceinline__ uint64_t draw_bits(uint64_t seed, uint64_t sid, uint64_t t) {
    U4 c{(uint32_t)t, (uint32_t)(t >> 32), (uint32_t)sid, (uint32_t)(sid >> 32)};
    U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((uint64_t)o.y << 32) | (uint64_t)o.x;
}

// ---------------------------------------------------------------- diagnostics
// Kernels launched by this library since it was loaded (read by bmm_launch_count).
inline std::atomic<unsigned long long>& launch_counter() {
    static std::atomic<unsigned long long> n{0};
    return n;
}
inline void count_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------------- misc
__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace bmm
