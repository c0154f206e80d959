// phase_ops.cuh -- complex helpers of the phase iterator kernels (k_phase.cu,
// k_phase_grid.cu).
#pragma once

#include <cuda_runtime.h>

namespace grv {
namespace ph {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dcmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// e^{i a} in FP64
__device__ __forceinline__ double2 expi(double a) {
    double s, c;
    sincos(a, &s, &c);
    return make_double2(c, s);
}
// a complex FP64 value as an unevaluated sum of float pairs (re hi, re lo, im hi, im lo)
__device__ __forceinline__ float4 split_hilo(double2 v) {
    const float hr = (float)v.x, hi = (float)v.y;
    return make_float4(hr, (float)(v.x - (double)hr), hi, (float)(v.y - (double)hi));
}
// c - k for k given as a float pair: the shared rounding of k is not repeated
__device__ __forceinline__ float2 sub_hilo(float2 c, float4 k) {
    return make_float2((c.x - k.x) - k.y, (c.y - k.z) - k.w);
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// ---- float-float numbers: hi + lo with |lo| <= ulp(hi) / 2, about 48
// significant bits from FP32 operations alone (error-free sums after Knuth
// and Dekker, products with one FMA).  The per-step constants of the on-chip
// sweeps are formed this way: FP64 on the GB300 costs ~100-175 cycles of
// latency per operation.  The _rn intrinsics keep the compiler from
// contracting or reordering the error-free steps.
// Rounded FP32 operations that neither the device nor the host compiler may
// contract or reorder (the float-float helpers also compile for the host,
// where a unit test checks their error bounds).
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}
__host__ __device__ __forceinline__ float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return __builtin_fmaf(a, b, c);
#endif
}

struct ff {
    float hi, lo;
};
__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = add_rn(a, b), bb = sub_rn(s, a);
    return ff{s, add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb))};
}
__host__ __device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = add_rn(a, b);
    return ff{s, sub_rn(b, sub_rn(s, a))};
}
__host__ __device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi), t = ff_two_sum(a.lo, b.lo);
    const ff u = ff_fast_two_sum(s.hi, add_rn(s.lo, t.hi));
    return ff_fast_two_sum(u.hi, add_rn(u.lo, t.lo));
}
__host__ __device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = mul_rn(a.hi, b.hi);
    float e = fma_rn(a.hi, b.hi, -p);
    e = fma_rn(a.hi, b.lo, e);
    e = fma_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
// a double as a float-float (FP64: for constants formed off the critical path)
__host__ __device__ __forceinline__ ff ff_of(double v) {
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}

struct cff {
    ff re, im;
};
__host__ __device__ __forceinline__ cff cff_add(cff a, cff b) { return cff{ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__host__ __device__ __forceinline__ cff cff_mul(cff a, cff b) {
    return cff{ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__host__ __device__ __forceinline__ cff cff_conj(cff a) { return cff{a.re, ff_neg(a.im)}; }
// (re hi, re lo, im hi, im lo): the layout sub_hilo consumes
__host__ __device__ __forceinline__ float4 cff_pack(cff a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__host__ __device__ __forceinline__ cff cff_unpack(float4 p) { return cff{ff{p.x, p.y}, ff{p.z, p.w}}; }

template <int G> __device__ __forceinline__ float pairwise(const float *v) {
    if constexpr (G == 1) return v[0];
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

}  // namespace ph
}  // namespace grv
