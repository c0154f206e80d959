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
template <int G> __device__ __forceinline__ float pairwise(const float *v) {
    if constexpr (G == 1) return v[0];
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

}  // namespace ph
}  // namespace grv
