// fixed_sum.cuh -- exact fixed-point summation on the integer pipe.
//
// The mean of the inversion about the mean (Algorithm "n-qubit Inversion about
// Mean") needs sums of up to 2^33 complex amplitudes.  On the GB300 the FP64
// pipe delivers ~1.7 adds per clock per SM, so FP64 running sums compete with
// the update itself; here values are added as signed integers in units of
// 2^-100 instead:
//   * fix_add<E>: x with |x| < 2^E is added as round-toward-zero(x * 2^100)
//     into a 128-bit accumulator (the dropped part is below 2^-100); larger
//     magnitudes, Inf and NaN go to an FP64 side sum;
//   * warp / block sums of the 128-bit accumulators are integer additions, and
//     the sum over CTAs uses 192 bits, so every reduction is exact and its
//     result does not depend on the order of the additions;
//   * i192_to_double rounds the final sum once (round to nearest).
// Callers choose E so that no 128-bit partial can overflow: a thread adds at
// most 2^16 values below 2^(100+E), and a CTA has 256 threads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace grv {

typedef unsigned __int128 u128;
constexpr int kFixFrac = 100;

// The rare out-of-window path is a real call: if it were inlined, the compiler
// would predicate its FP64 add and issue it for every value.
static __device__ __noinline__ double side_add(double side, double x) { return side + x; }

template <int E> __device__ __forceinline__ void fix_add(u128 &acc, double &side, double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e >= 1023u + E) {
        side = side_add(side, x);
        return;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0u) << 52);
    const int sh = (int)e - (1075 - kFixFrac);  // x = m * 2^(sh - 100)
    u128 v;
    if (sh >= 0) v = (u128)m << sh;
    else v = sh > -64 ? (u128)(m >> (-sh)) : (u128)0;
    const u128 neg = (u128)(__int128)((long long)b >> 63);
    acc += (v ^ neg) - neg;
}

template <int E> __device__ __forceinline__ void fix_add(u128 &acc, double &side, float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xFFu;
    if (e >= 127u + E) {
        side = side_add(side, (double)x);
        return;
    }
    const unsigned long long m = (b & 0x7FFFFFu) | ((unsigned)(e != 0u) << 23);
    const int sh = (int)e - (150 - kFixFrac);
    u128 v;
    if (sh >= 0) v = (u128)m << sh;
    else v = sh > -24 ? (u128)(m >> (-sh)) : (u128)0;
    const u128 neg = (u128)(__int128)((int)b >> 31);
    acc += (v ^ neg) - neg;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    return ((u128)__shfl_xor_sync(0xffffffffu, hi, o) << 64) | __shfl_xor_sync(0xffffffffu, lo, o);
}
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
    return v;
}

// 192-bit two's complement integer.
struct I192 {
    unsigned long long w0, w1, w2;
};
__device__ __forceinline__ I192 i192_from(u128 x) {
    const unsigned long long hi = (unsigned long long)(x >> 64);
    return I192{(unsigned long long)x, hi, (unsigned long long)((long long)hi >> 63)};
}
__device__ __forceinline__ void i192_add(I192 &a, const I192 &b) {
    asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}
__device__ __forceinline__ I192 shfl_xor_i192(const I192 &v, int o) {
    return I192{__shfl_xor_sync(0xffffffffu, v.w0, o), __shfl_xor_sync(0xffffffffu, v.w1, o),
                __shfl_xor_sync(0xffffffffu, v.w2, o)};
}
__device__ __forceinline__ I192 warp_sum_i192(I192 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) i192_add(v, shfl_xor_i192(v, o));
    return v;
}

// Rounds a 192-bit integer to the nearest double: the top 64 significant bits
// with the remaining bits folded into the lowest one (a sticky bit below the
// rounding position), converted with round to nearest, then scaled exactly.
__device__ __forceinline__ double i192_to_double(I192 x) {
    const bool neg = (long long)x.w2 < 0;
    if (neg) {
        x.w0 = ~x.w0;
        x.w1 = ~x.w1;
        x.w2 = ~x.w2;
        i192_add(x, I192{1ull, 0ull, 0ull});
    }
    int shift;
    unsigned long long top, rest;
    if (x.w2) {
        const int lz = __clzll((long long)x.w2);
        shift = 128 - lz;
        top = lz ? (x.w2 << lz) | (x.w1 >> (64 - lz)) : x.w2;
        rest = (lz ? (x.w1 << lz) : x.w1) | x.w0;
    } else if (x.w1) {
        const int lz = __clzll((long long)x.w1);
        shift = 64 - lz;
        top = lz ? (x.w1 << lz) | (x.w0 >> (64 - lz)) : x.w1;
        rest = lz ? (x.w0 << lz) : x.w0;
    } else {
        shift = 0;
        top = x.w0;
        rest = 0;
    }
    const double v = __ull2double_rn(top | (rest != 0ull ? 1ull : 0ull)) * __hiloint2double((1023 + shift) << 20, 0);
    return neg ? -v : v;
}

}  // namespace grv
