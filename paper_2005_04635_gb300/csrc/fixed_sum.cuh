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

// round-toward-zero(x 2^100) of an FP32 x with |x| < 2^54 as t 2^50 + l (both
// of the sign of x): x 2^100 = t 2^50 + r 2^100, t = trunc(x 2^50) and
// r = x - t 2^-50 exact in FP32, so trunc(x 2^100) = t 2^50 + trunc(r 2^100);
// |l| < 2^50.  Float-to-integer conversions replace a variable 128-bit shift.
__host__ __device__ __forceinline__ void fix_parts(float x, long long &t, long long &l) {
    const float tf = truncf(x * 0x1p50f);
    t = (long long)tf;
    l = (long long)(fmaf(tf, -0x1p-50f, x) * 0x1p100f);
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

// The same sum as fix_add for FP32 values |x| < 2^E, E <= 4, with the value
// split by fix_parts (two float-to-integer conversions) instead of a variable
// shift.  Measured on GB300: faster in the HBM-bound streaming pass (n = 33:
// 6710 against 6654 GB/s), slower in the on-chip iterators, where the
// conversions' latency lies on the critical path (grid iterator n = 20: 3.48
// against 3.15 us per iteration), which therefore keep fix_add.
template <int E> __device__ __forceinline__ void fix_add_cvt(u128 &acc, double &side, float x) {
    static_assert(E <= 4, "fix_parts needs |x| < 2^54 and the 2^-50 part below 2^54");
    const unsigned b = __float_as_uint(x);
    if (((b >> 23) & 0xFFu) >= 127u + E) {
        side = side_add(side, (double)x);
        return;
    }
    long long t, l;
    fix_parts(x, t, l);
    acc += (u128)((__int128)t << 50) + (u128)(__int128)l;
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
// Scaled by 2^e (folded into the exponent; the result must stay normal).
__device__ __forceinline__ double i192_to_double(I192 x, int e = 0) {
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
    const double v = __ull2double_rn(top | (rest != 0ull ? 1ull : 0ull)) * __hiloint2double((1023 + shift + e) << 20, 0);
    return neg ? -v : v;
}

// The float-pair conversion below also compiles for the host, where a unit
// test checks it against exact rounding.
__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}
__host__ __device__ __forceinline__ float float_from_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, sizeof f);
    return f;
#endif
}

// a != 0 shifted left so that bit 127 is set: returns the shift, H:L the result.
__host__ __device__ __forceinline__ int norm128(u128 a, unsigned long long &H, unsigned long long &L) {
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    if (hi) {
        const int lz = clz64(hi);
        H = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
        L = lo << lz;
        return lz;
    }
    const int lz = clz64(lo);
    H = lo << lz;
    L = 0;
    return 64 + lz;
}

// Rounds a normalised H:L to its top 24 bits (ties to even): returns m, set
// up when the rounding went up (m may then reach 2^24).
__host__ __device__ __forceinline__ uint32_t top24_rn(unsigned long long H, unsigned long long L, bool &up) {
    const uint32_t m = (uint32_t)(H >> 40);
    up = ((H >> 39) & 1ull) && ((H & ((1ull << 39) - 1)) | L | (m & 1u));
    return m + (up ? 1u : 0u);
}

// x * 2^s for a signed 128-bit integer x as an unevaluated float pair:
// hi = RN(x 2^s), lo = RN(x 2^s - hi), ties to even.  Integer work only, the
// float bits assembled directly (on the GB300 a single FP64 operation costs
// about as much latency as this whole routine).  Every nonzero value involved
// must be a normal float: the caller keeps s >= -126 and |x| 2^s < 2^127.
__host__ __device__ __forceinline__ float2 fix_to_f32_pair(u128 x, int s) {
    if (x == 0) return make_float2(0.f, 0.f);
    const uint32_t sign = (uint32_t)((unsigned long long)(x >> 64) >> 63) << 31;
    unsigned long long H, L;
    const int lz = norm128(sign ? (u128)0 - x : x, H, L);
    bool up;
    const uint32_t m = top24_rn(H, L, up);
    // a float m * 2^E with 2^23 <= m <= 2^24 has the bits ((E + 149) << 23) + m
    const uint32_t hb = ((uint32_t)(104 - lz + s + 149) << 23) + m;
    // |x| - hi in units of the normalised frame (below 2^104, at most 2^103 after rounding up)
    u128 r = ((u128)(H & ((1ull << 40) - 1)) << 64) | L;
    if (up) r = ((u128)1 << 104) - r;
    uint32_t lb = 0;
    if (r != 0) {
        unsigned long long H2, L2;
        const int lz2 = norm128(r, H2, L2);
        bool up2;
        const uint32_t m2 = top24_rn(H2, L2, up2);
        lb = ((((uint32_t)(104 - lz2 - lz + s + 149) << 23) + m2) | ((up ? 1u : 0u) << 31)) ^ sign;
    }
    return make_float2(float_from_bits(hb | sign), float_from_bits(lb));
}

}  // namespace grv
