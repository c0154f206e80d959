// grid_exchange.cuh -- exact grid-wide sums between the CTAs of a persistent
// cooperative launch, through global memory.
//
// Every CTA contributes NV signed 128-bit fixed-point values (plus FP64 side
// values for magnitudes outside the fixed-point window).  One thread per CTA:
//   * adds the three 43-bit limbs of each value into 64-bit accumulators, each
//     on its own 128-byte line (integer adds: exact and independent of the
//     order; G <= 512 limbs sum to less than 2^52, so no add carries out);
//   * writes its side values to its slot, and counts a CTA with side values
//     in one more accumulator;
//   * adds 1 to an arrival counter with release semantics;
//   * polls the counter with acquire loads (at most wait_limit polls) until
//     it reads G * (xi + 1) for exchange number xi;
//   * reads the accumulators and takes the difference from what it read two
//     exchanges earlier (accumulator sets alternate by exchange parity and are
//     never reset within a launch), rebuilds each total modulo 2^128 (the true
//     total fits, so this is exact) and rounds it once to FP64; side values are
//     added in rank order when any CTA had some.
// Every CTA obtains the bitwise identical totals.  A set is written again only
// after the counter shows every CTA's next contribution, which each CTA makes
// only after it has read the set.  The accumulators and the counter must be
// zero at launch.
#pragma once

#include "fixed_sum.cuh"

namespace grv {

constexpr int kGxLine = 16;  // 64-bit words per 128-byte line

template <int NV> struct GxLayout {
    static constexpr int W = 3 * NV + 1;                                         // accumulators per set
    static constexpr size_t kAccBytes = sizeof(unsigned long long) * kGxLine * (2 * W + 1);  // + counter line
    static constexpr size_t side_bytes(unsigned G) { return sizeof(double) * 2 * (size_t)G * NV; }
};

__device__ __forceinline__ void gx_red_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void gx_red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gx_ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Called by one thread of each CTA.  region: accumulators [2][W] lines, then
// the counter line, then side slots [2][G][NV] doubles.  prev: per-thread
// copy of the accumulators' last values [2][W], zero at launch.  Returns
// false if the wait ran out (tot is then unset).
template <int NV>
__device__ bool gx_exchange(const u128 (&v)[NV], const double (&side)[NV], int any_side, unsigned long long *region,
                            unsigned long long (&prev)[2][3 * NV + 1], long long xi, unsigned G, unsigned rank,
                            long long wait_limit, bool withhold, double (&tot)[NV]) {
    constexpr int W = 3 * NV + 1;
    const int par = (int)(xi & 1);
    unsigned long long *acc = region + (size_t)par * W * kGxLine;
    unsigned long long *counter = region + (size_t)2 * W * kGxLine;
    double *slots = reinterpret_cast<double *>(region + (size_t)(2 * W + 1) * kGxLine);
    if (!withhold) {
        const u128 lm = ((u128)1 << 43) - 1;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const unsigned long long l0 = (unsigned long long)(v[q] & lm);
            const unsigned long long l1 = (unsigned long long)((v[q] >> 43) & lm);
            const unsigned long long l2 = (unsigned long long)(v[q] >> 86);
            if (l0) gx_red_add(acc + (3 * q + 0) * kGxLine, l0);
            if (l1) gx_red_add(acc + (3 * q + 1) * kGxLine, l1);
            if (l2) gx_red_add(acc + (3 * q + 2) * kGxLine, l2);
            slots[((size_t)par * G + rank) * NV + q] = side[q];
        }
        if (any_side) gx_red_add(acc + (3 * NV) * kGxLine, 1ull);
        gx_red_release_add(counter, 1ull);
    }
    const unsigned long long target = (unsigned long long)G * (unsigned long long)(xi + 1);
    long long polls = 0;
    while (gx_ld_acquire(counter) < target)
        if (++polls >= wait_limit) return false;
    unsigned long long d[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const unsigned long long cur = __ldcg(acc + w * kGxLine);
        d[w] = cur - prev[par][w];
        prev[par][w] = cur;
    }
    double sd[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sd[q] = 0.0;
    if (d[3 * NV]) {
        for (unsigned r = 0; r < G; ++r)
#pragma unroll
            for (int q = 0; q < NV; ++q) sd[q] += __ldcg(slots + ((size_t)par * G + r) * NV + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const u128 T = (u128)d[3 * q] + ((u128)d[3 * q + 1] << 43) + ((u128)d[3 * q + 2] << 86);
        tot[q] = i192_to_double(i192_from(T)) * 0x1p-100 + sd[q];
    }
    return true;
}

}  // namespace grv
