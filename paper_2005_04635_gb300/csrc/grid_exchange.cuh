// grid_exchange.cuh -- exact grid-wide sums between the CTAs of a persistent
// cooperative launch, through global memory.
//
// Every CTA contributes NV signed 128-bit fixed-point values (plus FP64 side
// values for magnitudes outside the fixed-point window).  One thread per CTA
// adds, into each of 3 NV + 1 64-bit accumulator words (one 128-byte line
// each), 2^52 plus its part: the three 43-bit limbs of each value, and for the
// last word whether it has side values.  A word's top 12 bits thus count the
// CTAs that have contributed and its low 52 bits hold their exact limb sum
// (G <= 512 limbs of 43 bits stay below 2^52).  The same thread then polls the
// words (acquire loads, at most wait_limit rounds) until each has risen by
// G * 2^52 plus a limb sum since it last read it: completion and the data
// arrive in one read, with no separate counter.  It rebuilds each total modulo
// 2^128 (the true total fits, so this is exact) and rounds it once to FP64;
// side values (written to per-CTA slots before the release-ordered add to the
// last word) are added in rank order when any CTA had some.  Every CTA obtains
// the bitwise identical totals.
// Words alternate between two sets by exchange parity and are never reset
// within a launch (each thread keeps what it read two exchanges earlier).  A
// CTA adds to a set again only after it has read every CTA's contribution to
// the exchange in between, which each CTA makes only after it has read the
// set, so no read can see a later exchange's contributions.  The words must be
// zero at launch.
#pragma once

#include "fixed_sum.cuh"

namespace grv {

constexpr int kGxLine = 16;  // 64-bit words per 128-byte line

template <int NV> struct GxLayout {
    static constexpr int W = 3 * NV + 1;                                         // words per set
    static constexpr size_t kAccBytes = sizeof(unsigned long long) * kGxLine * (2 * W + 1);
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
__device__ __forceinline__ unsigned long long gx_ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Called by one thread of each CTA.  region: word sets [2][W] lines, one spare
// line, then side slots [2][G][NV] doubles.  prev: this thread's copy of the
// words' last values [2][W], zero at launch.  Returns false if the wait ran
// out (tot is then unset).
template <int NV>
__device__ bool gx_exchange(const u128 (&v)[NV], const double (&side)[NV], int any_side, unsigned long long *region,
                            unsigned long long (&prev)[2][3 * NV + 1], long long xi, unsigned G, unsigned rank,
                            long long wait_limit, bool withhold, double (&tot)[NV]) {
    constexpr int W = 3 * NV + 1;
    constexpr unsigned long long kOne = 1ull << 52, kLow = kOne - 1;
    const int par = (int)(xi & 1);
    unsigned long long *acc = region + (size_t)par * W * kGxLine;
    double *slots = reinterpret_cast<double *>(region + (size_t)(2 * W + 1) * kGxLine);
    if (!withhold) {
        const u128 lm = ((u128)1 << 43) - 1;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            slots[((size_t)par * G + rank) * NV + q] = side[q];
            gx_red_add(acc + (3 * q + 0) * kGxLine, kOne + (unsigned long long)(v[q] & lm));
            gx_red_add(acc + (3 * q + 1) * kGxLine, kOne + (unsigned long long)((v[q] >> 43) & lm));
            gx_red_add(acc + (3 * q + 2) * kGxLine, kOne + (unsigned long long)(v[q] >> 86));
        }
        // release: the side slots are visible to whoever sees this count
        gx_red_release_add(acc + (3 * NV) * kGxLine, kOne + (any_side ? 1ull : 0ull));
    }
    unsigned long long d[W];
    for (long long polls = 0;; ++polls) {
        bool all = true;
        d[3 * NV] = gx_ld_acquire(acc + (3 * NV) * kGxLine) - prev[par][3 * NV];
        all = (d[3 * NV] >> 52) == G;
#pragma unroll
        for (int w = 0; w < 3 * NV; ++w) {
            d[w] = gx_ld_relaxed(acc + w * kGxLine) - prev[par][w];
            all = all && (d[w] >> 52) == G;
        }
        if (all) break;
        if (polls + 1 >= wait_limit) return false;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) prev[par][w] += d[w];
    double sd[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sd[q] = 0.0;
    if (d[3 * NV] & kLow) {
        for (unsigned r = 0; r < G; ++r)
#pragma unroll
            for (int q = 0; q < NV; ++q) sd[q] += __ldcg(slots + ((size_t)par * G + r) * NV + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const u128 T = (u128)(d[3 * q] & kLow) + ((u128)(d[3 * q + 1] & kLow) << 43) +
                       ((u128)(d[3 * q + 2] & kLow) << 86);
        tot[q] = i192_to_double(i192_from(T)) * 0x1p-100 + sd[q];
    }
    return true;
}

}  // namespace grv
