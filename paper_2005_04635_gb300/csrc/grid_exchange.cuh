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
// words (relaxed loads issued together, at most wait_limit rounds) until each
// has risen by G * 2^52 plus a limb sum since it last read it: completion and
// the data arrive in one read, with no separate counter and no fence, since
// everything a reader needs is inside the words it reads.  It rebuilds each
// exact total modulo 2^128 (the true total fits) and hands it back as an
// integer, with the FP64 side sum; the caller rounds it as it needs.
// Side values are rare (only non-normalised states reach them).  When the
// counts show that some CTA has any, every CTA (they all read the same sums)
// takes a second round: it writes its side values to its slot, makes a
// release-ordered arrival on a further word, waits for all G arrivals and
// fences (acquire) before it sums the slots in rank order.  Every CTA obtains
// the bitwise identical totals.
// Words alternate between two sets by exchange parity and are never reset
// within a launch (each thread keeps what it read two exchanges earlier).  A
// CTA adds to a set again only after it has read every CTA's contribution to
// the exchange in between, which each CTA issues only after its reads of the
// set have returned (the poll loop's exit depends on them), so no read can see
// a later exchange's contributions.  The words must be zero at launch.
#pragma once

#include "fixed_sum.cuh"

namespace grv {

constexpr int kGxLine = 16;  // 64-bit words per 128-byte line

template <int NV> struct GxLayout {
    static constexpr int W = 3 * NV + 2;  // words per set: limbs, arrivals (+ side flags), side-round arrivals
    static constexpr size_t kAccBytes = sizeof(unsigned long long) * kGxLine * 2 * W;
    static constexpr size_t side_bytes(unsigned G) { return sizeof(double) * 2 * (size_t)G * NV; }
};

__device__ __forceinline__ void gx_red_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void gx_red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gx_ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void gx_fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Called by one thread of each CTA.  region: word sets [2][W] lines, then side
// slots [2][G][NV] doubles.  prev: this thread's copy of the words' last values
// [2][W], zero at launch.  On return tot holds the exact integer totals (units
// of 2^-100, two's complement) and sd the side sums.  Returns false if a wait
// ran out (tot and sd are then unset).
template <int NV>
__device__ bool gx_exchange(const u128 (&v)[NV], const double (&side)[NV], int any_side, unsigned long long *region,
                            unsigned long long (&prev)[2][GxLayout<NV>::W], long long xi, unsigned G, unsigned rank,
                            long long wait_limit, bool withhold, u128 (&tot)[NV], double (&sd)[NV]) {
    constexpr int W1 = 3 * NV + 1;  // words of the first round
    constexpr unsigned long long kOne = 1ull << 52, kLow = kOne - 1;
    const int par = (int)(xi & 1);
    unsigned long long *acc = region + (size_t)par * GxLayout<NV>::W * kGxLine;
    double *slots = reinterpret_cast<double *>(region + (size_t)2 * GxLayout<NV>::W * kGxLine);
    if (!withhold) {
        const u128 lm = ((u128)1 << 43) - 1;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            gx_red_add(acc + (3 * q + 0) * kGxLine, kOne + (unsigned long long)(v[q] & lm));
            gx_red_add(acc + (3 * q + 1) * kGxLine, kOne + (unsigned long long)((v[q] >> 43) & lm));
            gx_red_add(acc + (3 * q + 2) * kGxLine, kOne + (unsigned long long)(v[q] >> 86));
        }
        gx_red_add(acc + (3 * NV) * kGxLine, kOne + (any_side ? 1ull : 0ull));
    }
    unsigned long long d[W1];
    for (long long polls = 0;; ++polls) {
        bool all = true;
#pragma unroll
        for (int w = 0; w < W1; ++w) {
            d[w] = gx_ld_relaxed(acc + w * kGxLine) - prev[par][w];
            all = all && (d[w] >> 52) == G;
        }
        if (all) break;
        if (polls + 1 >= wait_limit) return false;
    }
#pragma unroll
    for (int w = 0; w < W1; ++w) prev[par][w] += d[w];
#pragma unroll
    for (int q = 0; q < NV; ++q) sd[q] = 0.0;
    if (d[3 * NV] & kLow) {
        // second round, taken by every CTA: slots, release arrival, acquire
        double *mine = slots + ((size_t)par * G + rank) * NV;
#pragma unroll
        for (int q = 0; q < NV; ++q) mine[q] = side[q];
        unsigned long long *cnt = acc + W1 * kGxLine;
        gx_red_release_add(cnt, kOne);
        unsigned long long c;
        for (long long polls = 0;; ++polls) {
            c = gx_ld_relaxed(cnt) - prev[par][W1];
            if ((c >> 52) == G) break;
            if (polls + 1 >= wait_limit) return false;
        }
        prev[par][W1] += c;
        gx_fence_acquire();
        for (unsigned r = 0; r < G; ++r)
#pragma unroll
            for (int q = 0; q < NV; ++q) sd[q] += __ldcg(slots + ((size_t)par * G + r) * NV + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
        tot[q] = (u128)(d[3 * q] & kLow) + ((u128)(d[3 * q + 1] & kLow) << 43) + ((u128)(d[3 * q + 2] & kLow) << 86);
    return true;
}

}  // namespace grv
