// k_resident.cu -- persistent on-chip Grover iterators for small and mid-size
// states: one thread-block cluster (k_resident_cluster) or the whole grid
// (k_resident_grid, further down).
//
// One thread-block cluster of C CTAs (C <= 16) runs all k iterations of the
// proposed grover_search loop in one launch.  CTA r keeps amplitudes
// [r*L, (r+1)*L) in its shared memory from the first load to the final store,
// together with a bitmask of the marked indices of its slice (the oracle's
// solution list, Algorithm "n-qubit Oracle").  Each iteration (Algorithm
// "n-qubit Inversion about Mean"):
//   1. every thread updates its amplitudes in shared memory,
//        c <- 2 mu - O c,
//      and adds O c_new into a 128-bit fixed-point sum (exact: 100 fractional
//      bits; complex64 adds the FP32 pairwise sum of each 8-amplitude group,
//      16 in the grid iterator's wide slices);
//   2. the CTA reduces its threads' sums exactly (integer shuffles) into a
//      partial in its own shared memory;
//   3. a hardware cluster barrier (release / acquire), then every CTA reads
//      the C partials through distributed shared memory and adds them in
//      integers, so all CTAs obtain the bitwise identical next mean without
//      any global-memory round trip or spin-wait.
// Partials are double buffered, so one barrier per iteration suffices: a CTA
// can overwrite a slot only after every CTA has passed the next barrier, which
// each CTA reaches only after it has read that slot.
//
// The fixed-point window is |x| < 16: for N <= 2^22 the whole state sums to
// less than 2^26 in magnitude, so no 128-bit sum can overflow.  Larger
// magnitudes, Inf and NaN go to an FP64 side sum combined in a fixed order.
#include <cooperative_groups.h>

#include "fixed_sum.cuh"
#include "grid_exchange.cuh"
#include "grover_internal.cuh"

namespace grv {
namespace {

namespace cg = cooperative_groups;

constexpr int kResThreads = 256;
constexpr int kResWarps = kResThreads / 32;

template <class T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int APV = 2;
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int APV = 1;
};

__device__ __forceinline__ float flip(float x, uint32_t f) { return __uint_as_float(__float_as_uint(x) ^ (f << 31)); }
__device__ __forceinline__ double flip(double x, uint32_t f) {
    return __hiloint2double(__double2hiint(x) ^ (int)(f << 31), __double2loint(x));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Nonzero side sums, tested on the bits (an FP64 compare would sit on the slow
// FP64 pipe; -0.0 merely takes the FP64 route below).
__device__ __forceinline__ bool has_side(double a, double b) {
    return (__double_as_longlong(a) | __double_as_longlong(b)) != 0;
}

// The mean from the exact sums r, i (units 2^-100) and the side sums sr, si,
// N = 2^n.  Without side sums, mu = RN(sum / N) straight from the integers, and
// the complex64 update's float pair for 2 mu is RN(2 mu exact) plus the
// rounded rest, built with integer operations only (GB300's FP64 pipe would
// put ~1500 cycles of latency on every iteration).  With side sums (non-
// normalised states) everything goes through FP64: (RN(r 2^-100) + sr) / N.
__device__ __forceinline__ void write_mean_slot(MeanSlot *ms, u128 r, u128 i, double sr, double si, int n,
                                                bool need_f32, bool need_f64) {
    if (!has_side(sr, si)) {
        if (need_f32) {
            const float2 pr = fix_to_f32_pair(r, -99 - n), pi = fix_to_f32_pair(i, -99 - n);
            ms->two32 = make_float4(pr.x, pr.y, pi.x, pi.y);
        }
        if (need_f64) {
            const double tr = i192_to_double(i192_from(r), -99 - n), ti = i192_to_double(i192_from(i), -99 - n);
            ms->two = make_double2(tr, ti);
            ms->mu = make_double2(0.5 * tr, 0.5 * ti);
        }
        return;
    }
    const double inv_n = __hiloint2double((1023 - n) << 20, 0);
    const double mr = (i192_to_double(i192_from(r), -100) + sr) * inv_n;
    const double mi = (i192_to_double(i192_from(i), -100) + si) * inv_n;
    const double tr = 2.0 * mr, ti = 2.0 * mi;
    const float hr = (float)tr, hi = (float)ti;
    ms->mu = make_double2(mr, mi);
    ms->two = make_double2(tr, ti);
    ms->two32 = make_float4(hr, (float)(tr - (double)hr), hi, (float)(ti - (double)hi));
}

// Sums behind the last mean, kept by the thread that built it, so that the
// full slot (FP64 mean included) is written once, after the last iteration.
struct LastSums {
    u128 r = 0, i = 0;
    double sr = 0.0, si = 0.0;
};

template <int G, class T> __device__ __forceinline__ T pairwise(const T *v) {
    if constexpr (G == 1) return v[0];
    else if constexpr (G == 2) return v[0] + v[1];
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

struct Part {
    unsigned long long rl, rh, il, ih;
    double sr, si;
    int side;  // any side sum in this CTA
};

template <class T>
__global__ void __launch_bounds__(kResThreads) k_resident_cluster(ResArgs a) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    constexpr int U = 4;  // vectors per thread per group
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), C = cl.num_blocks();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    V *sl = reinterpret_cast<V *>(smem);
    const uint32_t nv = a.slice_vecs;
    const uint32_t nbits = nv * APV, nwords = (nbits + 31) / 32;
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + (size_t)nv * sizeof(V));
    __shared__ Part part[2];
    __shared__ unsigned long long wint[kResWarps][4];
    __shared__ double wside[kResWarps][2];
    __shared__ MeanSlot s_mu;

    V *g = static_cast<V *>(a.amps) + (size_t)rank * nv;
    const uint64_t a0 = (uint64_t)rank * nbits;

    for (uint32_t j = threadIdx.x; j < nv; j += kResThreads) sl[j] = g[j];
    for (uint32_t w = threadIdx.x; w < nwords; w += kResThreads) fm[w] = 0u;
    __syncthreads();
    if (a.mk.mode == MARK_LIST) {
        for (uint64_t i = threadIdx.x; i < a.mk.m; i += kResThreads) {
            const uint64_t x = a.mk.list[i];
            if (x >= a0 && x < a0 + nbits) atomicOr(fm + ((x - a0) >> 5), 1u << (uint32_t)((x - a0) & 31));
        }
    } else if (a.mk.mode == MARK_BITS) {
        for (uint32_t e = threadIdx.x; e < nbits; e += kResThreads) {
            const uint64_t x = a0 + e;
            if ((a.mk.words[x >> 5] >> (uint32_t)(x & 31)) & 1u) atomicOr(fm + (e >> 5), 1u << (e & 31));
        }
    }
    __syncthreads();

    LastSums last;
    // t = -1 computes the first mean, t = 0..k-1 are the iterations
    for (long long t = -1; t < (long long)a.k; ++t) {
        const bool upd = t >= 0;
        const int slot = (int)((t + 1) & 1);
        T two_re = T(0), two_im = T(0), lo_re = T(0), lo_im = T(0);
        if (upd) {
            if constexpr (APV == 2) {
                two_re = s_mu.two32.x;
                lo_re = s_mu.two32.y;
                two_im = s_mu.two32.z;
                lo_im = s_mu.two32.w;
            } else {
                two_re = s_mu.two.x;
                two_im = s_mu.two.y;
            }
        }
        u128 ar = 0, ai = 0;
        double sr = 0.0, si = 0.0;
        for (uint32_t j0 = threadIdx.x; j0 < nv; j0 += U * kResThreads) {
            T gr[U * APV], gi[U * APV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * kResThreads;
                if (j >= nv) {
#pragma unroll
                    for (int q = 0; q < APV; ++q) gr[u * APV + q] = gi[u * APV + q] = T(0);
                    continue;
                }
                V c = sl[j];
                const uint32_t e = j * APV;
                const uint32_t f = (fm[e >> 5] >> (e & 31)) & ((1u << APV) - 1u);
                if constexpr (APV == 2) {
                    const uint32_t f0 = f & 1u, f1 = f >> 1;
                    if (upd) {
                        c.x = (two_re - flip(c.x, f0)) + lo_re;
                        c.y = (two_im - flip(c.y, f0)) + lo_im;
                        c.z = (two_re - flip(c.z, f1)) + lo_re;
                        c.w = (two_im - flip(c.w, f1)) + lo_im;
                        sl[j] = c;
                    }
                    gr[2 * u] = flip(c.x, f0);
                    gi[2 * u] = flip(c.y, f0);
                    gr[2 * u + 1] = flip(c.z, f1);
                    gi[2 * u + 1] = flip(c.w, f1);
                } else {
                    if (upd) {
                        c.x = two_re - flip(c.x, f);
                        c.y = two_im - flip(c.y, f);
                        sl[j] = c;
                    }
                    gr[u] = flip(c.x, f);
                    gi[u] = flip(c.y, f);
                }
            }
            if constexpr (APV == 2) {
                fix_add<4>(ar, sr, pairwise<U * APV>(gr));
                fix_add<4>(ai, si, pairwise<U * APV>(gi));
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    fix_add<4>(ar, sr, gr[u]);
                    fix_add<4>(ai, si, gi[u]);
                }
            }
        }
        // CTA partial: exact integer sums, side sums (if any) in a fixed tree order
        ar = warp_sum_u128(ar);
        ai = warp_sum_u128(ai);
        if (__any_sync(0xffffffffu, has_side(sr, si))) {
            sr = warp_sum(sr);
            si = warp_sum(si);
        }
        if (lane == 0) {
            wint[warp][0] = (unsigned long long)ar;
            wint[warp][1] = (unsigned long long)(ar >> 64);
            wint[warp][2] = (unsigned long long)ai;
            wint[warp][3] = (unsigned long long)(ai >> 64);
            wside[warp][0] = sr;
            wside[warp][1] = si;
        }
        __syncthreads();
        if (warp == 0) {
            u128 r = 0, i = 0;
            double s1 = 0.0, s2 = 0.0;
            if (lane < kResWarps) {
                r = ((u128)wint[lane][1] << 64) | wint[lane][0];
                i = ((u128)wint[lane][3] << 64) | wint[lane][2];
                s1 = wside[lane][0];
                s2 = wside[lane][1];
            }
            r = warp_sum_u128(r);
            i = warp_sum_u128(i);
            const int any_side = __any_sync(0xffffffffu, has_side(s1, s2));
            if (any_side) {
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
            }
            if (lane == 0) part[slot] = Part{(unsigned long long)r, (unsigned long long)(r >> 64),
                                             (unsigned long long)i, (unsigned long long)(i >> 64), s1, s2, any_side};
        }
        cl.sync();
        if (warp == 0) {
            u128 r = 0, i = 0;
            double s1 = 0.0, s2 = 0.0;
            int side = 0;
            if (lane < (int)C) {
                const Part *rp = cl.map_shared_rank(&part[slot], lane);
                r = ((u128)rp->rh << 64) | rp->rl;
                i = ((u128)rp->ih << 64) | rp->il;
                s1 = rp->sr;
                s2 = rp->si;
                side = rp->side;
            }
            r = warp_sum_u128(r);
            i = warp_sum_u128(i);
            if (__any_sync(0xffffffffu, side)) {
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
            }
            if (lane == 0) {
                write_mean_slot(&s_mu, r, i, s1, s2, a.n, APV == 2, APV == 1);
                last = LastSums{r, i, s1, s2};
            }
        }
        __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < nv; j += kResThreads) g[j] = sl[j];
    if (rank == 0 && threadIdx.x == 0) {
        write_mean_slot(&s_mu, last.r, last.i, last.sr, last.si, a.n, true, true);
        *a.mu_out = s_mu;
    }
    cl.sync();  // keep every CTA's partial slots alive until all have read them
}

// ---- grid-wide variant ----------------------------------------------------------------
// The same iteration over all SMs: a cooperative launch of G CTAs (one per SM,
// all co-resident), CTA r keeping vectors [r*L, min((r+1)*L, nvec)) in shared
// memory.  There is no hardware barrier across the grid, so the exact CTA
// partials meet in global memory through grid_exchange.cuh: limb sums and
// arrival counts share 64-bit words, one thread per CTA polls them (bounded)
// and rebuilds the exact total, so every CTA holds the bitwise identical mean.
// A wait that runs out sets *status = 3 and the CTA leaves the loop (the
// others then run out too).
static_assert(kRgBytes >= GxLayout<2>::kAccBytes + GxLayout<2>::side_bytes(kRgMaxGrid),
              "the grid iterator's exchange region is too small");
constexpr int kRgThreads = 512;
constexpr int kRgWarps = kRgThreads / 32;

// U vectors per thread per summation group: complex64 slices of at least
// kRgWideVecs vectors take U = 8, one FP32 pairwise sum of 16 amplitudes per
// exact fixed-point add (half the adds: 7-11 % faster per iteration at
// n = 20-22 on GB300), smaller slices U = 4 (8 amplitudes), where threads hold
// too few vectors to fill a group of 16.
constexpr uint32_t kRgWideVecs = 6 * kRgThreads;

template <class T, int U>
__global__ void __launch_bounds__(kRgThreads, 1) k_resident_grid(ResGridArgs a) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    const unsigned rank = blockIdx.x, G = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    V *sl = reinterpret_cast<V *>(smem);
    const uint64_t start = (uint64_t)rank * a.slice_vecs;
    const uint32_t nv = start >= a.nvec ? 0u
                        : (uint32_t)((a.nvec - start) < a.slice_vecs ? (a.nvec - start) : a.slice_vecs);
    const uint32_t nbits = nv * APV, nwords = (a.slice_vecs * APV + 31) / 32;
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + (size_t)a.slice_vecs * sizeof(V));
    __shared__ unsigned long long wint[kRgWarps][4];
    __shared__ double wside[kRgWarps][2];
    __shared__ unsigned long long s_prev[2][GxLayout<2>::W];
    __shared__ MeanSlot s_mu;
    __shared__ int s_abort;

    V *g = static_cast<V *>(a.amps) + start;
    const uint64_t a0 = start * APV;
    for (uint32_t j = threadIdx.x; j < nv; j += kRgThreads) sl[j] = g[j];
    for (uint32_t w = threadIdx.x; w < nwords; w += kRgThreads) fm[w] = 0u;
    if (threadIdx.x == 0) s_abort = 0;
    if (threadIdx.x < 2 * GxLayout<2>::W) s_prev[threadIdx.x / GxLayout<2>::W][threadIdx.x % GxLayout<2>::W] = 0ull;
    __syncthreads();
    if (a.mk.mode == MARK_LIST) {
        for (uint64_t i = threadIdx.x; i < a.mk.m; i += kRgThreads) {
            const uint64_t x = a.mk.list[i];
            if (x >= a0 && x < a0 + nbits) atomicOr(fm + ((x - a0) >> 5), 1u << (uint32_t)((x - a0) & 31));
        }
    } else if (a.mk.mode == MARK_BITS) {
        for (uint32_t e = threadIdx.x; e < nbits; e += kRgThreads) {
            const uint64_t x = a0 + e;
            if ((a.mk.words[x >> 5] >> (uint32_t)(x & 31)) & 1u) atomicOr(fm + (e >> 5), 1u << (e & 31));
        }
    }
    __syncthreads();

    LastSums last;
    for (long long t = -1; t < (long long)a.k; ++t) {
        const bool upd = t >= 0;
        T two_re = T(0), two_im = T(0), lo_re = T(0), lo_im = T(0);
        if (upd) {
            if constexpr (APV == 2) {
                two_re = s_mu.two32.x;
                lo_re = s_mu.two32.y;
                two_im = s_mu.two32.z;
                lo_im = s_mu.two32.w;
            } else {
                two_re = s_mu.two.x;
                two_im = s_mu.two.y;
            }
        }
        u128 ar = 0, ai = 0;
        double sr = 0.0, si = 0.0;
        for (uint32_t j0 = threadIdx.x; j0 < nv; j0 += U * kRgThreads) {
            T gr[U * APV], gi[U * APV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * kRgThreads;
                if (j >= nv) {
#pragma unroll
                    for (int q = 0; q < APV; ++q) gr[u * APV + q] = gi[u * APV + q] = T(0);
                    continue;
                }
                V c = sl[j];
                const uint32_t e = j * APV;
                const uint32_t f = (fm[e >> 5] >> (e & 31)) & ((1u << APV) - 1u);
                if constexpr (APV == 2) {
                    const uint32_t f0 = f & 1u, f1 = f >> 1;
                    if (upd) {
                        c.x = (two_re - flip(c.x, f0)) + lo_re;
                        c.y = (two_im - flip(c.y, f0)) + lo_im;
                        c.z = (two_re - flip(c.z, f1)) + lo_re;
                        c.w = (two_im - flip(c.w, f1)) + lo_im;
                        sl[j] = c;
                    }
                    gr[2 * u] = flip(c.x, f0);
                    gi[2 * u] = flip(c.y, f0);
                    gr[2 * u + 1] = flip(c.z, f1);
                    gi[2 * u + 1] = flip(c.w, f1);
                } else {
                    if (upd) {
                        c.x = two_re - flip(c.x, f);
                        c.y = two_im - flip(c.y, f);
                        sl[j] = c;
                    }
                    gr[u] = flip(c.x, f);
                    gi[u] = flip(c.y, f);
                }
            }
            if constexpr (APV == 2) {
                fix_add<4>(ar, sr, pairwise<U * APV>(gr));
                fix_add<4>(ai, si, pairwise<U * APV>(gi));
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    fix_add<4>(ar, sr, gr[u]);
                    fix_add<4>(ai, si, gi[u]);
                }
            }
        }
        // CTA partial (exact), written to its slot
        ar = warp_sum_u128(ar);
        ai = warp_sum_u128(ai);
        if (__any_sync(0xffffffffu, has_side(sr, si))) {
            sr = warp_sum(sr);
            si = warp_sum(si);
        }
        if (lane == 0) {
            wint[warp][0] = (unsigned long long)ar;
            wint[warp][1] = (unsigned long long)(ar >> 64);
            wint[warp][2] = (unsigned long long)ai;
            wint[warp][3] = (unsigned long long)(ai >> 64);
            wside[warp][0] = sr;
            wside[warp][1] = si;
        }
        __syncthreads();
        if (warp == 0) {
            u128 r = 0, i = 0;
            double s1 = 0.0, s2 = 0.0;
            if (lane < kRgWarps) {
                r = ((u128)wint[lane][1] << 64) | wint[lane][0];
                i = ((u128)wint[lane][3] << 64) | wint[lane][2];
                s1 = wside[lane][0];
                s2 = wside[lane][1];
            }
            r = warp_sum_u128(r);
            i = warp_sum_u128(i);
            const int any_side = __any_sync(0xffffffffu, has_side(s1, s2));
            if (any_side) {
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
            }
            const bool withhold = a.stall && t == -1 && rank == 0;  // test hook: this partial never arrives
            if (lane == 0) {
                const u128 v[2] = {r, i};
                const double sdv[2] = {s1, s2};
                u128 tot[2];
                double tsd[2];
                const bool ok = gx_exchange<2>(v, sdv, any_side, a.region, s_prev, t + 1, G, rank, a.wait_limit,
                                               withhold, tot, tsd);
                s_abort = ok ? 0 : 1;
                if (ok) {
                    write_mean_slot(&s_mu, tot[0], tot[1], tsd[0], tsd[1], a.n, APV == 2, APV == 1);
                    last = LastSums{tot[0], tot[1], tsd[0], tsd[1]};
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) atomicExch(a.status, 3);
            break;
        }
    }
    for (uint32_t j = threadIdx.x; j < nv; j += kRgThreads) g[j] = sl[j];
    if (rank == 0 && threadIdx.x == 0 && !s_abort) {
        write_mean_slot(&s_mu, last.r, last.i, last.sr, last.si, a.n, true, true);
        *a.mu_out = s_mu;
    }
}

template <class T> cudaError_t launch_grid_t(const ResGridArgs &a, unsigned G, size_t smem, cudaStream_t st) {
    void (*kern)(ResGridArgs) = k_resident_grid<T, 4>;
    if constexpr (Vec<T>::APV == 2)
        if (a.slice_vecs >= kRgWideVecs) kern = k_resident_grid<T, 8>;
    cudaError_t e;
    if ((e = raise_smem_limit(kern, smem)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRgThreads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kRgThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all G CTAs co-resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class T> cudaError_t launch_cluster_t(const ResArgs &a, unsigned C, size_t smem, cudaStream_t st) {
    auto kern = k_resident_cluster<T>;
    cudaError_t e;
    if ((e = raise_smem_limit(kern, smem)) != cudaSuccess) return e;
    if (C > 8 && (e = raise_func_attr(reinterpret_cast<const void *>(kern), cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1)) != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg)) != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorNotSupported;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

// Chooses the cluster size: enough CTAs for the state to fit their shared
// memory, and up to one 16-byte vector per thread to spread the arithmetic.
bool resident_plan(int n, grover_dtype dt, unsigned *C_out, uint32_t *slice_vecs, size_t *smem_out) {
    const uint64_t N = 1ull << n;
    const int apv = dt == GROVER_C64 ? 2 : 1;
    const uint64_t nvec = N / apv;
    for (unsigned C = 1; C <= (unsigned)kResMaxCluster; C <<= 1) {
        if (nvec % C) break;
        const uint64_t nv = nvec / C;
        const size_t smem = (size_t)nv * 16 + ((nv * apv + 31) / 32) * 4;
        if (smem > kResSmemMax) continue;
        // spread small states over more CTAs while each thread keeps >= 1 vector
        unsigned Cw = C;
        while (Cw < (unsigned)kResMaxCluster && nvec / (Cw * 2) >= (uint64_t)kResThreads && nvec % (Cw * 2) == 0) Cw <<= 1;
        const uint64_t nvw = nvec / Cw;
        *C_out = Cw;
        *slice_vecs = (uint32_t)nvw;
        *smem_out = (size_t)nvw * 16 + ((nvw * apv + 31) / 32) * 4;
        return true;
    }
    return false;
}

// Grid-wide variant: one CTA per SM; the slices (and their marked bitmasks)
// must fit one CTA's shared memory.
// Small states run on fewer, fuller CTAs: one exchange costs about 0.8 us with
// 16-38 CTAs, 1.0 us with 76 and 1.45 us with 152 on a GB300, while the update
// shrinks with the slice.  Measured best: complex64 a quarter of the SMs for
// n <= 17 and half for n = 18; complex128 (slower FP64 update) half for
// n <= 16; all SMs above.
bool resident_grid_plan(int n, grover_dtype dt, int sm_count, unsigned *G_out, uint32_t *slice_vecs,
                        size_t *smem_out) {
    const uint64_t N = 1ull << n;
    const int apv = dt == GROVER_C64 ? 2 : 1;
    const uint64_t nvec = N / apv;
    if (sm_count < 1 || sm_count > kRgThreads) return false;
    int ctas = sm_count;
    if (dt == GROVER_C64 ? n <= 17 : n <= 16) ctas = sm_count / (dt == GROVER_C64 ? 4 : 2);
    else if (dt == GROVER_C64 && n == 18) ctas = sm_count / 2;
    if (ctas < 1) ctas = 1;
    if (nvec < (uint64_t)ctas) return false;
    const uint64_t L = (nvec + ctas - 1) / ctas;
    const size_t smem = (size_t)L * 16 + ((L * apv + 31) / 32) * 4;
    if (smem > kRgSmemMax) return false;
    *G_out = (unsigned)((nvec + L - 1) / L);
    *slice_vecs = (uint32_t)L;
    *smem_out = smem;
    return true;
}

cudaError_t launch_resident_grid(const ResGridArgs &a, grover_dtype dt, unsigned G, size_t smem, cudaStream_t st) {
    if (dt == GROVER_C64) return launch_grid_t<float>(a, G, smem, st);
    return launch_grid_t<double>(a, G, smem, st);
}

cudaError_t launch_resident(const ResArgs &a, grover_dtype dt, unsigned C, size_t smem, cudaStream_t st) {
    if (dt == GROVER_C64) return launch_cluster_t<float>(a, C, smem, st);
    return launch_cluster_t<double>(a, C, smem, st);
}

}  // namespace grv
