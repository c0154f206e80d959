// k_batch_group.cu -- the large instances of a batch kept on chip by groups
// of CTAs.
//
// A state of 2^n complex64 amplitudes with n >= 15 does not fit one CTA's
// shared memory, but it fits that of G = ceil(8 * 2^n / 225 KiB) SMs (n = 20:
// 37).  One cooperative launch per instance size n runs P = floor(SMs / G)
// groups of G CTAs; group g runs, one after the other, the instances the host
// assigned to it (longest processing time first).  For each instance the CTA of
// rank r keeps vectors [r L, (r + 1) L) of the state in shared memory from the
// uniform start to the end of its search -- the proposed grover_search loop,
// Algorithm "n-qubit Oracle" then Algorithm "n-qubit Inversion about Mean", k_i
// times -- and writes them to the batch buffer once.  Per iteration the CTA
// updates its slice, c <- 2 mu - O c, adds O c_new into exact 128-bit
// fixed-point sums (FP32 pairwise sums of 16-amplitude groups), reduces them
// in integers and exchanges them with the other G - 1 CTAs
// of its group through global memory (grid_exchange.cuh: limb sums and arrival
// counts in shared words, bounded polls), so every CTA of the group obtains the
// bitwise identical next mean; 2 mu becomes a float pair with integer
// operations.  The success probability sum over marked x of |c_x|^2 goes
// through the exchange's FP64 side round, summed in rank order.  Groups never
// wait for one another; the cooperative launch keeps all CTAs resident.  A wait
// that runs out sets the status word (3) and the CTA leaves.
#include "fixed_sum.cuh"
#include "grid_exchange.cuh"
#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kBgWarps = kBatchGroupThreads / 32;
// vectors per thread per summation group: one FP32 pairwise sum of 16
// amplitudes per exact fixed-point add (against 8: half the adds, 8 % faster
// over the batch on GB300)
constexpr int kBgU = 8;

__device__ __forceinline__ float bg_flip(float x, uint32_t f) { return __uint_as_float(__float_as_uint(x) ^ (f << 31)); }

template <int G> __device__ __forceinline__ float bg_pairwise(const float *v) {
    if constexpr (G == 1) return v[0];
    else return bg_pairwise<G / 2>(v) + bg_pairwise<G / 2>(v + G / 2);
}

__device__ __forceinline__ double bg_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool bg_has_side(double a, double b) {
    return (__double_as_longlong(a) | __double_as_longlong(b)) != 0;
}

// 2 mu as a float pair (re hi, re lo, im hi, im lo) from the exact sums r, i
// (units 2^-100) and the FP64 side sums, N = 2^n: integer operations only
// when there are no side sums (normalised states), else FP64.
__device__ __forceinline__ float4 two_mu_pair(u128 r, u128 i, double sr, double si, int n) {
    if (!bg_has_side(sr, si)) {
        const float2 pr = fix_to_f32_pair(r, -99 - n), pi = fix_to_f32_pair(i, -99 - n);
        return make_float4(pr.x, pr.y, pi.x, pi.y);
    }
    const double inv_n = ldexp(1.0, -n);
    const double tr = 2.0 * ((i192_to_double(i192_from(r), -100) + sr) * inv_n);
    const double ti = 2.0 * ((i192_to_double(i192_from(i), -100) + si) * inv_n);
    const float hr = (float)tr, hi = (float)ti;
    return make_float4(hr, (float)(tr - (double)hr), hi, (float)(ti - (double)hi));
}

__global__ void __launch_bounds__(kBatchGroupThreads, 1) k_batch_group(BatchGroupLaunch L) {
    const unsigned G = L.group_ctas, g = blockIdx.x / G, rank = blockIdx.x % G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *sl = reinterpret_cast<float4 *>(smem);
    // the marked vectors of the slice, ascending, with their amplitude bits
    // (1: the first of the vector's two amplitudes, 2: the second)
    __shared__ uint32_t s_mv[kBatchMaxMarked], s_mf[kBatchMaxMarked];
    __shared__ uint32_t s_mcnt;
    __shared__ unsigned long long wint[kBgWarps][4];
    __shared__ double wside[kBgWarps][2];
    __shared__ unsigned long long s_prev[2][GxLayout<2>::W];
    __shared__ float4 s_two;
    __shared__ int s_abort;

    unsigned long long *region = L.region + (size_t)g * L.region_words;
    if (tid < 2 * GxLayout<2>::W) s_prev[tid / GxLayout<2>::W][tid % GxLayout<2>::W] = 0ull;
    if (tid == 0) s_abort = 0;
    __syncthreads();
    long long xi = 0;  // exchanges so far (the same sequence in every CTA of the group)
    const uint32_t i0 = L.goff[g], i1 = L.goff[g + 1];

    for (uint32_t ii = i0; ii < i1; ++ii) {
        const uint32_t id = L.glist[ii];
        const BatchInst I = L.inst[id];
        const uint64_t nvec = (1ull << I.n) / 2;
        const uint64_t per = (nvec + G - 1) / G;  // <= L.slice_vecs (host)
        const uint64_t start = (uint64_t)rank * per;
        const uint32_t nv = start >= nvec ? 0u : (uint32_t)(nvec - start < per ? nvec - start : per);
        const float a0 = (float)(1.0 / sqrt((double)(1ull << I.n)));  // IEEE sqrt and division
        for (uint32_t j = tid; j < nv; j += kBatchGroupThreads) sl[j] = make_float4(a0, 0.f, a0, 0.f);
        const uint64_t e0 = 2 * start;  // first amplitude of the slice
        if (tid == 0) {
            // the instance's list is sorted and unique: one pass
            uint32_t c = 0;
            for (uint32_t i = 0; i < I.m; ++i) {
                const uint64_t x = L.marked[I.mark_off + i];
                if (x < e0 || x >= e0 + 2ull * nv) continue;
                const uint32_t j = (uint32_t)((x - e0) >> 1), bit = 1u << (uint32_t)((x - e0) & 1);
                if (c && s_mv[c - 1] == j) s_mf[c - 1] |= bit;
                else {
                    s_mv[c] = j;
                    s_mf[c] = bit;
                    ++c;
                }
            }
            s_mcnt = c;
        }
        __syncthreads();
        const uint32_t mcnt = s_mcnt;

        for (long long t = -1; t < (long long)I.k; ++t) {
            const bool upd = t >= 0;
            float two_re = 0.f, lo_re = 0.f, two_im = 0.f, lo_im = 0.f;
            if (upd) {
                const float4 h = s_two;
                two_re = h.x;
                lo_re = h.y;
                two_im = h.z;
                lo_im = h.w;
            }
            u128 ar = 0, ai = 0;
            double sr = 0.0, si = 0.0;
            // a thread visits its vectors in increasing order: a cursor into the
            // marked vectors finds the rare ones, the others take no flips
            uint32_t cur = 0;
            while (cur < mcnt && s_mv[cur] < (uint32_t)tid) ++cur;
            uint32_t nextj = cur < mcnt ? s_mv[cur] : 0xFFFFFFFFu;
            for (uint32_t j0 = tid; j0 < nv; j0 += kBgU * kBatchGroupThreads) {
                float gr[2 * kBgU], gi[2 * kBgU];
#pragma unroll
                for (int u = 0; u < kBgU; ++u) {
                    const uint32_t j = j0 + u * kBatchGroupThreads;
                    if (j >= nv) {
                        gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                        continue;
                    }
                    float4 c = sl[j];
                    while (nextj < j) {  // marked vectors of other threads
                        ++cur;
                        nextj = cur < mcnt ? s_mv[cur] : 0xFFFFFFFFu;
                    }
                    if (j != nextj) {
                        if (upd) {
                            c.x = (two_re - c.x) + lo_re;
                            c.y = (two_im - c.y) + lo_im;
                            c.z = (two_re - c.z) + lo_re;
                            c.w = (two_im - c.w) + lo_im;
                            sl[j] = c;
                        }
                        gr[2 * u] = c.x;
                        gi[2 * u] = c.y;
                        gr[2 * u + 1] = c.z;
                        gi[2 * u + 1] = c.w;
                    } else {
                        const uint32_t f = s_mf[cur];
                        const uint32_t f0 = f & 1u, f1 = f >> 1;
                        if (upd) {
                            c.x = (two_re - bg_flip(c.x, f0)) + lo_re;
                            c.y = (two_im - bg_flip(c.y, f0)) + lo_im;
                            c.z = (two_re - bg_flip(c.z, f1)) + lo_re;
                            c.w = (two_im - bg_flip(c.w, f1)) + lo_im;
                            sl[j] = c;
                        }
                        gr[2 * u] = bg_flip(c.x, f0);
                        gi[2 * u] = bg_flip(c.y, f0);
                        gr[2 * u + 1] = bg_flip(c.z, f1);
                        gi[2 * u + 1] = bg_flip(c.w, f1);
                    }
                }
                fix_add<4>(ar, sr, bg_pairwise<2 * kBgU>(gr));
                fix_add<4>(ai, si, bg_pairwise<2 * kBgU>(gi));
            }
            // the CTA's exact partial
            ar = warp_sum_u128(ar);
            ai = warp_sum_u128(ai);
            if (__any_sync(0xffffffffu, bg_has_side(sr, si))) {
                sr = bg_warp_sum(sr);
                si = bg_warp_sum(si);
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
                if (lane < kBgWarps) {
                    r = ((u128)wint[lane][1] << 64) | wint[lane][0];
                    i = ((u128)wint[lane][3] << 64) | wint[lane][2];
                    s1 = wside[lane][0];
                    s2 = wside[lane][1];
                }
                r = warp_sum_u128(r);
                i = warp_sum_u128(i);
                const int any_side = __any_sync(0xffffffffu, bg_has_side(s1, s2));
                if (any_side) {
                    s1 = bg_warp_sum(s1);
                    s2 = bg_warp_sum(s2);
                }
                if (lane == 0) {
                    const u128 v[2] = {r, i};
                    const double sdv[2] = {s1, s2};
                    u128 tot[2];
                    double tsd[2];
                    const bool withhold = L.stall && g == 0 && rank == 0 && xi == 0;  // test hook
                    const bool ok = gx_exchange<2>(v, sdv, any_side, region, s_prev, xi, G, rank, L.wait_limit,
                                                   withhold, tot, tsd);
                    if (ok) s_two = two_mu_pair(tot[0], tot[1], tsd[0], tsd[1], I.n);
                    else s_abort = 1;
                }
            }
            ++xi;
            __syncthreads();
            if (s_abort) break;
        }
        if (s_abort) break;
        float4 *gdst = L.amps + I.amp_off / 2 + start;
        for (uint32_t j = tid; j < nv; j += kBatchGroupThreads) gdst[j] = sl[j];
        // success probability: this CTA's marked amplitudes in list order, then
        // the group's partials in rank order (the exchange's side round)
        if (warp == 0) {
            double p = 0.0;
            for (uint32_t i = lane; i < I.m; i += 32) {
                const uint64_t x = L.marked[I.mark_off + i];
                if (x < e0 || x >= e0 + 2ull * nv) continue;
                const float4 c = sl[(x - e0) >> 1];
                const float re = (x & 1) ? c.z : c.x, im = (x & 1) ? c.w : c.y;
                p += __dadd_rn(__dmul_rn((double)re, (double)re), __dmul_rn((double)im, (double)im));
            }
            p = bg_warp_sum(p);
            if (lane == 0) {
                const u128 v[2] = {0, 0};
                const double sdv[2] = {p, 0.0};
                u128 tot[2];
                double tsd[2];
                const bool ok =
                    gx_exchange<2>(v, sdv, 1, region, s_prev, xi, G, rank, L.wait_limit, false, tot, tsd);
                if (!ok) s_abort = 1;
                else if (rank == 0) L.psucc[id] = tsd[0];
            }
        }
        ++xi;
        __syncthreads();
        if (s_abort) break;
    }
    if (s_abort && tid == 0) atomicExch(L.status, 3);
}

}  // namespace

int batch_group_ctas(int n, size_t smem_max) {
    const uint64_t nvec = (1ull << n) / 2;
    for (uint64_t G = 1; G <= 1024; ++G) {
        const uint64_t per = (nvec + G - 1) / G;
        if (per * sizeof(float4) <= smem_max) return (int)G;
    }
    return 0;
}

size_t batch_group_region_words(int group_ctas) {
    return (GxLayout<2>::kAccBytes + GxLayout<2>::side_bytes((unsigned)group_ctas)) / sizeof(unsigned long long);
}

cudaError_t prepare_batch_group(size_t smem, int *per_sm) {
    cudaError_t e = raise_smem_limit(k_batch_group, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_group, kBatchGroupThreads, smem);
}

cudaError_t enqueue_batch_group(const BatchGroupLaunch &L, unsigned groups, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(L.region, 0, (size_t)groups * L.region_words * sizeof(unsigned long long), st);
    if (e != cudaSuccess || groups == 0) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups * L.group_ctas);
    cfg.blockDim = dim3(kBatchGroupThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_group, L);
}

}  // namespace grv
