// k_batch.cu -- many independent Grover searches in one persistent launch.
//
// Each instance i is a complex64 state of 2^n_i amplitudes at its own offset of
// one batch buffer, with its own sorted marked list and iteration count k_i.
// A persistent grid (resident CTAs only) takes instances from an atomic work
// counter in the order the host sorted them (largest N*k first, so the long
// searches start early and the short ones fill the tail), and one CTA runs an
// instance's whole search: the uniform initial state, k_i iterations of the
// proposed grover_search loop (Algorithm "n-qubit Oracle", Algorithm "n-qubit
// Inversion about Mean"), then P_success = sum over marked x of |c_x|^2.  The
// mean of every iteration is a CTA-wide reduction only, so no CTA ever waits
// for another.  Instances of at most `onchip_vecs` 16-byte vectors stay in
// shared memory for all iterations; larger ones stream through L2 / HBM.
// Sums are exact as in the single-instance pass: FP32 pairwise sums of each
// thread's 8-amplitude group added as 128-bit fixed point, reduced in integers.
#include <cooperative_groups.h>

#include "fixed_sum.cuh"
#include "grover_internal.cuh"

namespace grv {
namespace {

__device__ __forceinline__ float flip(float x, uint32_t f) { return __uint_as_float(__float_as_uint(x) ^ (f << 31)); }

template <int G> __device__ __forceinline__ float pairwise(const float *v) {
    if constexpr (G == 1) return v[0];
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cursor into the instance's sorted marked list (in shared memory): a thread
// visits its vectors in increasing order, so the cursor only moves forward.
struct SmCursor {
    const uint64_t *list;
    uint32_t m, p;
    __device__ __forceinline__ void init(const uint64_t *l, uint32_t mm, uint64_t first) {
        list = l;
        m = mm;
        p = 0;
        while (p < m && list[p] < first) ++p;
    }
    __device__ __forceinline__ uint32_t bits2(uint64_t a0) {  // amplitudes a0, a0 + 1
        while (p < m && list[p] < a0) ++p;
        uint32_t f = 0;
        uint32_t q = p;
        while (q < m && list[q] < a0 + 2) {
            f |= 1u << (uint32_t)(list[q] - a0);
            ++q;
        }
        return f;
    }
};

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_batch(float4 *amps, const BatchInst *inst, const uint32_t *order, uint32_t count, const uint64_t *marked,
        unsigned *next, double *psucc, uint32_t onchip_vecs) {
    constexpr int WARPS = THREADS / 32;
    constexpr int U = 4;  // vectors per thread per group
    extern __shared__ __align__(16) float4 sm[];
    __shared__ uint64_t s_list[kBatchMaxMarked];
    __shared__ unsigned long long s_int[WARPS][4];
    __shared__ double s_side[WARPS][2];
    __shared__ float4 s_two;  // (re hi, re lo, im hi, im lo) of 2 mu
    __shared__ uint32_t s_idx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_idx = atomicAdd(next, 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= count) break;
        const BatchInst I = inst[order[idx]];
        const uint64_t N = 1ull << I.n;
        const uint32_t nvec = (uint32_t)(N / 2);
        const bool onchip = nvec <= onchip_vecs;
        float4 *g = amps + I.amp_off / 2;
        float4 *st = onchip ? sm : g;
        for (uint32_t i = tid; i < I.m; i += THREADS) s_list[i] = marked[I.mark_off + i];
        // uniform initial state 1/sqrt(N) (IEEE sqrt and division, rounded to FP32)
        const float a0 = (float)(1.0 / sqrt((double)N));
        for (uint32_t j = tid; j < nvec; j += THREADS) st[j] = make_float4(a0, 0.f, a0, 0.f);
        __syncthreads();

        // t = -1: mean of O c of the initial state; t = 0..k-1: iterations
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
            SmCursor cur;
            cur.init(s_list, I.m, 2ull * tid);
            u128 ar = 0, ai = 0;
            double sr = 0.0, si = 0.0;
            for (uint32_t j0 = tid; j0 < nvec; j0 += U * THREADS) {
                float gr[2 * U], gi[2 * U];
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * THREADS;
                    if (j < nvec) v[u] = onchip ? st[j] : __ldcg(st + j);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * THREADS;
                    if (j >= nvec) {
                        gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                        continue;
                    }
                    float4 c = v[u];
                    const uint32_t f = cur.bits2(2ull * j);
                    const uint32_t f0 = f & 1u, f1 = f >> 1;
                    if (upd) {
                        c.x = (two_re - flip(c.x, f0)) + lo_re;
                        c.y = (two_im - flip(c.y, f0)) + lo_im;
                        c.z = (two_re - flip(c.z, f1)) + lo_re;
                        c.w = (two_im - flip(c.w, f1)) + lo_im;
                        if (onchip) st[j] = c;
                        else __stcg(st + j, c);
                    }
                    gr[2 * u] = flip(c.x, f0);
                    gi[2 * u] = flip(c.y, f0);
                    gr[2 * u + 1] = flip(c.z, f1);
                    gi[2 * u + 1] = flip(c.w, f1);
                }
                fix_add<4>(ar, sr, pairwise<2 * U>(gr));
                fix_add<4>(ai, si, pairwise<2 * U>(gi));
            }
            // CTA reduction (exact integers; FP64 side sums only if present)
            ar = warp_sum_u128(ar);
            ai = warp_sum_u128(ai);
            const int any_side = __syncthreads_or(sr != 0.0 || si != 0.0);
            if (any_side) {
                sr = warp_sum_d(sr);
                si = warp_sum_d(si);
            }
            if (lane == 0) {
                s_int[warp][0] = (unsigned long long)ar;
                s_int[warp][1] = (unsigned long long)(ar >> 64);
                s_int[warp][2] = (unsigned long long)ai;
                s_int[warp][3] = (unsigned long long)(ai >> 64);
                s_side[warp][0] = sr;
                s_side[warp][1] = si;
            }
            __syncthreads();
            if (warp == 0) {
                u128 r = 0, i = 0;
                double xr = 0.0, xi = 0.0;
                if (lane < WARPS) {
                    r = ((u128)s_int[lane][1] << 64) | s_int[lane][0];
                    i = ((u128)s_int[lane][3] << 64) | s_int[lane][2];
                    xr = s_side[lane][0];
                    xi = s_side[lane][1];
                }
                r = warp_sum_u128(r);
                i = warp_sum_u128(i);
                if (any_side) {
                    xr = warp_sum_d(xr);
                    xi = warp_sum_d(xi);
                }
                if (lane == 0) {
                    const double inv_n = ldexp(1.0, -I.n);
                    const double mr = (i192_to_double(i192_from(r)) * 0x1p-100 + xr) * inv_n;
                    const double mi = (i192_to_double(i192_from(i)) * 0x1p-100 + xi) * inv_n;
                    const double tr = 2.0 * mr, ti = 2.0 * mi;
                    const float hr = (float)tr, hi = (float)ti;
                    s_two = make_float4(hr, (float)(tr - (double)hr), hi, (float)(ti - (double)hi));
                }
            }
            __syncthreads();
        }
        // success probability (FP64 squares, fixed order) and store back
        if (warp == 0) {
            double p = 0.0;
            for (uint32_t i = lane; i < I.m; i += 32) {
                const uint64_t x = s_list[i];
                const float4 c = onchip ? st[x >> 1] : __ldcg(st + (x >> 1));
                const float re = (x & 1) ? c.z : c.x, im = (x & 1) ? c.w : c.y;
                p += __dadd_rn(__dmul_rn((double)re, (double)re), __dmul_rn((double)im, (double)im));
            }
            p = warp_sum_d(p);
            if (lane == 0) psucc[order[idx]] = p;
        }
        if (onchip)
            for (uint32_t j = tid; j < nvec; j += THREADS) g[j] = sm[j];
        __syncthreads();
    }
}

// ---- large instances: one thread-block cluster per instance ---------------------
// CTA r of a cluster holds vectors [r L, (r + 1) L) of the instance's state,
// L = (N / 2) / kBatchClusterSize: in shared memory when L fits, else streamed
// through L2 (at most one large state per cluster is live, so the clusters'
// states stay in L2).  Per iteration: the update and exact partial sums as in
// k_batch, the CTA's partial into its own shared memory (double buffered), a
// hardware cluster barrier, then every CTA adds the kBatchClusterSize partials
// read through distributed shared memory in rank order -- the same mean in
// every CTA without a global-memory round trip.
namespace cg = cooperative_groups;
constexpr int kBcThreads = 512;
constexpr int kBcWarps = kBcThreads / 32;

struct BcPart {
    unsigned long long rl, rh, il, ih;
    double sr, si;
    int side;
};

__global__ void __launch_bounds__(kBcThreads, 1) k_batch_cluster(BatchClusterLaunch L) {
    constexpr int U = 4;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), CS = cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) float4 smb[];
    __shared__ uint64_t s_list[kBatchMaxMarked];
    __shared__ unsigned long long s_int[kBcWarps][4];
    __shared__ double s_side[kBcWarps][2];
    __shared__ BcPart part[2];
    __shared__ float4 s_two;
    __shared__ uint32_t s_idx;
    __shared__ double s_p;

    cl.sync();  // every CTA of the cluster runs before distributed shared memory is written
    for (;;) {
        if (rank == 0 && tid == 0) {
            const uint32_t v = atomicAdd(L.next, 1u);
            for (unsigned r = 0; r < CS; ++r) *cl.map_shared_rank(&s_idx, r) = v;
        }
        cl.sync();
        const uint32_t idx = s_idx;
        if (idx >= L.count) break;
        const BatchInst I = L.inst[L.order[idx]];
        const uint64_t N = 1ull << I.n;
        const uint32_t nv = (uint32_t)(N / 2 / CS);
        const uint64_t v0 = (uint64_t)rank * nv;  // first vector of this CTA's slice
        const bool onchip = nv <= kBatchClusterOnchipVecs;
        float4 *g = L.amps + I.amp_off / 2 + v0;
        float4 *st = onchip ? smb : g;
        for (uint32_t i = tid; i < I.m; i += kBcThreads) s_list[i] = L.marked[I.mark_off + i];
        const float a0 = (float)(1.0 / sqrt((double)N));
        for (uint32_t j = tid; j < nv; j += kBcThreads) {
            if (onchip) st[j] = make_float4(a0, 0.f, a0, 0.f);
            else __stcg(st + j, make_float4(a0, 0.f, a0, 0.f));
        }
        __syncthreads();
        for (long long t = -1; t < (long long)I.k; ++t) {
            const bool upd = t >= 0;
            const int slot = (int)((t + 1) & 1);
            float two_re = 0.f, lo_re = 0.f, two_im = 0.f, lo_im = 0.f;
            if (upd) {
                const float4 h = s_two;
                two_re = h.x;
                lo_re = h.y;
                two_im = h.z;
                lo_im = h.w;
            }
            SmCursor cur;
            cur.init(s_list, I.m, 2ull * (v0 + tid));
            u128 ar = 0, ai = 0;
            double sr = 0.0, si = 0.0;
            for (uint32_t j0 = tid; j0 < nv; j0 += U * kBcThreads) {
                float gr[2 * U], gi[2 * U];
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * kBcThreads;
                    if (j < nv) v[u] = onchip ? st[j] : __ldcg(st + j);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * kBcThreads;
                    if (j >= nv) {
                        gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                        continue;
                    }
                    float4 c = v[u];
                    const uint32_t f = cur.bits2(2ull * (v0 + j));
                    const uint32_t f0 = f & 1u, f1 = f >> 1;
                    if (upd) {
                        c.x = (two_re - flip(c.x, f0)) + lo_re;
                        c.y = (two_im - flip(c.y, f0)) + lo_im;
                        c.z = (two_re - flip(c.z, f1)) + lo_re;
                        c.w = (two_im - flip(c.w, f1)) + lo_im;
                        if (onchip) st[j] = c;
                        else __stcg(st + j, c);
                    }
                    gr[2 * u] = flip(c.x, f0);
                    gi[2 * u] = flip(c.y, f0);
                    gr[2 * u + 1] = flip(c.z, f1);
                    gi[2 * u + 1] = flip(c.w, f1);
                }
                fix_add<4>(ar, sr, pairwise<2 * U>(gr));
                fix_add<4>(ai, si, pairwise<2 * U>(gi));
            }
            // CTA partial (exact integers; FP64 side sums in a fixed order)
            ar = warp_sum_u128(ar);
            ai = warp_sum_u128(ai);
            const int any_side = __syncthreads_or(sr != 0.0 || si != 0.0);
            if (any_side) {
                sr = warp_sum_d(sr);
                si = warp_sum_d(si);
            }
            if (lane == 0) {
                s_int[warp][0] = (unsigned long long)ar;
                s_int[warp][1] = (unsigned long long)(ar >> 64);
                s_int[warp][2] = (unsigned long long)ai;
                s_int[warp][3] = (unsigned long long)(ai >> 64);
                s_side[warp][0] = sr;
                s_side[warp][1] = si;
            }
            __syncthreads();
            if (warp == 0) {
                u128 r = 0, i = 0;
                double xr = 0.0, xi = 0.0;
                if (lane < kBcWarps) {
                    r = ((u128)s_int[lane][1] << 64) | s_int[lane][0];
                    i = ((u128)s_int[lane][3] << 64) | s_int[lane][2];
                    xr = s_side[lane][0];
                    xi = s_side[lane][1];
                }
                r = warp_sum_u128(r);
                i = warp_sum_u128(i);
                if (any_side) {
                    xr = warp_sum_d(xr);
                    xi = warp_sum_d(xi);
                }
                if (lane == 0)
                    part[slot] = BcPart{(unsigned long long)r, (unsigned long long)(r >> 64), (unsigned long long)i,
                                        (unsigned long long)(i >> 64), xr, xi, any_side};
            }
            cl.sync();
            if (warp == 0) {
                I192 r{0, 0, 0}, i{0, 0, 0};
                double xr = 0.0, xi = 0.0;
                int side = 0;
                if (lane < (int)CS) {
                    const BcPart *q = cl.map_shared_rank(&part[slot], lane);
                    r = i192_from(((u128)q->rh << 64) | q->rl);
                    i = i192_from(((u128)q->ih << 64) | q->il);
                    xr = q->sr;
                    xi = q->si;
                    side = q->side;
                }
                r = warp_sum_i192(r);
                i = warp_sum_i192(i);
                const int side_any = __any_sync(0xffffffffu, side);
                if (side_any) {
                    xr = warp_sum_d(xr);
                    xi = warp_sum_d(xi);
                }
                if (lane == 0) {
                    if (!side_any) {
                        // 2 mu = total 2^(1 - 100 - n) as a float pair, formed with
                        // integer operations from the exact total (which fits 128
                        // bits): no FP64 latency on the iteration's critical path
                        const float2 pr = fix_to_f32_pair(((u128)r.w1 << 64) | r.w0, -99 - I.n);
                        const float2 pi = fix_to_f32_pair(((u128)i.w1 << 64) | i.w0, -99 - I.n);
                        s_two = make_float4(pr.x, pr.y, pi.x, pi.y);
                    } else {
                        const double inv_n = ldexp(1.0, -I.n);
                        const double tr = 2.0 * ((i192_to_double(r) * 0x1p-100 + xr) * inv_n);
                        const double ti = 2.0 * ((i192_to_double(i) * 0x1p-100 + xi) * inv_n);
                        const float hr = (float)tr, hi = (float)ti;
                        s_two = make_float4(hr, (float)(tr - (double)hr), hi, (float)(ti - (double)hi));
                    }
                }
            }
            __syncthreads();
        }
        // success probability: each CTA its marked amplitudes, then rank order
        if (warp == 0) {
            double p = 0.0;
            const uint64_t lo = 2 * v0, hi = 2 * (v0 + nv);
            for (uint32_t i = lane; i < I.m; i += 32) {
                const uint64_t x = s_list[i];
                if (x < lo || x >= hi) continue;
                const uint64_t j = (x - lo) >> 1;
                const float4 c = onchip ? st[j] : __ldcg(st + j);
                const float re = (x & 1) ? c.z : c.x, im = (x & 1) ? c.w : c.y;
                p += __dadd_rn(__dmul_rn((double)re, (double)re), __dmul_rn((double)im, (double)im));
            }
            p = warp_sum_d(p);
            if (lane == 0) s_p = p;
        }
        if (onchip)
            for (uint32_t j = tid; j < nv; j += kBcThreads) g[j] = smb[j];
        cl.sync();
        if (rank == 0 && tid == 0) {
            double p = 0.0;
            for (unsigned r = 0; r < CS; ++r) p += *cl.map_shared_rank(&s_p, r);
            L.psucc[L.order[idx]] = p;
        }
        cl.sync();  // s_p, s_idx and the partials are reused by the next instance
    }
}

template <int THREADS> cudaError_t prepare_t(const BatchLaunch &L, int sm_count, unsigned *grid) {
    auto kern = k_batch<THREADS>;
    const size_t smem = (size_t)L.onchip_vecs * sizeof(float4);
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = (unsigned)(per_sm * sm_count);
    return cudaSuccess;
}

template <int THREADS> cudaError_t enqueue_t(const BatchLaunch &L, unsigned grid, cudaStream_t st) {
    const size_t smem = (size_t)L.onchip_vecs * sizeof(float4);
    k_batch<THREADS><<<grid, THREADS, smem, st>>>(L.amps, L.inst, L.order, L.count, L.marked, L.next, L.psucc,
                                                  L.onchip_vecs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_batch(const BatchLaunch &L, int sm_count, unsigned *grid) {
    switch (L.threads) {
    case 256: return prepare_t<256>(L, sm_count, grid);
    case 512: return prepare_t<512>(L, sm_count, grid);
    default: return prepare_t<1024>(L, sm_count, grid);
    }
}

static cudaLaunchConfig_t cluster_config(int clusters, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * kBatchClusterSize));
    cfg.blockDim = dim3(kBcThreads);
    cfg.dynamicSmemBytes = (size_t)kBatchClusterOnchipVecs * sizeof(float4);
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kBatchClusterSize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t prepare_batch_cluster(int *clusters) {
    *clusters = 0;
    cudaError_t e;
    if ((e = raise_smem_limit(k_batch_cluster, (size_t)kBatchClusterOnchipVecs * sizeof(float4))) != cudaSuccess)
        return e;
    if (kBatchClusterSize > 8 &&
        (e = raise_func_attr(reinterpret_cast<const void *>(k_batch_cluster),
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(1, 0, attr);
    int n = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&n, k_batch_cluster, &cfg)) != cudaSuccess) return e;
    *clusters = n;
    return cudaSuccess;
}

cudaError_t enqueue_batch_cluster(const BatchClusterLaunch &L, int clusters, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(L.next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (L.count == 0 || clusters < 1) return cudaSuccess;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(clusters, st, attr);
    return cudaLaunchKernelEx(&cfg, k_batch_cluster, L);
}

cudaError_t enqueue_batch(const BatchLaunch &L, unsigned grid, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(L.next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    switch (L.threads) {
    case 256: return enqueue_t<256>(L, grid, st);
    case 512: return enqueue_t<512>(L, grid, st);
    default: return enqueue_t<1024>(L, grid, st);
    }
}

}  // namespace grv
