// k_measure.cu -- measurement kernels (section "Simulation Results",
// measurement outcome: the probability |c_x|^2 of every basis state).
//
//   k_probs         p_i = |c_i|^2 in FP64 (no FMA contraction, so complex64
//                   squares are exact and complex128 ones are rounded exactly
//                   like a plain re*re + im*im)
//   k_norm_success  norm = sum_i |c_i|^2 and P_success = sum_marked |c_x|^2,
//                   FP64 accumulation, last-CTA fixed-order combine
//   k_topm          the m most probable states, ordered (p desc, index asc):
//                   per-thread sorted candidate lists, warp and block merges,
//                   then a merge of all blocks' lists by the last CTA
#include "grover_internal.cuh"

namespace grv {
namespace {

template <class T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int APV = 2;
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int APV = 1;
};

__device__ __forceinline__ double sq(double re, double im) {
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

template <class S> __device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class S> __device__ __forceinline__ S block_sum(S v, S *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < kThreads / 32) ? sm[lane] : S(0);
        v = warp_sum(v);
    }
    return v;
}

// ---- probabilities ------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) k_probs(const T *amps, uint64_t first, uint64_t count, double *out) {
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < count; i += (uint64_t)gridDim.x * kThreads) {
        const uint64_t x = first + i;
        out[i] = sq((double)amps[2 * x], (double)amps[2 * x + 1]);
    }
}

// ---- norm and success probability --------------------------------------------------
// complex64 squares are formed in FP32 per 16-byte vector and accumulated in
// FP64 above that; complex128 squares and sums are FP64.
constexpr int kMUnroll = 4;

template <class T, bool BITS>
__global__ void __launch_bounds__(kThreads)
k_norm_success(const T *amps, uint64_t nvec, const uint32_t *words, double2 *partials, unsigned *ticket,
               double2 *out) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    const V *v = reinterpret_cast<const V *>(amps);
    const uint64_t tile = (uint64_t)kThreads * kMUnroll;
    double nrm = 0.0, suc = 0.0;
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < nvec; base += (uint64_t)gridDim.x * tile) {
        V c[kMUnroll];
#pragma unroll
        for (int u = 0; u < kMUnroll; ++u) {
            const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
            if (i < nvec) c[u] = __ldcs(v + i);
        }
        if constexpr (APV == 2) {
            // squares in FP32, the 8 of one tile summed pairwise, FP64 above
            float q[kMUnroll];
#pragma unroll
            for (int u = 0; u < kMUnroll; ++u) {
                const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
                q[u] = i < nvec ? fmaf(c[u].x, c[u].x, c[u].y * c[u].y) + fmaf(c[u].z, c[u].z, c[u].w * c[u].w) : 0.f;
                if (BITS && i < nvec) {
                    const uint32_t w = words[(i * 2) >> 5] >> (uint32_t)((i * 2) & 31);
                    if (w & 1u) suc += sq(c[u].x, c[u].y);
                    if (w & 2u) suc += sq(c[u].z, c[u].w);
                }
            }
            nrm += (double)((q[0] + q[1]) + (q[2] + q[3]));
        } else {
#pragma unroll
            for (int u = 0; u < kMUnroll; ++u) {
                const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
                if (i >= nvec) continue;
                const double p = sq(c[u].x, c[u].y);
                nrm += p;
                if (BITS && ((words[i >> 5] >> (uint32_t)(i & 31)) & 1u)) suc += p;
            }
        }
    }
    __shared__ double sm[kThreads / 32];
    __shared__ unsigned s_last;
    nrm = block_sum(nrm, sm);
    suc = block_sum(suc, sm);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = make_double2(nrm, suc);
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kThreads) {
        const double2 q = __ldcg(partials + j);
        a += q.x;
        b += q.y;
    }
    a = block_sum(a, sm);
    b = block_sum(b, sm);
    if (threadIdx.x == 0) {
        out[0].x = a;
        if (BITS) out[0].y = b;
        *ticket = 0u;
    }
}

// Success probability over a sorted list: one CTA, fixed order.
template <class T> __global__ void __launch_bounds__(kThreads) k_success_list(const T *amps, const uint64_t *list, uint64_t m, double2 *out) {
    __shared__ double sm[kThreads / 32];
    double s = 0.0;
    for (uint64_t i = threadIdx.x; i < m; i += kThreads) {
        const uint64_t x = list[i];
        s += sq((double)amps[2 * x], (double)amps[2 * x + 1]);
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) out[0].y = s;
}

// ---- top-m ----------------------------------------------------------------------------------
__device__ __forceinline__ bool better(double p, uint64_t i, double q, uint64_t j) {
    return p > q || (p == q && i < j);
}

template <int K> struct TopK {
    double p[K];
    uint64_t i[K];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            p[j] = -1.0;
            i[j] = ~0ull;
        }
    }
    // returns false when (pv, iv) does not enter the list
    __device__ __forceinline__ bool insert(double pv, uint64_t iv) {
        if (!better(pv, iv, p[K - 1], i[K - 1])) return false;
        p[K - 1] = pv;
        i[K - 1] = iv;
#pragma unroll
        for (int j = K - 1; j > 0; --j) {
            if (better(p[j], i[j], p[j - 1], i[j - 1])) {
                double tp = p[j];
                p[j] = p[j - 1];
                p[j - 1] = tp;
                uint64_t ti = i[j];
                i[j] = i[j - 1];
                i[j - 1] = ti;
            }
        }
        return true;
    }
    // FP32 prefilter bound: a value whose FP32 estimate is below it cannot
    // enter the list (the estimate is within 2^-22 of the exact square).
    __device__ __forceinline__ float bound32() const {
        return p[K - 1] < 0.0 ? -1.0f : __double2float_rd(p[K - 1] * (1.0 - 0x1p-20));
    }
};

// Merges the sorted lists of a warp's lanes: K rounds, each takes the best
// head.  Lane 0 ends with the warp's top K in out.
template <int K> __device__ __forceinline__ void warp_merge(TopK<K> &t, TopK<K> &out) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        // the list is kept sorted with its head at index 0
        double bp = t.p[0];
        uint64_t bi = t.i[0];
        int bl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double op = __shfl_xor_sync(0xffffffffu, bp, o);
            uint64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (better(op, oi, bp, bi) || (op == bp && oi == bi && ol < bl)) {
                bp = op;
                bi = oi;
                bl = ol;
            }
        }
        if (lane == 0) {
            out.p[r] = bp;
            out.i[r] = bi;
        }
        if (lane == bl) {  // pop the head
#pragma unroll
            for (int j = 0; j < K - 1; ++j) {
                t.p[j] = t.p[j + 1];
                t.i[j] = t.i[j + 1];
            }
            t.p[K - 1] = -2.0;
            t.i[K - 1] = ~0ull;
        }
    }
}

// Block merge: warps' lists through shared memory, warp 0 merges them.
template <int K> __device__ void block_merge(TopK<K> &t, Cand *dst) {
    __shared__ Cand sm[(kThreads / 32) * K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TopK<K> w;
    w.init();
    warp_merge<K>(t, w);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < K; ++j) sm[warp * K + j] = Cand{w.p[j], w.i[j]};
    }
    __syncthreads();
    if (warp == 0) {
        TopK<K> mine;
        mine.init();
        for (int j = lane; j < (kThreads / 32) * K; j += 32) mine.insert(sm[j].p, sm[j].idx);
        TopK<K> res;
        res.init();
        warp_merge<K>(mine, res);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < K; ++j) dst[j] = Cand{res.p[j], res.i[j]};
        }
    }
}

template <class T, int K>
__global__ void __launch_bounds__(kThreads)
k_topm(const T *amps, uint64_t nvec, Cand *cand, unsigned *ticket, Cand *final_out) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    const V *v = reinterpret_cast<const V *>(amps);
    TopK<K> t;
    t.init();
    // A thread visits indices in increasing order, so an amplitude equal to one
    // that already failed to enter can never enter later (its probability ties
    // and its index is larger): equal magnitudes are skipped by comparing bits.
    // Four vectors per thread are loaded before any is examined (more 16-byte
    // loads in flight for the HBM stream), then examined in increasing order.
    constexpr int KU = 4;
    float b32 = -1.0f;
    uint64_t seen_hi = ~0ull, seen_lo = ~0ull;
    auto visit = [&](const V c, uint64_t i) {
        if constexpr (APV == 2) {
            const float e0 = fmaf(c.x, c.x, c.y * c.y);
            const float e1 = fmaf(c.z, c.z, c.w * c.w);
            if (e0 >= b32) {
                const uint64_t key = ((uint64_t)(__float_as_uint(c.x) & 0x7fffffffu) << 32) | (__float_as_uint(c.y) & 0x7fffffffu);
                if (key != seen_lo) {
                    if (!t.insert(sq(c.x, c.y), 2 * i)) seen_lo = key;
                    b32 = t.bound32();
                }
            }
            if (e1 >= b32) {
                const uint64_t key = ((uint64_t)(__float_as_uint(c.z) & 0x7fffffffu) << 32) | (__float_as_uint(c.w) & 0x7fffffffu);
                if (key != seen_lo) {
                    if (!t.insert(sq(c.z, c.w), 2 * i + 1)) seen_lo = key;
                    b32 = t.bound32();
                }
            }
        } else {
            const uint64_t kh = (uint64_t)__double_as_longlong(c.x) & 0x7fffffffffffffffull;
            const uint64_t kl = (uint64_t)__double_as_longlong(c.y) & 0x7fffffffffffffffull;
            if (kh != seen_hi || kl != seen_lo) {
                if (!t.insert(sq(c.x, c.y), i)) {
                    seen_hi = kh;
                    seen_lo = kl;
                }
            }
        }
    };
    const uint64_t S = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i0 < nvec; i0 += KU * S) {
        V cc[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u)
            if (i0 + u * S < nvec) cc[u] = __ldcs(v + i0 + u * S);
#pragma unroll
        for (int u = 0; u < KU; ++u)
            if (i0 + u * S < nvec) visit(cc[u], i0 + u * S);
    }
    block_merge<K>(t, cand + (size_t)blockIdx.x * K);

    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    TopK<K> all;
    all.init();
    for (unsigned j = threadIdx.x; j < gridDim.x * K; j += kThreads) {
        const double2 raw = __ldcg(reinterpret_cast<const double2 *>(cand) + j);
        all.insert(raw.x, (uint64_t)__double_as_longlong(raw.y));
    }
    __syncthreads();
    block_merge<K>(all, final_out);
    if (threadIdx.x == 0) *ticket = 0u;
}

unsigned grid_for(uint64_t work, const Geometry &g, int per_sm) {
    uint64_t need = (work + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)g.sm_count * per_sm;
    if (cap > (uint64_t)kMaxGrid) cap = kMaxGrid;
    unsigned grid = (unsigned)(need < cap ? need : cap);
    return grid ? grid : 1;
}

}  // namespace

cudaError_t launch_probs(const void *amps, grover_dtype dt, uint64_t first, uint64_t count, double *out,
                         cudaStream_t st, const Geometry &g) {
    unsigned grid = grid_for(count, g, 8);
    if (dt == GROVER_C64) k_probs<float><<<grid, kThreads, 0, st>>>((const float *)amps, first, count, out);
    else k_probs<double><<<grid, kThreads, 0, st>>>((const double *)amps, first, count, out);
    return cudaGetLastError();
}

cudaError_t launch_norm_success(const void *amps, int n, grover_dtype dt, const MarkedDev &mk, Scratch &sc,
                                cudaStream_t st, const Geometry &g) {
    const uint64_t N = 1ull << n;
    const uint64_t nvec = dt == GROVER_C64 ? N / 2 : N;
    unsigned grid = grid_for(nvec, g, 8);
    cudaError_t e = cudaMemsetAsync(sc.red, 0, sizeof(double2), st);
    if (e != cudaSuccess) return e;
    const bool bits = mk.mode == MARK_BITS && mk.m > 0;
    if (dt == GROVER_C64) {
        if (bits) k_norm_success<float, true><<<grid, kThreads, 0, st>>>((const float *)amps, nvec, mk.words, sc.partials, sc.ticket, sc.red);
        else k_norm_success<float, false><<<grid, kThreads, 0, st>>>((const float *)amps, nvec, nullptr, sc.partials, sc.ticket, sc.red);
    } else {
        if (bits) k_norm_success<double, true><<<grid, kThreads, 0, st>>>((const double *)amps, nvec, mk.words, sc.partials, sc.ticket, sc.red);
        else k_norm_success<double, false><<<grid, kThreads, 0, st>>>((const double *)amps, nvec, nullptr, sc.partials, sc.ticket, sc.red);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || bits || mk.m == 0) return e;
    if (dt == GROVER_C64) k_success_list<float><<<1, kThreads, 0, st>>>((const float *)amps, mk.list, mk.m, sc.red);
    else k_success_list<double><<<1, kThreads, 0, st>>>((const double *)amps, mk.list, mk.m, sc.red);
    return cudaGetLastError();
}

template <int K>
static cudaError_t topm_k(const void *amps, uint64_t nvec, grover_dtype dt, Scratch &sc, cudaStream_t st,
                          const Geometry &g) {
    unsigned grid = grid_for(nvec, g, 4);
    if (grid > (unsigned)kTopMGrid) grid = kTopMGrid;
    Cand *final_out = sc.cand + (size_t)kTopMGrid * kTopMMax;
    if (dt == GROVER_C64) k_topm<float, K><<<grid, kThreads, 0, st>>>((const float *)amps, nvec, sc.cand, sc.ticket, final_out);
    else k_topm<double, K><<<grid, kThreads, 0, st>>>((const double *)amps, nvec, sc.cand, sc.ticket, final_out);
    return cudaGetLastError();
}

cudaError_t launch_topm(const void *amps, int n, grover_dtype dt, int m, Scratch &sc, cudaStream_t st,
                        const Geometry &g) {
    const uint64_t N = 1ull << n;
    const uint64_t nvec = dt == GROVER_C64 ? N / 2 : N;
    if (m <= 1) return topm_k<1>(amps, nvec, dt, sc, st, g);
    if (m <= 4) return topm_k<4>(amps, nvec, dt, sc, st, g);
    return topm_k<16>(amps, nvec, dt, sc, st, g);
}

}  // namespace grv
