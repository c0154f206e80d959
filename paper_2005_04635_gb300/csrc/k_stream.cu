// k_stream.cu -- streaming kernels of the equivalent-operator Grover iterator.
//
//   k_init_uniform   psi = H^{(x)n}|0>, written directly as 1/sqrt(N)
//   k_oracle_*       Algorithm "n-qubit Oracle": c_x <- -c_x for marked x
//   k_pass<UPDATE>   one fused HBM pass of the proposed grover_search loop:
//                      c' = O c          (marked-set test, sign bit flip)
//                      c  <- 2 mu - c'   (Algorithm "n-qubit Inversion about
//                                         Mean", update loop)
//                    and, in the same pass, the partial sums of O c_new that
//                    give the next iteration's mean (the algorithm's sum loop),
//                    reduced warp -> block -> grid.  Without UPDATE the kernel
//                    is the sum loop alone.
//
// Layout: the state is N interleaved complex amplitudes; every thread moves
// 16-byte vectors (float4 = 2 complex64, double2 = 1 complex128), U vectors per
// tile, tiles strided over a grid sized to the resident-CTA capacity of the
// SMs.  The grid combine is a last-CTA-done ticket: the final CTA sums the
// per-CTA partials in a fixed order, so the mean is bitwise reproducible and no
// CTA ever waits on another.
#include "fixed_sum.cuh"
#include "grover_internal.cuh"

#include <math.h>

namespace grv {
namespace {

template <class T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int APV = 2;  // amplitudes per vector
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int APV = 1;
};

constexpr int kUnroll = 4;

// ---- programmatic dependent launch --------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- sign flips on the integer pipe --------------------------------------------
__device__ __forceinline__ float flip(float x, uint32_t f) {
    return __uint_as_float(__float_as_uint(x) ^ (f << 31));
}
__device__ __forceinline__ double flip(double x, uint32_t f) {
    return __hiloint2double(__double2hiint(x) ^ (int)(f << 31), __double2loint(x));
}

// ---- loads / stores ----------------------------------------------------------------
template <bool STREAM> __device__ __forceinline__ float4 ldv(const float4 *p) {
    if (STREAM) return __ldcs(p);
    return *p;
}
template <bool STREAM> __device__ __forceinline__ double2 ldv(const double2 *p) {
    if (STREAM) return __ldcs(p);
    return *p;
}
template <bool STREAM> __device__ __forceinline__ void stv(float4 *p, float4 v) {
    if (STREAM) __stcs(p, v);
    else *p = v;
}
template <bool STREAM> __device__ __forceinline__ void stv(double2 *p, double2 v) {
    if (STREAM) __stcs(p, v);
    else *p = v;
}

// ---- marked-set test ------------------------------------------------------------------
// A thread visits its vectors in increasing index order, so a cursor into the
// sorted list only moves forward; a stale cursor catches up by binary search.
struct ListCursor {
    const uint64_t *list;
    uint64_t m, p, nxt;

    __device__ __forceinline__ uint64_t at(uint64_t i) const { return i < m ? __ldg(list + i) : ~0ull; }
    __device__ __forceinline__ uint64_t lower_bound(uint64_t lo, uint64_t x) const {
        uint64_t hi = m;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (__ldg(list + mid) < x) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    }
    __device__ __forceinline__ void init(const uint64_t *l, uint64_t mm, uint64_t first) {
        list = l;
        m = mm;
        p = lower_bound(0, first);
        nxt = at(p);
    }
    // bit j set <=> amplitude a0 + j is marked, 0 <= j < APV
    template <int APV> __device__ __forceinline__ uint32_t bits(uint64_t a0) {
        uint32_t f = 0;
        if (nxt < a0 + APV) {
            if (nxt < a0) {
                p = lower_bound(p + 1, a0);
                nxt = at(p);
            }
            while (nxt < a0 + APV) {
                f |= 1u << (uint32_t)(nxt - a0);
                ++p;
                nxt = at(p);
            }
        }
        return f;
    }
};

template <int APV> __device__ __forceinline__ uint32_t mask_bits(const uint32_t *w, uint64_t a0) {
    uint32_t word = __ldg(w + (a0 >> 5));
    return (word >> (uint32_t)(a0 & 31)) & ((1u << APV) - 1u);
}

// ---- accumulators of the complex sum ------------------------------------------------
// A thread sums the G = kUnroll * APV values of one tile ("load group") and
// adds that to its running sum.  Pairwise summation of a group is exact when
// the values are equal, which they are for every unmarked amplitude of a
// uniform-start search: no rounding bias repeats across the N/G groups.
template <int G, class T> __device__ __forceinline__ T pairwise(const T *v) {
    if constexpr (G == 1) return v[0];
    else if constexpr (G == 2) return v[0] + v[1];
    else if constexpr (G == 4) return (v[0] + v[1]) + (v[2] + v[3]);
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

// Internal accumulation mode of the complex64 default: FP32 pairwise group
// sums, added exactly as fixed point above the group.
constexpr int ACC_HYBRID = 16;

// FP modes: running sums in S, block tree in S, per-CTA partial in FP64.
// complex128, GROVER_ACC_FP64: FP64 pairwise group sum, FP64 running sum.
struct AccD {
    double re = 0.0, im = 0.0;
    template <int G> __device__ __forceinline__ void add_group(const double *r, const double *i) {
        re += pairwise<G>(r);
        im += pairwise<G>(i);
    }
};
// complex64, GROVER_ACC_FP64: FP32 pairwise group sum, FP64 running sum.
struct AccF64 {
    double re = 0.0, im = 0.0;
    template <int G> __device__ __forceinline__ void add_group(const float *r, const float *i) {
        re += (double)pairwise<G>(r);
        im += (double)pairwise<G>(i);
    }
};
// complex64, GROVER_ACC_FP32: plain FP32 running sum, element by element.
struct AccF32 {
    float re = 0.f, im = 0.f;
    template <int G> __device__ __forceinline__ void add_group(const float *r, const float *i) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            re += r[j];
            im += i[j];
        }
    }
};
// complex64, GROVER_ACC_KAHAN: Neumaier-compensated FP32 running sum, element
// by element.
struct AccKahan {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    __device__ __forceinline__ static void neu(float &s, float &c, float x) {
        float t = __fadd_rn(s, x);
        float e = (fabsf(s) >= fabsf(x)) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
        c = __fadd_rn(c, e);
        s = t;
    }
    template <int G> __device__ __forceinline__ void add_group(const float *r, const float *i) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            neu(sr, cr, r[j]);
            neu(si, ci, i[j]);
        }
    }
};
__device__ __forceinline__ double2 acc_value(const AccD &a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ double2 acc_value(const AccF64 &a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ float2 acc_value(const AccF32 &a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ float2 acc_value(const AccKahan &a) {
    return make_float2(__fadd_rn(a.sr, a.cr), __fadd_rn(a.si, a.ci));
}

// Integer modes (fixed_sum.cuh).  Window exponents keep every 128-bit CTA
// partial in range: per element |x| < 1 (GROVER_ACC_EXACT), per 8-value FP32
// group |x| < 16 (ACC_HYBRID).
struct AccX {  // GROVER_ACC_EXACT: every amplitude exactly
    u128 r = 0, i = 0;
    double side_r = 0.0, side_i = 0.0;
    template <int G, class T> __device__ __forceinline__ void add_group(const T *re, const T *im) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            fix_add<0>(r, side_r, re[j]);
            fix_add<0>(i, side_i, im[j]);
        }
    }
};
struct AccH {  // ACC_HYBRID: FP32 pairwise group, exact above
    u128 r = 0, i = 0;
    double side_r = 0.0, side_i = 0.0;
    template <int G> __device__ __forceinline__ void add_group(const float *re, const float *im) {
        fix_add_cvt<4>(r, side_r, pairwise<G>(re));
        fix_add_cvt<4>(i, side_i, pairwise<G>(im));
    }
};

template <class T, int ACC> struct AccSel;
template <int ACC> struct AccSel<double, ACC> { using A = AccD; using S = double; static constexpr bool INT = false; };
template <> struct AccSel<double, GROVER_ACC_EXACT> { using A = AccX; using S = double; static constexpr bool INT = true; };
template <> struct AccSel<float, GROVER_ACC_EXACT> { using A = AccX; using S = double; static constexpr bool INT = true; };
template <> struct AccSel<float, ACC_HYBRID> { using A = AccH; using S = double; static constexpr bool INT = true; };
template <> struct AccSel<float, GROVER_ACC_FP64> { using A = AccF64; using S = double; static constexpr bool INT = false; };
template <> struct AccSel<float, GROVER_ACC_FP32> { using A = AccF32; using S = float; static constexpr bool INT = false; };
template <> struct AccSel<float, GROVER_ACC_KAHAN> { using A = AccKahan; using S = float; static constexpr bool INT = false; };

// ---- deterministic block reduction (result valid in thread 0) -----------------------
template <class S> __device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class S> __device__ __forceinline__ S block_sum(S v, S *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();  // sm may be reused by the caller's previous reduction
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < kThreads / 32) ? sm[lane] : S(0);
        v = warp_sum(v);
    }
    return v;
}

// The producer of a mean also stores what the consumers need, so that no
// consuming thread spends FP64 instructions on it.
__device__ __forceinline__ void write_mean(MeanSlot *ms, double mr, double mi) {
    const double tr = 2.0 * mr, ti = 2.0 * mi;
    const float hr = (float)tr, hi = (float)ti;
    ms->mu = make_double2(mr, mi);
    ms->two = make_double2(tr, ti);
    ms->two32 = make_float4(hr, (float)(tr - (double)hr), hi, (float)(ti - (double)hi));
}

// FP modes: per-CTA partial -> partials[], last CTA combines in FP64 in a
// fixed order.
__device__ __forceinline__ void grid_combine(double2 part, const PassArgs &a) {
    __shared__ double sm[kThreads / 32];
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = part;
        __threadfence();
        unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sr = 0.0, si = 0.0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kThreads) {
        double2 q = __ldcg(a.partials + j);
        sr += q.x;
        si += q.y;
    }
    sr = block_sum(sr, sm);
    si = block_sum(si, sm);
    if (threadIdx.x == 0) {
        write_mean(a.mu_out, sr * a.inv_n, si * a.inv_n);
        *a.ticket = 0u;
    }
}

// Integer modes: the CTA's exact partial (two 128-bit integers) and its FP64
// side sums go to partials[3b .. 3b+2]; the last CTA adds the integers in 192
// bits (exact, any order) and the side sums in a fixed order, and rounds once.
__device__ __forceinline__ void int_combine(u128 r, u128 i, double sr, double si, const PassArgs &a) {
    __shared__ unsigned long long wi[kThreads / 32][6];
    __shared__ double wsd[kThreads / 32][2];
    __shared__ unsigned s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // CTA partial (thread 0)
    r = warp_sum_u128(r);
    i = warp_sum_u128(i);
    const int any_side = __syncthreads_or(sr != 0.0 || si != 0.0);
    if (any_side) {
        sr = warp_sum(sr);
        si = warp_sum(si);
    }
    if (lane == 0) {
        wi[warp][0] = (unsigned long long)r;
        wi[warp][1] = (unsigned long long)(r >> 64);
        wi[warp][2] = (unsigned long long)i;
        wi[warp][3] = (unsigned long long)(i >> 64);
        wsd[warp][0] = sr;
        wsd[warp][1] = si;
    }
    __syncthreads();
    if (warp == 0) {
        u128 br = 0, bi = 0;
        double bsr = 0.0, bsi = 0.0;
        if (lane < kThreads / 32) {
            br = ((u128)wi[lane][1] << 64) | wi[lane][0];
            bi = ((u128)wi[lane][3] << 64) | wi[lane][2];
            bsr = wsd[lane][0];
            bsi = wsd[lane][1];
        }
        br = warp_sum_u128(br);
        bi = warp_sum_u128(bi);
        if (any_side) {
            bsr = warp_sum(bsr);
            bsi = warp_sum(bsi);
        }
        if (lane == 0) {
            double2 *p = a.partials + 3 * blockIdx.x;
            p[0] = make_double2(__longlong_as_double((long long)(unsigned long long)br),
                                __longlong_as_double((long long)(unsigned long long)(br >> 64)));
            p[1] = make_double2(__longlong_as_double((long long)(unsigned long long)bi),
                                __longlong_as_double((long long)(unsigned long long)(bi >> 64)));
            p[2] = make_double2(bsr, bsi);
            __threadfence();
            s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    I192 tr{0, 0, 0}, ti{0, 0, 0};
    double ssr = 0.0, ssi = 0.0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kThreads) {
        const double2 q0 = __ldcg(a.partials + 3 * j), q1 = __ldcg(a.partials + 3 * j + 1),
                      q2 = __ldcg(a.partials + 3 * j + 2);
        i192_add(tr, i192_from(((u128)(unsigned long long)__double_as_longlong(q0.y) << 64) |
                               (unsigned long long)__double_as_longlong(q0.x)));
        i192_add(ti, i192_from(((u128)(unsigned long long)__double_as_longlong(q1.y) << 64) |
                               (unsigned long long)__double_as_longlong(q1.x)));
        ssr += q2.x;
        ssi += q2.y;
    }
    const int any = __syncthreads_or(ssr != 0.0 || ssi != 0.0);
    tr = warp_sum_i192(tr);
    ti = warp_sum_i192(ti);
    if (any) {
        ssr = warp_sum(ssr);
        ssi = warp_sum(ssi);
    }
    if (lane == 0) {
        wi[warp][0] = tr.w0;
        wi[warp][1] = tr.w1;
        wi[warp][2] = tr.w2;
        wi[warp][3] = ti.w0;
        wi[warp][4] = ti.w1;
        wi[warp][5] = ti.w2;
        wsd[warp][0] = ssr;
        wsd[warp][1] = ssi;
    }
    __syncthreads();
    if (warp == 0) {
        I192 xr{0, 0, 0}, xi{0, 0, 0};
        double yr = 0.0, yi = 0.0;
        if (lane < kThreads / 32) {
            xr = I192{wi[lane][0], wi[lane][1], wi[lane][2]};
            xi = I192{wi[lane][3], wi[lane][4], wi[lane][5]};
            yr = wsd[lane][0];
            yi = wsd[lane][1];
        }
        xr = warp_sum_i192(xr);
        xi = warp_sum_i192(xi);
        if (any) {
            yr = warp_sum(yr);
            yi = warp_sum(yi);
        }
        if (lane == 0) {
            const double sum_r = i192_to_double(xr) * 0x1p-100, sum_i = i192_to_double(xi) * 0x1p-100;
            write_mean(a.mu_out, (sum_r + yr) * a.inv_n, (sum_i + yi) * a.inv_n);
            *a.ticket = 0u;
        }
    }
}

// ---- the fused pass -------------------------------------------------------------------
template <class T, int MARK, int ACC, bool STREAM, bool UPDATE>
__global__ void __launch_bounds__(kThreads) k_pass(PassArgs a) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    using Acc = typename AccSel<T, ACC>::A;
    using S = typename AccSel<T, ACC>::S;

    V *amps = static_cast<V *>(a.amps);
    const uint64_t nvec = a.nvec;
    const uint64_t tile = (uint64_t)kThreads * kUnroll;
    const uint64_t stride = (uint64_t)gridDim.x * tile;
    const uint64_t first = (uint64_t)blockIdx.x * tile + threadIdx.x;

    ListCursor cur;
    if (MARK == MARK_LIST) cur.init(a.mk.list, a.mk.m, first * APV);

    griddep_wait();  // previous pass: its stores and its mean are visible
    griddep_launch_dependents();

    // 2 mu in the storage type; for complex64 as an unevaluated sum hi + lo of
    // two floats, so the update is not shifted by one shared rounding of 2 mu.
    T two_re = T(0), two_im = T(0), lo_re = T(0), lo_im = T(0);
    if (UPDATE) {
        if constexpr (APV == 2) {
            const float4 h = a.mu_in->two32;
            two_re = h.x;
            lo_re = h.y;
            two_im = h.z;
            lo_im = h.w;
        } else {
            const double2 t2 = a.mu_in->two;
            two_re = t2.x;
            two_im = t2.y;
        }
    }
    auto upd = [&](T x, T two, T lo) -> T {
        if constexpr (APV == 2) return (two - x) + lo;
        else return two - x;
    };

    constexpr int G = kUnroll * APV;
    Acc acc;
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < nvec; base += stride) {
        V v[kUnroll];
        uint32_t f[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
            f[u] = 0;
            if (i < nvec) {
                v[u] = ldv<STREAM>(amps + i);
                if (MARK == MARK_BITS) f[u] = mask_bits<APV>(a.mk.words, i * APV);
            }
        }
        if (MARK == MARK_LIST) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
                if (i < nvec) f[u] = cur.template bits<APV>(i * APV);
            }
        }
        T gr[G], gi[G];  // O c_new of this tile, summed pairwise
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = base + (uint64_t)u * kThreads + threadIdx.x;
            if (i >= nvec) {
#pragma unroll
                for (int j = 0; j < APV; ++j) gr[u * APV + j] = gi[u * APV + j] = T(0);
                continue;
            }
            V c = v[u];
            if constexpr (APV == 2) {
                const uint32_t f0 = f[u] & 1u, f1 = f[u] >> 1;
                if (UPDATE) {
                    // c' = O c ; c <- 2 mu - c'
                    c.x = upd(flip(c.x, f0), two_re, lo_re);
                    c.y = upd(flip(c.y, f0), two_im, lo_im);
                    c.z = upd(flip(c.z, f1), two_re, lo_re);
                    c.w = upd(flip(c.w, f1), two_im, lo_im);
                    stv<STREAM>(amps + i, c);
                }
                gr[2 * u] = flip(c.x, f0);
                gi[2 * u] = flip(c.y, f0);
                gr[2 * u + 1] = flip(c.z, f1);
                gi[2 * u + 1] = flip(c.w, f1);
            } else {
                const uint32_t f0 = f[u];
                if (UPDATE) {
                    c.x = upd(flip(c.x, f0), two_re, lo_re);
                    c.y = upd(flip(c.y, f0), two_im, lo_im);
                    stv<STREAM>(amps + i, c);
                }
                gr[u] = flip(c.x, f0);
                gi[u] = flip(c.y, f0);
            }
        }
        acc.template add_group<G>(gr, gi);
    }

    if constexpr (AccSel<T, ACC>::INT) {
        int_combine(acc.r, acc.i, acc.side_r, acc.side_i, a);
    } else {
        // block tree in S precision, then FP64 partial
        __shared__ S sm[kThreads / 32];
        const auto val = acc_value(acc);
        S r = block_sum((S)val.x, sm);
        S im = block_sum((S)val.y, sm);
        grid_combine(make_double2((double)r, (double)im), a);
    }
}

// ---- the fused pass, staged through shared memory ---------------------------------------------
// The same pass for states larger than L2, with the state moved by the bulk
// copy engine instead of per-thread loads: CTAs stream chunks of
// kUnroll * kThreads vectors (16 KiB, the tile of k_pass, so every thread
// works on the same vectors and groups as there and the results are bitwise
// those of k_pass) through kBulkStages shared-memory buffers.  Thread 0 keeps
// the next chunk loads in flight (cp.async.bulk, completion counted on an
// mbarrier per buffer); every thread waits for its buffer (bounded), updates
// it in place, one block barrier, and thread 0 writes the buffer back with one
// bulk store and refills the buffer of the chunk before, whose store has been
// reading it meanwhile.
// Shape, measured on GB300 (n = 29 / 32 / 33 complex64, GB/s per pass): two
// stages and 8 CTAs launched per SM (4 resident at 62 registers a thread)
// 6722 / 6680 / 6717 against 6386 / 6376 / 6383 with per-thread 16-byte
// loads and stores; one CTA per SM with 4-8 stages is faster at some sizes
// and slower at others (6789 at n = 29, 6007 at n = 33 with 6 stages).
constexpr int kBulkStages = 2;
constexpr int kBulkCtasPerSm = 8;
constexpr int kBulkChunk = kThreads * kUnroll;  // vectors per chunk (16 KiB)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, unsigned parity) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_addr(b)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes) : "memory");
}

template <class T, int MARK, int ACC>
__global__ void __launch_bounds__(kThreads) k_pass_bulk(PassArgs a) {
    using V = typename Vec<T>::V;
    constexpr int APV = Vec<T>::APV;
    constexpr unsigned kBytes = kBulkChunk * sizeof(V);
    using Acc = typename AccSel<T, ACC>::A;
    using S = typename AccSel<T, ACC>::S;
    extern __shared__ __align__(128) unsigned char stage[];  // [kBulkStages][kBytes]
    __shared__ __align__(8) uint64_t bar[kBulkStages];
    __shared__ int s_bad;

    V *amps = static_cast<V *>(a.amps);
    const uint64_t G = gridDim.x, nchunks = a.nvec / kBulkChunk;
    const uint64_t mine = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / G + 1 : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBulkStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_bad = 0;
    }
    ListCursor cur;
    if (MARK == MARK_LIST) cur.init(a.mk.list, a.mk.m, ((uint64_t)blockIdx.x * kBulkChunk + threadIdx.x) * APV);
    __syncthreads();

    griddep_wait();  // previous pass: its stores and its mean are visible
    griddep_launch_dependents();
    uint64_t issued = 0;  // chunk loads issued (thread 0)
    if (threadIdx.x == 0)
        for (; issued < (uint64_t)kBulkStages && issued < mine; ++issued) {
            mbar_expect_tx(&bar[issued], kBytes);
            if (a.stall && blockIdx.x == 0 && issued == 0) continue;  // test hook: this copy never comes
            bulk_load(stage + issued * kBytes, amps + (blockIdx.x + issued * G) * kBulkChunk, kBytes, &bar[issued]);
        }

    T two_re = T(0), two_im = T(0), lo_re = T(0), lo_im = T(0);
    if constexpr (APV == 2) {
        const float4 h = a.mu_in->two32;
        two_re = h.x;
        lo_re = h.y;
        two_im = h.z;
        lo_im = h.w;
    } else {
        const double2 t2 = a.mu_in->two;
        two_re = t2.x;
        two_im = t2.y;
    }
    auto upd = [&](T x, T two, T lo) -> T {
        if constexpr (APV == 2) return (two - x) + lo;
        else return two - x;
    };

    constexpr int G8 = kUnroll * APV;
    Acc acc;
    uint64_t i = 0;
    for (; i < mine; ++i) {
        const int s = (int)(i % kBulkStages);
        const unsigned parity = (unsigned)((i / kBulkStages) & 1);
        const uint64_t base = (blockIdx.x + i * G) * kBulkChunk;
        // the marked flags need no data: take them before waiting
        uint32_t f[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t v = base + (uint64_t)u * kThreads + threadIdx.x;
            f[u] = 0;
            if (MARK == MARK_BITS) f[u] = mask_bits<APV>(a.mk.words, v * APV);
            if (MARK == MARK_LIST) f[u] = cur.template bits<APV>(v * APV);
        }
        int timed_out = 0;
        for (long long polls = 0; !mbar_try_wait(&bar[s], parity);)
            if (++polls >= a.wait_limit) {
                timed_out = 1;
                break;
            }
        V *buf = reinterpret_cast<V *>(stage + (size_t)s * kBytes);
        T gr[G8], gi[G8];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            V c = buf[u * kThreads + threadIdx.x];
            if constexpr (APV == 2) {
                const uint32_t f0 = f[u] & 1u, f1 = f[u] >> 1;
                c.x = upd(flip(c.x, f0), two_re, lo_re);
                c.y = upd(flip(c.y, f0), two_im, lo_im);
                c.z = upd(flip(c.z, f1), two_re, lo_re);
                c.w = upd(flip(c.w, f1), two_im, lo_im);
                buf[u * kThreads + threadIdx.x] = c;
                gr[2 * u] = flip(c.x, f0);
                gi[2 * u] = flip(c.y, f0);
                gr[2 * u + 1] = flip(c.z, f1);
                gi[2 * u + 1] = flip(c.w, f1);
            } else {
                const uint32_t f0 = f[u];
                c.x = upd(flip(c.x, f0), two_re, lo_re);
                c.y = upd(flip(c.y, f0), two_im, lo_im);
                buf[u * kThreads + threadIdx.x] = c;
                gr[u] = flip(c.x, f0);
                gi[u] = flip(c.y, f0);
            }
        }
        acc.template add_group<G8>(gr, gi);
        // this thread's shared-memory writes, before the bulk store reads them;
        // the barrier also tells every thread whether any wait of this chunk
        // ran out, so all leave the loop at the same chunk
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) s_bad = 1;
            break;
        }
        if (threadIdx.x == 0) {
            bulk_store(amps + base, buf, kBytes);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            // refill the buffer of the previous chunk, whose store has had a
            // whole chunk's compute time to read it (only the newest store may
            // still be reading)
            if (i >= 1 && i - 1 + kBulkStages < mine) {
                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                const int sp = (int)((i - 1) % kBulkStages);
                mbar_expect_tx(&bar[sp], kBytes);
                bulk_load(stage + (size_t)sp * kBytes, amps + (blockIdx.x + (i - 1 + kBulkStages) * G) * kBulkChunk,
                          kBytes, &bar[sp]);
                ++issued;
            }
        }
    }
    if (threadIdx.x == 0) {
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete before the combine
        if (s_bad) {
            // chunk i's wait ran out: report it, and let the loads still in
            // flight (chunks i .. issued - 1) land before the CTA's shared
            // memory is released.  The pass has failed already, so this wait
            // gets 64 times the normal bound: a copy that is merely slow lands
            // here rather than in the shared memory of a later CTA.  The copy
            // the test hook withheld is never issued and is not waited for.
            if (a.status) atomicExch(a.status, 5);
            const long long drain_limit = a.wait_limit * 64;
            for (uint64_t j = i; j < issued; ++j) {
                if (j == 0 && a.stall && blockIdx.x == 0) continue;
                for (long long polls = 0;
                     !mbar_try_wait(&bar[j % kBulkStages], (unsigned)((j / kBulkStages) & 1));)
                    if (++polls >= drain_limit) break;
            }
        }
    }

    if constexpr (AccSel<T, ACC>::INT) {
        int_combine(acc.r, acc.i, acc.side_r, acc.side_i, a);
    } else {
        __shared__ S sm[kThreads / 32];
        const auto val = acc_value(acc);
        S r = block_sum((S)val.x, sm);
        S im = block_sum((S)val.y, sm);
        grid_combine(make_double2((double)r, (double)im), a);
    }
}

// ---- initialisation / oracle -----------------------------------------------------------------
template <class T> __global__ void __launch_bounds__(kThreads) k_init_uniform(void *amps, uint64_t nvec, int n) {
    using V = typename Vec<T>::V;
    const double a = 1.0 / sqrt((double)(1ull << n));  // IEEE sqrt and division
    const T t = (T)a;
    V v;
    if constexpr (Vec<T>::APV == 2) v = make_float4(t, 0.f, t, 0.f);
    else v = make_double2(t, 0.0);
    V *p = static_cast<V *>(amps);
    griddep_wait();
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < nvec; i += (uint64_t)gridDim.x * kThreads)
        p[i] = v;
}

template <class T> __global__ void k_oracle_list(T *amps, const uint64_t *list, uint64_t m) {
    griddep_wait();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = list[i];
        amps[2 * x] = -amps[2 * x];
        amps[2 * x + 1] = -amps[2 * x + 1];
    }
}

template <class T> __global__ void k_oracle_bits(T *amps, const uint32_t *words, uint64_t nwords, uint64_t N) {
    griddep_wait();
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = words[w];
        while (b) {
            const int j = __ffs(b) - 1;
            b &= b - 1;
            const uint64_t x = w * 32 + j;
            if (x < N) {
                amps[2 * x] = -amps[2 * x];
                amps[2 * x + 1] = -amps[2 * x + 1];
            }
        }
    }
}

__global__ void k_bits_from_list(uint32_t *words, const uint64_t *list, uint64_t m) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = list[i];
        atomicOr(words + (x >> 5), 1u << (uint32_t)(x & 31));
    }
}

__global__ void k_bits_check_count(const uint32_t *words, uint64_t nwords, uint64_t N,
                                   unsigned long long *count, int *bad) {
    unsigned long long c = 0;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = words[w];
        if (N < 32 && w == 0 && (b >> N) != 0u) atomicExch(bad, 1);
        c += __popc(b);
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// ---- launch helpers ---------------------------------------------------------------------------
bool pdl_enabled() {
    // read once per process (initialisation of a local static is thread-safe)
    static const bool v = [] {
        const char *e = getenv("GROVER_PDL");
        return !(e && e[0] == '0');
    }();
    return v;
}

template <class... KArgs, class... Args>
cudaError_t launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Most CTAs a pass may launch: the partial-sum slots it writes (integer modes
// take three per CTA: two 128-bit integers and the FP64 side sums).
template <class T, int ACC> int slot_cap(const Geometry &g) {
    const int per_cta = AccSel<T, ACC>::INT ? 3 : 1;
    const int c = g.partial_slots / per_cta;
    return c < kMaxGrid ? c : kMaxGrid;
}

// CTAs of `kernel` resident on the handle's device at once (queried on every
// launch: occupancy depends on the device, and a process may drive several).
template <class K> int resident_ctas(K kernel, const Geometry &g) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const long long r = (long long)per_sm * g.sm_count;
    return (int)(r > kMaxGrid ? kMaxGrid : r);
}

template <class T, int MARK, int ACC, bool STREAM, bool UPDATE>
cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st, const Geometry &g) {
    auto kern = k_pass<T, MARK, ACC, STREAM, UPDATE>;
    int cap = resident_ctas(kern, g);
    const int slots = slot_cap<T, ACC>(g);
    if (cap > slots) cap = slots;
    const uint64_t tile = (uint64_t)kThreads * kUnroll;
    uint64_t need = (a.nvec + tile - 1) / tile;
    unsigned grid = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
    if (grid == 0) grid = 1;
    return launch(kern, grid, kThreads, st, a);
}

template <class T, int MARK, int ACC>
cudaError_t launch_bulk_t(const PassArgs &a, cudaStream_t st, const Geometry &g) {
    auto kern = k_pass_bulk<T, MARK, ACC>;
    constexpr size_t smem = (size_t)kBulkStages * kBulkChunk * 16;
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    const uint64_t nchunks = a.nvec / kBulkChunk, cap = (uint64_t)g.sm_count * kBulkCtasPerSm;
    unsigned grid = (unsigned)(nchunks < cap ? nchunks : cap);
    const unsigned slots = (unsigned)slot_cap<T, ACC>(g);
    if (grid > slots) grid = slots;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class T, int ACC, bool UPDATE>
cudaError_t dispatch_mark(const PassArgs &a, cudaStream_t st, const Geometry &g) {
    const bool s = a.stream_hint;
    // the staged pass for complex64 states larger than L2 / 2 (whole chunks
    // only); complex128 (FP64 update, every amplitude summed exactly) keeps
    // the per-thread pass unless asked: staged it measured 5.3 against
    // 6.3 TB/s at n = 28, the work per byte wants more warps than two stages
    // per CTA leave
    const bool automatic = s && sizeof(T) == 4;
    if (UPDATE && (a.staged == 1 || (a.staged < 0 && automatic)) && a.nvec >= (uint64_t)kBulkChunk &&
        a.nvec % kBulkChunk == 0) {
        switch (a.mk.mode) {
        case MARK_LIST: return launch_bulk_t<T, MARK_LIST, ACC>(a, st, g);
        case MARK_BITS: return launch_bulk_t<T, MARK_BITS, ACC>(a, st, g);
        default: return launch_bulk_t<T, MARK_NONE, ACC>(a, st, g);
        }
    }
    switch (a.mk.mode) {
    case MARK_LIST:
        return s ? launch_pass_t<T, MARK_LIST, ACC, true, UPDATE>(a, st, g)
                 : launch_pass_t<T, MARK_LIST, ACC, false, UPDATE>(a, st, g);
    case MARK_BITS:
        return s ? launch_pass_t<T, MARK_BITS, ACC, true, UPDATE>(a, st, g)
                 : launch_pass_t<T, MARK_BITS, ACC, false, UPDATE>(a, st, g);
    default:
        return s ? launch_pass_t<T, MARK_NONE, ACC, true, UPDATE>(a, st, g)
                 : launch_pass_t<T, MARK_NONE, ACC, false, UPDATE>(a, st, g);
    }
}

template <bool UPDATE>
cudaError_t dispatch(const PassArgs &a, grover_dtype dt, grover_accum acc, cudaStream_t st, const Geometry &g) {
    if (dt == GROVER_C128) {
        // complex128 default: exact integer accumulation (the FP64 pipe is the
        // bottleneck of the pass otherwise)
        if (acc == GROVER_ACC_FP64) return dispatch_mark<double, GROVER_ACC_FP64, UPDATE>(a, st, g);
        return dispatch_mark<double, GROVER_ACC_EXACT, UPDATE>(a, st, g);
    }
    switch (acc) {
    case GROVER_ACC_FP32: return dispatch_mark<float, GROVER_ACC_FP32, UPDATE>(a, st, g);
    case GROVER_ACC_KAHAN: return dispatch_mark<float, GROVER_ACC_KAHAN, UPDATE>(a, st, g);
    case GROVER_ACC_EXACT: return dispatch_mark<float, GROVER_ACC_EXACT, UPDATE>(a, st, g);
    case GROVER_ACC_FP64: return dispatch_mark<float, GROVER_ACC_FP64, UPDATE>(a, st, g);
    default: return dispatch_mark<float, ACC_HYBRID, UPDATE>(a, st, g);
    }
}

}  // namespace

// ---- host launchers ------------------------------------------------------------------------------
cudaError_t launch_init_uniform(void *amps, int n, grover_dtype dt, cudaStream_t st, const Geometry &g) {
    const uint64_t N = 1ull << n;
    const uint64_t nvec = dt == GROVER_C64 ? N / 2 : N;
    uint64_t need = (nvec + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)g.sm_count * 8;
    unsigned grid = (unsigned)(need < cap ? need : cap);
    if (dt == GROVER_C64) return launch(k_init_uniform<float>, grid, kThreads, st, amps, nvec, n);
    return launch(k_init_uniform<double>, grid, kThreads, st, amps, nvec, n);
}

cudaError_t launch_pass(const PassArgs &a, grover_dtype dt, grover_accum acc, cudaStream_t st,
                        const Geometry &g) {
    return dispatch<true>(a, dt, acc, st, g);
}

cudaError_t launch_reduce(const PassArgs &a, grover_dtype dt, grover_accum acc, cudaStream_t st,
                          const Geometry &g) {
    return dispatch<false>(a, dt, acc, st, g);
}

cudaError_t launch_oracle(void *amps, int n, grover_dtype dt, const MarkedDev &mk, cudaStream_t st,
                          const Geometry &g) {
    const uint64_t N = 1ull << n;
    if (mk.m == 0) return cudaSuccess;
    if (mk.mode == MARK_BITS) {
        const uint64_t nwords = (N + 31) / 32;
        uint64_t need = (nwords + kThreads - 1) / kThreads;
        const uint64_t cap = (uint64_t)g.sm_count * 8;
        unsigned grid = (unsigned)(need < cap ? need : cap);
        if (dt == GROVER_C64)
            return launch(k_oracle_bits<float>, grid, kThreads, st, (float *)amps, mk.words, nwords, N);
        return launch(k_oracle_bits<double>, grid, kThreads, st, (double *)amps, mk.words, nwords, N);
    }
    unsigned grid = (unsigned)((mk.m + 127) / 128);
    if (grid > 1024) grid = 1024;
    if (dt == GROVER_C64) return launch(k_oracle_list<float>, grid, 128, st, (float *)amps, mk.list, mk.m);
    return launch(k_oracle_list<double>, grid, 128, st, (double *)amps, mk.list, mk.m);
}

cudaError_t launch_bits_from_list(uint32_t *words, uint64_t nwords, const uint64_t *list, uint64_t m,
                                  cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(words, 0, nwords * sizeof(uint32_t), st);
    if (e != cudaSuccess || m == 0) return e;
    unsigned grid = (unsigned)((m + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_bits_from_list<<<grid, 256, 0, st>>>(words, list, m);
    return cudaGetLastError();
}

cudaError_t launch_bits_check_count(const uint32_t *words, uint64_t nwords, int n, unsigned long long *count_out,
                                    int *bad_out, cudaStream_t st) {
    unsigned grid = (unsigned)((nwords + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_bits_check_count<<<grid, 256, 0, st>>>(words, nwords, 1ull << n, count_out, bad_out);
    return cudaGetLastError();
}

}  // namespace grv
