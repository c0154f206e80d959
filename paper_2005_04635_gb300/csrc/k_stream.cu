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
// adds that to its running sum.  Pairwise summation of the group is exact when
// the values are equal, which they are for every unmarked amplitude of a
// uniform-start search: no rounding bias repeats across the N/G groups.
template <int G, class T> __device__ __forceinline__ T pairwise(const T *v) {
    if constexpr (G == 1) return v[0];
    else if constexpr (G == 2) return v[0] + v[1];
    else if constexpr (G == 4) return (v[0] + v[1]) + (v[2] + v[3]);
    else return pairwise<G / 2>(v) + pairwise<G / 2>(v + G / 2);
}

// complex128: FP64 pairwise group sum, FP64 running sum.
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

// GROVER_ACC_EXACT: magnitudes below 1 are added exactly as 128-bit integers
// in units of 2^-100 (bits below 2^-100 are dropped: < 2^-100 per amplitude),
// on the integer pipe; larger magnitudes, Inf and NaN go to an FP64 side sum.
// A thread's integer sum stays below 2^115 for any 2^32 amplitudes.
constexpr int kFixLsb = 100;
__device__ __forceinline__ void fix_add(unsigned __int128 &acc, double &side, double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e >= 1023u) {
        side += x;
        return;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0u) << 52);
    const int sh = (int)e - (1075 - kFixLsb);  // x = m * 2^(sh - kFixLsb)
    unsigned __int128 v;
    if (sh >= 0) v = (unsigned __int128)m << sh;
    else v = sh > -64 ? (unsigned __int128)(m >> (-sh)) : (unsigned __int128)0;
    const unsigned __int128 neg = (unsigned __int128)(__int128)((long long)b >> 63);
    acc += (v ^ neg) - neg;
}
__device__ __forceinline__ void fix_add(unsigned __int128 &acc, double &side, float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xFFu;
    if (e >= 127u) {
        side += (double)x;
        return;
    }
    const unsigned long long m = (b & 0x7FFFFFu) | ((unsigned)(e != 0u) << 23);
    const int sh = (int)e - (150 - kFixLsb);
    unsigned __int128 v;
    if (sh >= 0) v = (unsigned __int128)m << sh;
    else v = sh > -24 ? (unsigned __int128)(m >> (-sh)) : (unsigned __int128)0;
    const unsigned __int128 neg = (unsigned __int128)(__int128)((int)b >> 31);
    acc += (v ^ neg) - neg;
}
struct AccX {
    unsigned __int128 r = 0, i = 0;
    double side_r = 0.0, side_i = 0.0;
    template <int G, class T> __device__ __forceinline__ void add_group(const T *re, const T *im) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            fix_add(r, side_r, re[j]);
            fix_add(i, side_i, im[j]);
        }
    }
};

// double-double arithmetic for combining exact per-thread sums (plain adds only)
struct DD {
    double h, l;
};
__device__ __forceinline__ DD dd_add(DD a, DD b) {
    const double s = __dadd_rn(a.h, b.h);
    const double bb = __dsub_rn(s, a.h);
    double e = __dadd_rn(__dsub_rn(a.h, __dsub_rn(s, bb)), __dsub_rn(b.h, bb));
    e = __dadd_rn(e, __dadd_rn(a.l, b.l));
    const double h = __dadd_rn(s, e);
    return DD{h, __dsub_rn(e, __dsub_rn(h, s))};
}
__device__ __forceinline__ DD dd_from_fix(unsigned __int128 u, double side) {
    const __int128 x = (__int128)u;
    const double h = (double)x;
    const double l = (double)(x - (__int128)h);
    return dd_add(DD{h * 0x1p-100, l * 0x1p-100}, DD{side, 0.0});
}

template <class T, int ACC> struct AccSel;
template <int ACC> struct AccSel<double, ACC> { using A = AccD; using S = double; };
template <> struct AccSel<double, GROVER_ACC_EXACT> { using A = AccX; using S = double; };
template <> struct AccSel<float, GROVER_ACC_EXACT> { using A = AccX; using S = double; };
template <> struct AccSel<float, GROVER_ACC_FP64> { using A = AccF64; using S = double; };
template <> struct AccSel<float, GROVER_ACC_FP32> { using A = AccF32; using S = float; };
template <> struct AccSel<float, GROVER_ACC_KAHAN> { using A = AccKahan; using S = float; };

__device__ __forceinline__ double2 acc_value(const AccD &a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ double2 acc_value(const AccF64 &a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ float2 acc_value(const AccF32 &a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ float2 acc_value(const AccKahan &a) {
    return make_float2(__fadd_rn(a.sr, a.cr), __fadd_rn(a.si, a.ci));
}

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

// Per-CTA partial -> partials[], last CTA combines in FP64 in a fixed order.
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
        *a.mu_out = make_double2(sr * a.inv_n, si * a.inv_n);
        *a.ticket = 0u;
    }
}

__device__ __forceinline__ DD warp_dd(DD v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = dd_add(v, DD{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
    return v;
}
__device__ __forceinline__ DD block_dd(DD v, DD *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_dd(v);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < kThreads / 32) ? sm[lane] : DD{0.0, 0.0};
        v = warp_dd(v);
    }
    return v;
}
// Exact mode: per-CTA double-double partials in partials[2b], partials[2b+1];
// the last CTA adds them in a fixed order in double-double.
__device__ __forceinline__ void grid_combine_dd(DD re, DD im, const PassArgs &a) {
    __shared__ DD sm[kThreads / 32];
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
        a.partials[2 * blockIdx.x] = make_double2(re.h, re.l);
        a.partials[2 * blockIdx.x + 1] = make_double2(im.h, im.l);
        __threadfence();
        unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    DD sr{0.0, 0.0}, si{0.0, 0.0};
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kThreads) {
        const double2 qr = __ldcg(a.partials + 2 * j), qi = __ldcg(a.partials + 2 * j + 1);
        sr = dd_add(sr, DD{qr.x, qr.y});
        si = dd_add(si, DD{qi.x, qi.y});
    }
    sr = block_dd(sr, sm);
    si = block_dd(si, sm);
    if (threadIdx.x == 0) {
        *a.mu_out = make_double2(__dadd_rn(sr.h, sr.l) * a.inv_n, __dadd_rn(si.h, si.l) * a.inv_n);
        *a.ticket = 0u;
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
        const double2 mu = *a.mu_in;
        two_re = (T)(2.0 * mu.x);
        two_im = (T)(2.0 * mu.y);
        lo_re = (T)(2.0 * mu.x - (double)two_re);
        lo_im = (T)(2.0 * mu.y - (double)two_im);
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

    if constexpr (ACC == GROVER_ACC_EXACT) {
        __shared__ DD smd[kThreads / 32];
        const DD r = block_dd(dd_from_fix(acc.r, acc.side_r), smd);
        const DD im = block_dd(dd_from_fix(acc.i, acc.side_i), smd);
        grid_combine_dd(r, im, a);
    } else {
        // block tree in S precision, then FP64 partial
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
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("GROVER_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
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

template <class K> int resident_ctas(K kernel, const Geometry &g) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long r = (long long)per_sm * g.sm_count;
    return (int)(r > kMaxGrid ? kMaxGrid : r);
}

template <class T, int MARK, int ACC, bool STREAM, bool UPDATE>
cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st, const Geometry &g) {
    auto kern = k_pass<T, MARK, ACC, STREAM, UPDATE>;
    static int cap = 0;
    if (cap == 0) cap = resident_ctas(kern, g);
    const uint64_t tile = (uint64_t)kThreads * kUnroll;
    uint64_t need = (a.nvec + tile - 1) / tile;
    unsigned grid = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
    if (grid == 0) grid = 1;
    return launch(kern, grid, kThreads, st, a);
}

template <class T, int ACC, bool UPDATE>
cudaError_t dispatch_mark(const PassArgs &a, cudaStream_t st, const Geometry &g) {
    const bool s = a.stream_hint;
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
    default: return dispatch_mark<float, GROVER_ACC_FP64, UPDATE>(a, st, g);
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
