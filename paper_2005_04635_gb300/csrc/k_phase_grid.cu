// k_phase_grid.cu -- the phase iterator and its adjoint with the state kept in
// shared memory across all SMs (complex64, states that fit on chip).
//
// Same arithmetic as k_phase.cu (oracle phase e^{i phi_t} on marked
// amplitudes, c <- c - (1 - e^{i vphi_t}) <c>; adjoint through the inverse
// iterators), but one cooperative launch per sweep: CTA r keeps vectors
// [r L, (r + 1) L) of the state (and, backward, of the adjoint) in shared
// memory for all K iterations, and the per-iteration sums over all N
// amplitudes meet through grid_exchange.cuh (exact integer limbs, an arrival
// counter, bounded waits).
// Every CTA also keeps a replica of the M <= 256 marked amplitudes and applies
// to it the same operations, with the same constants and explicitly rounded
// arithmetic, as the CTA that owns them, so the replicas stay bitwise equal to
// the owners' values.  The marked sums the method needs (the oracle term of
// the next mean, P, and the phi gradient's sum) are then computed in every CTA
// without communication, and the exchange carries only the full sums: forward
// the state sum, backward the sums of the state and of the adjoint.  Every CTA
// forms the next pass's constants itself, the same operations in every CTA, so
// the same values.  No FP64 operation sits between an exchange and the next
// pass (each costs ~100-175 cycles of latency on the GB300): the exact integer
// totals become float pairs with integer operations, the constants are formed
// in float-float arithmetic, the per-step phase factors come as float pairs
// from a table filled before the launch, and the FP64 work that remains (the
// replica's sums, the gradients) runs in warps 1 and 2 while warp 0 waits for
// the other CTAs.
// The backward sweep carries lambda~ = sqrt(P) lambda, whose entries are at
// most 1 in magnitude (|lambda~_K,x| = |psi_x| / sqrt(P) <= 1 and the sweep is
// unitary), so its sums stay inside the fixed-point window whatever P is; the
// gradients and the stored lambda_0 are scaled back by 1 / sqrt(P).
#include "fixed_sum.cuh"
#include "grid_exchange.cuh"
#include "grover_internal.cuh"
#include "phase_ops.cuh"

namespace grv {
namespace {

using ph::cff_mul;
using ph::cff_add;
using ph::cff_pack;
using ph::expi;
using ph::pairwise;
using ph::sub_hilo;
using ph::warp_sum_d;

constexpr int kPgThreads = 512;
constexpr int kPgWarps = kPgThreads / 32;
constexpr int kNVmax = 4;  // sums per exchange: 2 forward, 4 backward
constexpr int kU = 4;      // vectors per thread per group

// complex product with every operation rounded on its own (no contraction),
// so an owner and a replica compute bitwise the same value
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b) {
    return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                       __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

// The two exchange series in the region: one of two sums (the forward sweep;
// the backward sweep's first exchange), then one of four (the backward passes).
__device__ __forceinline__ unsigned long long *series2(const PhaseGridArgs &a) { return a.region; }
__device__ __forceinline__ unsigned long long *series4(const PhaseGridArgs &a) {
    return a.region + (GxLayout<2>::kAccBytes + GxLayout<2>::side_bytes(512)) / sizeof(unsigned long long);
}

// Warps 0 and 1 meet at named barrier 1 (warp 1 arrives, warp 0 waits).
__device__ __forceinline__ void pair_arrive() { asm volatile("bar.arrive 1, 64;" ::: "memory"); }
__device__ __forceinline__ void pair_wait() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// nonzero side sum, tested on the bits (an FP64 compare is slow on the GB300)
__device__ __forceinline__ bool has_side(double v) { return __double_as_longlong(v) != 0; }

// (r 2^-100 + side) / N as a float-float: from the integer alone (exact
// rounding, integer operations) unless there is a side sum.
__device__ __forceinline__ ph::ff mean_ff(u128 r, double side, int n) {
    if (!has_side(side)) {
        const float2 p = fix_to_f32_pair(r, -100 - n);
        return ph::ff{p.x, p.y};
    }
    return ph::ff_of((i192_to_double(i192_from(r), -100) + side) * __hiloint2double((1023 - n) << 20, 0));
}
__device__ __forceinline__ double sum_d(u128 r, double side) {
    return i192_to_double(i192_from(r), -100) + side;
}

// The CTA's NV exact sums (side sums, if any, in a fixed tree order), then the
// grid exchange by thread 0.  Meanwhile warp 1 runs job() (it must leave its
// results in shared memory and not touch wint / wsd) and warp 2 aside().
// After both the exchange and job(), thread 0 runs post(T, S) with the exact
// integer totals (units 2^-100, the same in every CTA) and their side sums;
// post writes the next pass's constants to shared memory.  Two block barriers
// per exchange.  Returns false in every thread if a wait ran out (the status
// word is set and post did not run).
template <int NV, class Job, class Aside, class Post>
__device__ bool cta_exchange(u128 (&v)[NV], double (&sd)[NV], const PhaseGridArgs &a, unsigned long long *region,
                             long long xi, unsigned long long (&prev)[2][GxLayout<NV>::W], bool withhold, Job job,
                             Aside aside, Post post) {
    __shared__ unsigned long long wint[kPgWarps][kNVmax][2];
    __shared__ double wsd[kPgWarps][kNVmax];
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int local_side = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        v[q] = warp_sum_u128(v[q]);
        local_side |= has_side(sd[q]);
    }
    const bool warp_side = __any_sync(0xffffffffu, local_side);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        if (warp_side) sd[q] = warp_sum_d(sd[q]);
        if (lane == 0) {
            wint[warp][q][0] = (unsigned long long)v[q];
            wint[warp][q][1] = (unsigned long long)(v[q] >> 64);
            wsd[warp][q] = sd[q];
        }
    }
    __syncthreads();
    if (warp == 1) {
        job();
        pair_arrive();
    } else if (warp == 2) {
        aside();
    } else if (warp == 0) {
        u128 t[NV];
        double ts[NV];
        int side = 0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            t[q] = 0;
            ts[q] = 0.0;
            if (lane < kPgWarps) {
                t[q] = ((u128)wint[lane][q][1] << 64) | wint[lane][q][0];
                ts[q] = wsd[lane][q];
                side |= has_side(ts[q]);
            }
        }
        const int any_side = __any_sync(0xffffffffu, side);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            t[q] = warp_sum_u128(t[q]);
            if (any_side) ts[q] = warp_sum_d(ts[q]);
        }
        u128 T[NV];
        double S[NV];
        bool ok = false;
        if (lane == 0)
            ok = gx_exchange<NV>(t, ts, any_side, region, prev, xi, gridDim.x, blockIdx.x, a.wait_limit, withhold, T, S);
        pair_wait();
        if (lane == 0) {
            if (ok) post(T, S);
            else atomicExch(a.status, 3);
            s_ok = ok;
        }
    }
    __syncthreads();
    return s_ok != 0;
}

// Marked bitmask of this CTA's slice (amplitudes [a0, a0 + nbits)) in shared memory.
__device__ void build_mask(uint32_t *fm, uint32_t nwords, const PhaseGridArgs &a, uint64_t a0, uint32_t nbits) {
    for (uint32_t w = threadIdx.x; w < nwords; w += kPgThreads) fm[w] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < a.m; i += kPgThreads) {
        const uint64_t x = a.list[i];
        if (x >= a0 && x < a0 + nbits) atomicOr(fm + ((x - a0) >> 5), 1u << (uint32_t)((x - a0) & 31));
    }
    __syncthreads();
}

// The constants of step t from phi_t, vphi_t (FP64 sincos, then float pairs).
__device__ PhaseFac make_fac(double phi, double vphi) {
    const double2 e = expi(phi), ev = expi(vphi);
    PhaseFac f;
    f.em1 = cff_pack(ph::cff{ph::ff_of(e.x - 1.0), ph::ff_of(e.y)});
    f.omv = cff_pack(ph::cff{ph::ff_of(1.0 - ev.x), ph::ff_of(-ev.y)});
    f.rot = make_float2((float)e.x, (float)e.y);
    f.pad = make_float2(0.f, 0.f);
    return f;
}
// from the table the launcher filled, else formed here
__device__ __forceinline__ PhaseFac fac_of(const PhaseGridArgs &a, long long t) {
    if (a.table) {
        const float4 *p = reinterpret_cast<const float4 *>(a.table + t);
        PhaseFac f;
        f.em1 = __ldg(p);
        f.omv = __ldg(p + 1);
        const float4 r = __ldg(p + 2);
        f.rot = make_float2(r.x, r.y);
        f.pad = make_float2(0.f, 0.f);
        return f;
    }
    return make_fac(a.phi[t], a.vphi[t]);
}

__global__ void k_phase_table(const double *phi, const double *vphi, long long K, PhaseFac *table) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    table[t] = make_fac(phi[t], vphi[t]);
}

__device__ __forceinline__ uint32_t mark2(const uint32_t *fm, uint32_t j) {
    const uint32_t e = 2 * j;
    return (fm[e >> 5] >> (e & 31)) & 3u;
}

// Exact sums of a replica by one warp: Re, Im (and |c|^2 when want_p) as
// 128-bit integers (units 2^-100) with side sums; every lane gets them.
struct RepSums {
    u128 r = 0, i = 0, p = 0;
    double sr = 0.0, si = 0.0, sp = 0.0;
};
__device__ RepSums replica_sums(const float2 *rep, uint32_t m, bool want_p) {
    const int lane = threadIdx.x & 31;
    RepSums o;
    for (uint32_t q = lane; q < m; q += 32) {
        const float2 c = rep[q];
        fix_add<4>(o.r, o.sr, c.x);
        fix_add<4>(o.i, o.si, c.y);
        if (want_p) fix_add<4>(o.p, o.sp, (double)c.x * c.x + (double)c.y * c.y);
    }
    o.r = warp_sum_u128(o.r);
    o.i = warp_sum_u128(o.i);
    if (__any_sync(0xffffffffu, has_side(o.sr) || has_side(o.si))) {
        o.sr = warp_sum_d(o.sr);
        o.si = warp_sum_d(o.si);
    }
    if (want_p) {
        o.p = warp_sum_u128(o.p);
        o.sp = warp_sum_d(o.sp);
    }
    return o;
}

// ---- forward sweep -----------------------------------------------------------
// U vectors per thread per summation group: slices of at least kPgWideVecs
// vectors take U = 8, one FP32 pairwise sum of 16 amplitudes per exact add
// (half the adds), smaller ones U = 4, whose threads hold too few vectors.
constexpr uint32_t kPgWideVecs = 6 * kPgThreads;

template <int U>
__global__ void __launch_bounds__(kPgThreads, 1) k_phase_grid_fwd(PhaseGridArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float4 s_kap, s_can;
    __shared__ float2 s_rot;
    __shared__ PhaseFac s_fac;
    __shared__ float2 rep[kPhaseMaxMarked];
    __shared__ unsigned long long prev[2][GxLayout<2>::W];
    const unsigned rank = blockIdx.x;
    float4 *sl = reinterpret_cast<float4 *>(smem);
    const uint64_t start = (uint64_t)rank * a.slice_vecs;
    const uint32_t nv = start >= a.nvec ? 0u
                        : (uint32_t)((a.nvec - start) < a.slice_vecs ? (a.nvec - start) : a.slice_vecs);
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + (size_t)a.slice_vecs * 16);
    const uint32_t nwords = (a.slice_vecs * 2 + 31) / 32;
    float4 *g = static_cast<float4 *>(a.psi) + start;
    const float2 *g2 = static_cast<const float2 *>(a.psi);
    for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) sl[j] = g[j];
    for (uint32_t q = threadIdx.x; q < a.m; q += kPgThreads) rep[q] = g2[a.list[q]];
    if (threadIdx.x < 2 * GxLayout<2>::W) prev[threadIdx.x / GxLayout<2>::W][threadIdx.x % GxLayout<2>::W] = 0ull;
    build_mask(fm, nwords, a, start * 2, nv * 2);
    bool ok = true;
    for (long long t = -1; t < a.K && ok; ++t) {
        const bool upd = t >= 0;
        float4 kap = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 rot = make_float2(1.f, 0.f);
        if (upd) {
            kap = s_kap;
            rot = s_rot;
        }
        u128 v[2] = {0, 0};
        double sd[2] = {0.0, 0.0};
        for (uint32_t j0 = threadIdx.x; j0 < nv; j0 += U * kPgThreads) {
            float gr[2 * U], gi[2 * U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = j0 + u * kPgThreads;
                if (j >= nv) {
                    gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                    continue;
                }
                const float4 c = sl[j];
                float2 c0 = make_float2(c.x, c.y), c1 = make_float2(c.z, c.w);
                if (upd) {
                    const uint32_t f = mark2(fm, j);
                    if (f & 1u) c0 = cmul_rn(c0, rot);
                    if (f & 2u) c1 = cmul_rn(c1, rot);
                    c0 = sub_hilo(c0, kap);
                    c1 = sub_hilo(c1, kap);
                    sl[j] = make_float4(c0.x, c0.y, c1.x, c1.y);
                }
                gr[2 * u] = c0.x;
                gi[2 * u] = c0.y;
                gr[2 * u + 1] = c1.x;
                gi[2 * u + 1] = c1.y;
            }
            fix_add<4>(v[0], sd[0], pairwise<2 * U>(gr));
            fix_add<4>(v[1], sd[1], pairwise<2 * U>(gi));
        }
        const long long nxt = t + 1;
        const bool last = nxt >= a.K;
        // warp 1, while the exchange waits: the replica of the marked
        // amplitudes goes through the same update; its sum A gives the oracle
        // term (e^{i phi} - 1) A / N of the next mean (float pairs)
        auto job = [&]() {
            if (upd)
                for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) rep[q] = sub_hilo(cmul_rn(rep[q], rot), kap);
            __syncwarp();
            const RepSums rs = replica_sums(rep, a.m, last);
            if ((threadIdx.x & 31) == 0) {
                if (!last) {
                    const PhaseFac f = fac_of(a, nxt);
                    s_fac = f;
                    const ph::cff A{mean_ff(rs.r, rs.sr, a.n), mean_ff(rs.i, rs.si, a.n)};
                    s_can = cff_pack(cff_mul(ph::cff_unpack(f.em1), A));
                } else if (rank == 0 && a.stats) {
                    const double P = sum_d(rs.p, rs.sp);
                    a.stats[0] = P;
                    a.stats[1] = -log(P);
                }
            }
        };
        // thread 0: mean of O(phi_{t+1}) c = S / N + (e^{i phi} - 1) A / N, and
        // the diffusion constant (1 - e^{i vphi}) times it
        auto post = [&](const u128 (&T)[2], const double (&S)[2]) {
            if (last) return;
            const ph::cff mu = cff_add(ph::cff{mean_ff(T[0], S[0], a.n), mean_ff(T[1], S[1], a.n)}, ph::cff_unpack(s_can));
            s_kap = cff_pack(cff_mul(ph::cff_unpack(s_fac.omv), mu));
            s_rot = s_fac.rot;
        };
        ok = cta_exchange<2>(v, sd, a, series2(a), t + 1, prev, a.stall && t == -1 && rank == 0, job, [] {}, post);
    }
    for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) g[j] = sl[j];
}

// ---- backward sweep ----------------------------------------------------------
__global__ void __launch_bounds__(kPgThreads, 1) k_phase_grid_bwd(PhaseGridArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float4 s_kp, s_kl;
    __shared__ float2 s_rot;
    __shared__ double s_is;
    __shared__ PhaseFac s_fac;
    __shared__ RepSums s_rs;
    // an exchange's totals, for the vphi gradient warp 2 computes during the
    // next exchange (rank 0); two slots by exchange parity, so that a post
    // never overwrites what a running aside reads
    __shared__ unsigned long long s_pend[2][4][2];
    __shared__ double s_pend_sd[2][4];
    __shared__ long long s_pend_t[2];
    __shared__ float2 repp[kPhaseMaxMarked], repl[kPhaseMaxMarked];
    __shared__ unsigned long long prev2[2][GxLayout<2>::W], prev4[2][GxLayout<4>::W];
    const unsigned rank = blockIdx.x;
    float4 *sp = reinterpret_cast<float4 *>(smem);
    float4 *sm = sp + a.slice_vecs;
    const uint64_t start = (uint64_t)rank * a.slice_vecs;
    const uint32_t nv = start >= a.nvec ? 0u
                        : (uint32_t)((a.nvec - start) < a.slice_vecs ? (a.nvec - start) : a.slice_vecs);
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + (size_t)a.slice_vecs * 32);
    const uint32_t nwords = (a.slice_vecs * 2 + 31) / 32;
    float4 *gp = static_cast<float4 *>(a.psi) + start;
    float4 *gl = static_cast<float4 *>(a.lam) + start;
    const float2 *g2 = static_cast<const float2 *>(a.psi);
    for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) sp[j] = gp[j];
    for (uint32_t q = threadIdx.x; q < a.m; q += kPgThreads) repp[q] = g2[a.list[q]];
    if (threadIdx.x < 2 * GxLayout<2>::W) prev2[threadIdx.x / GxLayout<2>::W][threadIdx.x % GxLayout<2>::W] = 0ull;
    if (threadIdx.x < 2 * GxLayout<4>::W) prev4[threadIdx.x / GxLayout<4>::W][threadIdx.x % GxLayout<4>::W] = 0ull;
    if (threadIdx.x < 2) s_pend_t[threadIdx.x] = -1;
    build_mask(fm, nwords, a, start * 2, nv * 2);
    const double N = ldexp(1.0, a.n), inv_n = ldexp(1.0, -a.n);
    // P from the replica (every CTA), lambda~_K = -(marked psi_K) / sqrt(P)
    if ((threadIdx.x >> 5) == 1) {
        const RepSums rs = replica_sums(repp, a.m, true);
        if ((threadIdx.x & 31) == 0) s_is = 1.0 / sqrt(sum_d(rs.p, rs.sp));
    }
    __syncthreads();
    const double is = s_is;
    for (uint32_t q = threadIdx.x; q < a.m; q += kPgThreads)
        repl[q] = make_float2((float)(-(double)repp[q].x * is), (float)(-(double)repp[q].y * is));
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) {
        const uint32_t f = mark2(fm, j);
        float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (f) {
            const float4 c = sp[j];
            if (f & 1u) {
                l.x = (float)(-(double)c.x * is);
                l.y = (float)(-(double)c.y * is);
            }
            if (f & 2u) {
                l.z = (float)(-(double)c.z * is);
                l.w = (float)(-(double)c.w * is);
            }
        }
        sm[j] = l;
    }
    // exchange 0: the sum of psi_K (the adjoint's sum is the replica's)
    bool ok;
    {
        u128 v[2] = {0, 0};
        double sd[2] = {0.0, 0.0};
        for (uint32_t j0 = threadIdx.x; j0 < nv; j0 += kU * kPgThreads) {
            float gr[2 * kU], gi[2 * kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t j = j0 + u * kPgThreads;
                if (j >= nv) {
                    gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                    continue;
                }
                const float4 c = sp[j];
                gr[2 * u] = c.x;
                gi[2 * u] = c.y;
                gr[2 * u + 1] = c.z;
                gi[2 * u + 1] = c.w;
            }
            fix_add<4>(v[0], sd[0], pairwise<2 * kU>(gr));
            fix_add<4>(v[1], sd[1], pairwise<2 * kU>(gi));
        }
        auto job = [&]() {
            const RepSums rs = replica_sums(repl, a.m, false);
            if ((threadIdx.x & 31) == 0) {
                s_rs = rs;
                if (a.K > 0) s_fac = fac_of(a, a.K - 1);
            }
        };
        auto post = [&](const u128 (&T)[2], const double (&S)[2]) {
            if (a.K == 0) return;
            if (rank == 0) {
                const double2 mp = make_double2(sum_d(T[0], S[0]) * inv_n, sum_d(T[1], S[1]) * inv_n);
                const double2 ml = make_double2(sum_d(s_rs.r, s_rs.sr) * inv_n, sum_d(s_rs.i, s_rs.si) * inv_n);
                a.grad_vphi[a.K - 1] = -2.0 * N * (ml.x * mp.y - ml.y * mp.x) * is;
            }
            // conjugates: e^{-i phi}, 1 - e^{-i vphi}
            const ph::cff w = ph::cff_conj(ph::cff_unpack(s_fac.omv));
            const ph::cff mp{mean_ff(T[0], S[0], a.n), mean_ff(T[1], S[1], a.n)};
            const ph::cff ml{mean_ff(s_rs.r, s_rs.sr, a.n), mean_ff(s_rs.i, s_rs.si, a.n)};
            s_kp = cff_pack(cff_mul(w, mp));
            s_kl = cff_pack(cff_mul(w, ml));
            s_rot = make_float2(s_fac.rot.x, -s_fac.rot.y);
        };
        ok = cta_exchange<2>(v, sd, a, series2(a), 0, prev2, a.stall && rank == 0, job, [] {}, post);
    }
    // ---- the K adjoint passes (exchanges 1..K of the second counter series) ----
    long long xi = 0;
    for (long long t = a.K - 1; t >= 0 && ok; --t, ++xi) {
        const float4 kp = s_kp, kl = s_kl;
        const float2 rot = s_rot;
        u128 v[4] = {0, 0, 0, 0};
        double sd[4] = {0.0, 0.0, 0.0, 0.0};
        for (uint32_t j0 = threadIdx.x; j0 < nv; j0 += kU * kPgThreads) {
            float pr[2 * kU], pi[2 * kU], lr[2 * kU], li[2 * kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t j = j0 + u * kPgThreads;
                if (j >= nv) {
                    pr[2 * u] = pr[2 * u + 1] = pi[2 * u] = pi[2 * u + 1] = 0.f;
                    lr[2 * u] = lr[2 * u + 1] = li[2 * u] = li[2 * u + 1] = 0.f;
                    continue;
                }
                const float4 c = sp[j], l = sm[j];
                const uint32_t f = mark2(fm, j);
                float2 c0 = sub_hilo(make_float2(c.x, c.y), kp), c1 = sub_hilo(make_float2(c.z, c.w), kp);
                float2 l0 = sub_hilo(make_float2(l.x, l.y), kl), l1 = sub_hilo(make_float2(l.z, l.w), kl);
                if (f & 1u) {
                    c0 = cmul_rn(c0, rot);
                    l0 = cmul_rn(l0, rot);
                }
                if (f & 2u) {
                    c1 = cmul_rn(c1, rot);
                    l1 = cmul_rn(l1, rot);
                }
                sp[j] = make_float4(c0.x, c0.y, c1.x, c1.y);
                sm[j] = make_float4(l0.x, l0.y, l1.x, l1.y);
                pr[2 * u] = c0.x;
                pi[2 * u] = c0.y;
                pr[2 * u + 1] = c1.x;
                pi[2 * u + 1] = c1.y;
                lr[2 * u] = l0.x;
                li[2 * u] = l0.y;
                lr[2 * u + 1] = l1.x;
                li[2 * u + 1] = l1.y;
            }
            fix_add<4>(v[0], sd[0], pairwise<2 * kU>(pr));
            fix_add<4>(v[1], sd[1], pairwise<2 * kU>(pi));
            fix_add<4>(v[2], sd[2], pairwise<2 * kU>(lr));
            fix_add<4>(v[3], sd[3], pairwise<2 * kU>(li));
        }
        // warp 1, while the exchange waits: replicas of psi and lambda~ on the
        // marked set, the phi gradient (rank 0) from its sum
        // sum_marked Im(conj(lambda~) psi), and the next pass's constants
        auto job = [&]() {
            u128 gs = 0;
            double gsd = 0.0;
            for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) {
                const float2 c = cmul_rn(sub_hilo(repp[q], kp), rot), l = cmul_rn(sub_hilo(repl[q], kl), rot);
                repp[q] = c;
                repl[q] = l;
                fix_add<4>(gs, gsd, (double)l.x * c.y - (double)l.y * c.x);
            }
            gs = warp_sum_u128(gs);
            if (__any_sync(0xffffffffu, has_side(gsd))) gsd = warp_sum_d(gsd);
            if ((threadIdx.x & 31) == 0) {
                // dL/dphi_t = -2 Im(sum_marked conj(lambda_t) psi_t)
                if (rank == 0) a.grad_phi[t] = -2.0 * sum_d(gs, gsd) * is;
                if (t > 0) s_fac = fac_of(a, t - 1);
            }
        };
        // warp 2 (rank 0): dL/dvphi_{s-1} = -2 N Im(conj(<lambda_s>) <psi_s>)
        // from the totals the previous exchange left
        const int ps = (int)((xi + 1) & 1);  // the slot the previous exchange's post filled
        auto aside = [&]() {
            if (rank != 0 || (threadIdx.x & 31) != 0 || s_pend_t[ps] < 0) return;
            u128 T[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) T[q] = ((u128)s_pend[ps][q][1] << 64) | s_pend[ps][q][0];
            const double *sdp = s_pend_sd[ps];
            const double2 mp = make_double2(sum_d(T[0], sdp[0]) * inv_n, sum_d(T[1], sdp[1]) * inv_n);
            const double2 ml = make_double2(sum_d(T[2], sdp[2]) * inv_n, sum_d(T[3], sdp[3]) * inv_n);
            a.grad_vphi[s_pend_t[ps]] = -2.0 * N * (ml.x * mp.y - ml.y * mp.x) * is;
        };
        auto post = [&](const u128 (&T)[4], const double (&S)[4]) {
            if (t == 0) return;
            const ph::cff w = ph::cff_conj(ph::cff_unpack(s_fac.omv));
            const ph::cff mp{mean_ff(T[0], S[0], a.n), mean_ff(T[1], S[1], a.n)};
            const ph::cff ml{mean_ff(T[2], S[2], a.n), mean_ff(T[3], S[3], a.n)};
            s_kp = cff_pack(cff_mul(w, mp));
            s_kl = cff_pack(cff_mul(w, ml));
            s_rot = make_float2(s_fac.rot.x, -s_fac.rot.y);
            if (rank == 0) {
                const int w = (int)(xi & 1);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    s_pend[w][q][0] = (unsigned long long)T[q];
                    s_pend[w][q][1] = (unsigned long long)(T[q] >> 64);
                    s_pend_sd[w][q] = S[q];
                }
                s_pend_t[w] = t - 1;
            }
        };
        ok = cta_exchange<4>(v, sd, a, series4(a), xi, prev4, false, job, aside, post);
    }
    // psi_0 (rewound) and lambda_0 = lambda~_0 / sqrt(P); after a wait that
    // ran out the results are undefined and lambda is left as it was
    for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) gp[j] = sp[j];
    if (ok) {
        for (uint32_t j = threadIdx.x; j < nv; j += kPgThreads) {
            const float4 l = sm[j];
            gl[j] = make_float4((float)(l.x * is), (float)(l.y * is), (float)(l.z * is), (float)(l.w * is));
        }
    }
}

template <class F> cudaError_t launch_coop(F kern, unsigned G, size_t smem, cudaStream_t st, const PhaseGridArgs &a) {
    cudaError_t e;
    if ((e = raise_smem_limit(kern, smem)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPgThreads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kPgThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all G CTAs co-resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

bool phase_grid_plan(int n, bool backward, int sm_count, unsigned *G, uint32_t *slice_vecs, size_t *smem) {
    const uint64_t nvec = (1ull << n) / 2;
    if (n < 2 || sm_count < 1 || sm_count > 512 || nvec < (uint64_t)sm_count) return false;
    const uint64_t L = (nvec + sm_count - 1) / sm_count;
    const size_t bytes = (size_t)L * 16 * (backward ? 2 : 1) + ((L * 2 + 31) / 32) * 4;
    if (bytes > kPhaseGridSmemMax) return false;
    *G = (unsigned)((nvec + L - 1) / L);
    *slice_vecs = (uint32_t)L;
    *smem = bytes;
    return true;
}

// Two exchange series: one of two sums (the forward sweep; the backward
// sweep's first exchange), one of four (the backward passes).
size_t phase_grid_region_bytes(unsigned G) {
    return GxLayout<2>::kAccBytes + GxLayout<2>::side_bytes(G) + GxLayout<4>::kAccBytes + GxLayout<4>::side_bytes(G);
}
size_t phase_grid_zero_bytes() { return phase_grid_region_bytes(512); }

cudaError_t launch_phase_table(const double *phi, const double *vphi, long long K, PhaseFac *table, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    k_phase_table<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(phi, vphi, K, table);
    return cudaGetLastError();
}

cudaError_t launch_phase_grid(const PhaseGridArgs &a, bool backward, unsigned G, size_t smem, cudaStream_t st) {
    if (backward) return launch_coop(k_phase_grid_bwd, G, smem, st, a);
    if (a.slice_vecs >= kPgWideVecs) return launch_coop(k_phase_grid_fwd<8>, G, smem, st, a);
    return launch_coop(k_phase_grid_fwd<4>, G, smem, st, a);
}

}  // namespace grv
