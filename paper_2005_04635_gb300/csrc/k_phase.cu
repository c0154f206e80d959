// k_phase.cu -- generalised phase Grover iterator and its adjoint (complex64).
//
// The paper's iterator G = D O (section "Proposed Simulation Method") with the
// oracle's sign and the inversion's factor 2 replaced by learnable phases:
//   O(phi):  c_x <- e^{i phi} c_x for marked x,
//   D(vphi): c_i <- c_i - kappa,  kappa = (1 - e^{i vphi}) <c>,
// so that D(pi) O(pi) = -G.  Both are unitary with O(phi)^-1 = O(-phi) and
// D(vphi)^-1 = D(-vphi), so the backward pass recomputes every intermediate
// state by applying the inverse iterators to the final state instead of
// storing K states.  With lambda = dL/d(conj psi) (Wirtinger derivative) and
// a step psi_out = U psi_in, lambda_in = U^H lambda_out and
//   dL/dvphi_t = 2 Re(i N conj(<lambda_{t+1}>) <psi_{t+1}>),
//   dL/dphi_t  = 2 Re(i sum_marked conj(lambda_t,x) psi_t,x),
// where <.> is the mean over all N amplitudes.  For L = -log sum_marked |c_x|^2,
// lambda_K = -(marked part of psi_K) / P.
//
// Forward pass t: c <- O(phi_t) c - kappa_t, store, and the exact sum of the new
// state; the last CTA adds (e^{i phi_{t+1}} - 1) sum_marked c_x (M gathered
// values) to obtain the mean of O(phi_{t+1}) c, and writes kappa_{t+1} and
// e^{i phi_{t+1}} for the next pass.  Backward pass t: psi and lambda both go
// through D(-vphi_t) then O(-phi_t) with exact sums of both; the last CTA forms
// the gradients and the next pass's constants.  Sums: FP32 pairwise groups of 8
// amplitudes added as 128-bit fixed point (fixed_sum.cuh).
#include "fixed_sum.cuh"
#include "grover_internal.cuh"
#include "phase_ops.cuh"

namespace grv {
namespace {

constexpr int kPhThreads = 256;
constexpr int kPhUnroll = 4;

// Cursor into the sorted marked list: a thread visits its vectors in
// increasing order, so the cursor only moves forward (by binary search when it
// has fallen behind); `nxt` caches the next marked index.
struct ListCur {
    const uint64_t *list;
    uint32_t m, p;
    uint64_t nxt;
    __device__ __forceinline__ uint64_t at(uint32_t i) const { return i < m ? __ldg(list + i) : ~0ull; }
    __device__ __forceinline__ uint32_t lower_bound(uint32_t lo, uint64_t x) const {
        uint32_t hi = m;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(list + mid) < x) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    }
    __device__ __forceinline__ void init(const uint64_t *l, uint32_t mm, uint64_t first) {
        list = l;
        m = mm;
        p = lower_bound(0, first);
        nxt = at(p);
    }
    // bit j set <=> amplitude a0 + j is marked (j = 0, 1)
    __device__ __forceinline__ uint32_t bits2(uint64_t a0) {
        uint32_t f = 0;
        if (nxt < a0 + 2) {
            if (nxt < a0) {
                p = lower_bound(p + 1, a0);
                nxt = at(p);
            }
            while (nxt < a0 + 2) {
                f |= 1u << (uint32_t)(nxt - a0);
                nxt = at(++p);
            }
        }
        return f;
    }
};

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <bool STREAM> __device__ __forceinline__ float4 ldv(const float4 *p) {
    if (STREAM) return __ldcs(p);
    return *p;
}
template <bool STREAM> __device__ __forceinline__ void stv(float4 *p, float4 v) {
    if (STREAM) __stcs(p, v);
    else *p = v;
}

using ph::cmul;
using ph::dcmul;
using ph::expi;
using ph::pairwise;
using ph::split_hilo;
using ph::sub_hilo;
using ph::warp_sum_d;

// Grid sums of NS complex fixed-point accumulators, in two steps.
// grid_arrive: every CTA reduces its accumulators (integers exactly, FP64
// side sums in a fixed order) and writes 3 double2 slots per sum to
// partials; returns true (in every thread) in the CTA that arrives last.
template <int NS>
__device__ bool grid_arrive(u128 (&r)[NS], u128 (&i)[NS], double (&sr)[NS], double (&si)[NS], double2 *partials,
                            unsigned *ticket) {
    __shared__ unsigned long long wi[kPhThreads / 32][NS][4];
    __shared__ double wsd[kPhThreads / 32][NS][2];
    __shared__ unsigned s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __threadfence();  // this thread's amplitude stores before the ticket (the last CTA reads marked ones)
    int any = 0;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        r[q] = warp_sum_u128(r[q]);
        i[q] = warp_sum_u128(i[q]);
        any |= (sr[q] != 0.0 || si[q] != 0.0);
    }
    any = __syncthreads_or(any);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        if (any) {
            sr[q] = warp_sum_d(sr[q]);
            si[q] = warp_sum_d(si[q]);
        }
        if (lane == 0) {
            wi[warp][q][0] = (unsigned long long)r[q];
            wi[warp][q][1] = (unsigned long long)(r[q] >> 64);
            wi[warp][q][2] = (unsigned long long)i[q];
            wi[warp][q][3] = (unsigned long long)(i[q] >> 64);
            wsd[warp][q][0] = sr[q];
            wsd[warp][q][1] = si[q];
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            u128 br = 0, bi = 0;
            double xr = 0.0, xi = 0.0;
            if (lane < kPhThreads / 32) {
                br = ((u128)wi[lane][q][1] << 64) | wi[lane][q][0];
                bi = ((u128)wi[lane][q][3] << 64) | wi[lane][q][2];
                xr = wsd[lane][q][0];
                xi = wsd[lane][q][1];
            }
            br = warp_sum_u128(br);
            bi = warp_sum_u128(bi);
            if (any) {
                xr = warp_sum_d(xr);
                xi = warp_sum_d(xi);
            }
            if (lane == 0) {
                double2 *p = partials + (size_t)(3 * NS) * blockIdx.x + 3 * q;
                p[0] = make_double2(__longlong_as_double((long long)(unsigned long long)br),
                                    __longlong_as_double((long long)(unsigned long long)(br >> 64)));
                p[1] = make_double2(__longlong_as_double((long long)(unsigned long long)bi),
                                    __longlong_as_double((long long)(unsigned long long)(bi >> 64)));
                p[2] = make_double2(xr, xi);
            }
        }
        if (lane == 0) {
            __threadfence();
            s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
        }
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    return true;
}

// grid_total (last CTA, all threads): the totals of the NS sums -- the 192-bit
// integer sums rounded once to FP64 plus the side sums -- valid in warp 0.
// Resets the ticket.
template <int NS>
__device__ void grid_total(const double2 *partials, unsigned *ticket, double2 (&tot)[NS]) {
    __shared__ unsigned long long w3[kPhThreads / 32][NS][6];
    __shared__ double wsd[kPhThreads / 32][NS][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    I192 tr[NS], ti[NS];
    double ssr[NS], ssi[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        tr[q] = ti[q] = I192{0, 0, 0};
        ssr[q] = ssi[q] = 0.0;
    }
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kPhThreads) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const double2 *p = partials + (size_t)(3 * NS) * j + 3 * q;
            const double2 q0 = __ldcg(p), q1 = __ldcg(p + 1), q2 = __ldcg(p + 2);
            i192_add(tr[q], i192_from(((u128)(unsigned long long)__double_as_longlong(q0.y) << 64) |
                                      (unsigned long long)__double_as_longlong(q0.x)));
            i192_add(ti[q], i192_from(((u128)(unsigned long long)__double_as_longlong(q1.y) << 64) |
                                      (unsigned long long)__double_as_longlong(q1.x)));
            ssr[q] += q2.x;
            ssi[q] += q2.y;
        }
    }
    int anys = 0;
#pragma unroll
    for (int q = 0; q < NS; ++q) anys |= (ssr[q] != 0.0 || ssi[q] != 0.0);
    anys = __syncthreads_or(anys);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        tr[q] = warp_sum_i192(tr[q]);
        ti[q] = warp_sum_i192(ti[q]);
        if (anys) {
            ssr[q] = warp_sum_d(ssr[q]);
            ssi[q] = warp_sum_d(ssi[q]);
        }
        if (lane == 0) {
            w3[warp][q][0] = tr[q].w0;
            w3[warp][q][1] = tr[q].w1;
            w3[warp][q][2] = tr[q].w2;
            w3[warp][q][3] = ti[q].w0;
            w3[warp][q][4] = ti[q].w1;
            w3[warp][q][5] = ti[q].w2;
            wsd[warp][q][0] = ssr[q];
            wsd[warp][q][1] = ssi[q];
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            I192 xr{0, 0, 0}, xi{0, 0, 0};
            double yr = 0.0, yi = 0.0;
            if (lane < kPhThreads / 32) {
                xr = I192{w3[lane][q][0], w3[lane][q][1], w3[lane][q][2]};
                xi = I192{w3[lane][q][3], w3[lane][q][4], w3[lane][q][5]};
                yr = wsd[lane][q][0];
                yi = wsd[lane][q][1];
            }
            xr = warp_sum_i192(xr);
            xi = warp_sum_i192(xi);
            if (anys) {
                yr = warp_sum_d(yr);
                yi = warp_sum_d(yi);
            }
            tot[q] = make_double2(i192_to_double(xr) * 0x1p-100 + yr, i192_to_double(xi) * 0x1p-100 + yi);
        }
        if (lane == 0) *ticket = 0u;
    }
}

// Side work of a last CTA, done by warps 1 and 2 while the others start the
// grid total: e^{i a} for two angles (lanes 0, 1 of warp 1).
__device__ __forceinline__ void side_expi(double a0, double a1, double2 *out) {
    if ((threadIdx.x >> 5) == 1 && (threadIdx.x & 31) < 2) out[threadIdx.x & 1] = expi((threadIdx.x & 1) ? a1 : a0);
}

// ---- forward pass ----------------------------------------------------------
template <bool UPDATE, bool STREAM>
__global__ void __launch_bounds__(kPhThreads) k_phase_fwd(PhaseArgs a) {
    float4 *psi = reinterpret_cast<float4 *>(a.psi);
    const uint64_t tile = (uint64_t)kPhThreads * kPhUnroll;
    ListCur cur;
    if (UPDATE) cur.init(a.list, a.m, 2 * ((uint64_t)blockIdx.x * tile + threadIdx.x));
    griddep_wait();  // the previous pass: its stores and constants are visible
    griddep_launch_dependents();
    float4 kap = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 rot = make_float2(1.f, 0.f);
    if (UPDATE) {
        kap = a.cin->kpsi;
        rot = a.cin->rot;
    }
    u128 r[1] = {0}, i[1] = {0};
    double sr[1] = {0.0}, si[1] = {0.0};
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < a.nvec; base += (uint64_t)gridDim.x * tile) {
        float4 v[kPhUnroll];
        uint32_t f[kPhUnroll];
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            if (j < a.nvec) v[u] = ldv<STREAM>(psi + j);
        }
        if (UPDATE) {
#pragma unroll
            for (int u = 0; u < kPhUnroll; ++u) {
                const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
                f[u] = j < a.nvec ? cur.bits2(2 * j) : 0u;
            }
        }
        float gr[2 * kPhUnroll], gi[2 * kPhUnroll];
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            if (j >= a.nvec) {
                gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                continue;
            }
            float2 c0 = make_float2(v[u].x, v[u].y), c1 = make_float2(v[u].z, v[u].w);
            if (UPDATE) {
                if (f[u] & 1u) c0 = cmul(c0, rot);
                if (f[u] & 2u) c1 = cmul(c1, rot);
                c0 = sub_hilo(c0, kap);
                c1 = sub_hilo(c1, kap);
                stv<STREAM>(psi + j, make_float4(c0.x, c0.y, c1.x, c1.y));
            }
            gr[2 * u] = c0.x;
            gi[2 * u] = c0.y;
            gr[2 * u + 1] = c1.x;
            gi[2 * u + 1] = c1.y;
        }
        fix_add<4>(r[0], sr[0], pairwise<2 * kPhUnroll>(gr));
        fix_add<4>(i[0], si[0], pairwise<2 * kPhUnroll>(gi));
    }
    if (!grid_arrive<1>(r, i, sr, si, a.partials, a.ticket)) return;
    // last CTA: the constants of the next pass
    __shared__ double2 s_e[2];
    __shared__ double s_g[3];  // sum over marked of Re c, Im c, |c|^2
    const long long nxt = UPDATE ? a.t + 1 : 0;
    if (nxt < a.K) side_expi(a.phi[nxt], a.vphi[nxt], s_e);
    if ((threadIdx.x >> 5) == 2) {
        const float2 *pc = reinterpret_cast<const float2 *>(a.psi);
        double gr = 0.0, gi = 0.0, gp = 0.0;
        for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) {
            const float2 v = __ldcg(pc + a.list[q]);
            gr += (double)v.x;
            gi += (double)v.y;
            gp += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        gr = warp_sum_d(gr);
        gi = warp_sum_d(gi);
        gp = warp_sum_d(gp);
        if ((threadIdx.x & 31) == 0) {
            s_g[0] = gr;
            s_g[1] = gi;
            s_g[2] = gp;
        }
    }
    double2 tot[1];
    grid_total<1>(a.partials, a.ticket, tot);
    if (threadIdx.x != 0) return;
    const double inv_n = ldexp(1.0, -a.n);
    PhaseConst out = {};
    if (nxt < a.K) {
        // mean of O(phi_{t+1}) c: the sum plus (e^{i phi} - 1) sum over marked of c
        const double2 e = s_e[0], ev = s_e[1];
        const double cr = (e.x - 1.0) * s_g[0] - e.y * s_g[1];
        const double ci = (e.x - 1.0) * s_g[1] + e.y * s_g[0];
        const double2 mu = make_double2((tot[0].x + cr) * inv_n, (tot[0].y + ci) * inv_n);
        out.kpsi = split_hilo(dcmul(make_double2(1.0 - ev.x, -ev.y), mu));
        out.rot = make_float2((float)e.x, (float)e.y);
        out.mean_psi = mu;
    } else {
        out.mean_psi = make_double2(tot[0].x * inv_n, tot[0].y * inv_n);
        out.p_success = s_g[2];
        if (a.stats) {
            a.stats[0] = s_g[2];
            a.stats[1] = -log(s_g[2]);
        }
    }
    *a.cout = out;
}

// ---- backward pass ---------------------------------------------------------
template <bool STREAM>
__global__ void __launch_bounds__(kPhThreads) k_phase_bwd(PhaseArgs a) {
    float4 *psi = reinterpret_cast<float4 *>(a.psi);
    float4 *lam = reinterpret_cast<float4 *>(a.lam);
    const uint64_t tile = (uint64_t)kPhThreads * kPhUnroll;
    ListCur cur;
    cur.init(a.list, a.m, 2 * ((uint64_t)blockIdx.x * tile + threadIdx.x));
    griddep_wait();
    griddep_launch_dependents();
    const float4 kp = a.cin->kpsi, kl = a.cin->klam;
    const float2 rot = a.cin->rot;  // e^{-i phi_t}
    u128 r[2] = {0, 0}, i[2] = {0, 0};
    double sr[2] = {0.0, 0.0}, si[2] = {0.0, 0.0};
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < a.nvec; base += (uint64_t)gridDim.x * tile) {
        float4 vp[kPhUnroll], vl[kPhUnroll];
        uint32_t f[kPhUnroll];
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            if (j < a.nvec) {
                vp[u] = ldv<STREAM>(psi + j);
                vl[u] = ldv<STREAM>(lam + j);
            }
        }
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            f[u] = j < a.nvec ? cur.bits2(2 * j) : 0u;
        }
        float pr[2 * kPhUnroll], pi[2 * kPhUnroll], lr[2 * kPhUnroll], li[2 * kPhUnroll];
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            if (j >= a.nvec) {
                pr[2 * u] = pr[2 * u + 1] = pi[2 * u] = pi[2 * u + 1] = 0.f;
                lr[2 * u] = lr[2 * u + 1] = li[2 * u] = li[2 * u + 1] = 0.f;
                continue;
            }
            float2 c0 = sub_hilo(make_float2(vp[u].x, vp[u].y), kp), c1 = sub_hilo(make_float2(vp[u].z, vp[u].w), kp);
            float2 l0 = sub_hilo(make_float2(vl[u].x, vl[u].y), kl), l1 = sub_hilo(make_float2(vl[u].z, vl[u].w), kl);
            if (f[u] & 1u) {
                c0 = cmul(c0, rot);
                l0 = cmul(l0, rot);
            }
            if (f[u] & 2u) {
                c1 = cmul(c1, rot);
                l1 = cmul(l1, rot);
            }
            stv<STREAM>(psi + j, make_float4(c0.x, c0.y, c1.x, c1.y));
            stv<STREAM>(lam + j, make_float4(l0.x, l0.y, l1.x, l1.y));
            pr[2 * u] = c0.x;
            pi[2 * u] = c0.y;
            pr[2 * u + 1] = c1.x;
            pi[2 * u + 1] = c1.y;
            lr[2 * u] = l0.x;
            li[2 * u] = l0.y;
            lr[2 * u + 1] = l1.x;
            li[2 * u + 1] = l1.y;
        }
        fix_add<4>(r[0], sr[0], pairwise<2 * kPhUnroll>(pr));
        fix_add<4>(i[0], si[0], pairwise<2 * kPhUnroll>(pi));
        fix_add<4>(r[1], sr[1], pairwise<2 * kPhUnroll>(lr));
        fix_add<4>(i[1], si[1], pairwise<2 * kPhUnroll>(li));
    }
    if (!grid_arrive<2>(r, i, sr, si, a.partials, a.ticket)) return;
    __shared__ double2 s_e[2];
    __shared__ double s_g;  // sum over marked of Im(conj(lambda_x) psi_x)
    if (a.t > 0) side_expi(-a.phi[a.t - 1], -a.vphi[a.t - 1], s_e);
    if ((threadIdx.x >> 5) == 2) {
        const float2 *pc = reinterpret_cast<const float2 *>(a.psi);
        const float2 *lc = reinterpret_cast<const float2 *>(a.lam);
        double g = 0.0;
        for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) {
            const uint64_t x = a.list[q];
            const float2 p = __ldcg(pc + x), l = __ldcg(lc + x);
            g += (double)l.x * (double)p.y - (double)l.y * (double)p.x;
        }
        g = warp_sum_d(g);
        if ((threadIdx.x & 31) == 0) s_g = g;
    }
    double2 tot[2];
    grid_total<2>(a.partials, a.ticket, tot);
    if (threadIdx.x != 0) return;
    const double N = ldexp(1.0, a.n), inv_n = ldexp(1.0, -a.n);
    const double2 mp = make_double2(tot[0].x * inv_n, tot[0].y * inv_n);
    const double2 ml = make_double2(tot[1].x * inv_n, tot[1].y * inv_n);
    // dL/dphi_t = 2 Re(i sum_marked conj(lambda_t,x) psi_t,x) = -2 Im(sum conj(l) p)
    a.grad_phi[a.t] = -2.0 * s_g;
    PhaseConst out = {};
    out.mean_psi = mp;
    out.mean_lam = ml;
    if (a.t > 0) {
        // dL/dvphi_{t-1} = 2 Re(i N conj(<lambda_t>) <psi_t>) = -2 N Im(conj(ml) mp)
        a.grad_vphi[a.t - 1] = -2.0 * N * (ml.x * mp.y - ml.y * mp.x);
        const double2 ev = s_e[1];
        const double2 one_m = make_double2(1.0 - ev.x, -ev.y);
        out.kpsi = split_hilo(dcmul(one_m, mp));
        out.klam = split_hilo(dcmul(one_m, ml));
        out.rot = make_float2((float)s_e[0].x, (float)s_e[0].y);
    }
    *a.cout = out;
}

// Start of the backward sweep: lambda <- 0 everywhere and the exact sum of
// psi_K; the last CTA sets lambda_K = -(marked part of psi_K) / P, forms
// dL/dvphi_{K-1} and the constants of backward pass K-1.
template <bool STREAM>
__global__ void __launch_bounds__(kPhThreads) k_phase_bwd_start(PhaseArgs a) {
    const float4 *psi = reinterpret_cast<const float4 *>(a.psi);
    float4 *lam = reinterpret_cast<float4 *>(a.lam);
    const uint64_t tile = (uint64_t)kPhThreads * kPhUnroll;
    griddep_wait();
    griddep_launch_dependents();
    u128 r[1] = {0}, i[1] = {0};
    double sr[1] = {0.0}, si[1] = {0.0};
    for (uint64_t base = (uint64_t)blockIdx.x * tile; base < a.nvec; base += (uint64_t)gridDim.x * tile) {
        float gr[2 * kPhUnroll], gi[2 * kPhUnroll];
#pragma unroll
        for (int u = 0; u < kPhUnroll; ++u) {
            const uint64_t j = base + (uint64_t)u * kPhThreads + threadIdx.x;
            if (j >= a.nvec) {
                gr[2 * u] = gr[2 * u + 1] = gi[2 * u] = gi[2 * u + 1] = 0.f;
                continue;
            }
            const float4 c = ldv<STREAM>(psi + j);
            stv<STREAM>(lam + j, make_float4(0.f, 0.f, 0.f, 0.f));
            gr[2 * u] = c.x;
            gi[2 * u] = c.y;
            gr[2 * u + 1] = c.z;
            gi[2 * u + 1] = c.w;
        }
        fix_add<4>(r[0], sr[0], pairwise<2 * kPhUnroll>(gr));
        fix_add<4>(i[0], si[0], pairwise<2 * kPhUnroll>(gi));
    }
    if (!grid_arrive<1>(r, i, sr, si, a.partials, a.ticket)) return;
    __shared__ double2 s_e[2];
    __shared__ double s_g[3];  // P and the sum over marked of lambda_K
    if (a.K > 0) side_expi(-a.phi[a.K - 1], -a.vphi[a.K - 1], s_e);
    if ((threadIdx.x >> 5) == 2) {
        const float2 *pc = reinterpret_cast<const float2 *>(a.psi);
        float2 *lc = reinterpret_cast<float2 *>(a.lam);
        double p = 0.0;
        for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) {
            const float2 v = __ldcg(pc + a.list[q]);
            p += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        p = warp_sum_d(p);
        double slr = 0.0, sli = 0.0;
        for (uint32_t q = threadIdx.x & 31; q < a.m; q += 32) {
            const uint64_t x = a.list[q];
            const float2 v = __ldcg(pc + x);
            const float2 l = make_float2((float)(-(double)v.x / p), (float)(-(double)v.y / p));
            lc[x] = l;
            slr += (double)l.x;
            sli += (double)l.y;
        }
        slr = warp_sum_d(slr);
        sli = warp_sum_d(sli);
        if ((threadIdx.x & 31) == 0) {
            s_g[0] = p;
            s_g[1] = slr;
            s_g[2] = sli;
        }
    }
    double2 tot[1];
    grid_total<1>(a.partials, a.ticket, tot);
    if (threadIdx.x != 0) return;
    const double N = ldexp(1.0, a.n), inv_n = ldexp(1.0, -a.n);
    const double2 mp = make_double2(tot[0].x * inv_n, tot[0].y * inv_n);
    const double2 ml = make_double2(s_g[1] * inv_n, s_g[2] * inv_n);
    PhaseConst out = {};
    out.mean_psi = mp;
    out.mean_lam = ml;
    out.p_success = s_g[0];
    if (a.K > 0) {
        a.grad_vphi[a.K - 1] = -2.0 * N * (ml.x * mp.y - ml.y * mp.x);
        const double2 one_m = make_double2(1.0 - s_e[1].x, -s_e[1].y);
        out.kpsi = split_hilo(dcmul(one_m, mp));
        out.klam = split_hilo(dcmul(one_m, ml));
        out.rot = make_float2((float)s_e[0].x, (float)s_e[0].y);
    }
    *a.cout = out;
}

// CTAs of a streaming launch: resident CTAs only, at most one per tile.
unsigned phase_grid(int per_sm, uint64_t nvec, int sm_count) {
    const uint64_t tile = (uint64_t)kPhThreads * kPhUnroll;
    const uint64_t need = (nvec + tile - 1) / tile;
    uint64_t cap = (uint64_t)(per_sm < 1 ? 1 : per_sm) * (uint64_t)sm_count;
    if (cap > (uint64_t)kPhaseMaxGrid) cap = kPhaseMaxGrid;
    const uint64_t g = need < cap ? need : cap;
    return (unsigned)(g ? g : 1);
}

template <class F> int occupancy(F kern) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPhThreads, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

// Launch with programmatic stream serialisation: the kernel's CTAs may be
// scheduled while the previous kernel drains; every kernel here executes
// griddepcontrol.wait before it touches memory the previous one wrote.
cudaError_t launch_pdl(void (*kern)(PhaseArgs), unsigned grid, cudaStream_t st, const PhaseArgs &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPhThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

// The resident CTAs per SM are queried at every launch (for the current
// device), not cached in the process.
cudaError_t launch_phase_fwd(const PhaseArgs &a, bool update, bool stream, cudaStream_t st, int sm_count) {
    void (*kern[4])(PhaseArgs) = {k_phase_fwd<false, false>, k_phase_fwd<false, true>, k_phase_fwd<true, false>,
                                  k_phase_fwd<true, true>};
    const int w = (update ? 2 : 0) + (stream ? 1 : 0);
    return launch_pdl(kern[w], phase_grid(occupancy(kern[w]), a.nvec, sm_count), st, a);
}

cudaError_t launch_phase_bwd(const PhaseArgs &a, bool stream, cudaStream_t st, int sm_count) {
    void (*kern[2])(PhaseArgs) = {k_phase_bwd<false>, k_phase_bwd<true>};
    return launch_pdl(kern[stream], phase_grid(occupancy(kern[stream]), a.nvec, sm_count), st, a);
}

cudaError_t launch_phase_bwd_start(const PhaseArgs &a, bool stream, cudaStream_t st, int sm_count) {
    void (*kern[2])(PhaseArgs) = {k_phase_bwd_start<false>, k_phase_bwd_start<true>};
    return launch_pdl(kern[stream], phase_grid(occupancy(kern[stream]), a.nvec, sm_count), st, a);
}

}  // namespace grv
