// k_circuit.cu -- the conventional circuit gate by gate (section "Background").
//
// A gate-level state-vector simulator applies every gate of the circuit as
// its own pass over the state: the paper's cost model O([f_o(n) + f_c(n) + 2n]
// N^{3/2}).  Here:
//   * X and H on one qubit q (Algorithm "1-qubit Unitary Operation" with
//     U = X or H): pairs (x, x + 2^q) with bit q of x clear, each pair read
//     and written once (16-byte vectors, streaming);
//   * the multi-controlled Z of Fig. oracle1 (the register side of the
//     multi-controlled NOT onto an ancilla in (|0> - |1>)/sqrt(2)): with all n
//     qubits as controls its subspace is the single amplitude |1...1>, which a
//     controlled-gate kernel restricted to that subspace touches alone.
// The global factor -1 of 2|0><0| - I = -X^n MCZ X^n is folded into the scale
// of the next Hadamard pass.
#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kCircThreads = 256;
// pairs per thread per loop step: 8 (16 vectors in flight per thread) measured
// 6.42 TB/s per pass at n = 28 complex64 against 6.07 with 2
constexpr int kCircUnroll = 8;

template <bool STREAM, class V> __device__ __forceinline__ V ld(const V *p) {
    if (STREAM) return __ldcs(p);
    return *p;
}
template <bool STREAM, class V> __device__ __forceinline__ void st(V *p, V v) {
    if (STREAM) __stcs(p, v);
    else *p = v;
}

// (a, b) -> (b, a) for X, ((a + b) s, (a - b) s) for H with scale s
template <int OP, class T> __device__ __forceinline__ void pair_op(T &ar, T &ai, T &br, T &bi, T s) {
    if (OP == 0) {
        const T tr = ar, ti = ai;
        ar = br;
        ai = bi;
        br = tr;
        bi = ti;
    } else {
        const T sr = (ar + br) * s, si = (ai + bi) * s;
        const T dr = (ar - br) * s, di = (ai - bi) * s;
        ar = sr;
        ai = si;
        br = dr;
        bi = di;
    }
}

// complex64, qubit 0: both amplitudes of a pair share one float4
template <int OP, bool STREAM>
__global__ void __launch_bounds__(kCircThreads) k_gate1_c64_q0(float4 *v, uint64_t nvec, float s) {
    const uint64_t stride = (uint64_t)gridDim.x * kCircThreads * kCircUnroll;
    for (uint64_t j0 = (uint64_t)blockIdx.x * kCircThreads * kCircUnroll + threadIdx.x; j0 < nvec; j0 += stride) {
        float4 c[kCircUnroll];
#pragma unroll
        for (int u = 0; u < kCircUnroll; ++u) {
            const uint64_t j = j0 + (uint64_t)u * kCircThreads;
            if (j < nvec) c[u] = ld<STREAM>(v + j);
        }
#pragma unroll
        for (int u = 0; u < kCircUnroll; ++u) {
            const uint64_t j = j0 + (uint64_t)u * kCircThreads;
            if (j >= nvec) continue;
            pair_op<OP>(c[u].x, c[u].y, c[u].z, c[u].w, s);
            st<STREAM>(v + j, c[u]);
        }
    }
}

// pairs of 16-byte vectors (j, j + h) with bit log2(h) of j clear: complex64
// with q >= 1 (h = 2^(q-1) vectors of two amplitudes), complex128 with any q
// (h = 2^q vectors of one amplitude)
template <int OP, bool STREAM, class V, class T>
__global__ void __launch_bounds__(kCircThreads) k_gate1_pairs(V *v, uint64_t npairs, int hb, T s) {
    const uint64_t h = 1ull << hb, lowmask = h - 1;
    const uint64_t stride = (uint64_t)gridDim.x * kCircThreads * kCircUnroll;
    for (uint64_t t0 = (uint64_t)blockIdx.x * kCircThreads * kCircUnroll + threadIdx.x; t0 < npairs; t0 += stride) {
        V a[kCircUnroll], b[kCircUnroll];
        uint64_t j[kCircUnroll];
#pragma unroll
        for (int u = 0; u < kCircUnroll; ++u) {
            const uint64_t t = t0 + (uint64_t)u * kCircThreads;
            j[u] = ((t >> hb) << (hb + 1)) | (t & lowmask);
            if (t < npairs) {
                a[u] = ld<STREAM>(v + j[u]);
                b[u] = ld<STREAM>(v + j[u] + h);
            }
        }
#pragma unroll
        for (int u = 0; u < kCircUnroll; ++u) {
            const uint64_t t = t0 + (uint64_t)u * kCircThreads;
            if (t >= npairs) continue;
            if constexpr (sizeof(V) == 16 && sizeof(T) == 4) {  // float4: two amplitudes each
                pair_op<OP>(a[u].x, a[u].y, b[u].x, b[u].y, s);
                pair_op<OP>(a[u].z, a[u].w, b[u].z, b[u].w, s);
            } else {
                pair_op<OP>(a[u].x, a[u].y, b[u].x, b[u].y, s);
            }
            st<STREAM>(v + j[u], a[u]);
            st<STREAM>(v + j[u] + h, b[u]);
        }
    }
}

// multi-controlled Z on all n qubits: the amplitude |1...1> only
template <class T> __global__ void k_mcz_all(T *amps, uint64_t N) {
    amps[2 * (N - 1)] = -amps[2 * (N - 1)];
    amps[2 * (N - 1) + 1] = -amps[2 * (N - 1) + 1];
}

template <class K> unsigned grid_for(K kern, uint64_t items, uint64_t per_cta, const Geometry &g) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCircThreads, 0) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const uint64_t need = (items + per_cta - 1) / per_cta;
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)g.sm_count;
    const uint64_t gr = need < cap ? need : cap;
    return (unsigned)(gr ? gr : 1);
}

template <int OP, bool STREAM>
cudaError_t gate1_t(void *amps, int n, grover_dtype dt, int q, double scale, cudaStream_t st, const Geometry &g) {
    const uint64_t N = 1ull << n;
    if (dt == GROVER_C64) {
        float4 *v = static_cast<float4 *>(amps);
        const uint64_t nvec = N / 2;
        if (q == 0) {
            auto kern = k_gate1_c64_q0<OP, STREAM>;
            kern<<<grid_for(kern, nvec, (uint64_t)kCircThreads * kCircUnroll, g), kCircThreads, 0, st>>>(
                v, nvec, (float)scale);
        } else {
            auto kern = k_gate1_pairs<OP, STREAM, float4, float>;
            const uint64_t np = nvec / 2;
            kern<<<grid_for(kern, np, (uint64_t)kCircThreads * kCircUnroll, g), kCircThreads, 0, st>>>(
                v, np, q - 1, (float)scale);
        }
    } else {
        double2 *v = static_cast<double2 *>(amps);
        auto kern = k_gate1_pairs<OP, STREAM, double2, double>;
        const uint64_t np = N / 2;
        kern<<<grid_for(kern, np, (uint64_t)kCircThreads * kCircUnroll, g), kCircThreads, 0, st>>>(v, np, q, scale);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gate1(void *amps, int n, grover_dtype dt, int op, int q, double scale, cudaStream_t st,
                         const Geometry &g) {
    const bool stream = (long long)((1ull << n) * (dt == GROVER_C64 ? 8 : 16)) > g.l2_bytes / 2;
    if (op == 0) return stream ? gate1_t<0, true>(amps, n, dt, q, scale, st, g) : gate1_t<0, false>(amps, n, dt, q, scale, st, g);
    return stream ? gate1_t<1, true>(amps, n, dt, q, scale, st, g) : gate1_t<1, false>(amps, n, dt, q, scale, st, g);
}

cudaError_t launch_mcz_all(void *amps, int n, grover_dtype dt, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    if (dt == GROVER_C64) k_mcz_all<float><<<1, 1, 0, st>>>(static_cast<float *>(amps), N);
    else k_mcz_all<double><<<1, 1, 0, st>>>(static_cast<double *>(amps), N);
    return cudaGetLastError();
}

}  // namespace grv
