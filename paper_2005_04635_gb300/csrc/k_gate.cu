// k_gate.cu -- the conventional Grover circuit on CUDA cores (section
// "Background", conventional grover_search): per iteration the oracle O,
// H^{(x)n}, the conditional phase shift 2|0><0| - I and H^{(x)n} again.
//
// H^{(x)n} is applied as a product of Walsh-Hadamard transforms on groups of
// up to 8 index bits (the groups commute).  H = 2^(-n/2) W with W the +-1
// Walsh-Hadamard matrix, so the iterator H(2|0><0|-I)H = 2^-n W(2|0><0|-I)W:
// the passes of the first transform scale by 2^-kb (exact), those of the
// second do not.  A pass over the group of bits [lo, lo+kb) reads and writes
// the state once:
//   * a tile is 16 "columns" x 2^kb "mids": for lo >= 4, 16 consecutive
//     amplitudes (the bits below lo) at each of the 2^kb mid values; for
//     lo = 0, 16 consecutive blocks of 2^kb contiguous amplitudes;
//   * phase 1: each thread loads 2^a mids of one column (stride 2^b mids) and
//     runs the butterflies of the top a bits in registers, the tile goes to
//     shared memory; phase 2: each thread takes 2^b consecutive mids of one
//     column and runs the butterflies of the low b bits (a + b = kb,
//     b = min(kb, 4)); the tile is stored from shared memory with the
//     coalesced mapping of phase 1;
//   * the last pass of the first transform also applies 2|0><0| - I (every
//     amplitude but index 0 negated);
//   * each thread loads its phase-1 values of the CTA's next tile into
//     registers before the current tile's shared-memory phase and store, so
//     the loads of one tile overlap the rest of the previous one (at n = 28
//     to 33: 5.3-5.7 TB/s per pass, against 4.2-4.5 without).
// Butterflies are (x, y) -> (x + y, x - y) on real and imaginary parts.
#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kGateThreads = 256;
constexpr int kPad = 1;  // complex elements of padding per shared-memory row

template <class T> struct C2 {
    T re, im;
};

template <int LOG, class T> __device__ __forceinline__ void wht_regs(C2<T> *v) {
#pragma unroll
    for (int s = 0; s < LOG; ++s) {
        const int h = 1 << s;
#pragma unroll
        for (int i = 0; i < (1 << LOG); ++i) {
            if (i & h) continue;
            const C2<T> x = v[i], y = v[i + h];
            v[i] = C2<T>{x.re + y.re, x.im + y.im};
            v[i + h] = C2<T>{x.re - y.re, x.im - y.im};
        }
    }
}

// LOW: the group starts at bit 0 (columns are consecutive blocks of 2^KB);
// otherwise lo >= 4 (columns are COLS consecutive amplitudes).  WIDE (6-bit
// groups above bit 0, lo >= 5): 32 columns and 3 + 3 bits per phase, so every
// thread keeps eight loads in flight as in the 7-bit passes instead of four.
template <class T, int KB, bool LOW, bool WIDE>
__global__ void __launch_bounds__(kGateThreads)
k_wht(C2<T> *amps, int lo, uint64_t ntiles, int cols, T scale, int negate_but_zero) {
    static_assert(!WIDE || (KB == 6 && !LOW), "the wide mapping is for 6-bit groups above bit 0");
    constexpr int kCols = WIDE ? 32 : 16;
    constexpr int B = WIDE ? 3 : (KB < 4 ? KB : 4);
    constexpr int A = KB - B;
    constexpr int NA = 1 << A, NB = 1 << B, MIDS = 1 << KB;
    static_assert(LOW || kCols * NB <= kGateThreads, "at most one phase-1 value row per thread");
    constexpr int ROW = kCols + kPad;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T> *sm = reinterpret_cast<C2<T> *>(smraw);  // [MIDS][ROW]

    const int t = threadIdx.x;
    // load / store mapping (coalesced): LOW -> mids fastest, else columns fastest
    const int lc = LOW ? t / NB : t % kCols;
    const int lr = LOW ? t % NB : t / kCols;
    const bool lact = LOW ? (lc < cols) : (lr < NB);
    // phase-2 mapping: thread owns NB consecutive mids of one column
    const int pc = t % kCols, pq = t / kCols;
    const bool pact = pq < NA && pc < cols;
    const uint64_t stride = LOW ? 1ull : (1ull << lo);

    auto tile_base = [&](uint64_t tile) -> uint64_t {
        if (LOW) return tile * (uint64_t)kCols * MIDS;
        const uint64_t chunks = (1ull << lo) / kCols;
        return ((tile / chunks) << (lo + KB)) | ((tile % chunks) * kCols);
    };
    const uint64_t col_off = LOW ? (uint64_t)lc * MIDS : (uint64_t)lc;
    // phase-1 values of the current tile; the next tile's are loaded while
    // this one goes through shared memory and back to HBM
    C2<T> v[NA];
    uint64_t tile = blockIdx.x;
    if (lact && tile < ntiles) {
        const uint64_t base = tile_base(tile);
#pragma unroll
        for (int j = 0; j < NA; ++j) v[j] = amps[base + col_off + (uint64_t)(lr + NB * j) * stride];
    }
    for (; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = tile_base(tile);
        if (lact) {
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = C2<T>{v[j].re * scale, v[j].im * scale};
            wht_regs<A>(v);
#pragma unroll
            for (int j = 0; j < NA; ++j) sm[(lr + NB * j) * ROW + lc] = v[j];
        }
        __syncthreads();
        const uint64_t next = tile + gridDim.x;
        if (lact && next < ntiles) {
            const uint64_t nb = tile_base(next);
#pragma unroll
            for (int j = 0; j < NA; ++j) v[j] = amps[nb + col_off + (uint64_t)(lr + NB * j) * stride];
        }
        if (pact) {
            C2<T> w[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) w[i] = sm[(NB * pq + i) * ROW + pc];
            wht_regs<B>(w);
#pragma unroll
            for (int i = 0; i < NB; ++i) sm[(NB * pq + i) * ROW + pc] = w[i];
        }
        __syncthreads();
        if (lact) {
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const uint64_t g = base + col_off + (uint64_t)(lr + NB * j) * stride;
                C2<T> x = sm[(lr + NB * j) * ROW + lc];
                if (negate_but_zero && g != 0) x = C2<T>{-x.re, -x.im};
                amps[g] = x;
            }
        }
        __syncthreads();
    }
}

template <class T, int KB, bool LOW, bool WIDE>
cudaError_t launch_wht_w(void *amps, int n, int lo, T scale, bool negate, cudaStream_t st, const Geometry &g) {
    constexpr int kCols = WIDE ? 32 : 16;
    constexpr int MIDS = 1 << KB;
    const size_t smem = (size_t)MIDS * (kCols + kPad) * sizeof(C2<T>);
    auto kern = k_wht<T, KB, LOW, WIDE>;
    {
        cudaError_t e = raise_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t N = 1ull << n;
    int cols = kCols;
    uint64_t ntiles;
    if (LOW) {
        const uint64_t blocks = N / MIDS;  // blocks of 2^KB contiguous amplitudes
        if (blocks < (uint64_t)kCols) cols = (int)blocks;
        ntiles = (blocks + kCols - 1) / kCols;
    } else {
        ntiles = N / ((uint64_t)MIDS * kCols);
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGateThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const uint64_t cap = (uint64_t)per_sm * g.sm_count;
    const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
    kern<<<grid, kGateThreads, smem, st>>>(static_cast<C2<T> *>(amps), lo, ntiles, cols, scale, negate ? 1 : 0);
    return cudaGetLastError();
}

template <class T, int KB, bool LOW>
cudaError_t launch_wht_t(void *amps, int n, int lo, T scale, bool negate, cudaStream_t st, const Geometry &g) {
    if constexpr (KB == 6 && !LOW) {
        if (lo >= 5) return launch_wht_w<T, KB, LOW, true>(amps, n, lo, scale, negate, st, g);
    }
    return launch_wht_w<T, KB, LOW, false>(amps, n, lo, scale, negate, st, g);
}

template <class T, bool LOW>
cudaError_t dispatch_kb(int kb, void *amps, int n, int lo, T scale, bool negate, cudaStream_t st, const Geometry &g) {
    switch (kb) {
    case 1: return launch_wht_t<T, 1, LOW>(amps, n, lo, scale, negate, st, g);
    case 2: return launch_wht_t<T, 2, LOW>(amps, n, lo, scale, negate, st, g);
    case 3: return launch_wht_t<T, 3, LOW>(amps, n, lo, scale, negate, st, g);
    case 4: return launch_wht_t<T, 4, LOW>(amps, n, lo, scale, negate, st, g);
    case 5: return launch_wht_t<T, 5, LOW>(amps, n, lo, scale, negate, st, g);
    case 6: return launch_wht_t<T, 6, LOW>(amps, n, lo, scale, negate, st, g);
    case 7: return launch_wht_t<T, 7, LOW>(amps, n, lo, scale, negate, st, g);
    default: return launch_wht_t<T, 8, LOW>(amps, n, lo, scale, negate, st, g);
    }
}

}  // namespace

// One Walsh-Hadamard pass over bits [lo, lo + kb) (kb <= 8; lo = 0 or lo >= 4),
// scaled by 2^-kb if `scaled`, optionally negating every amplitude but index 0.
cudaError_t launch_wht_pass(void *amps, int n, grover_dtype dt, int lo, int kb, bool scaled, bool negate,
                            cudaStream_t st, const Geometry &g) {
    if (dt == GROVER_C64) {
        const float s = scaled ? ldexpf(1.0f, -kb) : 1.0f;
        return lo == 0 ? dispatch_kb<float, true>(kb, amps, n, lo, s, negate, st, g)
                       : dispatch_kb<float, false>(kb, amps, n, lo, s, negate, st, g);
    }
    const double s = scaled ? ldexp(1.0, -kb) : 1.0;
    return lo == 0 ? dispatch_kb<double, true>(kb, amps, n, lo, s, negate, st, g)
                   : dispatch_kb<double, false>(kb, amps, n, lo, s, negate, st, g);
}

}  // namespace grv
