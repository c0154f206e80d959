// k_gate_tc.cu -- Walsh-Hadamard passes of the conventional circuit on the
// 5th-generation tensor cores (tcgen05), complex64 states.
//
// A pass applies W (the +-1 Walsh-Hadamard matrix of order K = 2^kb,
// kb in {5, 6, 7}) to the index bits [lo, lo + kb): for every (outer, inner)
// position the 2^kb amplitudes along those bits are multiplied by W, i.e. a
// batched dense contraction.  A CTA tile holds 128 real columns x K mids:
//   * upper groups (lo >= 7): 64 consecutive amplitudes (re and im = 128
//     columns) below bit lo, at all K mid values; D = X^T W, so TMEM lane =
//     column and a warp's stores for one output mid are 128 contiguous bytes;
//   * the lowest group (lo = 0, kb = 7): 64 consecutive blocks of 128
//     amplitudes (column = (block, re/im)); D = W X, so TMEM lane = output mid
//     and each thread stores (re, im) pairs, 256 contiguous bytes per warp.
// W is exact in bf16.  Each FP32 amplitude is split into three bf16 slices
// x = b0 + b1 + b2 (each the round-to-nearest of the remainder), and the three
// slice products accumulate into one FP32 accumulator in tensor memory.
// Operands live in shared memory in the no-swizzle K-major layout (8 x 16-byte
// core matrices; leading byte offset = 128 B between core matrices along K,
// stride byte offset = 8-row group stride); one thread issues
// 3 x K/16 tcgen05.mma (M = 128, N = K or 128, K = 16 each) and a
// tcgen05.commit to an mbarrier; the epilogue reads the accumulator with
// tcgen05.ld, applies the pass scale (exact power of two) and the phase shift
// 2|0><0| - I where asked, and stores.  Every wait on the mbarrier is bounded:
// on expiry the kernel sets the status word, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kCols = 128;          // real columns per tile (= MMA M or N)
constexpr uint32_t kTmemCols = 128; // accumulator columns allocated
constexpr long long kWaitLimit = 1ll << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// byte offset of element (row, k) in a K-major no-swizzle bf16 operand with K columns
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K) {
    return (uint32_t)((row >> 3) * ((K >> 3) * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split3(float x, float &b0, float &b1, float &b2) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(h0);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(r);
    r -= __bfloat162float(h1);
    b0 = __bfloat162float(h0);
    b1 = __bfloat162float(h1);
    b2 = r;  // rounded to bf16 when packed
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}
// stores 8 consecutive-k values of one column (row) into the three slices
__device__ __forceinline__ void put8(unsigned char *xs, size_t slice_bytes, int row, int k0, int K, const float *v) {
    float b[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split3(v[j], b[0][j], b[1][j], b[2][j]);
    const uint32_t off = kmaj_off(row, k0, K);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        uint4 q;
        q.x = pack2(b[s][0], b[s][1]);
        q.y = pack2(b[s][2], b[s][3]);
        q.z = pack2(b[s][4], b[s][5]);
        q.w = pack2(b[s][6], b[s][7]);
        *reinterpret_cast<uint4 *>(xs + s * slice_bytes + off) = q;
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int KB, bool LOW>
__global__ void __launch_bounds__(kTcThreads, 1)
k_wht_tc(float *amps, int lo, uint64_t ntiles, float scale, int negate_but_zero, int *status) {
    constexpr int K = 1 << KB;
    constexpr size_t SLICE = (size_t)kCols * K * 2;  // bytes of one bf16 slice of the tile
    constexpr uint32_t SBO = (K / 8) * 128;
    constexpr uint32_t LBO = 128;
    constexpr int M_MMA = 128;
    constexpr int N_MMA = LOW ? kCols : K;
    static_assert(!LOW || KB == 7, "the lowest group uses W as the 128-row operand");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *xs = smem;                 // [3][SLICE] state slices
    unsigned char *ws = smem + 3 * SLICE;     // W, K x K bf16
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tslot;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // W[n][k] = (-1)^popcount(n & k), K-major
    for (int i = tid; i < K * K / 8; i += kTcThreads) {
        const int n = i / (K / 8), k0 = (i % (K / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (__popc(n & (k0 + j)) & 1) ? -1.0f : 1.0f;
        uint4 q;
        q.x = pack2(v[0], v[1]);
        q.y = pack2(v[2], v[3]);
        q.z = pack2(v[4], v[5]);
        q.w = pack2(v[6], v[7]);
        *reinterpret_cast<uint4 *>(ws + kmaj_off(n, k0, K)) = q;
    }
    if (tid == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t taddr = tslot;
    uint32_t phase = 0;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- tile geometry (amplitude indices) ----
        uint64_t abase;       // first amplitude of the tile
        uint64_t mid_stride;  // amplitude stride between consecutive mids
        if (LOW) {
            abase = tile * (uint64_t)(kCols / 2) * K;  // 64 blocks of K amplitudes
            mid_stride = 1;
        } else {
            const uint64_t chunks = (1ull << lo) / (kCols / 2);
            abase = ((tile / chunks) << (lo + KB)) | ((tile % chunks) * (kCols / 2));
            mid_stride = 1ull << lo;
        }
        // ---- producer: global fp32 -> three bf16 slices in shared memory ----
        if (LOW) {
            // unit = (block o of 64, k-group of 8 mids): 8 complex = 4 float4 contiguous
            for (int u = tid; u < (kCols / 2) * (K / 8); u += kTcThreads) {
                const int kg = u % (K / 8), o = u / (K / 8);
                const float4 *src = reinterpret_cast<const float4 *>(amps + 2 * (abase + (uint64_t)o * K + kg * 8));
                float re[8], im[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 c = __ldcs(src + q);
                    re[2 * q] = c.x;
                    im[2 * q] = c.y;
                    re[2 * q + 1] = c.z;
                    im[2 * q + 1] = c.w;
                }
                put8(xs, SLICE, 2 * o, kg * 8, K, re);
                put8(xs, SLICE, 2 * o + 1, kg * 8, K, im);
            }
        } else {
            // unit = (k-group of 8 mids, float4 column group): 8 rows x 16 bytes
            for (int u = tid; u < (K / 8) * (kCols / 4); u += kTcThreads) {
                const int c4 = u % (kCols / 4), kg = u / (kCols / 4);
                float col[4][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint64_t a = abase + (uint64_t)(kg * 8 + j) * mid_stride;
                    const float4 c = __ldcs(reinterpret_cast<const float4 *>(amps + 2 * a) + c4);
                    col[0][j] = c.x;
                    col[1][j] = c.y;
                    col[2][j] = c.z;
                    col[3][j] = c.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) put8(xs, SLICE, 4 * c4 + q, kg * 8, K, col[q]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        // ---- MMA: one thread issues 3 slices x K/16 steps, then commits ----
        if (tid == 0) {
            constexpr uint32_t idesc = idesc_bf16(M_MMA, N_MMA);
#pragma unroll 1
            for (int s = 0; s < 3; ++s) {
#pragma unroll 1
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint32_t xa = su32(xs + s * SLICE) + kk * 2 * LBO;
                    const uint32_t wa = su32(ws) + kk * 2 * LBO;
                    const uint64_t da = LOW ? smem_desc(wa, LBO, SBO) : smem_desc(xa, LBO, SBO);
                    const uint64_t db = LOW ? smem_desc(xa, LBO, SBO) : smem_desc(wa, LBO, SBO);
                    const uint32_t acc = (s | kk) != 0;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(taddr), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar))
                         : "memory");
        }
        // ---- bounded wait for the accumulator ----
        uint32_t done = 0;
        for (long long it = 0; it < kWaitLimit && !done; ++it) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(su32(&bar)), "r"(phase) : "memory");
            if (!done) __nanosleep(32);
        }
        if (!done) {
            atomicExch(status, 2);
            s_abort = 1;
        }
        phase ^= 1u;
        fence_after();
        __syncthreads();
        if (s_abort) break;
        // ---- epilogue: TMEM -> registers -> global ----
        {
            const int lg = warp & 3, cg = warp >> 2;  // TMEM lane group, 32-column chunk
            constexpr int NCH = N_MMA / 32;
            if (cg < NCH) {
                uint32_t v[32];
                tmem_ld32(taddr + ((uint32_t)(32 * lg) << 16) + (uint32_t)(32 * cg), v);
                const int row = 32 * lg + lane;
                if (LOW) {
                    // row = output mid, registers = columns 32cg .. 32cg+31 = 16 blocks x (re, im)
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const uint64_t a = abase + (uint64_t)(16 * cg + q) * K + row;
                        float re = __uint_as_float(v[2 * q]) * scale, im = __uint_as_float(v[2 * q + 1]) * scale;
                        if (negate_but_zero && a != 0) {
                            re = -re;
                            im = -im;
                        }
                        __stcs(reinterpret_cast<float2 *>(amps) + a, make_float2(re, im));
                    }
                } else {
                    // row = column (re/im of amplitude row/2), registers = output mids 32cg + j
                    const uint64_t a0 = abase + (uint64_t)(row >> 1);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const uint64_t a = a0 + (uint64_t)(32 * cg + j) * mid_stride;
                        float x = __uint_as_float(v[j]) * scale;
                        if (negate_but_zero && a != 0) x = -x;
                        __stcs(amps + 2 * a + (row & 1), x);
                    }
                }
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

template <int KB, bool LOW>
cudaError_t launch_tc_t(void *amps, int n, int lo, float scale, bool negate, int *status, cudaStream_t st,
                        const Geometry &g) {
    constexpr int K = 1 << KB;
    const size_t smem = 3 * (size_t)kCols * K * 2 + (size_t)K * K * 2;
    auto kern = k_wht_tc<KB, LOW>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint64_t N = 1ull << n;
    const uint64_t ntiles = N / ((uint64_t)(kCols / 2) * K);
    const uint64_t grid = ntiles < (uint64_t)g.sm_count ? ntiles : (uint64_t)g.sm_count;
    kern<<<(unsigned)grid, kTcThreads, smem, st>>>(static_cast<float *>(amps), lo, ntiles, scale, negate ? 1 : 0,
                                                   status);
    return cudaGetLastError();
}

}  // namespace

bool tc_pass_supported(int n, int lo, int kb) {
    if (lo == 0) return kb == 7 && n >= 13;          // 64 blocks of 128 amplitudes per tile
    return kb >= 5 && kb <= 7 && lo >= 6;            // 64 consecutive amplitudes below lo
}

cudaError_t launch_wht_tc_pass(void *amps, int n, int lo, int kb, bool scaled, bool negate, int *status,
                               cudaStream_t st, const Geometry &g) {
    const float s = scaled ? ldexpf(1.0f, -kb) : 1.0f;
    if (lo == 0) return launch_tc_t<7, true>(amps, n, lo, s, negate, status, st, g);
    switch (kb) {
    case 5: return launch_tc_t<5, false>(amps, n, lo, s, negate, status, st, g);
    case 6: return launch_tc_t<6, false>(amps, n, lo, s, negate, status, st, g);
    default: return launch_tc_t<7, false>(amps, n, lo, s, negate, status, st, g);
    }
}

}  // namespace grv
