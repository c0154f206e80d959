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
// x = b0 + b1 + b2 (each the round-to-nearest of the remainder).  The b0
// products accumulate in one FP32 tensor-memory accumulator (A0), the b1 and b2
// products in a second (A12, about 2^-8 of A0, so the accumulator's own
// rounding there is below 2^-32 of the result instead of biasing the large
// one); the epilogue adds A12 + A0 with round to nearest.  Two such pairs
// (512 TMEM columns) alternate between tiles, so the epilogue of one tile
// runs while the tensor cores multiply the next.
// Pipeline per CTA (one per SM): the next tile streams into an fp32 staging
// buffer by TMA (one tiled cp.async.bulk.tensor copy per tile; the lowest
// group's with the 128-byte swizzle so its reads are free of bank conflicts;
// mbarrier transaction count) while the current tile is multiplied and stored.  Operands live in shared memory in
// the no-swizzle K-major layout (8 x 16-byte core matrices; leading byte
// offset = 144 B between core matrices along K, stride byte offset = 8-row
// group stride, both padded against bank conflicts); one thread issues 3 x K/16 tcgen05.mma (M = 128, N = K or
// 128, K = 16 each) and a tcgen05.commit to an mbarrier; the epilogue reads
// the accumulators with tcgen05.ld, applies the pass scale (exact power of
// two) and the phase shift 2|0><0| - I where asked, and stores.  Every
// mbarrier wait is bounded: on expiry the kernel sets the status word, waits
// (bounded) for its own copies and MMAs in flight, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <mutex>

#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kTcThreads = 512;
constexpr int kCols = 128;          // real columns per tile (= MMA M or N)
constexpr uint32_t kTmemCols = 512; // three accumulators of up to 128 columns


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
// Padded no-swizzle K-major operand layout.  A core matrix (8 rows x 8 bf16
// along K) is 128 contiguous bytes; core matrices adjacent along K are LBO =
// 144 bytes apart and 8-row groups SBO bytes apart, SBO = 18 K rounded up to
// 16 (mod 128).  The 16-byte pads put the eight k-groups of one row, and the
// rows 4c..4c+3 of eight consecutive c, on distinct bank groups, so the
// slice stores below are free of shared-memory bank conflicts (unpadded, the
// k-groups of a row were all 128 bytes apart, on the same banks).
constexpr uint32_t kLBO = 144;
__host__ __device__ constexpr uint32_t sbo_of(int K) {
    return 18u * (uint32_t)K + ((16u - ((18u * (uint32_t)K) & 127u)) & 127u);
}
// byte offset of element (row, k) in that layout for a K-column operand
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K) {
    return (uint32_t)((row >> 3) * sbo_of(K) + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// 128-byte-swizzle K-major operand layout (groups of 6 and 7 bits, K >= 64):
// a row's 64 elements of one K chunk fill 128 bytes, 8 rows form a 1024-byte
// atom, and the 16-byte chunk c of row r sits at chunk c ^ (r % 8); the K
// chunks of an R-row operand follow one another, R / 8 atoms each.  The
// tensor cores read it at full shared-memory width (the padded layout's
// 144-byte core-matrix stride straddles 128-byte lines), and stores whose 8
// rows differ in r % 8, or whose 8 chunks differ, are conflict-free.
__device__ __forceinline__ uint32_t sw_off(int row, int k, int R) {
    const int kc = k >> 6, kin = k & 63;
    return (uint32_t)(kc * (R >> 3) * 1024 + (row >> 3) * 1024 + (row & 7) * 128) +
           ((uint32_t)((kin >> 3) ^ (row & 7)) << 4) + (uint32_t)(kin & 7) * 2;
}
// descriptor of that layout: SBO 1024 B between 8-row atoms, LBO unused (16),
// layout field 2 (128-byte swizzle); atoms start on 1024-byte boundaries
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
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
// stores 8 consecutive-k values of one column (row) into the three slices at
// byte offset off (16-byte aligned) of each
__device__ __forceinline__ void put8(unsigned char *xs, size_t slice_bytes, uint32_t off, const float *v) {
    float b[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split3(v[j], b[0][j], b[1][j], b[2][j]);
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

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long limit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(su32(bar)), "r"(parity) : "memory");
        if (!done) __nanosleep(32);
    }
    return done != 0;
}

// Real columns of a tile: 128 for the lowest group (64 blocks x re/im); for an
// upper group 128 x 128 / K, so every tile holds 8192 amplitudes (64 KiB) and
// a K < 128 pass runs 128 / K column blocks of 128 through the MMAs.
template <int KB, bool LOW> __host__ __device__ constexpr int tile_cols() { return LOW ? kCols : kCols * (128 >> KB); }
// box width (floats) of one tensor copy of an upper-group tile (at most 256)
template <int KB> __host__ __device__ constexpr int box_cols() {
    return tile_cols<KB, false>() < 256 ? tile_cols<KB, false>() : 256;
}

// Tile geometry: first amplitude of the tile (the mids are 2^lo apart).
template <int KB, bool LOW> __device__ __forceinline__ uint64_t tile_base(uint64_t tile, int lo) {
    constexpr int K = 1 << KB;
    if (LOW) return tile * (uint64_t)(kCols / 2) * K;  // 64 blocks of K amplitudes
    constexpr int AMPS = tile_cols<KB, false>() / 2;
    const uint64_t chunks = (1ull << lo) / AMPS;
    return ((tile / chunks) << (lo + KB)) | ((tile % chunks) * AMPS);
}

// Warp 0 streams one tile of fp32 amplitudes into the staging buffer: the
// lowest group is one contiguous block, an upper group K rows of 512 bytes.
template <int KB, bool LOW>
__device__ __forceinline__ void issue_tile_load(const float *amps, const CUtensorMap *tmap, uint64_t tile, int lo,
                                                unsigned char *stage, unsigned long long *bar, int lane) {
    constexpr int K = 1 << KB;
    constexpr uint32_t TILEB = (uint32_t)K * tile_cols<KB, LOW>() * 4;  // 64 KiB
    const uint64_t abase = tile_base<KB, LOW>(tile, lo);
    if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(TILEB) : "memory");
    __syncwarp();
    if (LOW) {
        // one tiled copy with the 128-byte swizzle: box {32 floats, 8 lines,
        // 64 blocks} of the view [block][8 lines][32 floats]; x = 0, y = 0,
        // z = first block of the tile
        if (lane == 0) {
            const int z = (int)(abase / K);
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                         "[%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(su32(stage)), "l"(tmap), "r"(0), "r"(0), "r"(z), "r"(su32(bar)) : "memory");
        }
    } else if (lane == 0) {
        // tiled copies of box {BOX floats, K mids, 1 outer} of the view
        // [outer][mid][2^(lo+1) floats]; x = chunk * COLS + b * BOX floats (a
        // multiple of 16 bytes), y = 0, z = outer; copy b lands as its own
        // [K][BOX] block of the stage
        constexpr int COLS = tile_cols<KB, false>(), BOX = box_cols<KB>();
        const uint64_t chunks = (1ull << lo) / (COLS / 2);
        const int z = (int)(tile / chunks);
#pragma unroll
        for (int b = 0; b < COLS / BOX; ++b) {
            const int x = (int)((tile % chunks) * COLS) + b * BOX;
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                         "[%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(su32(stage + (size_t)b * K * BOX * 4)), "l"(tmap), "r"(x), "r"(0), "r"(z),
                           "r"(su32(bar)) : "memory");
        }
    }
    (void)amps;
}

template <int KB, bool LOW>
__global__ void __launch_bounds__(kTcThreads, 1)
k_wht_tc(float *amps, const __grid_constant__ CUtensorMap tmap, int lo, uint64_t ntiles, float scale,
         int negate_but_zero, int *status, long long wait_limit, int stall) {
    constexpr int K = 1 << KB;
    constexpr int COLS = tile_cols<KB, LOW>();            // real columns (operand rows)
    constexpr int NB = COLS / kCols;                        // column blocks of 128 (MMA M)
    constexpr bool SW = KB >= 6;                            // 128-byte-swizzle operands
    constexpr size_t STAGE = (size_t)K * COLS * 4;          // fp32 tile, 64 KiB
    constexpr uint32_t SBO = sbo_of(K);
    constexpr uint32_t LBO = kLBO;
    constexpr size_t SLICE = SW ? (size_t)COLS * K * 2 : (size_t)(COLS / 8) * SBO;  // one bf16 slice of the tile
    constexpr int M_MMA = 128;
    constexpr int N_MMA = LOW ? kCols : K;                  // accumulator columns; A12 sits N_MMA after A0
    static_assert(!LOW || KB == 7, "the lowest group uses W as the 128-row operand");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *stage = smem;                        // fp32 tile from global
    unsigned char *xs = smem + STAGE;                   // [3][SLICE] bf16 slices
    unsigned char *ws = smem + STAGE + 3 * SLICE;       // W, K x K bf16
    __shared__ __align__(8) unsigned long long tma_bar, mma_bar;
    __shared__ uint32_t tslot;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the 128-byte swizzle of the staged tile repeats every 1024 bytes: the
    // stage must start on such a boundary (the reads undo the pattern from
    // offsets relative to it)
    if (su32(stage) & 1023u) {
        if (tid == 0) atomicExch(status, 4);
        return;
    }
    for (int i = tid; i < K * K / 8; i += kTcThreads) {  // W[n][k] = (-1)^popcount(n & k)
        const int n = i / (K / 8), k0 = (i % (K / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (__popc(n & (k0 + j)) & 1) ? -1.0f : 1.0f;
        uint4 q;
        q.x = pack2(v[0], v[1]);
        q.y = pack2(v[2], v[3]);
        q.z = pack2(v[4], v[5]);
        q.w = pack2(v[6], v[7]);
        *reinterpret_cast<uint4 *>(ws + (SW ? sw_off(n, k0, K) : kmaj_off(n, k0, K))) = q;
    }
    if (tid == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tma_bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mma_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t taddr = tslot;
    // loads_done / mmas_done count completed phases of the two mbarriers; the
    // parity of the next phase to wait for is the count's low bit
    uint32_t loads_done = 0, mmas_done = 0;
    bool load_pending = blockIdx.x < ntiles, mma_pending = false;
    if (warp == 0 && load_pending) issue_tile_load<KB, LOW>(amps, &tmap, blockIdx.x, lo, stage, &tma_bar, lane);

    // Epilogue of a finished tile from TMEM buffer `buf`: A12 + A0 (one
    // rounding), scale, phase shift, store.
    auto epilogue = [&](uint64_t etile, uint32_t buf) {
        const uint64_t abase = tile_base<KB, LOW>(etile, lo);
        const int lg = warp & 3, cw = warp >> 2;
        constexpr int CPB = N_MMA / 32;  // 32-column chunks per column block
        if (cw < NB * CPB) {
            const int blk = cw / CPB, cg = cw % CPB;
            uint32_t a[32], b[32];
            const uint32_t t0 = taddr + 256u * buf + ((uint32_t)(32 * lg) << 16) + (uint32_t)(blk * 2 * N_MMA + 32 * cg);
            tmem_ld32(t0 + (uint32_t)N_MMA, a);
            tmem_ld32(t0, b);
#pragma unroll
            for (int j = 0; j < 32; ++j) a[j] = __float_as_uint(__uint_as_float(a[j]) + __uint_as_float(b[j]));
            const int row = 32 * lg + lane;
            if (LOW) {
                // row = output mid, registers = 16 blocks x (re, im); lanes 2l and
                // 2l + 1 hold mids r and r + 1: the even lane stores both for the
                // even blocks, the odd lane for the odd blocks (16-byte stores)
                const bool odd = lane & 1;
                const int r0 = row & ~1;
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const float e0 = __uint_as_float(a[4 * p]), e1 = __uint_as_float(a[4 * p + 1]);
                    const float o0 = __uint_as_float(a[4 * p + 2]), o1 = __uint_as_float(a[4 * p + 3]);
                    // even lane gives its odd-block pair, odd lane its even-block pair
                    const float g0 = __shfl_xor_sync(0xffffffffu, odd ? e0 : o0, 1);
                    const float g1 = __shfl_xor_sync(0xffffffffu, odd ? e1 : o1, 1);
                    // (mid r0: re, im), (mid r0 + 1: re, im) of block 2p + odd
                    float4 v = odd ? make_float4(g0, g1, o0, o1) : make_float4(e0, e1, g0, g1);
                    const uint64_t a0 = abase + (uint64_t)(16 * cg + 2 * p + (odd ? 1 : 0)) * K + r0;
                    v.x *= scale;
                    v.y *= scale;
                    v.z *= scale;
                    v.w *= scale;
                    if (negate_but_zero) {
                        if (a0 != 0) {
                            v.x = -v.x;
                            v.y = -v.y;
                        }
                        v.z = -v.z;
                        v.w = -v.w;
                    }
                    __stcs(reinterpret_cast<float4 *>(amps) + a0 / 2, v);
                }
            } else {
                // row = column (re or im of amplitude col / 2), registers = output
                // mids; lanes 2l and 2l + 1 hold re and im of one amplitude: they
                // swap halves so each stores (re, im) pairs for 16 mids
                const int col = kCols * blk + row;
                const uint64_t ar = abase + (uint64_t)(col >> 1);
                const bool odd = lane & 1;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    // even lane keeps mid 2j (its re) and receives the im of mid 2j;
                    // odd lane keeps mid 2j + 1 (its im) and receives the re of mid 2j + 1
                    const float mine_e = __uint_as_float(a[2 * j]), mine_o = __uint_as_float(a[2 * j + 1]);
                    const float give = odd ? mine_e : mine_o;
                    const float got = __shfl_xor_sync(0xffffffffu, give, 1);
                    const int mid = 32 * cg + 2 * j + (odd ? 1 : 0);
                    const uint64_t a0 = ar + ((uint64_t)mid << lo);
                    float re = (odd ? got : mine_e) * scale, im = (odd ? mine_o : got) * scale;
                    if (negate_but_zero && a0 != 0) {
                        re = -re;
                        im = -im;
                    }
                    __stcs(reinterpret_cast<float2 *>(amps) + a0, make_float2(re, im));
                }
            }
        }
    };

    // Per tile i: build the slices of tile i; issue the load of tile i + 1 and
    // the MMAs of tile i into TMEM buffer i & 1; while they run, the epilogue
    // of tile i - 1 drains buffer (i - 1) & 1; then wait for the MMAs (the
    // slices are free again).
    uint64_t prev = ~0ull;
    uint32_t it = 0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        // ---- staged fp32 tile -> three bf16 slices ----
        if (!mbar_wait(&tma_bar, loads_done & 1, wait_limit)) {
            atomicExch(status, 2);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        ++loads_done;
        load_pending = false;
        if (LOW) {
            // unit = (block o, k-group of 8 mids): 8 complex = 4 float4 contiguous
            // the stage holds 128-byte lines whose 16-byte chunks the copy
            // permuted: chunk c of line L sits at chunk c ^ (L & 7); the eight
            // threads of a load phase then read eight different bank groups
            for (int u = tid; u < (kCols / 2) * (K / 8); u += kTcThreads) {
                const int kg = u % (K / 8), o = u / (K / 8);
                float re[8], im[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t logical = (uint32_t)o * (K * 8) + (uint32_t)kg * 64 + (uint32_t)q * 16;
                    const uint32_t phys = logical ^ (((logical >> 7) & 7u) << 4);
                    const float4 c = *reinterpret_cast<const float4 *>(stage + phys);
                    re[2 * q] = c.x;
                    im[2 * q] = c.y;
                    re[2 * q + 1] = c.z;
                    im[2 * q + 1] = c.w;
                }
                put8(xs, SLICE, SW ? sw_off(2 * o, kg * 8, COLS) : kmaj_off(2 * o, kg * 8, K), re);
                put8(xs, SLICE, SW ? sw_off(2 * o + 1, kg * 8, COLS) : kmaj_off(2 * o + 1, kg * 8, K), im);
            }
        } else {
            // copy b of the tile holds columns [b BOX, (b + 1) BOX) as a [K][BOX] block
            constexpr int BOX = box_cols<KB>();
            if constexpr (SW) {
                // unit = (k-group of 8 mids, column): consecutive threads read
                // consecutive columns of each mid row and store rows whose r % 8
                // differ (both conflict-free)
                const float *stf = reinterpret_cast<const float *>(stage);
                for (int u = tid; u < (K / 8) * COLS; u += kTcThreads) {
                    const int c = u % COLS, kg = u / COLS;
                    const float *src = stf + (size_t)(c / BOX) * K * BOX + (size_t)(kg * 8) * BOX + (c % BOX);
                    float col[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) col[j] = src[(size_t)j * BOX];
                    put8(xs, SLICE, sw_off(c, kg * 8, COLS), col);
                }
            } else
            // unit = (k-group of 8 mids, float4 column group)
            for (int u = tid; u < (K / 8) * (COLS / 4); u += kTcThreads) {
                const int c4 = u % (COLS / 4), kg = u / (COLS / 4);
                const int bx = (4 * c4) / BOX, w4 = ((4 * c4) % BOX) / 4;
                const float4 *blk4 = reinterpret_cast<const float4 *>(stage) + (size_t)bx * K * (BOX / 4);
                float col[4][8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 c = blk4[(size_t)(kg * 8 + j) * (BOX / 4) + w4];
                    col[0][j] = c.x;
                    col[1][j] = c.y;
                    col[2][j] = c.z;
                    col[3][j] = c.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) put8(xs, SLICE, kmaj_off(4 * c4 + q, kg * 8, K), col[q]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        // ---- next tile's load ----
        const uint64_t next = tile + gridDim.x;
        if (warp == 0 && next < ntiles) issue_tile_load<KB, LOW>(amps, &tmap, next, lo, stage, &tma_bar, lane);
        load_pending = next < ntiles;
        // ---- MMA into buffer it & 1: A0 = W b0 (or b0 W), A12 = W (b1 + b2) ----
        if (tid == 0) {
            constexpr uint32_t idesc = idesc_bf16(M_MMA, N_MMA);
            const uint32_t tb = taddr + 256u * (it & 1u);
#pragma unroll 1
            for (int blk = 0; blk < NB; ++blk) {
#pragma unroll 1
                for (int s = 0; s < 3; ++s) {
#pragma unroll 1
                    for (int kk = 0; kk < K / 16; ++kk) {
                        // column block blk: operand rows [128 blk, 128 blk + 128)
                        uint64_t dx, dw;
                        if constexpr (SW) {
                            const uint32_t kin = (uint32_t)(kk & 3) * 32u, kc = (uint32_t)(kk >> 2);
                            dx = smem_desc_sw128(su32(xs + s * SLICE) + kc * (COLS / 8) * 1024u + (uint32_t)blk * 16u * 1024u +
                                                 kin);
                            dw = smem_desc_sw128(su32(ws) + kc * (K / 8) * 1024u + kin);
                        } else {
                            dx = smem_desc(su32(xs + s * SLICE) + (uint32_t)blk * 16u * SBO + kk * 2 * LBO, LBO, SBO);
                            dw = smem_desc(su32(ws) + kk * 2 * LBO, LBO, SBO);
                        }
                        const uint64_t da = LOW ? dw : dx;
                        const uint64_t db = LOW ? dx : dw;
                        const uint32_t acc = (s == 2) || kk != 0;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(tb + (uint32_t)(blk * 2 * N_MMA) + (s ? (uint32_t)N_MMA : 0u)), "l"(da),
                                       "l"(db), "r"(idesc), "r"(acc) : "memory");
                    }
                }
            }
            // test hook: without the commit nothing arrives on mma_bar
            if (!stall)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(su32(&mma_bar)) : "memory");
        }
        mma_pending = true;
        // ---- epilogue of the previous tile, overlapping the MMAs ----
        if (prev != ~0ull) epilogue(prev, (it - 1) & 1u);
        if (!mbar_wait(&mma_bar, mmas_done & 1, wait_limit)) {
            atomicExch(status, 2);
            s_abort = 1;
        }
        fence_before();
        __syncthreads();
        fence_after();
        if (s_abort) break;
        ++mmas_done;
        mma_pending = false;
        prev = tile;
    }
    if (!s_abort && prev != ~0ull) {
        epilogue(prev, (it - 1) & 1u);
        fence_before();
        __syncthreads();
    }
    // after an abort, wait (bounded) for this CTA's own load and MMA in flight
    // before the tensor memory is freed and the CTA exits
    if (tid == 0) {
        if (load_pending) (void)mbar_wait(&tma_bar, loads_done & 1, wait_limit);
        if (mma_pending) (void)mbar_wait(&mma_bar, mmas_done & 1, wait_limit);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// View of an n-qubit complex64 state for the pass over bits [lo, lo + kb):
// [outer][mid][2^(lo+1) floats], box {128, 2^kb, 1}.
cudaError_t encode_upper_map(CUtensorMap *m, void *amps, int n, int lo, int kb) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t inner = 1ull << (lo + 1);
    const cuuint64_t dims[3] = {inner, 1ull << kb, 1ull << (n - lo - kb)};
    const cuuint64_t strides[2] = {inner * 4, (inner << kb) * 4};
    const int cols = kCols * (128 >> kb);
    const cuuint32_t box[3] = {(cuuint32_t)(cols < 256 ? cols : 256), (cuuint32_t)(1u << kb), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, amps, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// View of the state for the lowest group: [block of 128 amplitudes][8 lines][32
// floats], box {32, 8, 64} with the 128-byte swizzle.
cudaError_t encode_low_map(CUtensorMap *m, void *amps, int n) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {32, 8, 1ull << (n - 7)};
    const cuuint64_t strides[2] = {128, 1024};
    const cuuint32_t box[3] = {32u, 8u, (cuuint32_t)(kCols / 2)};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, amps, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int KB, bool LOW>
cudaError_t launch_tc_t(void *amps, int n, int lo, float scale, bool negate, int *status, long long wait_limit,
                        int stall, cudaStream_t st, const Geometry &g) {
    constexpr int K = 1 << KB;
    // fp32 stage, three bf16 slices (128 rows), W (K rows), padded layout
    constexpr int COLS = tile_cols<KB, LOW>();
    const size_t smem = KB >= 6 ? (size_t)K * COLS * 4 + 3 * (size_t)COLS * K * 2 + (size_t)K * K * 2
                                : (size_t)K * COLS * 4 + 3 * (size_t)(COLS / 8) * sbo_of(K) + (size_t)(K / 8) * sbo_of(K);
    auto kern = k_wht_tc<KB, LOW>;
    {
        cudaError_t e = raise_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    {
        cudaError_t e = LOW ? encode_low_map(&tmap, amps, n) : encode_upper_map(&tmap, amps, n, lo, KB);
        if (e != cudaSuccess) return e;
    }
    const uint64_t N = 1ull << n;
    const uint64_t ntiles = N / ((uint64_t)(COLS / 2) * K);
    const uint64_t grid = ntiles < (uint64_t)g.sm_count ? ntiles : (uint64_t)g.sm_count;
    kern<<<(unsigned)grid, kTcThreads, smem, st>>>(static_cast<float *>(amps), tmap, lo, ntiles, scale,
                                                   negate ? 1 : 0, status, wait_limit, stall);
    return cudaGetLastError();
}

}  // namespace

bool tc_pass_supported(int n, int lo, int kb) {
    if (lo == 0) return kb == 7 && n >= 13;          // 64 blocks of 128 amplitudes per tile
    // 64 * 128 / K consecutive amplitudes below lo
    return kb >= 5 && kb <= 7 && lo >= 13 - kb && lo + kb <= n;
}

cudaError_t launch_wht_tc_pass(void *amps, int n, int lo, int kb, bool scaled, bool negate, int *status,
                               long long wait_limit, int stall, cudaStream_t st, const Geometry &g) {
    const float s = scaled ? ldexpf(1.0f, -kb) : 1.0f;
    if (lo == 0) return launch_tc_t<7, true>(amps, n, lo, s, negate, status, wait_limit, stall, st, g);
    switch (kb) {
    case 5: return launch_tc_t<5, false>(amps, n, lo, s, negate, status, wait_limit, stall, st, g);
    case 6: return launch_tc_t<6, false>(amps, n, lo, s, negate, status, wait_limit, stall, st, g);
    default: return launch_tc_t<7, false>(amps, n, lo, s, negate, status, wait_limit, stall, st, g);
    }
}

}  // namespace grv
