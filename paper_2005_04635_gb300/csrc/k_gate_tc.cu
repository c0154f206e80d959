// k_gate_tc.cu -- Walsh-Hadamard passes of the conventional circuit on the
// 5th-generation tensor cores (tcgen05), complex64 states.
//
// A pass applies W (the +-1 Walsh-Hadamard matrix of order K = 2^kb,
// kb in {5, 6, 7}) to the index bits [lo, lo + kb): for every (outer, inner)
// position the K amplitudes along those bits are multiplied by W, i.e. a
// batched dense contraction (Eq. unitary applied to kb qubits at once).  A
// tile is 8192 amplitudes = 128 x 128 / K real columns x K mids:
//   * upper groups (lo >= 13 - kb): 64 * 128 / K consecutive amplitudes below
//     bit lo (re and im = the columns) at all K mid values; D = X^T W per
//     block of 128 columns, so TMEM lane = column and a warp's stores for one
//     output mid are 128 contiguous bytes;
//   * the lowest group (lo = 0, kb = 7): 64 consecutive blocks of 128
//     amplitudes (column = (block, re/im)); D = W X, so TMEM lane = output mid
//     and a warp stores 32 consecutive amplitudes (256 bytes) at once.
// W is exact in bf16.  Each FP32 amplitude is split into three bf16 slices
// x = b0 + b1 + b2 (each the round-to-nearest of the remainder; the three hold
// all 24 bits).  The b0 products accumulate in one FP32 tensor-memory
// accumulator (A0), the b1 and b2 products in a second (A12, about 2^-8 of
// A0, so its own rounding is far below the result's); the epilogue adds
// A12 + A0 with one rounding, scales by an exact power of two and applies the
// phase shift 2|0><0| - I where asked.
//
// Pipeline.  A tile is cut into 8 chunks of 128 columns x 16 mids (one MMA K
// step each: 8 KiB of FP32, 3 x 4 KiB of bf16).  Warp roles, one CTA per SM:
//   * TMA warp: one tiled cp.async.bulk.tensor copy per chunk into a ring of
//     12 FP32 stages (mbarrier transaction counts; the lowest group's copies
//     with the 128-byte swizzle, so the converters' reads are spread over the
//     banks);
//   * 8 converter warps, each owning one slice slot: warp w converts chunks
//     w, w + 8, ... (eight chunks at once), frees the chunk's stage as soon
//     as the values are in registers, and writes the slices in the
//     no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
//     matrix, 128 bytes between the two K halves, 256 bytes between 8-row
//     groups);
//   * MMA warp: one thread issues the chunk's three tcgen05.mma (kind::f16,
//     M = 128, N = K or 128, K = 16) and a tcgen05.commit that frees the slot,
//     and after a tile's last chunk a commit that hands its accumulators on;
//     two accumulator pairs (512 TMEM columns) alternate between tiles;
//   * 4 epilogue warps (TMEM lanes 0..127): tcgen05.ld, sum, scale, phase
//     shift, streaming stores.
// So the copy of one chunk, the slices of the next and the MMAs and the
// epilogue of earlier ones all overlap.  Every mbarrier wait is bounded: on
// expiry the kernel sets the status word, every role leaves its loop, the
// copies and MMAs already issued are waited for (bounded) and the tensor
// memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <mutex>

#include "grover_internal.cuh"

namespace grv {
namespace {

constexpr int kEpiWarps = 4;    // warps 0-3: TMEM lanes 32 w .. 32 w + 31
constexpr int kTmaWarp = 4;
constexpr int kMmaWarp = 5;
constexpr int kConvWarp0 = 6;
constexpr int kConvWarps = 8;
constexpr int kTcThreads = 32 * (kConvWarp0 + kConvWarps);  // 448
constexpr int kSlots = kConvWarps;  // slice slots: converter warp w owns slot w
// FP32 chunk stages: 96 KiB of copies in flight per SM (as many as shared
// memory leaves beside the slots and a 7-bit W).  Chunk q uses stage q % 12 and
// is converted by warp q % 8; successive chunks of a stage belong to different
// warps, so before it waits for phase q / 12 of full[s] a converter waits until
// phase q / 12 - 1 of empty[s] has completed (that stage's previous chunk was
// read).  Both waits are then unambiguous by parity: phase q / 12 - 2 of a
// stage is chunk q - 24, which this warp itself converted earlier (24 is a
// multiple of 8).
constexpr int kRing = 12;
static_assert((2 * kRing) % kConvWarps == 0, "a stage's phase two back must be the same converter warp's");
constexpr int kRows = 128;       // real columns per chunk (MMA M, or N for the lowest group)
constexpr int kChunkK = 16;      // mids per chunk (one MMA K step)
constexpr int kChunksPerTile = 8;
constexpr uint32_t kStageBytes = kRows * kChunkK * 4;  // 8 KiB
constexpr uint32_t kSliceBytes = kRows * kChunkK * 2;  // 4 KiB
constexpr uint32_t kSlotBytes = 3 * kSliceBytes;
constexpr uint32_t kTmemCols = 512;                    // 2 tiles x (A0 + A12) x 128 columns
constexpr uint32_t kLBO = 128, kSBO = 256;             // core-matrix strides along K / along rows

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// byte offset of (row, k), k < 16, in a [rows][16] bf16 operand chunk
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}
// Three bf16 slices of two FP32 values x0, x1, packed in pairs (x0 in the low
// half): s0 = bf16(x), s1 = bf16(x - s0), s2 = bf16(x - s0 - s1), each the
// round-to-nearest of the remainder (the subtractions are exact, and the last
// remainder has at most 8 significant bits, so s0 + s1 + s2 = x).
__device__ __forceinline__ void split3x2(float x0, float x1, uint32_t &s0, uint32_t &s1, uint32_t &s2) {
    s0 = pack2(x0, x1);
    const float r0 = x0 - __uint_as_float(s0 << 16), r1 = x1 - __uint_as_float(s0 & 0xFFFF0000u);
    s1 = pack2(r0, r1);
    s2 = pack2(r0 - __uint_as_float(s1 << 16), r1 - __uint_as_float(s1 & 0xFFFF0000u));
}
// the three slices of 8 values (one 16-byte row of each slice)
__device__ __forceinline__ void split3x8(const float *x, uint4 &a, uint4 &b, uint4 &c) {
    split3x2(x[0], x[1], a.x, b.x, c.x);
    split3x2(x[2], x[3], a.y, b.y, c.y);
    split3x2(x[4], x[5], a.z, b.z, c.z);
    split3x2(x[6], x[7], a.w, b.w, c.w);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(su32(bar)), "r"(parity) : "memory");
    return done != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

struct TcShared {
    unsigned long long full[kRing], empty[kRing];    // FP32 stage loaded / read
    unsigned long long sfull[kSlots], sempty[kSlots];  // slices written / read by the MMAs
    unsigned long long accfull[2], accempty[2];      // accumulators complete / drained
    unsigned long long done;                         // every MMA issued has completed
    uint32_t tslot;
    volatile int abort;
};

// Bounded wait on phase `parity` of `bar` by one thread.  Gives up when
// another role has given up, or after `limit` polls (then it sets the status
// word and tells the other roles).
__device__ __forceinline__ bool wait_bar(TcShared &sh, unsigned long long *bar, uint32_t parity, long long limit,
                                         int *status) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (sh.abort) return false;
        __nanosleep(20);
    }
    atomicExch(status, 2);
    sh.abort = 1;
    return false;
}
// The same for a whole warp, with one outcome for all lanes: lane 0 polls;
// after a completed phase every lane observes it too (so each lane's reads of
// the data the phase guards are ordered after it; the phase cannot advance
// before this warp arrives on the barrier that frees it).
__device__ __forceinline__ bool warp_wait(TcShared &sh, unsigned long long *bar, uint32_t parity, long long limit,
                                          int *status) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = wait_bar(sh, bar, parity, limit, status) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) (void)mbar_try(bar, parity);
    return ok != 0;
}

// Real columns of a tile: 128 for the lowest group (64 blocks x re/im); for an
// upper group 128 x 128 / K, run as 128 / K blocks of 128 columns.
template <int KB, bool LOW> __host__ __device__ constexpr int tile_cols() { return LOW ? kRows : kRows * (128 >> KB); }

// First amplitude of a tile (the mids are 2^lo apart).
template <int KB, bool LOW> __device__ __forceinline__ uint64_t tile_base(uint64_t tile, int lo) {
    if (LOW) return tile * 8192ull;
    constexpr int AMPS = tile_cols<KB, false>() / 2;
    const uint64_t per_outer = (1ull << lo) / AMPS;
    return ((tile / per_outer) << (lo + KB)) | ((tile % per_outer) * AMPS);
}

template <int KB, bool LOW>
__global__ void __launch_bounds__(kTcThreads, 1)
k_wht_tc(float *amps, const __grid_constant__ CUtensorMap tmap, int lo, uint64_t ntiles, float scale,
         int negate_but_zero, int *status, long long wait_limit, int stall) {
    constexpr int K = 1 << KB;
    constexpr int KC = K / kChunkK;          // chunks per block of 128 columns
    constexpr int NB = kChunksPerTile / KC;  // blocks of 128 columns per tile
    constexpr int N_MMA = LOW ? kRows : K;   // accumulator columns per block
    constexpr int RING = kRing;
    static_assert(!LOW || KB == 7, "the lowest group uses W as the 128-row operand");
    static_assert(NB * 2 * N_MMA == 256, "one tile's accumulators fill 256 TMEM columns");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *ring = smem;                                 // [RING][8 KiB] FP32 chunks
    unsigned char *slots = smem + RING * kStageBytes;           // [kSlots][3][4 KiB] bf16 slices
    unsigned char *wsm = slots + kSlots * kSlotBytes;           // [KC][K rows][16] bf16 W
    TcShared &sh = *reinterpret_cast<TcShared *>(wsm + K * K * 2);  // barriers (all shared memory is dynamic)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the 128-byte swizzle of the lowest group's stages repeats every 1024
    // bytes: the ring must start on such a boundary
    if (su32(ring) & 1023u) {
        if (tid == 0) atomicExch(status, 4);
        return;
    }
    // W[n][k] = w (-1)^popcount(n & k), w = the pass scale (a power of two),
    // negated when the pass applies the phase shift 2|0><0| - I (every
    // amplitude but index 0 negated; the epilogue restores index 0): exact in
    // bf16, so the products and sums are those of the unscaled pass scaled
    const float wv = negate_but_zero ? -scale : scale;
    for (int i = tid; i < K * K / 8; i += kTcThreads) {
        const int n = i / (K / 8), k0 = (i % (K / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (__popc(n & (k0 + j)) & 1) ? -wv : wv;
        uint4 q;
        q.x = pack2(v[0], v[1]);
        q.y = pack2(v[2], v[3]);
        q.z = pack2(v[4], v[5]);
        q.w = pack2(v[6], v[7]);
        *reinterpret_cast<uint4 *>(wsm + (k0 >> 4) * (K * 32) + core_off(n, k0 & 15)) = q;
    }
    if (tid == 0) {
        sh.abort = 0;
        for (int s = 0; s < RING; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.empty[s])) : "memory");
        }
        for (int s = 0; s < kSlots; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.sfull[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.sempty[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.accfull[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sh.accempty[b])), "r"(kEpiWarps) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tslot)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W, for the tensor cores
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t taddr = sh.tslot;

    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t my_chunks = my_tiles * kChunksPerTile;

    if (warp == kTmaWarp) {
        // ---- producer: one tensor copy per chunk -------------------------------------
        uint64_t issued = 0;
        if (lane == 0) {
            for (uint64_t q = 0; q < my_chunks; ++q) {
                const int s = (int)(q % RING);
                if (q >= (uint64_t)RING &&
                    !wait_bar(sh, &sh.empty[s], (uint32_t)((q / RING - 1) & 1), wait_limit, status))
                    break;
                const uint64_t tile = blockIdx.x + (q / kChunksPerTile) * gridDim.x;
                const int j = (int)(q % kChunksPerTile), blk = j / KC, c = j % KC;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&sh.full[s])),
                             "r"(kStageBytes) : "memory");
                if (LOW) {
                    // view [block of 128 amplitudes][256 floats], box {32 floats, 64 blocks}
                    const int x = 32 * c, y = (int)(tile * 64);
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                                 "[%0], [%1, {%2, %3}], [%4];"
                                 ::"r"(su32(ring + s * kStageBytes)), "l"(&tmap), "r"(x), "r"(y), "r"(su32(&sh.full[s]))
                                 : "memory");
                } else {
                    // view [outer][K mids][2^(lo+1) floats], box {128 floats, 16 mids, 1}
                    constexpr int COLS = tile_cols<KB, false>();
                    const uint64_t per_outer = (1ull << (lo + 1)) / COLS;
                    const int x = (int)((tile % per_outer) * COLS) + blk * kRows, y = kChunkK * c;
                    const int z = (int)(tile / per_outer);
                    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                                 "[%0], [%1, {%2, %3, %4}], [%5];"
                                 ::"r"(su32(ring + s * kStageBytes)), "l"(&tmap), "r"(x), "r"(y), "r"(z),
                                   "r"(su32(&sh.full[s]))
                                 : "memory");
                }
                ++issued;
            }
            // every copy issued must have landed before the CTA's shared memory
            // is released (after an abort some may still be in flight); the
            // kernel has failed by then, so the wait may be long
            const uint64_t first = issued > (uint64_t)RING ? issued - RING : 0;
            for (uint64_t q = first; q < issued; ++q) {
                const int s = (int)(q % RING);
                for (long long it = 0; it < 64 * wait_limit && !mbar_try(&sh.full[s], (uint32_t)((q / RING) & 1)); ++it)
                    __nanosleep(20);
            }
        }
    } else if (warp == kMmaWarp) {
        // ---- MMA issue: one thread --------------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, N_MMA);
            uint64_t q = 0;
            bool ok = true;
            for (uint64_t i = 0; ok && i < my_tiles; ++i) {
                const uint32_t b = (uint32_t)(i & 1);
                if (i >= 2 && !wait_bar(sh, &sh.accempty[b], (uint32_t)((i / 2 - 1) & 1), wait_limit, status)) break;
                fence_after();
                for (int j = 0; j < kChunksPerTile; ++j, ++q) {
                    const int p = (int)(q % kSlots), blk = j / KC, c = j % KC;
                    if (!wait_bar(sh, &sh.sfull[p], (uint32_t)((q / kSlots) & 1), wait_limit, status)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t d0 = taddr + 256u * b + (uint32_t)(blk * 2 * N_MMA);
                    const uint64_t dw = smem_desc(su32(wsm + c * (K * 32)));
#pragma unroll
                    for (int sl = 0; sl < 3; ++sl) {
                        const uint64_t dx = smem_desc(su32(slots + p * kSlotBytes + sl * kSliceBytes));
                        const uint64_t da = LOW ? dw : dx, db = LOW ? dx : dw;
                        const uint32_t d = d0 + (sl ? (uint32_t)N_MMA : 0u);
                        const uint32_t acc = (sl == 2 || c != 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(d), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
                    }
                    mma_commit(&sh.sempty[p]);  // the slot is free once these MMAs have read it
                }
                if (!ok) break;
                // test hook: without this commit the epilogue's wait runs out
                if (!(stall && i == 0)) mma_commit(&sh.accfull[b]);
            }
            // every MMA issued has completed before the tensor memory is freed
            mma_commit(&sh.done);
            for (long long it = 0; it < 64 * wait_limit && !mbar_try(&sh.done, 0u); ++it) __nanosleep(20);
        }
    } else if (warp >= kConvWarp0) {
        // ---- converters: FP32 chunk -> three bf16 slices ---------------------------------
        // warp w converts chunks w, w + 8, ... from stage w into slot w, so eight
        // chunks are converted at once; lane l takes the columns l, l + 32,
        // l + 64, l + 96 (all 16 mids of each) and writes 16-byte rows, the 32
        // lanes of a store covering four whole 128-byte core-matrix rows
        const int w = warp - kConvWarp0;
        for (uint64_t q = (uint64_t)w; q < my_chunks; q += kConvWarps) {
            const uint32_t use = (uint32_t)(q / kConvWarps);  // uses of slot w so far
            const int s = (int)(q % RING);
            const uint32_t ph = (uint32_t)(q / RING);
            if (ph >= 1 && !warp_wait(sh, &sh.empty[s], (ph - 1) & 1u, wait_limit, status)) break;
            if (!warp_wait(sh, &sh.full[s], ph & 1u, wait_limit, status)) break;
            const unsigned char *st = ring + s * kStageBytes;
            unsigned char *slot = slots + w * kSlotBytes;
            if (LOW) {
                // unit u = lane + 32 r: block u / 2 (columns 2b = re, 2b + 1 = im),
                // mids 8 (u & 1) .. + 7, read as four 16-byte (re, im, re, im)
                // pieces; the stage holds 128-byte lines (one per block) whose
                // 16-byte chunks the copy permuted, chunk c of line L at
                // c ^ (L & 7), so the eight lanes of a load phase hit eight
                // different chunks
                float4 v[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int u = lane + 32 * r, b = u >> 1, h = u & 1;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        v[r][c] = *reinterpret_cast<const float4 *>(st + b * 128 +
                                                                    ((uint32_t)((4 * h + c) ^ (b & 7)) << 4));
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.empty[s]);  // the stage is read
                if (use >= 1 && !warp_wait(sh, &sh.sempty[w], (use - 1) & 1u, wait_limit, status)) break;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int u = lane + 32 * r, b = u >> 1, h = u & 1;
                    float re[8], im[8];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        re[2 * c] = v[r][c].x;
                        im[2 * c] = v[r][c].y;
                        re[2 * c + 1] = v[r][c].z;
                        im[2 * c + 1] = v[r][c].w;
                    }
                    uint4 a0, a1, a2;
                    split3x8(re, a0, a1, a2);
                    *reinterpret_cast<uint4 *>(slot + core_off(2 * b, 8 * h)) = a0;
                    *reinterpret_cast<uint4 *>(slot + kSliceBytes + core_off(2 * b, 8 * h)) = a1;
                    *reinterpret_cast<uint4 *>(slot + 2 * kSliceBytes + core_off(2 * b, 8 * h)) = a2;
                    split3x8(im, a0, a1, a2);
                    *reinterpret_cast<uint4 *>(slot + core_off(2 * b + 1, 8 * h)) = a0;
                    *reinterpret_cast<uint4 *>(slot + kSliceBytes + core_off(2 * b + 1, 8 * h)) = a1;
                    *reinterpret_cast<uint4 *>(slot + 2 * kSliceBytes + core_off(2 * b + 1, 8 * h)) = a2;
                }
            } else {
                // [16 mids][128 floats]; lane l takes columns l, l + 32, l + 64,
                // l + 96 (consecutive lanes: consecutive floats, whole 128-byte
                // rows of the core matrices on the stores)
                float v[4][16];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int mid = 0; mid < 16; ++mid)
                        v[r][mid] = reinterpret_cast<const float *>(st)[mid * kRows + lane + 32 * r];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.empty[s]);  // the stage is read
                if (use >= 1 && !warp_wait(sh, &sh.sempty[w], (use - 1) & 1u, wait_limit, status)) break;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint4 a0, a1, a2;
                        split3x8(&v[r][8 * h], a0, a1, a2);
                        const uint32_t off = core_off(lane + 32 * r, 8 * h);
                        *reinterpret_cast<uint4 *>(slot + off) = a0;
                        *reinterpret_cast<uint4 *>(slot + kSliceBytes + off) = a1;
                        *reinterpret_cast<uint4 *>(slot + 2 * kSliceBytes + off) = a2;
                    }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // slices, for the tensor cores
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.sfull[w]);
        }
    } else {
        // ---- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31 ------------------------
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        for (uint64_t i = 0; i < my_tiles; ++i) {
            const uint32_t b = (uint32_t)(i & 1);
            if (!warp_wait(sh, &sh.accfull[b], (uint32_t)((i / 2) & 1), wait_limit, status)) break;
            fence_after();
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            const uint64_t abase = tile_base<KB, LOW>(tile, lo);
            constexpr int GROUPS = NB * (N_MMA / 32);  // 32-column groups per accumulator
#pragma unroll 1
            for (int g = 0; g < GROUPS; ++g) {
                const int blk = g / (N_MMA / 32), cg = g % (N_MMA / 32);
                uint32_t a[32], z[32];
                const uint32_t t0 = taddr + lane_base + 256u * b + (uint32_t)(blk * 2 * N_MMA + 32 * cg);
                tmem_ld32(t0 + (uint32_t)N_MMA, a);  // A12
                tmem_ld32(t0, z);                    // A0
                tmem_wait_ld();
                if (g == GROUPS - 1) {
                    // the accumulators of this tile are read: hand them back
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.accempty[b]);
                }
                // W carried the scale and the phase-shift sign; only amplitude 0
                // (in tile 0, first group, warp 0) must not be negated
                const bool fix0 = negate_but_zero && tile == 0 && g == 0 && warp == 0;
                if (LOW) {
                    // lane = output mid r; registers = 16 blocks x (re, im):
                    // stores of 32 consecutive amplitudes per warp
                    const int r = 32 * warp + lane;
                    float2 *p = reinterpret_cast<float2 *>(amps) + abase + (uint64_t)(16 * cg) * 128 + r;
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        float re = __uint_as_float(a[2 * t]) + __uint_as_float(z[2 * t]);
                        float im = __uint_as_float(a[2 * t + 1]) + __uint_as_float(z[2 * t + 1]);
                        if (t == 0 && fix0 && lane == 0) {
                            re = -re;
                            im = -im;
                        }
                        __stcs(p + t * 128, make_float2(re, im));
                    }
                } else {
                    // lane = column (re or im of amplitude col / 2), registers =
                    // 32 consecutive output mids: each store writes 32
                    // consecutive floats of one mid
                    const int col = kRows * blk + 32 * warp + lane;
                    float *p = amps + 2 * abase + col + ((uint64_t)(32 * cg) << (lo + 1));
                    const uint64_t stride = 2ull << lo;  // floats between consecutive mids
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float x = __uint_as_float(a[j]) + __uint_as_float(z[j]);
                        if (j == 0 && fix0 && lane < 2) x = -x;
                        __stcs(p, x);
                        p += stride;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == kMmaWarp) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
    }
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
// [outer][mid][2^(lo+1) floats], box {128 floats, 16 mids, 1}.
cudaError_t encode_upper_map(CUtensorMap *m, void *amps, int n, int lo, int kb) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t inner = 1ull << (lo + 1);
    const cuuint64_t dims[3] = {inner, 1ull << kb, 1ull << (n - lo - kb)};
    const cuuint64_t strides[2] = {inner * 4, (inner << kb) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kRows, (cuuint32_t)kChunkK, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, amps, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// View of the state for the lowest group: [block of 128 amplitudes][256
// floats], box {32 floats, 64 blocks} with the 128-byte swizzle.
cudaError_t encode_low_map(CUtensorMap *m, void *amps, int n) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {256, 1ull << (n - 7)};
    const cuuint64_t strides[1] = {1024};
    const cuuint32_t box[2] = {32u, 64u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, amps, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int KB, bool LOW>
cudaError_t launch_tc_t(void *amps, int n, int lo, float scale, bool negate, int *status, long long wait_limit,
                        int stall, cudaStream_t st, const Geometry &g) {
    constexpr int K = 1 << KB;
    // stages, slots, W, barriers; at least 120 KiB so that one CTA runs per
    // SM (each allocates all 512 TMEM columns)
    size_t smem = (size_t)kRing * kStageBytes + (size_t)kSlots * kSlotBytes + (size_t)K * K * 2 + sizeof(TcShared);
    if (smem < 120 * 1024) smem = 120 * 1024;
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
    const uint64_t ntiles = (1ull << n) / 8192ull;
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
