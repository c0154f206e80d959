// k_noalloc.cu -- grover_iterate_noalloc: Grover iterations without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a framework's
// caching allocator owns the device memory budget, real-time loops that must
// not take the implicit device synchronisation of cudaMalloc/cudaFree, or
// plugins that are only handed device buffers.  grover_create allocates a
// small scratch area, so those callers cannot use a state handle.  This entry
// point runs the same fused iteration passes with their scratch (per-CTA
// partial sums, the double-buffered mean and the last-CTA ticket) in a
// file-scope __device__ array instead, which every GPU that loads the library
// holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks the
// array's device address up with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.  All calls on a device share the one
// array and it keeps the last call's contents, so each call clears the ticket
// it relies on; calls that overlap on the GPU (different streams, or host
// threads without ordering) race on the array and give wrong results.
#include <stdio.h>

#include <mutex>

#include "grover_internal.cuh"
#include "trace.cuh"

namespace {

constexpr int kNoAllocSlots = 2048;  // per-CTA partial sums: at most this many CTAs per pass
constexpr size_t kPartialsBytes = sizeof(double2) * kNoAllocSlots;
constexpr size_t kMuOffset = kPartialsBytes;           // MeanSlot mu[2] (96 bytes)
constexpr size_t kTicketOffset = kMuOffset + 256;      // unsigned ticket
constexpr size_t kNoAllocBytes = kTicketOffset + 256;  // 33,280 bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// The message is what grover_last_error(NULL) returns on this host thread.
grover_status noalloc_fail(grover_status st, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(buf, sizeof buf, "grover_iterate_noalloc: %s: %s", msg, cudaGetErrorString(e));
    } else {
        snprintf(buf, sizeof buf, "grover_iterate_noalloc: %s", msg);
    }
    grv::set_thread_error(buf);
    return st;
}

// Device address of the scratch array on device dev (dev must be current).
grover_status scratch_address(int dev, char **out) {
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(GROVER_EUNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(GROVER_ECUDA, "cudaGetSymbolAddress", e);
        g_scratch_addr[dev] = p;
    }
    *out = (char *)g_scratch_addr[dev];
    return GROVER_OK;
}

bool is_device_pointer(const void *p, int dev) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == dev;
}

}  // namespace

extern "C" grover_status grover_iterate_noalloc(void *dev_amps, int n, grover_dtype dtype,
                                                const uint64_t *dev_marked, size_t m, uint64_t k,
                                                void *cuda_stream) {
    GROVER_TRACE("grover_iterate_noalloc");
    using namespace grv;
    if (dtype != GROVER_C64 && dtype != GROVER_C128) return noalloc_fail(GROVER_EINVAL, "unknown dtype");
    const int nmax = dtype == GROVER_C64 ? 33 : 32;
    if (n < 1 || n > nmax) return noalloc_fail(GROVER_EINVAL, "n outside [1, 33] (complex64) / [1, 32] (complex128)");
    const uint64_t N = 1ull << n;
    if (m > N) return noalloc_fail(GROVER_ERANGE, "m exceeds 2^n");
    if (!dev_amps || (uintptr_t)dev_amps % 16 != 0)
        return noalloc_fail(GROVER_EINVAL, "amplitude buffer is NULL or not 16-byte aligned");
    if (m > 0 && (!dev_marked || (uintptr_t)dev_marked % 8 != 0))
        return noalloc_fail(GROVER_EINVAL, "marked list is NULL or not 8-byte aligned");
    if (k == 0) return GROVER_OK;

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(GROVER_ECUDA, "cudaGetDevice", e);
    if (!is_device_pointer(dev_amps, dev)) return noalloc_fail(GROVER_EINVAL, "amplitude buffer is not memory of the current device");
    if (m > 0 && !is_device_pointer(dev_marked, dev))
        return noalloc_fail(GROVER_EINVAL, "marked list is not memory of the current device");

    Geometry geo;
    int sms = 0, l2 = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev)) != cudaSuccess)
        return noalloc_fail(GROVER_ECUDA, "cudaDeviceGetAttribute", e);
    geo.sm_count = sms;
    geo.dev = dev;
    geo.l2_bytes = l2;
    // the pass launcher caps every grid at the slots of the static array
    // (one per CTA with FP64 partial sums), whatever the device could hold
    geo.partial_slots = kNoAllocSlots;

    char *base = nullptr;
    if (grover_status st = scratch_address(dev, &base)) return st;
    double2 *partials = (double2 *)base;
    MeanSlot *mu = (MeanSlot *)(base + kMuOffset);
    unsigned *ticket = (unsigned *)(base + kTicketOffset);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // the array keeps the previous call's contents: start from a zero ticket
    if ((e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream)) != cudaSuccess)
        return noalloc_fail(GROVER_ECUDA, "ticket reset", e);

    MarkedDev mk;
    mk.list = m ? dev_marked : nullptr;
    mk.words = nullptr;
    mk.m = m;
    mk.mode = m ? MARK_LIST : MARK_NONE;
    PassArgs a;
    a.amps = dev_amps;
    a.nvec = dtype == GROVER_C64 ? N / 2 : N;
    a.mk = mk;
    a.partials = partials;
    a.ticket = ticket;
    a.inv_n = ldexp(1.0, -n);
    a.stream_hint = (long long)(N * (dtype == GROVER_C64 ? 8 : 16)) > geo.l2_bytes / 2;
    a.status = nullptr;  // no status word: a staged wait that runs out is not reported here
    a.wait_limit = 1ll << 22;
    a.staged = 0;  // per-thread pass: the grid stays within the resident-CTA bound the scratch is sized for
    a.stall = 0;

    // mean of O c for the first iteration, then k fused passes; FP64
    // accumulation keeps one partial-sum slot per CTA
    const grover_accum acc = GROVER_ACC_FP64;
    a.mu_in = mu;
    a.mu_out = mu;
    if ((e = launch_reduce(a, dtype, acc, stream, geo)) != cudaSuccess)
        return noalloc_fail(GROVER_ECUDA, "mean reduction launch", e);
    int slot = 0;
    for (uint64_t t = 0; t < k; ++t) {
        a.mu_in = mu + slot;
        a.mu_out = mu + (slot ^ 1);
        if ((e = launch_pass(a, dtype, acc, stream, geo)) != cudaSuccess)
            return noalloc_fail(GROVER_ECUDA, "iteration pass launch", e);
        slot ^= 1;
    }
    return GROVER_OK;
}
