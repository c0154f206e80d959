// grover_batch.cu -- C ABI of the batched searches (declared in include/grover.h).
//
// Host side only: validation, the instance table on the device (largest N * k
// first), the autotuner over the kernel's thread count and on-chip threshold,
// and the CUDA graph that holds the one persistent launch.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "grover_internal.cuh"
#include "trace.cuh"

using namespace grv;

struct grover_batch {
    size_t count;
    cudaStream_t stream;
    int sm_count;
    float4 *amps;
    void *dev_mem;          // instance table, orders, marked lists, counters, results
    BatchLaunch L;          // small instances, one CTA each
    BatchClusterLaunch LC;  // large instances, one cluster each
    unsigned grid;
    int clusters;           // co-resident clusters (0: cluster packing unavailable)
    int packing;            // 0 / 1: one CTA per instance; kBatchClusterSize: clusters for the large
                            // instances; kBatchPackGroups: groups of CTAs for the large instances
    int pack_min_qubits;    // with packing: instances of at least this many qubits leave the one-CTA kernel
    // groups of CTAs (packing == kBatchPackGroups): one launch per instance size
    struct GroupClass {
        int n;
        unsigned groups, ctas;  // groups x CTAs per group
        uint32_t slice_vecs;
        size_t smem;
        uint32_t list_off, goff_off;  // into the device glist / goff arrays
    };
    std::vector<GroupClass> gclasses;
    void *group_mem;        // glist, goff, the exchange region, the status word
    unsigned long long *group_region;
    int *group_status;
    int group_per_sm;       // resident group-kernel CTAs per SM (0: groups unavailable)
    size_t glist_len;       // entries of the device glist (every class's lists)
    long long wait_limit;   // polls of a bounded wait in the group kernel
    int test_stall;         // test hook: group 0's first exchange never completes
    std::vector<uint64_t> kk;  // iterations per instance
    uint32_t *order_dev;    // [2 * count]: small order, then large order
    std::vector<uint32_t> order;  // all instances, largest N * k first
    std::vector<int> nq;    // qubits per instance
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ready;
    double work;            // sum of N * k
    char err[512];
};

namespace {

constexpr int kBatchPackGroups = 2;  // packing value of the CTA-group mode

grover_status bfail(grover_batch *b, grover_status st, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
        if (e == cudaErrorMemoryAllocation) st = GROVER_ENOMEM;
    } else {
        snprintf(buf, sizeof buf, "%s", msg);
    }
    set_thread_error(buf);
    if (b) snprintf(b->err, sizeof b->err, "%s", buf);
    return st;
}

// Splits the instances between the two kernels (large ones to clusters when
// packing is on and clusters can run) and uploads both orders.
// Instances of size n that the CTA-group kernel can hold (a group fits the GPU).
bool group_fits(const grover_batch *b, int n) {
    if (b->group_per_sm < 1 || n < kBatchGroupMinQubits) return false;
    const int G = batch_group_ctas(n, kBatchGroupSmemMax);
    return G > 0 && G <= b->sm_count;
}

// Group mode: the instances of each size n >= the threshold that a group can
// hold, spread over floor(SMs / G) groups, each next instance (largest k first)
// to the group with the least work so far; uploads the lists and sizes the
// exchange region for the largest class.
grover_status plan_groups(grover_batch *b, const std::vector<uint32_t> &large) {
    b->gclasses.clear();
    if (b->group_mem) {
        cudaFree(b->group_mem);
        b->group_mem = nullptr;
    }
    if (large.empty()) return GROVER_OK;
    std::vector<uint32_t> glist, goff;
    size_t region_words_max = 0;
    for (int n = kBatchMaxQubits; n >= kBatchGroupMinQubits; --n) {
        std::vector<uint32_t> cls;
        for (uint32_t i : large)
            if (b->nq[i] == n) cls.push_back(i);
        if (cls.empty()) continue;
        grover_batch::GroupClass gc;
        gc.n = n;
        gc.ctas = (unsigned)batch_group_ctas(n, kBatchGroupSmemMax);
        gc.groups = (unsigned)(b->sm_count / (int)gc.ctas);
        if (gc.groups > cls.size()) gc.groups = (unsigned)cls.size();
        const uint64_t nvec = (1ull << n) / 2;
        gc.slice_vecs = (uint32_t)((nvec + gc.ctas - 1) / gc.ctas);
        gc.smem = (size_t)gc.slice_vecs * 16;
        // longest processing time first: instances by k, largest first
        std::stable_sort(cls.begin(), cls.end(), [&](uint32_t x, uint32_t y) { return b->kk[x] > b->kk[y]; });
        std::vector<std::vector<uint32_t>> per(gc.groups);
        std::vector<double> load(gc.groups, 0.0);
        for (uint32_t i : cls) {
            const size_t g = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
            per[g].push_back(i);
            load[g] += (double)b->kk[i] + 1.0;
        }
        gc.list_off = (uint32_t)glist.size();
        gc.goff_off = (uint32_t)goff.size();
        uint32_t o = 0;
        for (unsigned g = 0; g < gc.groups; ++g) {
            goff.push_back(o);
            for (uint32_t i : per[g]) glist.push_back(i);
            o += (uint32_t)per[g].size();
        }
        goff.push_back(o);
        region_words_max = std::max(region_words_max, (size_t)gc.groups * batch_group_region_words((int)gc.ctas));
        b->gclasses.push_back(gc);
    }
    const size_t s_list = ((glist.size() * 4) + 255) & ~size_t(255), s_goff = ((goff.size() * 4) + 255) & ~size_t(255);
    const size_t s_region = ((region_words_max * 8) + 255) & ~size_t(255);
    char *mem = nullptr;
    cudaError_t e = cudaMalloc((void **)&mem, s_list + s_goff + s_region + 256);
    if (e != cudaSuccess) return bfail(b, GROVER_ENOMEM, "device allocation of the group tables", e);
    b->group_mem = mem;
    b->group_region = (unsigned long long *)(mem + s_list + s_goff);
    b->group_status = (int *)(mem + s_list + s_goff + s_region);
    if ((e = cudaMemcpy(mem, glist.data(), glist.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(mem + s_list, goff.data(), goff.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(b->group_status, 0, sizeof(int))) != cudaSuccess)
        return bfail(b, GROVER_ECUDA, "upload of the group tables", e);
    return GROVER_OK;
}

BatchGroupLaunch group_launch(const grover_batch *b, const grover_batch::GroupClass &gc) {
    const char *mem = (const char *)b->group_mem;
    const size_t s_list = ((b->glist_len * 4) + 255) & ~size_t(255);  // glist, then goff
    BatchGroupLaunch G;
    G.amps = b->amps;
    G.inst = b->L.inst;
    G.marked = b->L.marked;
    G.glist = (const uint32_t *)mem + gc.list_off;
    G.goff = (const uint32_t *)(mem + s_list) + gc.goff_off;
    G.psucc = b->L.psucc;
    G.region = b->group_region;
    G.region_words = batch_group_region_words((int)gc.ctas);
    G.group_ctas = gc.ctas;
    G.slice_vecs = gc.slice_vecs;
    G.status = b->group_status;
    G.wait_limit = b->wait_limit;
    G.stall = b->test_stall;
    return G;
}

grover_status split(grover_batch *b) {
    const bool clusters = b->packing == kBatchClusterSize && b->clusters > 0;
    const bool groups = b->packing == kBatchPackGroups && b->group_per_sm > 0;
    std::vector<uint32_t> small, large;
    for (uint32_t i : b->order) {
        const int n = b->nq[i];
        const bool big = (clusters && n >= std::max(b->pack_min_qubits, kBatchClusterMinQubits)) ||
                         (groups && n >= b->pack_min_qubits && group_fits(b, n));
        (big ? large : small).push_back(i);
    }
    if (groups) {
        b->glist_len = large.size();
        if (grover_status st = plan_groups(b, large)) return st;
        large.clear();  // the group launches take them; the cluster kernel gets none
    } else {
        b->gclasses.clear();
    }
    cudaError_t e = cudaSuccess;
    if (!small.empty())
        e = cudaMemcpy(b->order_dev, small.data(), small.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !large.empty())
        e = cudaMemcpy(b->order_dev + b->count, large.data(), large.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "upload of the batch orders", e);
    b->L.order = b->order_dev;
    b->L.count = (uint32_t)small.size();
    b->LC.order = b->order_dev + b->count;
    b->LC.count = (uint32_t)large.size();
    return GROVER_OK;
}

grover_status rebuild(grover_batch *b) {
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->graph_ready = false;
    }
    cudaError_t e = prepare_batch(b->L, b->sm_count, &b->grid);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "batch kernel set-up", e);
    if (grover_status st = split(b)) return st;
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return bfail(b, GROVER_ECUDA, "capture stream", e);
    size_t gsmem = 0;
    for (const auto &gc : b->gclasses) gsmem = std::max(gsmem, gc.smem);
    if (gsmem) {
        int per_sm = 0;
        if ((e = prepare_batch_group(gsmem, &per_sm)) != cudaSuccess) return bfail(b, GROVER_ECUDA, "group kernel set-up", e);
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // large instances first (they hold the longest runs), then the small ones
        cudaError_t e2 = cudaSuccess;
        for (const auto &gc : b->gclasses)
            if (e2 == cudaSuccess) e2 = enqueue_batch_group(group_launch(b, gc), gc.groups, gc.smem, cs);
        if (e2 == cudaSuccess && b->LC.count) e2 = enqueue_batch_cluster(b->LC, b->clusters, cs);
        if (e2 == cudaSuccess) e2 = enqueue_batch(b->L, b->grid, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e2 != cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "graph capture of the batch launch", e);
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(b->graph);
        return bfail(b, GROVER_ECUDA, "graph instantiation", e);
    }
    b->graph_ready = true;
    return GROVER_OK;
}

}  // namespace

extern "C" {

uint64_t grover_batch_amps_needed(size_t count, const int *n_qubits) {
    if (!n_qubits) return 0;
    uint64_t total = 0;
    for (size_t i = 0; i < count; ++i) {
        if (n_qubits[i] < 1 || n_qubits[i] > kBatchMaxQubits) return 0;
        total += 1ull << n_qubits[i];
    }
    return total;
}

grover_status grover_batch_create(grover_batch **out, size_t count, const int *n_qubits, const uint64_t *k,
                                  const uint64_t *marked, const uint64_t *marked_offsets, void *dev_amps,
                                  uint64_t amps_capacity, void *cuda_stream) {
    if (!out || !n_qubits || !k || !marked_offsets || !dev_amps)
        return bfail(nullptr, GROVER_EINVAL, "NULL argument");
    if (count == 0 || count > (1u << 30)) return bfail(nullptr, GROVER_EINVAL, "count must be in [1, 2^30]");
    if ((uintptr_t)dev_amps % 16) return bfail(nullptr, GROVER_EINVAL, "amplitude buffer is not 16-byte aligned");
    if (marked_offsets[0] != 0) return bfail(nullptr, GROVER_EINVAL, "marked_offsets[0] must be 0");
    std::vector<BatchInst> inst(count);
    uint64_t off = 0;
    double work = 0.0;
    for (size_t i = 0; i < count; ++i) {
        const int n = n_qubits[i];
        if (n < 1 || n > kBatchMaxQubits) return bfail(nullptr, GROVER_EINVAL, "an instance has n outside [1, 26]");
        const uint64_t N = 1ull << n;
        const uint64_t m0 = marked_offsets[i], m1 = marked_offsets[i + 1];
        if (m1 < m0) return bfail(nullptr, GROVER_EINVAL, "marked_offsets must not decrease");
        const uint64_t m = m1 - m0;
        if (m > kBatchMaxMarked) return bfail(nullptr, GROVER_EINVAL, "an instance has more than 64 marked indices");
        if (m && !marked) return bfail(nullptr, GROVER_EINVAL, "marked list is NULL");
        for (uint64_t j = 0; j < m; ++j) {
            const uint64_t x = marked[m0 + j];
            if (x >= N) return bfail(nullptr, GROVER_ERANGE, "a marked index is >= 2^n of its instance");
            if (j && x == marked[m0 + j - 1]) return bfail(nullptr, GROVER_EDUP, "a marked list holds an index twice");
            if (j && x < marked[m0 + j - 1]) return bfail(nullptr, GROVER_EUNSORTED, "a marked list decreases");
        }
        inst[i] = BatchInst{off, k[i], m0, (uint32_t)m, n};
        off += N;
        work += (double)N * (double)k[i];
    }
    if (off > amps_capacity) return bfail(nullptr, GROVER_EINVAL, "amplitude buffer smaller than the batch");
    const uint64_t total_marked = marked_offsets[count];
    std::vector<uint32_t> order(count);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return (double)(1ull << inst[a].n) * (double)(inst[a].k + 1) > (double)(1ull << inst[b].n) * (double)(inst[b].k + 1);
    });

    grover_batch *b = new (std::nothrow) grover_batch();
    if (!b) return bfail(nullptr, GROVER_ENOMEM, "host allocation of the batch");
    b->order = order;
    b->nq.resize(count);
    b->kk.resize(count);
    for (size_t i = 0; i < count; ++i) {
        b->nq[i] = inst[i].n;
        b->kk[i] = inst[i].k;
    }
    b->group_mem = nullptr;
    b->gclasses.clear();
    b->glist_len = 0;
    b->wait_limit = kDefaultWaitLimit;
    b->test_stall = 0;
    b->count = count;
    b->stream = (cudaStream_t)cuda_stream;
    b->amps = (float4 *)dev_amps;
    b->work = work;
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        delete b;
        return bfail(nullptr, GROVER_ECUDA, "device query", e);
    }
    const size_t s_inst = ((count * sizeof(BatchInst)) + 255) & ~size_t(255);
    const size_t s_order = ((2 * count * sizeof(uint32_t)) + 255) & ~size_t(255);
    const size_t s_mark = ((std::max<uint64_t>(total_marked, 1) * sizeof(uint64_t)) + 255) & ~size_t(255);
    const size_t s_next = 256, s_res = ((count * sizeof(double)) + 255) & ~size_t(255);
    char *mem = nullptr;
    if ((e = cudaMalloc((void **)&mem, s_inst + s_order + s_mark + s_next + s_res)) != cudaSuccess) {
        delete b;
        return bfail(nullptr, GROVER_ENOMEM, "device allocation of the batch tables", e);
    }
    b->dev_mem = mem;
    BatchLaunch &L = b->L;
    L.amps = b->amps;
    L.inst = (const BatchInst *)mem;
    L.order = (const uint32_t *)(mem + s_inst);
    L.marked = (const uint64_t *)(mem + s_inst + s_order);
    L.next = (unsigned *)(mem + s_inst + s_order + s_mark);
    L.psucc = (double *)(mem + s_inst + s_order + s_mark + s_next);
    L.count = (uint32_t)count;
    L.onchip_vecs = 8192;  // 128 KiB: instances up to n = 14
    L.threads = 512;
    b->order_dev = (uint32_t *)(mem + s_inst);
    BatchClusterLaunch &LC = b->LC;
    LC.amps = b->amps;
    LC.inst = L.inst;
    LC.marked = L.marked;
    LC.next = L.next + 32;  // its own counter, 128 bytes after the first
    LC.psucc = L.psucc;
    if (prepare_batch_cluster(&b->clusters) != cudaSuccess) {
        (void)cudaGetLastError();
        b->clusters = 0;
    }
    {
        int coop = 0, per_sm = 0;
        b->group_per_sm = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
            prepare_batch_group(kBatchGroupSmemMax, &per_sm) == cudaSuccess)
            b->group_per_sm = per_sm;
        (void)cudaGetLastError();
    }
    // default: groups of CTAs for the instances of at least 15 qubits where
    // cooperative launches run (measured faster than one CTA per instance for
    // every size from 15 to 20 qubits), else one CTA per instance;
    // grover_batch_tune also tries the other packings
    b->packing = b->group_per_sm > 0 ? kBatchPackGroups : 0;
    b->pack_min_qubits = b->group_per_sm > 0 ? kBatchGroupMinQubits : kBatchClusterMinQubits;
    if ((e = cudaMemcpy((void *)L.inst, inst.data(), count * sizeof(BatchInst), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (total_marked && (e = cudaMemcpy((void *)L.marked, marked, total_marked * sizeof(uint64_t),
                                         cudaMemcpyHostToDevice)) != cudaSuccess)) {
        cudaFree(mem);
        delete b;
        return bfail(nullptr, GROVER_ECUDA, "upload of the batch tables", e);
    }
    if (grover_status st = rebuild(b)) {
        cudaFree(mem);
        delete b;
        return st;
    }
    *out = b;
    return GROVER_OK;
}

grover_status grover_batch_run(grover_batch *b) {
    GROVER_TRACE("grover_batch_run");
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "batch graph launch", e);
    return GROVER_OK;
}

grover_status grover_batch_tune(grover_batch *b, int *threads_out, uint32_t *onchip_vecs_out) {
    GROVER_TRACE("grover_batch_tune");
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    static const int kThreadsOpts[] = {256, 512, 1024};
    static const uint32_t kOnchipOpts[] = {2048, 4096, 8192};  // 32, 64, 128 KiB
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return bfail(b, GROVER_ECUDA, "tuner events", e);
    // the one-CTA kernel's shape is tuned over every instance
    b->packing = 0;
    if (grover_status st = split(b)) return st;
    BatchLaunch best = b->L;
    float best_ms = 3.4e38f;
    for (int th : kThreadsOpts) {
        for (uint32_t oc : kOnchipOpts) {
            BatchLaunch L = b->L;
            L.threads = th;
            L.onchip_vecs = oc;
            unsigned grid = 0;
            if (prepare_batch(L, b->sm_count, &grid) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;
            }
            float ms = 0.f;
            bool ok = enqueue_batch(L, grid, b->stream) == cudaSuccess;  // warm-up
            ok = ok && cudaEventRecord(e0, b->stream) == cudaSuccess && enqueue_batch(L, grid, b->stream) == cudaSuccess &&
                 cudaEventRecord(e1, b->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (!ok) {
                (void)cudaGetLastError();
                continue;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = L;
            }
        }
    }
    if (best_ms > 3.3e38f) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return bfail(b, GROVER_ECUDA, "no batch configuration could run");
    }
    b->L = best;
    // then whole graphs: one CTA per instance against clusters for the large ones
    b->packing = 0;
    if (grover_status st = rebuild(b)) return st;
    if (b->clusters > 0 || b->group_per_sm > 0) {
        auto time_graph = [&](float *ms) {
            return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess && cudaEventRecord(e0, b->stream) == cudaSuccess &&
                   cudaGraphLaunch(b->exec, b->stream) == cudaSuccess && cudaEventRecord(e1, b->stream) == cudaSuccess &&
                   cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
        };
        // clusters for the instances of at least 17 or at least 19 qubits
        // (17-18 qubits fit the clusters' shared memory, 19-20 stream through
        // L2), or none
        float t_best = 0.f;
        const bool ok1 = time_graph(&t_best);
        int best_min = 0, best_mode = 0;
        grover_status st = GROVER_OK;
        if (ok1) {
            static const int kMinOpts[] = {kBatchClusterMinQubits, kBatchClusterMinQubits + 2};
            int nmax = 0;
            for (int q : b->nq) nmax = q > nmax ? q : nmax;
            for (int mq : kMinOpts) {
                if (mq > nmax) continue;  // no instance would change place
                b->packing = kBatchClusterSize;
                b->pack_min_qubits = mq;
                float t = 0.f;
                st = rebuild(b);
                if (st == GROVER_OK && time_graph(&t) && t < t_best) {
                    t_best = t;
                    best_min = mq;
                    best_mode = kBatchClusterSize;
                }
                (void)cudaGetLastError();
            }
            // groups of CTAs for the instances of at least 15, 17 or 19 qubits
            static const int kGroupMinOpts[] = {kBatchGroupMinQubits, kBatchGroupMinQubits + 2,
                                                kBatchGroupMinQubits + 4};
            for (int mq : kGroupMinOpts) {
                bool any = false;
                for (int q : b->nq) any = any || (q >= mq && group_fits(b, q));
                if (!any) continue;
                b->packing = kBatchPackGroups;
                b->pack_min_qubits = mq;
                float t = 0.f;
                st = rebuild(b);
                if (st == GROVER_OK && time_graph(&t) && t < t_best) {
                    t_best = t;
                    best_min = mq;
                    best_mode = kBatchPackGroups;
                }
                (void)cudaGetLastError();
            }
        } else {
            (void)cudaGetLastError();
        }
        b->packing = best_mode;
        b->pack_min_qubits = best_min ? best_min : kBatchClusterMinQubits;
        if ((st = rebuild(b)) != GROVER_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (threads_out) *threads_out = best.threads;
    if (onchip_vecs_out) *onchip_vecs_out = best.onchip_vecs;
    return GROVER_OK;
}

grover_status grover_batch_set_packing(grover_batch *b, int cluster_size) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    if (cluster_size != 0 && cluster_size != 1 && cluster_size != kBatchClusterSize && cluster_size != kBatchPackGroups)
        return bfail(b, GROVER_EINVAL, "packing must be 0, 1, 2 or 16");
    if (cluster_size == kBatchClusterSize && b->clusters == 0)
        return bfail(b, GROVER_EUNSUPPORTED, "clusters of 16 CTAs cannot run on this device");
    if (cluster_size == kBatchPackGroups && b->group_per_sm == 0)
        return bfail(b, GROVER_EUNSUPPORTED, "the CTA-group kernel cannot run on this device");
    b->packing = cluster_size;
    return rebuild(b);
}

grover_status grover_batch_set_packing_min_qubits(grover_batch *b, int min_qubits) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    if (min_qubits < kBatchGroupMinQubits || min_qubits > kBatchMaxQubits)
        return bfail(b, GROVER_EINVAL, "the packing threshold must be in [15, 26] qubits");
    b->pack_min_qubits = min_qubits;
    return rebuild(b);
}

grover_status grover_batch_set_option(grover_batch *b, grover_option opt, int64_t value) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    switch (opt) {
    case GROVER_OPT_WAIT_LIMIT:
        if (value < 1) return bfail(b, GROVER_EINVAL, "wait limit must be >= 1");
        b->wait_limit = value;
        break;
    case GROVER_OPT_TEST_STALL:
        if (value != 0 && value != 1) return bfail(b, GROVER_EINVAL, "test stall must be 0 or 1");
        b->test_stall = (int)value;
        break;
    default:
        return bfail(b, GROVER_EINVAL, "option not available for batches (wait limit and test stall are)");
    }
    return rebuild(b);
}

grover_status grover_batch_get_packing(const grover_batch *b, int *cluster_size, int *min_qubits) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    if (cluster_size) *cluster_size = b->packing > 1 ? b->packing : 1;  // 1, 2 (groups) or 16
    if (min_qubits) *min_qubits = b->pack_min_qubits;
    return GROVER_OK;
}

grover_status grover_batch_success(grover_batch *b, double *p_success) {
    if (!b || !p_success) return bfail(b, GROVER_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(p_success, b->L.psucc, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    int status = 0;
    if (e == cudaSuccess && b->group_mem)
        e = cudaMemcpyAsync(&status, b->group_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "batch result copy", e);
    if (status) {
        (void)cudaMemset(b->group_status, 0, sizeof(int));
        return bfail(b, GROVER_ETIMEOUT, "a bounded wait of a CTA group gave up; the results are undefined");
    }
    return GROVER_OK;
}

grover_status grover_batch_destroy(grover_batch *b) {
    if (!b) return GROVER_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
    }
    cudaFree(b->dev_mem);
    if (b->group_mem) cudaFree(b->group_mem);
    delete b;
    if (e != cudaSuccess) return bfail(nullptr, GROVER_ECUDA, "grover_batch_destroy", e);
    return GROVER_OK;
}

}  // extern "C"
