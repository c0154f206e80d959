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
    int packing;            // 0: one CTA per instance; kBatchClusterSize: clusters for large instances
    int pack_min_qubits;    // with packing: instances of at least this many qubits run on clusters
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
grover_status split(grover_batch *b) {
    const bool use = b->packing > 1 && b->clusters > 0;
    std::vector<uint32_t> small, large;
    for (uint32_t i : b->order) ((use && b->nq[i] >= b->pack_min_qubits) ? large : small).push_back(i);
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
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // large instances first (they hold the longest runs), then the small ones
        cudaError_t e2 = b->LC.count ? enqueue_batch_cluster(b->LC, b->clusters, cs) : cudaSuccess;
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
    for (size_t i = 0; i < count; ++i) b->nq[i] = inst[i].n;
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
    b->packing = 0;  // one CTA per instance; grover_batch_tune also tries clusters
    b->pack_min_qubits = kBatchClusterMinQubits;
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
    if (b->clusters > 0) {
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
        int best_min = 0;
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
                }
                (void)cudaGetLastError();
            }
        } else {
            (void)cudaGetLastError();
        }
        b->packing = best_min ? kBatchClusterSize : 0;
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
    if (cluster_size != 0 && cluster_size != 1 && cluster_size != kBatchClusterSize)
        return bfail(b, GROVER_EINVAL, "cluster size must be 0, 1 or 16");
    if (cluster_size == kBatchClusterSize && b->clusters == 0)
        return bfail(b, GROVER_EUNSUPPORTED, "clusters of 16 CTAs cannot run on this device");
    b->packing = cluster_size;
    return rebuild(b);
}

grover_status grover_batch_set_packing_min_qubits(grover_batch *b, int min_qubits) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    if (min_qubits < kBatchClusterMinQubits || min_qubits > kBatchMaxQubits)
        return bfail(b, GROVER_EINVAL, "the packing threshold must be in [17, 26] qubits");
    b->pack_min_qubits = min_qubits;
    return rebuild(b);
}

grover_status grover_batch_get_packing(const grover_batch *b, int *cluster_size, int *min_qubits) {
    if (!b) return bfail(nullptr, GROVER_EINVAL, "batch is NULL");
    if (cluster_size) *cluster_size = b->packing > 1 ? b->packing : 1;
    if (min_qubits) *min_qubits = b->pack_min_qubits;
    return GROVER_OK;
}

grover_status grover_batch_success(grover_batch *b, double *p_success) {
    if (!b || !p_success) return bfail(b, GROVER_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(p_success, b->L.psucc, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, GROVER_ECUDA, "batch result copy", e);
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
    delete b;
    if (e != cudaSuccess) return bfail(nullptr, GROVER_ECUDA, "grover_batch_destroy", e);
    return GROVER_OK;
}

}  // extern "C"
