// grover_api.cu -- the C ABI of libgrover (declared in include/grover.h).
//
// Host-side orchestration only: argument validation, scratch ownership, the
// cached complex mean, launch order on the caller's stream and error codes.
// All arithmetic on amplitudes runs in the kernels of k_stream.cu and
// k_measure.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "grover_internal.cuh"
#include "trace.cuh"

using namespace grv;

namespace {

thread_local char g_err[512] = "";
std::atomic<uint64_t> g_next_marked_id{1};

grover_status fail(grover_state *s, grover_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    snprintf(g_err, sizeof g_err, "%s", buf);
    if (s) snprintf(s->err, sizeof s->err, "%s", buf);
    return st;
}

grover_status cuda_fail(grover_state *s, cudaError_t e, const char *what) {
    (void)cudaGetLastError();  // clear a sticky launch error from the runtime's slot
    return fail(s, e == cudaErrorMemoryAllocation ? GROVER_ENOMEM : GROVER_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(s, expr, what)                                  \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, what); \
    } while (0)

int max_qubits(grover_dtype dt) { return dt == GROVER_C64 ? 33 : 32; }
size_t amp_bytes(grover_dtype dt) { return dt == GROVER_C64 ? 8 : 16; }
uint64_t nvec_of(const grover_state *s) { return s->dtype == GROVER_C64 ? s->N / 2 : s->N; }

// Scratch carve-up, 256-byte aligned pieces.
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
struct Layout {
    size_t partials, mu, ticket, status, cand, red, total;
};
Layout scratch_layout() {
    Layout L;
    size_t off = 0;
    L.partials = off; off += align256(sizeof(double2) * kMaxGrid);
    L.mu = off; off += align256(sizeof(MeanSlot) * 2);
    L.ticket = off; off += align256(sizeof(unsigned));
    L.status = off; off += align256(sizeof(int));
    L.cand = off; off += align256(sizeof(Cand) * (size_t)(kTopMGrid + 1) * kTopMMax);
    L.red = off; off += align256(sizeof(double2) * 4);
    L.total = off;
    return L;
}

PassArgs pass_args(grover_state *s, const MarkedDev &mk) {
    PassArgs a;
    a.amps = s->amps;
    a.nvec = nvec_of(s);
    a.mk = mk;
    a.mu_in = s->sc.mu + s->mu_slot;
    a.mu_out = s->sc.mu + (s->mu_slot ^ 1);
    a.partials = s->sc.partials;
    a.ticket = s->sc.ticket;
    a.inv_n = ldexp(1.0, -s->n);
    a.stream_hint = (long long)(s->N * amp_bytes(s->dtype)) > s->geo.l2_bytes / 2;
    a.status = s->sc.status;
    a.wait_limit = s->wait_limit;
    a.staged = s->staged;
    a.stall = 0;
    return a;
}

MarkedDev no_marks() {
    MarkedDev d;
    d.list = nullptr;
    d.words = nullptr;
    d.m = 0;
    d.mode = MARK_NONE;
    return d;
}

grover_status check_state(grover_state *s) {
    if (!s) return fail(nullptr, GROVER_EINVAL, "state handle is NULL");
    return GROVER_OK;
}

grover_status check_marked(grover_state *s, const grover_marked *mk) {
    if (!mk) return fail(s, GROVER_EINVAL, "marked set is NULL");
    if (mk->n != s->n)
        return fail(s, GROVER_EINVAL, "marked set built for n=%d used with a state of n=%d", mk->n, s->n);
    return GROVER_OK;
}

// Makes mu[slot] hold mean(O_mk c) (mk may be the empty view = mean of c).
grover_status ensure_mean(grover_state *s, const MarkedDev &mk, uint64_t key) {
    if (s->mu_valid && s->mu_key == key) return GROVER_OK;
    PassArgs a = pass_args(s, mk);
    a.mu_out = s->sc.mu + s->mu_slot;  // the reduction writes the current slot
    CK(s, launch_reduce(a, s->dtype, s->acc, s->stream, s->geo), "mean reduction launch");
    s->mu_valid = true;
    s->mu_key = key;
    return GROVER_OK;
}

}  // namespace

void grv::set_thread_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

cudaError_t grv::raise_func_attr(const void *kern, cudaFuncAttribute attr, int value) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int>, int> done;  // (kernel, device, attribute) -> value set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &cur = done[std::make_tuple(kern, dev, (int)attr)];
    if (cur >= value && cur != 0) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(kern, attr, value)) == cudaSuccess) cur = value;
    return e;
}

extern "C" {

const char *grover_status_string(grover_status st) {
    switch (st) {
    case GROVER_OK: return "GROVER_OK";
    case GROVER_EINVAL: return "GROVER_EINVAL";
    case GROVER_ENOMEM: return "GROVER_ENOMEM";
    case GROVER_ECUDA: return "GROVER_ECUDA";
    case GROVER_ETIMEOUT: return "GROVER_ETIMEOUT";
    case GROVER_EUNSORTED: return "GROVER_EUNSORTED";
    case GROVER_EDUP: return "GROVER_EDUP";
    case GROVER_ERANGE: return "GROVER_ERANGE";
    case GROVER_EUNSUPPORTED: return "GROVER_EUNSUPPORTED";
    }
    return "GROVER_<unknown>";
}

const char *grover_last_error(const grover_state *s) { return s ? s->err : g_err; }

uint64_t grover_optimal_iterations(int n_qubits, uint64_t m) {
    if (m == 0 || n_qubits < 1 || n_qubits > 63) return 0;
    const double r = sqrt(ldexp(1.0, n_qubits) / (double)m);
    return (uint64_t)floor(0.78539816339744830962 * r);
}

grover_status grover_create(grover_state **out, int n, grover_dtype dtype, void *dev_amps, void *cuda_stream) {
    if (!out) return fail(nullptr, GROVER_EINVAL, "out is NULL");
    if (dtype != GROVER_C64 && dtype != GROVER_C128) return fail(nullptr, GROVER_EINVAL, "unknown dtype %d", (int)dtype);
    if (n < 1 || n > max_qubits(dtype))
        return fail(nullptr, GROVER_EINVAL, "n=%d outside [1, %d] for this dtype", n, max_qubits(dtype));
    if (!dev_amps) return fail(nullptr, GROVER_EINVAL, "amplitude buffer is NULL");
    if ((uintptr_t)dev_amps % 16 != 0) return fail(nullptr, GROVER_EINVAL, "amplitude buffer is not 16-byte aligned");

    cudaPointerAttributes pa;
    cudaError_t e = cudaPointerGetAttributes(&pa, dev_amps);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaPointerGetAttributes");
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
        return fail(nullptr, GROVER_EINVAL, "amplitude buffer is not device memory");
    int cur = -1;
    if ((e = cudaGetDevice(&cur)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (cur != pa.device)
        return fail(nullptr, GROVER_EINVAL, "amplitude buffer lives on device %d, current device is %d", pa.device, cur);

    grover_state *s = (grover_state *)calloc(1, sizeof(grover_state));
    if (!s) return fail(nullptr, GROVER_ENOMEM, "host allocation of the handle failed");
    s->n = n;
    s->N = 1ull << n;
    s->dtype = dtype;
    s->acc = GROVER_ACC_DEFAULT;
    s->amps = dev_amps;
    s->stream = (cudaStream_t)cuda_stream;
    s->geo.dev = cur;
    int sms = 0, l2 = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, cur)) != cudaSuccess) {
        free(s);
        return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
    }
    s->geo.sm_count = sms;
    s->geo.l2_bytes = l2;
    s->geo.partial_slots = kMaxGrid;

    const Layout L = scratch_layout();
    char *base = nullptr;
    if ((e = cudaMalloc((void **)&base, L.total)) != cudaSuccess) {
        free(s);
        return cuda_fail(nullptr, e, "cudaMalloc(scratch)");
    }
    if ((e = cudaMemset(base, 0, L.total)) != cudaSuccess) {
        cudaFree(base);
        free(s);
        return cuda_fail(nullptr, e, "cudaMemset(scratch)");
    }
    s->scratch_base = base;
    s->sc.partials = (double2 *)(base + L.partials);
    s->sc.mu = (MeanSlot *)(base + L.mu);
    s->sc.ticket = (unsigned *)(base + L.ticket);
    s->sc.status = (int *)(base + L.status);
    s->sc.cand = (Cand *)(base + L.cand);
    s->sc.red = (double2 *)(base + L.red);
    s->sc.probs_tmp = nullptr;
    s->resident = -1;
    s->gate_engine = -1;
    s->staged = -1;
    s->wait_limit = kDefaultWaitLimit;
    s->test_stall = 0;
    s->mu_slot = 0;
    s->mu_valid = false;
    s->mu_key = 0;
    s->err[0] = 0;
    *out = s;
    return GROVER_OK;
}

grover_status grover_destroy(grover_state *s) {
    if (!s) return GROVER_OK;
    cudaError_t e1 = cudaStreamSynchronize(s->stream);
    cudaError_t e2 = cudaFree(s->scratch_base);
    cudaError_t e3 = s->sc.probs_tmp ? cudaFree(s->sc.probs_tmp) : cudaSuccess;
    if (s->phase_mem && e3 == cudaSuccess) e3 = cudaFree(s->phase_mem);
    if (s->rg_mem && e3 == cudaSuccess) e3 = cudaFree(s->rg_mem);
    free(s);
    cudaError_t e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "grover_destroy");
    return GROVER_OK;
}

grover_status grover_set_accum(grover_state *s, grover_accum mode) {
    if (grover_status st = check_state(s)) return st;
    if (mode < GROVER_ACC_DEFAULT || mode > GROVER_ACC_EXACT)
        return fail(s, GROVER_EINVAL, "unknown accumulation mode %d", (int)mode);
    if (s->dtype == GROVER_C128 && (mode == GROVER_ACC_FP32 || mode == GROVER_ACC_KAHAN))
        return fail(s, GROVER_EINVAL, "FP32 accumulation modes apply to complex64 states only");
    if (mode != s->acc) s->mu_valid = false;
    s->acc = mode;
    return GROVER_OK;
}

grover_status grover_set_option(grover_state *s, grover_option opt, int64_t value) {
    if (grover_status st = check_state(s)) return st;
    switch (opt) {
    case GROVER_OPT_RESIDENT:
        if (value < -1 || value > 2) return fail(s, GROVER_EINVAL, "GROVER_OPT_RESIDENT takes -1, 0, 1 or 2");
        s->resident = (int)value;
        return GROVER_OK;
    case GROVER_OPT_GATE_ENGINE:
        if (value < -1 || value > 1) return fail(s, GROVER_EINVAL, "option %d takes -1, 0 or 1", (int)opt);
        s->gate_engine = (int)value;
        return GROVER_OK;
    case GROVER_OPT_WAIT_LIMIT:
        if (value < 1) return fail(s, GROVER_EINVAL, "GROVER_OPT_WAIT_LIMIT must be positive");
        s->wait_limit = value;
        return GROVER_OK;
    case GROVER_OPT_TEST_STALL:
        if (value < 0 || value > 1) return fail(s, GROVER_EINVAL, "GROVER_OPT_TEST_STALL takes 0 or 1");
        s->test_stall = (int)value;
        return GROVER_OK;
    case GROVER_OPT_STAGED_PASS:
        if (value < -1 || value > 1) return fail(s, GROVER_EINVAL, "option %d takes -1, 0 or 1", (int)opt);
        s->staged = (int)value;
        return GROVER_OK;
    }
    return fail(s, GROVER_EINVAL, "unknown option %d", (int)opt);
}

grover_status grover_init_uniform(grover_state *s) {
    GROVER_TRACE("grover_init_uniform");
    if (grover_status st = check_state(s)) return st;
    CK(s, launch_init_uniform(s->amps, s->n, s->dtype, s->stream, s->geo), "init launch");
    s->mu_valid = false;
    return GROVER_OK;
}

grover_status grover_init_state(grover_state *s, const void *amps, int amps_on_device) {
    GROVER_TRACE("grover_init_state");
    if (grover_status st = check_state(s)) return st;
    if (!amps) return fail(s, GROVER_EINVAL, "source amplitudes are NULL");
    const size_t bytes = s->N * amp_bytes(s->dtype);
    CK(s, cudaMemcpyAsync(s->amps, amps, bytes, amps_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s->stream),
       "state copy");
    if (!amps_on_device) CK(s, cudaStreamSynchronize(s->stream), "state copy sync");
    s->mu_valid = false;
    return GROVER_OK;
}

grover_status grover_marked_from_list(grover_marked **out, int n, const uint64_t *idx, size_t m) {
    if (!out) return fail(nullptr, GROVER_EINVAL, "out is NULL");
    if (n < 1 || n > 33) return fail(nullptr, GROVER_EINVAL, "n=%d outside [1, 33]", n);
    if (m > 0 && !idx) return fail(nullptr, GROVER_EINVAL, "index list is NULL");
    const uint64_t N = 1ull << n;
    if (m > N) return fail(nullptr, GROVER_ERANGE, "m=%zu exceeds N=%llu", m, (unsigned long long)N);
    for (size_t i = 0; i < m; ++i) {
        if (idx[i] >= N)
            return fail(nullptr, GROVER_ERANGE, "marked index %llu at position %zu is >= N=%llu",
                        (unsigned long long)idx[i], i, (unsigned long long)N);
        if (i > 0 && idx[i] == idx[i - 1])
            return fail(nullptr, GROVER_EDUP, "marked index %llu appears twice", (unsigned long long)idx[i]);
        if (i > 0 && idx[i] < idx[i - 1])
            return fail(nullptr, GROVER_EUNSORTED, "marked list decreases at position %zu", i);
    }
    grover_marked *mk = (grover_marked *)calloc(1, sizeof(grover_marked));
    if (!mk) return fail(nullptr, GROVER_ENOMEM, "host allocation of the marked set failed");
    mk->n = n;
    mk->id = g_next_marked_id.fetch_add(1);
    mk->dev = no_marks();
    mk->dev.m = m;
    cudaError_t e;
    if (m > 0) {
        if ((e = cudaMalloc(&mk->list_mem, m * sizeof(uint64_t))) != cudaSuccess ||
            (e = cudaMemcpy(mk->list_mem, idx, m * sizeof(uint64_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
            grover_marked_destroy(mk);
            return cuda_fail(nullptr, e, "marked list upload");
        }
        mk->dev.list = (const uint64_t *)mk->list_mem;
        mk->dev.mode = MARK_LIST;
        mk->host_list = (uint64_t *)malloc(m * sizeof(uint64_t));
        if (!mk->host_list) {
            grover_marked_destroy(mk);
            return fail(nullptr, GROVER_ENOMEM, "host copy of the marked list");
        }
        memcpy(mk->host_list, idx, m * sizeof(uint64_t));
    }
    if (m > kListMax) {
        const uint64_t nwords = (N + 31) / 32;
        if ((e = cudaMalloc(&mk->words_mem, nwords * sizeof(uint32_t))) != cudaSuccess ||
            (e = launch_bits_from_list((uint32_t *)mk->words_mem, nwords, mk->dev.list, m, 0)) != cudaSuccess ||
            (e = cudaStreamSynchronize(0)) != cudaSuccess) {
            grover_marked_destroy(mk);
            return cuda_fail(nullptr, e, "marked bitmask build");
        }
        mk->dev.words = (const uint32_t *)mk->words_mem;
        mk->dev.mode = MARK_BITS;
    }
    *out = mk;
    return GROVER_OK;
}

grover_status grover_marked_from_bitmask(grover_marked **out, int n, const uint32_t *words, size_t nwords,
                                         int on_device) {
    if (!out) return fail(nullptr, GROVER_EINVAL, "out is NULL");
    if (n < 1 || n > 33) return fail(nullptr, GROVER_EINVAL, "n=%d outside [1, 33]", n);
    if (!words) return fail(nullptr, GROVER_EINVAL, "bitmask is NULL");
    const uint64_t N = 1ull << n;
    const uint64_t need = (N + 31) / 32;
    if (nwords != need)
        return fail(nullptr, GROVER_ERANGE, "bitmask has %zu words, 2^%d states need %llu", nwords, n,
                    (unsigned long long)need);
    grover_marked *mk = (grover_marked *)calloc(1, sizeof(grover_marked));
    if (!mk) return fail(nullptr, GROVER_ENOMEM, "host allocation of the marked set failed");
    mk->n = n;
    mk->id = g_next_marked_id.fetch_add(1);
    mk->dev = no_marks();
    cudaError_t e;
    unsigned long long *cnt = nullptr;
    int bad = 0;
    unsigned long long count = 0;
    if ((e = cudaMalloc(&mk->words_mem, nwords * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemcpy(mk->words_mem, words, nwords * sizeof(uint32_t),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc((void **)&cnt, 16)) != cudaSuccess || (e = cudaMemset(cnt, 0, 16)) != cudaSuccess ||
        (e = launch_bits_check_count((const uint32_t *)mk->words_mem, nwords, n, cnt, (int *)(cnt + 1), 0)) !=
            cudaSuccess ||
        (e = cudaMemcpy(&count, cnt, sizeof count, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(&bad, cnt + 1, sizeof bad, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        if (cnt) cudaFree(cnt);
        grover_marked_destroy(mk);
        return cuda_fail(nullptr, e, "marked bitmask upload");
    }
    cudaFree(cnt);
    if (bad) {
        grover_marked_destroy(mk);
        return fail(nullptr, GROVER_ERANGE, "bitmask marks an index >= N=%llu", (unsigned long long)N);
    }
    mk->dev.words = (const uint32_t *)mk->words_mem;
    mk->dev.m = count;
    mk->dev.mode = count ? MARK_BITS : MARK_NONE;
    *out = mk;
    return GROVER_OK;
}

grover_status grover_marked_count(const grover_marked *mk, uint64_t *m) {
    if (!mk || !m) return fail(nullptr, GROVER_EINVAL, "NULL argument");
    *m = mk->dev.m;
    return GROVER_OK;
}

grover_status grover_marked_destroy(grover_marked *mk) {
    if (!mk) return GROVER_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (mk->list_mem) cudaFree(mk->list_mem);
    if (mk->words_mem) cudaFree(mk->words_mem);
    free(mk->host_list);
    free(mk);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "grover_marked_destroy");
    return GROVER_OK;
}

grover_status grover_oracle(grover_state *s, const grover_marked *mk) {
    GROVER_TRACE("grover_oracle");
    if (grover_status st = check_state(s)) return st;
    if (grover_status st = check_marked(s, mk)) return st;
    if (mk->dev.m == 0) return GROVER_OK;
    CK(s, launch_oracle(s->amps, s->n, s->dtype, mk->dev, s->stream, s->geo), "oracle launch");
    // the cached mean of O c is the mean of the new state
    if (s->mu_valid && s->mu_key == mk->id) s->mu_key = 0;
    else s->mu_valid = false;
    return GROVER_OK;
}

grover_status grover_diffuse(grover_state *s) {
    GROVER_TRACE("grover_diffuse");
    if (grover_status st = check_state(s)) return st;
    const MarkedDev none = no_marks();
    if (grover_status st = ensure_mean(s, none, 0)) return st;
    PassArgs a = pass_args(s, none);
    CK(s, launch_pass(a, s->dtype, s->acc, s->stream, s->geo), "diffusion pass launch");
    s->mu_slot ^= 1;
    s->mu_valid = true;
    s->mu_key = 0;
    return GROVER_OK;
}

grover_status grover_iterate(grover_state *s, const grover_marked *mk, uint64_t k) {
    GROVER_TRACE("grover_iterate");
    if (grover_status st = check_state(s)) return st;
    if (grover_status st = check_marked(s, mk)) return st;
    if (k == 0) return GROVER_OK;
    if (s->resident != 0) {
        const bool exact_ok = s->acc == GROVER_ACC_DEFAULT || s->acc == GROVER_ACC_EXACT;
        unsigned C = 0, G = 0;
        uint32_t nv = 0, gv = 0;
        size_t smem = 0, gsmem = 0;
        const bool cluster_fits = exact_ok && resident_plan(s->n, s->dtype, &C, &nv, &smem);
        const bool grid_fits = exact_ok && resident_grid_plan(s->n, s->dtype, s->geo.sm_count, &G, &gv, &gsmem);
        // automatic choice, from per-iteration times measured on GB300: one
        // cluster up to cluster_max; the whole grid for [grid_min, grid_max]
        // (its exchange through global memory costs about 3.3 us per
        // iteration, against 2.7 us for the cluster's at small n); passes
        // otherwise
        const bool c64 = s->dtype == GROVER_C64;
        const int cluster_max = c64 ? 12 : 11, grid_min = c64 ? 13 : 12, grid_max = c64 ? 22 : 21;
        const bool use_cluster = cluster_fits && (s->resident == 1 || (s->resident == -1 && s->n <= cluster_max));
        const bool use_grid = !use_cluster && grid_fits &&
                              (s->resident >= 1 || (s->resident == -1 && s->n >= grid_min && s->n <= grid_max));
        if (use_cluster) {
            ResArgs r;
            r.amps = s->amps;
            r.slice_vecs = nv;
            r.mk = mk->dev;
            r.k = k;
            r.inv_n = ldexp(1.0, -s->n);
            r.n = s->n;
            r.mu_out = s->sc.mu + s->mu_slot;
            cudaError_t e = launch_resident(r, s->dtype, C, smem, s->stream);
            if (e == cudaSuccess) {
                s->mu_valid = true;
                s->mu_key = mk->id;
                return GROVER_OK;
            }
            (void)cudaGetLastError();
            if (s->resident == 1) return cuda_fail(s, e, "persistent iterator launch");
        } else if (use_grid) {
            if (!s->rg_mem) CK(s, cudaMalloc(&s->rg_mem, kRgBytes), "cudaMalloc(grid iterator region)");
            ResGridArgs r;
            r.amps = s->amps;
            r.nvec = nvec_of(s);
            r.slice_vecs = gv;
            r.mk = mk->dev;
            r.k = k;
            r.inv_n = ldexp(1.0, -s->n);
            r.n = s->n;
            r.mu_out = s->sc.mu + s->mu_slot;
            r.region = (unsigned long long *)s->rg_mem;
            r.status = s->sc.status;
            r.wait_limit = s->wait_limit;
            r.stall = s->test_stall;
            s->test_stall = 0;
            CK(s, cudaMemsetAsync(s->rg_mem, 0, kRgBytes, s->stream), "grid iterator reset");
            cudaError_t e = launch_resident_grid(r, s->dtype, G, gsmem, s->stream);
            if (e == cudaSuccess) {
                s->mu_valid = true;
                s->mu_key = mk->id;
                return GROVER_OK;
            }
            (void)cudaGetLastError();
            if (s->resident >= 1) return cuda_fail(s, e, "grid persistent iterator launch");
        } else if (s->resident >= 1) {
            return fail(s, GROVER_EUNSUPPORTED, "the persistent iterators need GROVER_ACC_DEFAULT or GROVER_ACC_EXACT "
                                                "and a state that fits the shared memory of one cluster (16 x 200 "
                                                "KiB) or of all SMs (%d x 226 KiB)", s->geo.sm_count);
        }
    }
    if (grover_status st = ensure_mean(s, mk->dev, mk->id)) return st;
    for (uint64_t t = 0; t < k; ++t) {
        PassArgs a = pass_args(s, mk->dev);
        a.stall = s->test_stall;  // test hook, taken by the first pass (staged passes only)
        s->test_stall = 0;
        cudaError_t e = launch_pass(a, s->dtype, s->acc, s->stream, s->geo);
        if (e != cudaSuccess) {
            s->mu_valid = false;
            return cuda_fail(s, e, "iteration pass launch");
        }
        s->mu_slot ^= 1;
    }
    s->mu_valid = true;
    s->mu_key = mk->id;
    return GROVER_OK;
}

grover_status grover_iterate_gate(grover_state *s, const grover_marked *mk, uint64_t k) {
    GROVER_TRACE("grover_iterate_gate");
    if (grover_status st = check_state(s)) return st;
    if (grover_status st = check_marked(s, mk)) return st;
    if (k == 0) return GROVER_OK;
    // Plans: CUDA cores take ceil(n / 8) index-bit groups of balanced sizes;
    // tensor cores 7 bits from bit 0 and the rest in 7-bit groups, or in
    // near-equal groups where that leaves fewer groups the tensor-core pass
    // cannot take.  Engine 0: the CUDA-core plan, all on CUDA cores.  Engine
    // 1: the tensor-core plan, every group the tensor-core pass takes on the
    // tensor cores, the rest on CUDA cores.  Default (-1): CUDA cores below
    // 2^26 complex64 amplitudes (there a tensor-core pass has fewer tiles than
    // its pipeline needs and measured slower); from 2^26 on, whichever plan
    // has fewer groups (ties: the tensor-core plan), with every group the
    // tensor-core pass takes on the tensor cores.
    const bool tc_possible = s->dtype == GROVER_C64 && s->n >= 13;
    if (s->gate_engine == 1 && !tc_possible)
        return fail(s, GROVER_EUNSUPPORTED, "the tensor-core gate path needs a complex64 state with n >= 13");
    int clo[8], ckb[8], tlo[8], tkb[8];  // n <= 33: at most 5 groups
    const int ncc = (s->n + 7) / 8;
    for (int gi = 0, lo = 0; gi < ncc; ++gi) {
        ckb[gi] = s->n / ncc + (gi < s->n % ncc ? 1 : 0);
        clo[gi] = lo;
        lo += ckb[gi];
    }
    int ntc = 0;
    if (tc_possible) {
        ntc = (s->n + 6) / 7;
        for (int gi = 0, lo = 0; gi < ntc; ++gi) {
            tkb[gi] = s->n - lo < 7 ? s->n - lo : 7;
            tlo[gi] = lo;
            lo += tkb[gi];
        }
        auto fallbacks = [&](const int *kbs) {
            int c = 0;
            for (int gi = 0, lo = 0; gi < ntc; lo += kbs[gi], ++gi) c += !tc_pass_supported(s->n, lo, kbs[gi]);
            return c;
        };
        const int rest = s->n - 7, parts = ntc - 1;
        if (parts > 0) {
            int bal[8];
            bal[0] = 7;
            for (int j = 0; j < parts; ++j) bal[j + 1] = rest / parts + (j < rest % parts ? 1 : 0);
            if (fallbacks(bal) < fallbacks(tkb))
                for (int gi = 0, lo = 0; gi < ntc; lo += bal[gi], ++gi) {
                    tlo[gi] = lo;
                    tkb[gi] = bal[gi];
                }
        }
    }
    const bool use_tc = s->gate_engine == 1 || (s->gate_engine < 0 && tc_possible && s->n >= kGateTcAutoMinQubits);
    const bool tc_plan = s->gate_engine == 1 || (use_tc && ntc <= ncc);
    const int ngroups = tc_plan ? ntc : ncc;
    const int *glo = tc_plan ? tlo : clo, *gkb = tc_plan ? tkb : ckb;
    s->mu_valid = false;
    for (uint64_t t = 0; t < k; ++t) {
        CK(s, launch_oracle(s->amps, s->n, s->dtype, mk->dev, s->stream, s->geo), "oracle launch");
        for (int pass = 0; pass < 2 * ngroups; ++pass) {
            const int gi = pass % ngroups, lo = glo[gi], kb = gkb[gi];
            const bool first = pass < ngroups;  // first H^{(x)n}: scaled by 2^-n in total
            const bool phase = pass == ngroups - 1;
            if (use_tc && tc_pass_supported(s->n, lo, kb)) {
                const int stall = s->test_stall;
                s->test_stall = 0;
                CK(s, launch_wht_tc_pass(s->amps, s->n, lo, kb, first, phase, s->sc.status, s->wait_limit, stall,
                                         s->stream, s->geo),
                   "tensor-core Walsh-Hadamard pass launch");
            } else {
                CK(s, launch_wht_pass(s->amps, s->n, s->dtype, lo, kb, first, phase, s->stream, s->geo),
                   "Walsh-Hadamard pass launch");
            }
        }
    }
    return GROVER_OK;
}

grover_status grover_iterate_circuit(grover_state *s, const grover_marked *mk, uint64_t k, uint64_t *gates_out,
                                     uint64_t *passes_out) {
    GROVER_TRACE("grover_iterate_circuit");
    if (grover_status st = check_state(s)) return st;
    if (grover_status st = check_marked(s, mk)) return st;
    if (mk->dev.m > 0 && !mk->host_list)
        return fail(s, GROVER_EUNSUPPORTED, "the gate-by-gate oracle needs a marked set built from a list");
    const double r = 0.70710678118654752440;  // 1/sqrt(2)
    uint64_t gates = 0, passes = 0;
    s->mu_valid = false;
    for (uint64_t t = 0; t < k; ++t) {
        // oracle (Fig. oracle1): X where the solution has a 0, MCZ, the same X
        for (uint64_t i = 0; i < mk->dev.m; ++i) {
            const uint64_t x = mk->host_list[i];
            for (int pass = 0; pass < 2; ++pass) {
                for (int q = 0; q < s->n; ++q) {
                    if ((x >> q) & 1) continue;
                    CK(s, launch_gate1(s->amps, s->n, s->dtype, 0, q, 1.0, s->stream, s->geo), "X gate launch");
                    ++gates;
                    ++passes;
                }
                if (pass == 0) {
                    CK(s, launch_mcz_all(s->amps, s->n, s->dtype, s->stream), "MCZ launch");
                    ++gates;
                }
            }
        }
        // H^{(x)n}
        for (int q = 0; q < s->n; ++q) {
            CK(s, launch_gate1(s->amps, s->n, s->dtype, 1, q, r, s->stream, s->geo), "H gate launch");
            ++gates;
            ++passes;
        }
        // 2|0><0| - I = -X^{(x)n} MCZ X^{(x)n}; the -1 rides on the next H
        for (int q = 0; q < s->n; ++q) {
            CK(s, launch_gate1(s->amps, s->n, s->dtype, 0, q, 1.0, s->stream, s->geo), "X gate launch");
            ++gates;
            ++passes;
        }
        CK(s, launch_mcz_all(s->amps, s->n, s->dtype, s->stream), "MCZ launch");
        ++gates;
        for (int q = 0; q < s->n; ++q) {
            CK(s, launch_gate1(s->amps, s->n, s->dtype, 0, q, 1.0, s->stream, s->geo), "X gate launch");
            ++gates;
            ++passes;
        }
        // H^{(x)n}, the first Hadamard also carrying the phase shift's -1
        for (int q = 0; q < s->n; ++q) {
            CK(s, launch_gate1(s->amps, s->n, s->dtype, 1, q, q == 0 ? -r : r, s->stream, s->geo), "H gate launch");
            ++gates;
            ++passes;
        }
    }
    if (gates_out) *gates_out = gates;
    if (passes_out) *passes_out = passes;
    return GROVER_OK;
}

grover_status grover_measure_probs(grover_state *s, double *out, int out_on_device) {
    GROVER_TRACE("grover_measure_probs");
    if (grover_status st = check_state(s)) return st;
    if (!out) return fail(s, GROVER_EINVAL, "output is NULL");
    if (out_on_device) {
        CK(s, launch_probs(s->amps, s->dtype, 0, s->N, out, s->stream, s->geo), "probability launch");
        return GROVER_OK;
    }
    if (!s->sc.probs_tmp) CK(s, cudaMalloc((void **)&s->sc.probs_tmp, kProbsChunk * sizeof(double)), "cudaMalloc(probs staging)");
    for (uint64_t first = 0; first < s->N; first += kProbsChunk) {
        const uint64_t cnt = (s->N - first) < kProbsChunk ? (s->N - first) : kProbsChunk;
        CK(s, launch_probs(s->amps, s->dtype, first, cnt, s->sc.probs_tmp, s->stream, s->geo), "probability launch");
        CK(s, cudaMemcpyAsync(out + first, s->sc.probs_tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
           "probability copy");
        CK(s, cudaStreamSynchronize(s->stream), "probability sync");
    }
    return GROVER_OK;
}

grover_status grover_measure_topm(grover_state *s, size_t m, uint64_t *idx, double *p) {
    GROVER_TRACE("grover_measure_topm");
    if (grover_status st = check_state(s)) return st;
    if (!idx || !p) return fail(s, GROVER_EINVAL, "output is NULL");
    if (m < 1 || m > (size_t)kTopMMax || m > s->N)
        return fail(s, GROVER_EINVAL, "m=%zu outside [1, min(%d, N)]", m, kTopMMax);
    CK(s, launch_topm(s->amps, s->n, s->dtype, (int)m, s->sc, s->stream, s->geo), "top-m launch");
    Cand host[kTopMMax];
    CK(s, cudaMemcpyAsync(host, s->sc.cand + (size_t)kTopMGrid * kTopMMax, m * sizeof(Cand), cudaMemcpyDeviceToHost,
                          s->stream),
       "top-m copy");
    CK(s, cudaStreamSynchronize(s->stream), "top-m sync");
    for (size_t j = 0; j < m; ++j) {
        idx[j] = host[j].idx;
        p[j] = host[j].p;
    }
    return GROVER_OK;
}

grover_status grover_success_prob(grover_state *s, const grover_marked *mk, double *p_success, double *norm) {
    GROVER_TRACE("grover_success_prob");
    if (grover_status st = check_state(s)) return st;
    if (grover_status st = check_marked(s, mk)) return st;
    CK(s, launch_norm_success(s->amps, s->n, s->dtype, mk->dev, s->sc, s->stream, s->geo), "norm launch");
    double2 r;
    CK(s, cudaMemcpyAsync(&r, s->sc.red, sizeof r, cudaMemcpyDeviceToHost, s->stream), "norm copy");
    CK(s, cudaStreamSynchronize(s->stream), "norm sync");
    if (norm) *norm = r.x;
    if (p_success) *p_success = r.y;
    return GROVER_OK;
}

grover_status grover_sync(grover_state *s) {
    if (grover_status st = check_state(s)) return st;
    CK(s, cudaStreamSynchronize(s->stream), "stream sync");
    int status = 0;
    CK(s, cudaMemcpy(&status, s->sc.status, sizeof status, cudaMemcpyDeviceToHost), "status read");
    if (status != 0) {
        CK(s, cudaMemset(s->sc.status, 0, sizeof(int)), "status reset");
        s->mu_valid = false;
        if (status == 4)
            return fail(s, GROVER_ECUDA, "tensor-core pass skipped: its staging buffer is not 1024-byte aligned");
        return fail(s, GROVER_ETIMEOUT, "a bounded device-side wait gave up (status %d: %s)", status,
                    status == 3 ? "grid persistent iterator"
                    : status == 5 ? "staged iteration pass" : "tensor-core pass");
    }
    return GROVER_OK;
}

}  // extern "C"
