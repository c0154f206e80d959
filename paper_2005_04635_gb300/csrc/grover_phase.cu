// grover_phase.cu -- C ABI of the generalised phase iterator and its adjoint
// (declared in include/grover.h).  Host-side validation and launch order
// only; the arithmetic is in k_phase.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "grover_internal.cuh"
#include "trace.cuh"

using namespace grv;

namespace {

grover_status pfail(grover_state *s, grover_status st, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(buf, sizeof buf, "%s: %s (%s)", msg, cudaGetErrorString(e), cudaGetErrorName(e));
        st = e == cudaErrorMemoryAllocation ? GROVER_ENOMEM : GROVER_ECUDA;
    } else {
        snprintf(buf, sizeof buf, "%s", msg);
    }
    set_thread_error(buf);
    if (s) snprintf(s->err, sizeof s->err, "%s", buf);
    return st;
}

// Scratch of the phase iterator inside s->phase_mem, 256-byte aligned pieces.
struct PhaseScratch {
    PhaseConst *c;      // [2] constants, ping-pong between passes
    unsigned *ticket;   // [1]
    double2 *partials;  // [6 * kPhaseMaxGrid]
    unsigned long long *region;  // exchange region of the on-chip sweeps
    PhaseFac *table;             // [kPhaseTableMax] per-step constants of the on-chip sweeps
};
constexpr size_t kPhOffTicket = 256, kPhOffPartials = 512;
constexpr size_t kPhOffRegion = kPhOffPartials + sizeof(double2) * 6 * (size_t)kPhaseMaxGrid;
size_t ph_off_table() { return (kPhOffRegion + phase_grid_region_bytes(512) + 255) & ~(size_t)255; }
size_t ph_bytes() { return ph_off_table() + sizeof(PhaseFac) * (size_t)kPhaseTableMax; }
static_assert(2 * sizeof(PhaseConst) <= kPhOffTicket, "phase constants overflow their slot");

grover_status phase_scratch(grover_state *s, PhaseScratch *out) {
    if (!s->phase_mem) {
        cudaError_t e = cudaMalloc(&s->phase_mem, ph_bytes());
        if (e != cudaSuccess) {
            s->phase_mem = nullptr;
            return pfail(s, GROVER_ECUDA, "cudaMalloc(phase scratch)", e);
        }
        if ((e = cudaMemsetAsync(s->phase_mem, 0, ph_bytes(), s->stream)) != cudaSuccess)
            return pfail(s, GROVER_ECUDA, "cudaMemsetAsync(phase scratch)", e);
    }
    char *b = (char *)s->phase_mem;
    out->c = (PhaseConst *)b;
    out->ticket = (unsigned *)(b + kPhOffTicket);
    out->partials = (double2 *)(b + kPhOffPartials);
    out->region = (unsigned long long *)(b + kPhOffRegion);
    out->table = (PhaseFac *)(b + ph_off_table());
    return GROVER_OK;
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == dev;
}

grover_status check_common(grover_state *s, const grover_marked *mk, const double *phi, const double *vphi,
                           uint64_t K) {
    if (!s) return pfail(nullptr, GROVER_EINVAL, "state handle is NULL");
    if (s->dtype != GROVER_C64)
        return pfail(s, GROVER_EUNSUPPORTED, "the phase iterator runs on complex64 states only");
    if (!mk) return pfail(s, GROVER_EINVAL, "marked set is NULL");
    if (mk->n != s->n) return pfail(s, GROVER_EINVAL, "marked set built for another number of qubits");
    if (mk->dev.m == 0 || !mk->dev.list || mk->dev.m > kPhaseMaxMarked)
        return pfail(s, GROVER_EUNSUPPORTED, "the phase iterator needs a marked list of 1 to 256 indices "
                                             "(built by grover_marked_from_list)");
    if (K > (uint64_t)1 << 40) return pfail(s, GROVER_ERANGE, "K is out of range");
    if (K > 0) {
        if (!phi || !vphi) return pfail(s, GROVER_EINVAL, "phase arrays are NULL");
        if (!on_device(phi, s->geo.dev) || !on_device(vphi, s->geo.dev))
            return pfail(s, GROVER_EINVAL, "phase arrays must be device memory of the state's device");
    }
    return GROVER_OK;
}

PhaseArgs base_args(grover_state *s, const grover_marked *mk, const double *phi, const double *vphi, uint64_t K,
                    const PhaseScratch &ps) {
    PhaseArgs a;
    memset(&a, 0, sizeof a);
    a.psi = s->amps;
    a.nvec = s->N / 2;
    a.n = s->n;
    a.list = mk->dev.list;
    a.m = (uint32_t)mk->dev.m;
    a.phi = phi;
    a.vphi = vphi;
    a.K = (long long)K;
    a.partials = ps.partials;
    a.ticket = ps.ticket;
    return a;
}

// The on-chip sweep (one cooperative launch) where the state -- backward: the
// state and the adjoint -- fits the SMs' shared memory, unless the handle's
// GROVER_OPT_RESIDENT is 0.  Returns cudaErrorNotSupported when it does not
// apply, so the caller runs the pass kernels.
cudaError_t try_grid(grover_state *s, const grover_marked *mk, const double *phi, const double *vphi, uint64_t K,
                     const PhaseScratch &ps, bool backward, void *lam, double *gphi, double *gvphi, double *stats) {
    unsigned G = 0;
    uint32_t L = 0;
    size_t smem = 0;
    if (s->resident == 0 || !phase_grid_plan(s->n, backward, s->geo.sm_count, &G, &L, &smem))
        return cudaErrorNotSupported;
    PhaseGridArgs g;
    memset(&g, 0, sizeof g);
    g.psi = s->amps;
    g.lam = lam;
    g.nvec = s->N / 2;
    g.slice_vecs = L;
    g.n = s->n;
    g.list = mk->dev.list;
    g.m = (uint32_t)mk->dev.m;
    g.phi = phi;
    g.vphi = vphi;
    g.K = (long long)K;
    g.region = ps.region;
    g.stats = stats;
    g.grad_phi = gphi;
    g.grad_vphi = gvphi;
    g.status = s->sc.status;
    g.wait_limit = s->wait_limit;
    g.stall = s->test_stall;
    cudaError_t e = cudaMemsetAsync(ps.region, 0, phase_grid_zero_bytes(), s->stream);
    if (e != cudaSuccess) return e;
    if (K <= (uint64_t)kPhaseTableMax) {
        if ((e = launch_phase_table(phi, vphi, (long long)K, ps.table, s->stream)) != cudaSuccess) return e;
        g.table = ps.table;
    }
    e = launch_phase_grid(g, backward, G, smem, s->stream);
    if (e == cudaSuccess) s->test_stall = 0;
    return e;
}

}  // namespace

extern "C" {

grover_status grover_phase_forward(grover_state *s, const grover_marked *mk, const double *phi, const double *vphi,
                                   uint64_t K, double *stats) {
    GROVER_TRACE("grover_phase_forward");
    if (grover_status st = check_common(s, mk, phi, vphi, K)) return st;
    if (stats && !on_device(stats, s->geo.dev))
        return pfail(s, GROVER_EINVAL, "stats must be device memory of the state's device");
    PhaseScratch ps;
    if (grover_status st = phase_scratch(s, &ps)) return st;
    s->mu_valid = false;
    cudaError_t eg = try_grid(s, mk, phi, vphi, K, ps, false, nullptr, nullptr, nullptr, stats);
    if (eg == cudaSuccess) return GROVER_OK;
    (void)cudaGetLastError();
    if (eg != cudaErrorNotSupported && s->resident >= 1) return pfail(s, GROVER_ECUDA, "on-chip phase sweep launch", eg);
    PhaseArgs a = base_args(s, mk, phi, vphi, K, ps);
    a.stats = stats;
    a.t = -1;
    a.cin = ps.c;
    a.cout = ps.c;
    const bool stream = (long long)(s->N * 8) > s->geo.l2_bytes / 2;
    cudaError_t e = launch_phase_fwd(a, false, stream, s->stream, s->geo.sm_count);
    if (e != cudaSuccess) return pfail(s, GROVER_ECUDA, "phase iterator reduction launch", e);
    for (uint64_t t = 0; t < K; ++t) {
        a.t = (long long)t;
        a.cin = ps.c + (t & 1);
        a.cout = ps.c + ((t + 1) & 1);
        if ((e = launch_phase_fwd(a, true, stream, s->stream, s->geo.sm_count)) != cudaSuccess)
            return pfail(s, GROVER_ECUDA, "phase iterator pass launch", e);
    }
    return GROVER_OK;
}

grover_status grover_phase_backward(grover_state *s, const grover_marked *mk, const double *phi, const double *vphi,
                                    uint64_t K, void *lam, double *grad_phi, double *grad_vphi) {
    GROVER_TRACE("grover_phase_backward");
    if (grover_status st = check_common(s, mk, phi, vphi, K)) return st;
    if (!lam || (uintptr_t)lam % 16 != 0 || !on_device(lam, s->geo.dev))
        return pfail(s, GROVER_EINVAL, "lambda must be 16-byte aligned device memory of the state's device");
    const uintptr_t l0 = (uintptr_t)lam, a0 = (uintptr_t)s->amps, bytes = (uintptr_t)(s->N * 8);
    if (l0 < a0 + bytes && a0 < l0 + bytes) return pfail(s, GROVER_EINVAL, "lambda overlaps the state");
    if (K > 0) {
        if (!grad_phi || !grad_vphi) return pfail(s, GROVER_EINVAL, "gradient arrays are NULL");
        if (!on_device(grad_phi, s->geo.dev) || !on_device(grad_vphi, s->geo.dev))
            return pfail(s, GROVER_EINVAL, "gradient arrays must be device memory of the state's device");
    }
    PhaseScratch ps;
    if (grover_status st = phase_scratch(s, &ps)) return st;
    s->mu_valid = false;
    cudaError_t eg = try_grid(s, mk, phi, vphi, K, ps, true, lam, grad_phi, grad_vphi, nullptr);
    if (eg == cudaSuccess) return GROVER_OK;
    (void)cudaGetLastError();
    if (eg != cudaErrorNotSupported && s->resident >= 1) return pfail(s, GROVER_ECUDA, "on-chip adjoint sweep launch", eg);
    PhaseArgs a = base_args(s, mk, phi, vphi, K, ps);
    a.lam = lam;
    a.grad_phi = grad_phi;
    a.grad_vphi = grad_vphi;
    a.t = (long long)K;
    a.cin = ps.c;
    a.cout = ps.c;
    const bool stream = (long long)(s->N * 16) > s->geo.l2_bytes / 2;  // state and adjoint
    cudaError_t e = launch_phase_bwd_start(a, stream, s->stream, s->geo.sm_count);
    if (e != cudaSuccess) return pfail(s, GROVER_ECUDA, "adjoint start launch", e);
    for (uint64_t i = 0; i < K; ++i) {
        a.t = (long long)(K - 1 - i);
        a.cin = ps.c + (i & 1);
        a.cout = ps.c + ((i + 1) & 1);
        if ((e = launch_phase_bwd(a, stream, s->stream, s->geo.sm_count)) != cudaSuccess)
            return pfail(s, GROVER_ECUDA, "adjoint pass launch", e);
    }
    return GROVER_OK;
}

}  // extern "C"
