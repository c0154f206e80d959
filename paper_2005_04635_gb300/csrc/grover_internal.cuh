// grover_internal.cuh -- types shared by the translation units of libgrover.
//
// Device-side views, the handle layout and the host-side launchers that the C
// ABI (grover_api.cu) calls.  Kernels live in k_stream.cu (init, oracle, fused
// iteration pass, mean reduction) and k_measure.cu (probabilities, norm,
// top-m).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "grover.h"

namespace grv {

constexpr int kThreads = 256;           // threads per CTA of the streaming kernels
constexpr int kMaxGrid = 4096;          // upper bound on CTAs of a streaming launch
constexpr uint64_t kListMax = 256;      // larger marked lists also get a bitmask
constexpr int kTopMMax = 16;            // grover_measure_topm limit
constexpr int kTopMGrid = 1024;         // CTAs of a top-m launch

enum MarkMode : int { MARK_NONE = 0, MARK_LIST = 1, MARK_BITS = 2 };

// Device view of a marked set.
struct MarkedDev {
    const uint64_t *list;   // sorted unique indices (MARK_LIST), else unused
    const uint32_t *words;  // bitmask (MARK_BITS), else unused
    uint64_t m;             // number of marked indices
    int mode;               // MarkMode used by the streaming kernels
};

// Candidate of the top-m selection.
struct Cand {
    double p;
    uint64_t idx;
};

// A complex mean as produced by one pass for the next: the mean itself, 2 mu,
// and 2 mu as an unevaluated sum of two floats (hi, lo) per component.
struct MeanSlot {
    double2 mu;
    double2 two;
    float4 two32;  // (re hi, re lo, im hi, im lo)
};

// Device scratch owned by one state handle (one cudaMalloc, carved up).
struct Scratch {
    double2 *partials;      // [kMaxGrid] per-CTA partial sums
    MeanSlot *mu;           // [2] double-buffered complex mean
    unsigned *ticket;       // [1] last-CTA-done counter (always left at 0)
    int *status;            // [1] device status word (0 = ok)
    Cand *cand;             // [(kTopMGrid + 1) * kTopMMax] per-CTA top-m candidates + result
    double2 *red;           // [4] reduction outputs (norm, success)
    double *probs_tmp;      // [kProbsChunk] staging for host probability output
};
constexpr size_t kProbsChunk = size_t(1) << 22;  // 32 MiB of doubles

// Launch geometry derived once per handle, for the device the handle lives on.
struct Geometry {
    int sm_count;
    int dev;
    long long l2_bytes;
    int partial_slots;      // double2 slots of the per-CTA partial-sum array a pass writes into
};

// Everything a streaming kernel launch needs.
struct PassArgs {
    void *amps;
    uint64_t nvec;          // number of 16-byte vectors in the state
    MarkedDev mk;
    const MeanSlot *mu_in;  // mean used by this pass (device)
    MeanSlot *mu_out;       // mean produced for the next pass (device)
    double2 *partials;
    unsigned *ticket;
    double inv_n;           // 1 / N
    bool stream_hint;       // state larger than L2: streaming cache hints
    int *status;            // device status word (5: a staged copy's wait ran out), or NULL
    long long wait_limit;   // polls of a bounded wait
    int staged;             // -1 staged above L2 / 2, 0 never, 1 whenever whole chunks
    int stall;              // test hook: CTA 0 of a staged pass withholds its first copy
};

// ---- launchers (k_stream.cu) ---------------------------------------------
cudaError_t launch_init_uniform(void *amps, int n, grover_dtype dt, cudaStream_t st,
                                const Geometry &g);
// One fused iteration pass: c <- 2*mu_in - flip(c), store, and
// mu_out = mean(flip(c_new)).
// Both flips use args.mk (MARK_NONE: no flip).
cudaError_t launch_pass(const PassArgs &a, grover_dtype dt, grover_accum acc, cudaStream_t st,
                        const Geometry &g);
// Mean only: mu_out = mean(flip(c)).
cudaError_t launch_reduce(const PassArgs &a, grover_dtype dt, grover_accum acc, cudaStream_t st,
                          const Geometry &g);
// Oracle alone: c_x <- -c_x for marked x.
cudaError_t launch_oracle(void *amps, int n, grover_dtype dt, const MarkedDev &mk,
                          cudaStream_t st, const Geometry &g);
// Bitmask helpers for marked sets.
cudaError_t launch_bits_from_list(uint32_t *words, uint64_t nwords, const uint64_t *list,
                                  uint64_t m, cudaStream_t st);
cudaError_t launch_bits_check_count(const uint32_t *words, uint64_t nwords, int n,
                                    unsigned long long *count_out, int *bad_out,
                                    cudaStream_t st);

// ---- launchers (k_measure.cu) --------------------------------------------
cudaError_t launch_probs(const void *amps, grover_dtype dt, uint64_t first, uint64_t count,
                         double *out, cudaStream_t st, const Geometry &g);
// red[0].x = norm, red[1].x = success probability
cudaError_t launch_norm_success(const void *amps, int n, grover_dtype dt, const MarkedDev &mk,
                                Scratch &sc, cudaStream_t st, const Geometry &g);
cudaError_t launch_topm(const void *amps, int n, grover_dtype dt, int m, Scratch &sc,
                        cudaStream_t st, const Geometry &g);

// ---- persistent on-chip iterator (k_resident.cu) ---------------------------
constexpr int kResMaxCluster = 16;          // CTAs per cluster (non-portable size)
constexpr size_t kResSmemMax = 200 * 1024;  // dynamic shared memory per CTA
struct ResArgs {
    void *amps;
    uint32_t slice_vecs;    // 16-byte vectors held by each CTA
    MarkedDev mk;
    uint64_t k;             // iterations
    double inv_n;           // 1 / N
    int n;                  // N = 2^n (n <= 27 keeps the float means normal)
    MeanSlot *mu_out;       // mean of O c after the last iteration
};
// false if the state does not fit one cluster's shared memory
bool resident_plan(int n, grover_dtype dt, unsigned *C, uint32_t *slice_vecs, size_t *smem);
cudaError_t launch_resident(const ResArgs &a, grover_dtype dt, unsigned C, size_t smem, cudaStream_t st);
// Grid-wide variant (cooperative launch, one CTA per SM, exact partials
// exchanged through global memory, grid_exchange.cuh).
constexpr size_t kRgSmemMax = 226 * 1024;  // dynamic shared memory per CTA
constexpr int kRgMaxGrid = 512;
// exchange region of two sums: two sets of 8 word lines, side slots for 512 CTAs
constexpr size_t kRgBytes = sizeof(unsigned long long) * 16 * (2 * 8) + sizeof(double) * 2 * kRgMaxGrid * 2;
struct ResGridArgs {
    void *amps;
    uint64_t nvec;          // 16-byte vectors in the state
    uint32_t slice_vecs;    // vectors per CTA (the last CTA may hold fewer)
    MarkedDev mk;
    uint64_t k;
    double inv_n;
    int n;                  // N = 2^n (n <= 27 keeps the float means normal)
    MeanSlot *mu_out;
    unsigned long long *region;  // exchange region (kRgBytes, zeroed before the launch)
    int *status;            // set to 3 if a wait runs out
    long long wait_limit;   // polls before giving up
    int stall;              // test hook: CTA 0 never reports its first partial
};
bool resident_grid_plan(int n, grover_dtype dt, int sm_count, unsigned *G, uint32_t *slice_vecs, size_t *smem);
cudaError_t launch_resident_grid(const ResGridArgs &a, grover_dtype dt, unsigned G, size_t smem, cudaStream_t st);

// ---- conventional circuit (k_gate.cu) ---------------------------------------
// One Walsh-Hadamard pass over index bits [lo, lo + kb) (kb <= 8; lo = 0 or
// lo >= 4), scaled by 2^-kb if `scaled`, negating every amplitude but index 0
// if `negate` (the conditional phase shift 2|0><0| - I).
cudaError_t launch_wht_pass(void *amps, int n, grover_dtype dt, int lo, int kb, bool scaled, bool negate,
                            cudaStream_t st, const Geometry &g);

// ---- conventional circuit on tensor cores (k_gate_tc.cu), complex64 ---------
// true if a tensor-core pass exists for bits [lo, lo + kb) of an n-qubit state
bool tc_pass_supported(int n, int lo, int kb);
// smallest n whose default gate path uses the tensor cores
constexpr int kGateTcAutoMinQubits = 26;
// Walsh-Hadamard pass on the tensor cores; a wait longer than wait_limit
// polls gives up and sets *status = 2; stall != 0 withholds the MMA
// completion signal (test hook for that path)
cudaError_t launch_wht_tc_pass(void *amps, int n, int lo, int kb, bool scaled, bool negate, int *status,
                               long long wait_limit, int stall, cudaStream_t st, const Geometry &g);
constexpr long long kDefaultWaitLimit = 1ll << 22;  // mbarrier polls (~0.4 s)

// ---- conventional circuit gate by gate (k_circuit.cu) ------------------------
// One single-qubit gate as one pass: op 0 = X, op 1 = H scaled by `scale`
// (+-1/sqrt(2)).
cudaError_t launch_gate1(void *amps, int n, grover_dtype dt, int op, int q, double scale, cudaStream_t st,
                         const Geometry &g);
// Multi-controlled Z on all n qubits: negates the amplitude |1...1>.
cudaError_t launch_mcz_all(void *amps, int n, grover_dtype dt, cudaStream_t st);

// ---- batched searches (k_batch.cu) ------------------------------------------
constexpr uint32_t kBatchMaxMarked = 64;  // marked indices per instance
constexpr int kBatchMaxQubits = 26;
struct BatchInst {
    uint64_t amp_off;   // first amplitude of the instance in the batch buffer
    uint64_t k;         // iterations
    uint64_t mark_off;  // first marked index in the concatenated lists
    uint32_t m;         // marked indices
    int n;              // qubits
};
struct BatchLaunch {
    float4 *amps;
    const BatchInst *inst;
    const uint32_t *order;  // instance indices, largest N * k first
    uint32_t count;
    const uint64_t *marked;
    unsigned *next;         // work counter
    double *psucc;          // [count] success probabilities
    uint32_t onchip_vecs;   // instances of at most this many 16-byte vectors stay in shared memory
    int threads;            // 256, 512 or 1024
};
// Sets the kernel attributes for L and returns the persistent grid size.
cudaError_t prepare_batch(const BatchLaunch &L, int sm_count, unsigned *grid);
// Resets the work counter and launches (capturable in a CUDA graph).
cudaError_t enqueue_batch(const BatchLaunch &L, unsigned grid, cudaStream_t st);

// Large instances run one per thread-block cluster of kBatchClusterSize CTAs
// (each CTA a slice of the state; exact partials combined through distributed
// shared memory after a hardware cluster barrier per iteration), the small
// ones one per CTA (k_batch).
constexpr int kBatchClusterSize = 16;
constexpr int kBatchClusterMinQubits = 17;     // smallest n run by a cluster
constexpr uint32_t kBatchClusterOnchipVecs = 12800;  // slice kept in shared memory up to 200 KiB
struct BatchClusterLaunch {
    float4 *amps;
    const BatchInst *inst;
    const uint32_t *order;  // the large instances, largest N * k first
    uint32_t count;
    const uint64_t *marked;
    unsigned *next;         // work counter
    double *psucc;
};
// Sets the attributes and returns the number of co-resident clusters (0 if
// clusters of kBatchClusterSize cannot run).
cudaError_t prepare_batch_cluster(int *clusters);
cudaError_t enqueue_batch_cluster(const BatchClusterLaunch &L, int clusters, cudaStream_t st);

// Large instances kept on chip by groups of CTAs (k_batch_group.cu): one
// cooperative launch per instance size n, groups of group_ctas CTAs, each
// running the instances glist[goff[g] .. goff[g + 1]) with exact per-iteration
// exchanges through its part of `region` (region_words words per group, zero
// at launch).
constexpr int kBatchGroupThreads = 512;
constexpr int kBatchGroupMinQubits = 15;   // smallest n a group may take
constexpr size_t kBatchGroupSmemMax = 225 * 1024;  // dynamic shared memory per CTA (227 KiB less static)
struct BatchGroupLaunch {
    float4 *amps;
    const BatchInst *inst;
    const uint64_t *marked;
    const uint32_t *glist;      // instance indices, group by group
    const uint32_t *goff;       // [groups + 1] offsets into glist
    double *psucc;
    unsigned long long *region; // exchange words, groups x region_words
    size_t region_words;
    unsigned group_ctas;
    uint32_t slice_vecs;        // shared-memory vectors per CTA (the largest slice of this size)
    int *status;                // 3 if a wait runs out
    long long wait_limit;
    int stall;                  // test hook: CTA 0 of group 0 withholds its first partial sums
};
// CTAs of one group for a 2^n-amplitude instance: the fewest whose slices fit
// smem_max bytes each.
int batch_group_ctas(int n, size_t smem_max);
size_t batch_group_region_words(int group_ctas);
// Sets the kernel's shared-memory limit; *per_sm = resident CTAs per SM.
cudaError_t prepare_batch_group(size_t smem, int *per_sm);
// Zeroes the region and launches groups x group_ctas CTAs (cooperative).
cudaError_t enqueue_batch_group(const BatchGroupLaunch &L, unsigned groups, size_t smem, cudaStream_t st);

// ---- generalised phase iterator and its adjoint (k_phase.cu), complex64 ----
constexpr int kPhaseMaxGrid = 2048;  // CTAs of a phase-iterator launch
constexpr uint64_t kPhaseMaxMarked = 256;
// Constants one pass hands to the next (written by the pass's last CTA).
struct PhaseConst {
    float4 kpsi;        // kappa applied to psi as (re hi, re lo, im hi, im lo)
    float4 klam;        // kappa applied to lambda (backward only)
    float2 rot;         // e^{i phi} (forward) or e^{-i phi} (backward) on marked amplitudes
    double2 mean_psi;   // mean of the state the pass produced
    double2 mean_lam;   // mean of the adjoint the pass produced (backward only)
    double p_success;   // sum over marked x of |psi_x|^2 (last forward pass, backward start)
};
struct PhaseArgs {
    void *psi;                  // complex64 state, nvec 16-byte vectors
    void *lam;                  // complex64 adjoint (backward)
    uint64_t nvec;
    int n;
    const uint64_t *list;       // sorted marked indices
    uint32_t m;
    const double *phi, *vphi;   // [K] phases (device)
    long long t;                // iteration this pass applies (forward: -1 = initial reduction)
    long long K;
    const PhaseConst *cin;
    PhaseConst *cout;
    double2 *partials;          // [3 * 2 * kPhaseMaxGrid]
    unsigned *ticket;           // last-CTA-done counter, left at 0
    double *grad_phi, *grad_vphi;  // [K] (backward, device)
    double *stats;              // [2] P_success and -log P_success, or NULL (forward)
};
// Forward pass t (update) or the initial reduction (t = -1, no update);
// stream: streaming cache hints (data larger than L2).
cudaError_t launch_phase_fwd(const PhaseArgs &a, bool update, bool stream, cudaStream_t st, int sm_count);
// Backward pass t: psi and lambda through D(-vphi_t) then O(-phi_t).
cudaError_t launch_phase_bwd(const PhaseArgs &a, bool stream, cudaStream_t st, int sm_count);
// lambda_K from psi_K, dL/dvphi_{K-1} and the constants of backward pass K-1.
cudaError_t launch_phase_bwd_start(const PhaseArgs &a, bool stream, cudaStream_t st, int sm_count);

// ---- the phase iterator kept on chip (k_phase_grid.cu), complex64 ------------
// Constants of one step t, as float pairs (re hi, re lo, im hi, im lo).
struct PhaseFac {
    float4 em1;  // e^{i phi_t} - 1
    float4 omv;  // 1 - e^{i vphi_t}
    float2 rot;  // e^{i phi_t} rounded to complex64
    float2 pad;
};
constexpr size_t kPhaseGridSmemMax = 232448 - 8192;  // dynamic shared memory per CTA (227 KiB less static)
struct PhaseGridArgs {
    void *psi;                  // state (forward: psi_0 -> psi_K; backward: psi_K -> psi_0)
    void *lam;                  // adjoint output lambda_0 (backward)
    uint64_t nvec;              // 16-byte vectors
    uint32_t slice_vecs;        // vectors per CTA (the last may hold fewer)
    int n;
    const uint64_t *list;       // sorted marked indices
    uint32_t m;
    const double *phi, *vphi;   // [K] phases (device)
    long long K;
    unsigned long long *region; // exchange region (accumulators + counter zeroed before the launch)
    double *stats;              // forward: [2] P, -log P, or NULL
    double *grad_phi, *grad_vphi;  // backward: [K]
    int *status;                // 3 if a wait runs out
    long long wait_limit;
    int stall;                  // test hook: CTA 0 withholds its first contribution
    const PhaseFac *table;      // [K] per-step constants, or NULL (then formed in the sweep)
};
constexpr long long kPhaseTableMax = 1ll << 14;  // table entries kept in the handle's scratch
// Fills table[t] from phi_t, vphi_t (FP64 sincos, then split into float pairs).
cudaError_t launch_phase_table(const double *phi, const double *vphi, long long K, PhaseFac *table, cudaStream_t st);
// false if the state (backward: state and adjoint) does not fit the SMs' shared memory
bool phase_grid_plan(int n, bool backward, int sm_count, unsigned *G, uint32_t *slice_vecs, size_t *smem);
size_t phase_grid_region_bytes(unsigned G);  // whole exchange region
size_t phase_grid_zero_bytes();              // its part that must be zero at launch
cudaError_t launch_phase_grid(const PhaseGridArgs &a, bool backward, unsigned G, size_t smem, cudaStream_t st);

// ---- errors (grover_api.cu) ------------------------------------------------
// Sets the message grover_last_error(NULL) returns on this host thread.
void set_thread_error(const char *msg);

// ---- kernel attributes (grover_api.cu) ----------------------------------------
// Raises a kernel attribute (a shared-memory limit, the non-portable cluster
// permission) on the current device to at least `value`, once per device:
// attributes belong to a device's context, so a process driving several GPUs
// sets them on each.  Thread-safe.
cudaError_t raise_func_attr(const void *kern, cudaFuncAttribute attr, int value);
template <class F> cudaError_t raise_smem_limit(F kern, size_t smem) {
    return raise_func_attr(reinterpret_cast<const void *>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace grv

// Handle layout (opaque in the C ABI).
struct grover_state {
    int n;
    uint64_t N;
    grover_dtype dtype;
    grover_accum acc;
    void *amps;
    cudaStream_t stream;
    grv::Geometry geo;
    void *scratch_base;
    grv::Scratch sc;
    int resident;           // -1 auto, 0 never, 1 required (grover_set_option)
    int gate_engine;        // -1 auto, 0 CUDA cores, 1 tensor cores (grover_set_option)
    int staged;             // GROVER_OPT_STAGED_PASS: -1 auto, 0 never, 1 whenever possible
    long long wait_limit;   // polls of a bounded device-side wait
    int test_stall;         // test hook: the next tensor-core pass withholds its MMA signal
    int mu_slot;            // which mu[] holds the current mean
    bool mu_valid;          // cached mean of flip_key(c) is valid
    uint64_t mu_key;        // 0: mean of c itself; else id of the marked set applied
    void *phase_mem;        // phase-iterator scratch (allocated on first use)
    void *rg_mem;           // grid-resident iterator accumulators, counter, side sums (first use)
    char err[512];
};

struct grover_marked {
    int n;
    uint64_t id;            // unique per marked set in this process
    grv::MarkedDev dev;
    void *list_mem;
    void *words_mem;
    uint64_t *host_list;    // host copy of a list-built set (the gate-by-gate oracle reads its bits)
};
