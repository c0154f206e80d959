/*
 * grover.h -- C ABI of libgrover.so, a GB300 (sm_103a) Grover search
 * state-vector simulator built around the equivalent-operator method of
 * Chattopadhyay & Menon, "Fast simulation of Grover's quantum search on
 * classical computer" (arXiv 2005.04635).
 *
 * The method (section "Proposed Simulation Method"): one Grover iteration
 * G = (2|psi><psi| - I) O is the oracle phase flip of the solution states
 * (Algorithm "n-qubit Oracle") followed by the inversion about the mean
 * (Algorithm "n-qubit Inversion about Mean"), c_x <- 2<c> - c_x with <c> the
 * complex arithmetic mean of all N = 2^n amplitudes.  The conventional circuit
 * (section "Background", conventional grover_search) applies H^{(x)n}, the
 * conditional phase shift 2|0><0| - I and H^{(x)n} instead of the inversion.
 *
 * Conventions for every call
 *   - State layout: N = 2^n interleaved complex amplitudes (re, im) in a
 *     caller-owned device buffer, complex64 (GROVER_C64, 8 B each) or
 *     complex128 (GROVER_C128, 16 B each), 16-byte aligned; the index is the
 *     basis state (section "Quantum State").
 *   - Streams: every call that launches work runs it on the stream given to
 *     grover_create (a cudaStream_t passed as void*; NULL = legacy default
 *     stream) and returns without waiting, unless stated otherwise.  Device-side
 *     failures (a bounded wait that gave up) are reported by grover_sync and by
 *     the calls that read results back.
 *   - Errors: every call returns a grover_status; nothing aborts or throws.
 *     grover_last_error gives a message for the last failure on a handle.
 *   - Threads: a handle or marked set must not be used by two host threads at
 *     once.  Handles on different streams are independent.
 *   - Sizes: 1 <= n <= 33 for GROVER_C64 and 1 <= n <= 32 for GROVER_C128,
 *     bounded in practice by device memory (n = 33 complex64 is 64 GiB).
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns GROVER_ECUDA.
 */
#ifndef GROVER_H
#define GROVER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GROVER_OK = 0,
    GROVER_EINVAL = 1,       /* bad argument: NULL pointer, n out of range, misaligned buffer */
    GROVER_ENOMEM = 2,       /* a host or device allocation failed */
    GROVER_ECUDA = 3,        /* a CUDA runtime call failed (message in grover_last_error) */
    GROVER_ETIMEOUT = 4,     /* a bounded device-side wait gave up (state is undefined) */
    GROVER_EUNSORTED = 5,    /* marked list not in increasing order */
    GROVER_EDUP = 6,         /* marked list holds an index twice */
    GROVER_ERANGE = 7,       /* marked index >= N, bitmask of the wrong size or with bits >= N */
    GROVER_EUNSUPPORTED = 8  /* valid request this build does not provide */
} grover_status;

typedef enum { GROVER_C64 = 0, GROVER_C128 = 1 } grover_dtype;

/* How the complex mean <c> is accumulated (section "Inversion About Mean
 * Operator"; the paper sums Re and Im separately in one running sum).  Every
 * mode combines per-block partial sums in a fixed order, so a result is
 * bitwise reproducible run to run.
 *   GROVER_ACC_DEFAULT: complex64: each thread's 8 amplitudes of a load group
 *                       (16 in the on-chip grid iterator from 6 vectors per
 *                       thread, n >= 20, and in the batches' groups of CTAs)
 *                       summed pairwise in FP32 (exact for equal values), each
 *                       such group sum added exactly as a fixed-point integer
 *                       with 100 fractional bits (group sums of magnitude 16
 *                       or more, Inf and NaN in FP64), threads and blocks
 *                       combined in integers,
 *                       one rounding at the end; complex128: GROVER_ACC_EXACT.
 *   GROVER_ACC_FP32:    complex64 only; plain FP32 running sum per thread and an
 *                       FP32 tree across the block, FP64 across blocks.
 *   GROVER_ACC_KAHAN:   complex64 only; Neumaier-compensated FP32 running sum
 *                       per thread and an FP32 tree across the block, FP64
 *                       across blocks.
 *   GROVER_ACC_FP64:    complex64: FP32 pairwise sum of each thread's 8
 *                       amplitudes per load group, FP64 above that;
 *                       complex128: FP64 throughout.
 *   GROVER_ACC_EXACT:   every amplitude of magnitude below 1 is added exactly as
 *                       a fixed-point integer with 100 fractional bits (larger
 *                       magnitudes in FP64); threads and blocks are combined in
 *                       double-double.  The sum is exact up to 2^-100 per
 *                       amplitude and a final double-double rounding. */
typedef enum {
    GROVER_ACC_DEFAULT = 0,
    GROVER_ACC_FP32 = 1,
    GROVER_ACC_KAHAN = 2,
    GROVER_ACC_FP64 = 3,
    GROVER_ACC_EXACT = 4
} grover_accum;

typedef struct grover_state grover_state;   /* opaque: n, dtype, buffer, stream, scratch, cached mean */
typedef struct grover_marked grover_marked; /* opaque: validated set of solution states on the device */

/* ---- handles ----------------------------------------------------------- */

/* Binds a state handle to a caller-owned device buffer of N = 2^n amplitudes
 * (section "Quantum State": psi[N], index = basis state).  dev_amps must be a
 * device pointer, 16-byte aligned, holding N elements of dtype; it is neither
 * initialised nor freed by the library.  cuda_stream is a cudaStream_t (or
 * NULL).  The library allocates a small device scratch area (< 1 MiB) that
 * grover_destroy frees.  *out is set only on GROVER_OK.  Synchronous. */
grover_status grover_create(grover_state **out, int n_qubits, grover_dtype dtype,
                            void *dev_amps, void *cuda_stream);

/* Waits for the handle's stream, then frees its scratch (not the amplitudes).
 * NULL is accepted. */
grover_status grover_destroy(grover_state *s);

/* Selects the accumulation of the complex mean (see grover_accum).
 * GROVER_EINVAL for FP32/KAHAN on a complex128 state. */
grover_status grover_set_accum(grover_state *s, grover_accum mode);

typedef enum {
    /* How grover_iterate runs.  Two persistent iterators keep the state in
     * shared memory for all k iterations and sum exactly (fixed point); they
     * need GROVER_ACC_DEFAULT or GROVER_ACC_EXACT.
     *   cluster: one thread-block cluster (16 CTAs x 200 KiB: n <= 18
     *            complex64, n <= 17 complex128), partials exchanged through
     *            distributed shared memory;
     *   grid:    up to one CTA per SM (cooperative launch; 152 x 226 KiB on
     *            GB300: n <= 22 complex64, n <= 21 complex128; small states
     *            use a quarter or half of the SMs, since the exchange costs
     *            more with more CTAs), partials added as integer limbs into
     *            global words that also count the arrivals, bounded waits (a
     *            wait that runs out sets the status word: GROVER_ETIMEOUT at
     *            grover_sync).
     *   -1 (default): the cluster iterator for n <= 12 (complex64) or n <= 11
     *                 (complex128); the grid iterator for 13 <= n <= 22
     *                 (complex64) or 12 <= n <= 21 (complex128); else one
     *                 fused pass per iteration (the faster choice at each n
     *                 as measured on GB300);
     *    0: always one fused pass per iteration;
     *    1: the cluster iterator where it fits, else the grid iterator
     *       (GROVER_EUNSUPPORTED where neither fits);
     *    2: the grid iterator (GROVER_EUNSUPPORTED where it does not fit). */
    GROVER_OPT_RESIDENT = 0,
    /* Engine of grover_iterate_gate's Walsh-Hadamard passes.
     *    0: CUDA cores, ceil(n/8) groups of balanced sizes;
     *    1: tensor cores, 7-bit groups (complex64; GROVER_EUNSUPPORTED for
     *       complex128 or n < 13); a group the tensor-core pass does not take
     *       (fewer than 5 bits above bit 0) runs on CUDA cores;
     *   -1 (default): complex64 with n >= 26: whichever of the two group plans
     *       has fewer groups (ties: the 7-bit one), every group of at most 7
     *       bits on the tensor cores and the 8-bit ones on CUDA cores; else
     *       CUDA cores.  Measured on GB300: at n >= 26 a tensor-core pass moves
     *       6.3-6.7 TB/s against 5.7-6.2 for a CUDA-core one; below, it has
     *       fewer tiles than its pipeline needs and is 1.4-3x slower. */
    GROVER_OPT_GATE_ENGINE = 1,
    /* Polls (about 0.1 us each) a bounded device-side wait makes before it
     * gives up; default 2^22.  A wait that gives up sets the device status
     * word, the kernel waits (bounded) for its own copies in flight, frees its
     * tensor memory and returns; grover_sync then returns GROVER_ETIMEOUT and
     * the state is undefined. */
    GROVER_OPT_WAIT_LIMIT = 2,
    /* Test hook for those failure paths: 1 makes the next tensor-core pass
     * of grover_iterate_gate withhold its MMA completion signal, the next
     * grid persistent launch (grover_iterate, or an on-chip phase sweep)
     * withhold CTA 0's first partial, or the next staged pass of
     * grover_iterate withhold CTA 0's first chunk copy, so a wait runs out
     * (reset to 0 once used).  Not for production use. */
    GROVER_OPT_TEST_STALL = 3,
    /* How an iteration pass of grover_iterate moves the state:
     *   -1 (default): complex64 states larger than half the L2 cache are
     *                 staged: CTAs stream 16 KiB chunks through two shared-
     *                 memory buffers each with bulk copies (cp.async.bulk; on
     *                 GB300 about 5 % more bandwidth than per-thread loads);
     *                 complex128 and smaller states use per-thread 16-byte
     *                 loads and stores;
     *    0: per-thread loads and stores always;
     *    1: staged whenever the state is a whole number of chunks (complex64
     *       n >= 11, complex128 n >= 10).
     * The results are the same bit for bit.  A staged copy whose wait runs
     * out sets the status word (GROVER_ETIMEOUT at grover_sync). */
    GROVER_OPT_STAGED_PASS = 4
} grover_option;

/* Sets an execution option of the handle (see grover_option).  GROVER_EINVAL
 * for an unknown option or value. */
grover_status grover_set_option(grover_state *s, grover_option opt, int64_t value);

/* ---- state preparation ------------------------------------------------- */

/* psi = H^{(x)n}|0...0>, written directly as c_i = 1/sqrt(N) rounded to the
 * storage type (both grover_search algorithms, first two steps). */
grover_status grover_init_uniform(grover_state *s);

/* Copies N amplitudes of the handle's dtype from amps (host memory if
 * amps_on_device == 0, device memory otherwise) into the state.  The copy is
 * not renormalised.  A host source is read before the call returns. */
grover_status grover_init_state(grover_state *s, const void *amps, int amps_on_device);

/* ---- marked sets (the oracle's data k[] in Algorithm "n-qubit Oracle") -- */

/* Builds a marked set for n-qubit states from a HOST list of m indices, which
 * must be strictly increasing (GROVER_EUNSORTED if an index is smaller than its
 * predecessor, GROVER_EDUP if equal) and < 2^n (GROVER_ERANGE).  m = 0 gives the
 * empty set (O = I).  The list is copied to the device; for m > 256 a bitmask
 * is built on the device as well.  *out is set only on GROVER_OK.  Synchronous. */
grover_status grover_marked_from_list(grover_marked **out, int n_qubits,
                                      const uint64_t *idx, size_t m);

/* Builds a marked set from a bitmask of nwords = ceil(2^n / 32) uint32 words:
 * index x is marked iff bit (x % 32) of word x / 32 is set.  words is host
 * memory if on_device == 0, else device memory.  GROVER_ERANGE if nwords is
 * wrong or a bit >= 2^n is set.  Synchronous (counts the set bits). */
grover_status grover_marked_from_bitmask(grover_marked **out, int n_qubits,
                                         const uint32_t *words, size_t nwords,
                                         int on_device);

/* Number of marked indices M. */
grover_status grover_marked_count(const grover_marked *mk, uint64_t *m);

/* Frees a marked set (waits for the device first).  NULL is accepted. */
grover_status grover_marked_destroy(grover_marked *mk);

/* ---- the Grover operators ---------------------------------------------- */

/* Algorithm "n-qubit Oracle": c_x <- -c_x for every marked x.  The marked set
 * must have been built for the state's n (GROVER_EINVAL otherwise). */
grover_status grover_oracle(grover_state *s, const grover_marked *mk);

/* Algorithm "n-qubit Inversion about Mean" (section "Inversion About Mean
 * Operator"): <c> = (1/N) sum_i c_i over ALL amplitudes, then
 * c_i <- 2<c> - c_i for all i.  Equals applying Delta = 2|psi><psi| - I. */
grover_status grover_diffuse(grover_state *s);

/* k Grover iterations of the proposed grover_search loop: each applies the
 * oracle then the inversion about the mean, as one fused device pass over the
 * state per iteration (the mean used by iteration t+1 is accumulated while
 * iteration t stores), or inside one persistent launch for states that fit
 * on chip (GROVER_OPT_RESIDENT).  k = 0 is a no-op. */
grover_status grover_iterate(grover_state *s, const grover_marked *mk, uint64_t k);

/* k iterations of the conventional circuit (section "Background",
 * conventional grover_search): oracle, H^{(x)n}, 2|0><0| - I, H^{(x)n}.
 * H^{(x)n} is a product of Walsh-Hadamard transforms on groups of index bits,
 * one read + write pass over the state per group, with exact power-of-two
 * scaling (2^-n per iteration in total); the phase shift is fused into the
 * last pass of the first transform.  Engines (GROVER_OPT_GATE_ENGINE): the
 * tensor cores (complex64: groups of 5-7 bits as dense +-1 matrix products,
 * operands split into three bf16 slices, FP32 accumulation) and CUDA cores
 * (+-1 butterflies); by default the tensor cores for complex64 states of
 * 2^26 amplitudes or more.  The result equals grover_iterate's up to
 * rounding (no global phase).  Invalidates the cached mean; a tensor-core wait
 * that gives up is reported by grover_sync (GROVER_ETIMEOUT). */
grover_status grover_iterate_gate(grover_state *s, const grover_marked *mk, uint64_t k);

/* k iterations of the conventional circuit GATE BY GATE, the way a gate-level
 * state-vector simulator runs it (section "Background", cost model
 * O([f_o(n) + f_c(n) + 2n] N^{3/2})): every single-qubit gate is one pass over
 * the state (Algorithm "1-qubit Unitary Operation").
 *   oracle      for each marked s (Fig. oracle1): X on every qubit where s has
 *               a 0, a multi-controlled Z on all n qubits (the register side
 *               of the multi-controlled NOT onto an ancilla in
 *               (|0> - |1>)/sqrt(2); it touches the single amplitude |1...1>),
 *               the same X gates again: f_o = sum_s (2 zeros(s) + 1) gates;
 *   H^{(x)n}    n Hadamards, scale 1/sqrt(2) rounded to the state's type;
 *   2|0><0| - I X^{(x)n}, MCZ, X^{(x)n} and a global -1 (carried by the next
 *               Hadamard's scale): f_c = 2n + 1 gates;
 *   H^{(x)n}.
 * gates_out / passes_out (optional, host): gates applied (the paper's count
 * f_o + f_c + 2n per iteration) and full passes over the state among them.
 * The marked set must be built from a list (GROVER_EUNSUPPORTED for bitmask
 * sets, whose indices are not on the host).  Asynchronous on the stream. */
grover_status grover_iterate_circuit(grover_state *s, const grover_marked *mk, uint64_t k,
                                     uint64_t *gates_out, uint64_t *passes_out);

/* floor(pi/4 * sqrt(2^n / m)), the iteration count that maximises the success
 * probability for m marked states out of 2^n (the paper's loop bound
 * pi*sqrt(N)/4 read as a floor, generalised to m solutions); 0 if m == 0 or
 * n is out of [1, 63]. */
uint64_t grover_optimal_iterations(int n_qubits, uint64_t m);

/* ---- measurement (section "Simulation Results", measurement outcome) --- */

/* p_i = |c_i|^2 in FP64 for all N basis states, written to out (N doubles;
 * host memory if out_on_device == 0, else device).  Synchronous for host
 * output. */
grover_status grover_measure_probs(grover_state *s, double *out, int out_on_device);

/* The m most probable basis states (1 <= m <= 16, m <= N) ordered by
 * (probability desc, index asc), written to HOST arrays idx[m], p[m]
 * (p in FP64).  Synchronous. */
grover_status grover_measure_topm(grover_state *s, size_t m, uint64_t *idx, double *p);

/* P_success = sum over marked x of |c_x|^2 and norm = sum over all i of
 * |c_i|^2, FP64 accumulation, written to HOST doubles (either may be NULL).
 * Synchronous. */
grover_status grover_success_prob(grover_state *s, const grover_marked *mk,
                                  double *p_success, double *norm);

/* ---- many independent searches in one launch ---------------------------- */

typedef struct grover_batch grover_batch; /* opaque: instance table, CUDA graph of the launch */

/* Amplitudes (complex64) a batch of `count` instances of n_qubits[i] qubits
 * needs: sum of 2^n_qubits[i]; 0 if some n is outside [1, 26]. */
uint64_t grover_batch_amps_needed(size_t count, const int *n_qubits);

/* Describes `count` independent searches, each the proposed grover_search
 * (section "Proposed Simulation Method") from the uniform state: instance i
 * has n_qubits[i] in [1, 26], k[i] iterations and the marked indices
 * marked[marked_offsets[i] .. marked_offsets[i+1]) (host arrays; each list
 * strictly increasing, < 2^n_qubits[i], at most 64 indices;
 * marked_offsets[0] = 0).  dev_amps is a caller-owned device buffer of
 * amps_capacity complex64 amplitudes, 16-byte aligned, at least
 * grover_batch_amps_needed(); instance i's state occupies 2^n_qubits[i]
 * amplitudes after those of instances 0..i-1.  The library copies the tables
 * to the device, orders the instances by decreasing N * k, and captures the
 * single persistent launch in a CUDA graph.  Synchronous. */
grover_status grover_batch_create(grover_batch **out, size_t count, const int *n_qubits, const uint64_t *k,
                                  const uint64_t *marked, const uint64_t *marked_offsets, void *dev_amps,
                                  uint64_t amps_capacity, void *cuda_stream);

/* Runs every instance: one launch of the captured graph on the batch's stream
 * (asynchronous).  A persistent grid takes instances from a work counter; one
 * thread block runs an instance's whole search (initial state, k iterations,
 * success probability), keeping it in shared memory when it fits the tuned
 * threshold; the large instances run as grover_batch_set_packing says (by
 * default on groups of CTAs, one cooperative launch per instance size, before
 * the small ones).  Sums are exact as in grover_iterate (complex64 default). */
grover_status grover_batch_run(grover_batch *b);

/* Times the batch under each thread count (256, 512, 1024) and on-chip
 * threshold (32, 64, 128 KiB) of the one-CTA kernel and keeps the fastest,
 * then times the whole batch with one CTA per instance against clusters of 16
 * for the instances of at least 17 or 19 qubits and groups of CTAs for those
 * of at least 15, 17 or 19 qubits (grover_batch_set_packing,
 * grover_batch_set_packing_min_qubits) and keeps the fastest (the batch runs
 * about 30 times); the one-CTA kernel's choice is returned if the pointers are
 * not NULL (grover_batch_get_packing gives the packing).  Synchronous. */
grover_status grover_batch_tune(grover_batch *b, int *threads, uint32_t *onchip_vecs);

/* How instances map to the GPU (default: 2 with threshold 15 where
 * cooperative launches run, else 1).  0 or 1: every instance on one CTA.
 * 16: each instance with n >= the packing threshold (at least 17) on one
 * thread-block cluster of 16 CTAs -- each CTA a slice of the state, in shared
 * memory up to 200 KiB per CTA (n <= 18), else streamed through L2 with one
 * large state per cluster live; the exact partial sums of an iteration meet
 * through distributed shared memory after a hardware cluster barrier -- and
 * the rest one per CTA.  2: each instance with n >= the threshold (at least
 * 15) whose state fits the shared memory of at most all SMs runs on a group of
 * G CTAs, G = ceil(state / 225 KiB) (n = 20: 37), the whole search in shared
 * memory, the exact partial sums exchanged through global memory every
 * iteration (bounded waits: grover_batch_success returns GROVER_ETIMEOUT if one
 * ran out); one cooperative launch per instance size, floor(SMs / G) groups
 * each taking its share of the instances; the rest one per CTA.  GROVER_EINVAL
 * for other values, GROVER_EUNSUPPORTED where clusters (16) or cooperative
 * launches (2) cannot run.  Rebuilds the captured graph. */
grover_status grover_batch_set_packing(grover_batch *b, int cluster_size);

/* Sets the packing threshold in qubits (15 to 26; clusters use at least 17).
 * GROVER_EINVAL outside that range.  Rebuilds the captured graph. */
grover_status grover_batch_set_packing_min_qubits(grover_batch *b, int min_qubits);

/* The packing in use: *cluster_size 1 (one CTA per instance), 2 (groups of
 * CTAs) or 16 (clusters), and the threshold in qubits (either pointer may be
 * NULL). */
grover_status grover_batch_get_packing(const grover_batch *b, int *cluster_size, int *min_qubits);

/* Options of the groups-of-CTAs launches: GROVER_OPT_WAIT_LIMIT (polls of a
 * bounded wait, default 2^22) and GROVER_OPT_TEST_STALL (1: in the next runs
 * the first CTA of the first group withholds its first partial sums, so that
 * group's waits run out and grover_batch_success returns GROVER_ETIMEOUT; the
 * other groups and the small instances are unaffected; 0: off).  GROVER_EINVAL
 * for other options or values.  Rebuilds the captured graph. */
grover_status grover_batch_set_option(grover_batch *b, grover_option opt, int64_t value);

/* Copies the count success probabilities sum_marked |c_x|^2 (FP64) of the last
 * run to the HOST array p_success.  Synchronous. */
grover_status grover_batch_success(grover_batch *b, double *p_success);

/* Waits for the batch's stream and frees its tables.  NULL is accepted. */
grover_status grover_batch_destroy(grover_batch *b);

/* ---- iteration without device allocation -------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory.  grover_create cudaMalloc's a small scratch
 * area, which some callers cannot do: code running while a framework's caching
 * allocator owns the device memory budget, loops that cannot take the implicit
 * device-wide synchronisation of cudaMalloc / cudaFree, or plug-ins that are
 * only handed device buffers.  This call performs k iterations like
 * grover_iterate (oracle then inversion about the mean, GROVER_ACC_FP64 sums)
 * on the caller's buffers and allocates nothing.
 *   dev_amps    device buffer of 2^n amplitudes of dtype, 16-byte aligned,
 *               updated in place;
 *   dev_marked  device array of m marked indices, strictly increasing and
 *               < 2^n (not checked: a list that breaks this gives wrong results
 *               but no out-of-bounds access); may be NULL when m == 0;
 *   cuda_stream the stream the work is queued on (asynchronous).
 * Its scratch (per-block partial sums, the mean, a counter) is a file-scope
 * device array of 33,280 bytes, which every GPU that loads the library holds
 * until the process exits; every pass it launches runs at most 2048 blocks,
 * one partial-sum slot each, whatever the device could hold at once.  n beyond
 * 33 (complex64) / 32 (complex128) is rejected with GROVER_EINVAL (message in
 * grover_last_error(NULL)).  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress) with that device current: make that first
 * call before any stream capture.  All calls on a device share the array and
 * it keeps the last call's contents (each call resets the counter it needs);
 * calls that overlap on the GPU -- on different streams, or from host threads
 * without ordering -- race on it and give wrong results. */
grover_status grover_iterate_noalloc(void *dev_amps, int n_qubits, grover_dtype dtype,
                                     const uint64_t *dev_marked, size_t m, uint64_t k,
                                     void *cuda_stream);

/* ---- generalised phase iterator and its adjoint ------------------------- */

/* A differentiable generalisation of the proposed grover_search loop (section
 * "Proposed Simulation Method"; the paper has no phases or gradients): the
 * oracle's sign flip becomes a phase and the inversion about the mean a
 * partial reflection,
 *   O(phi):  c_x <- e^{i phi} c_x for marked x        (Algorithm "n-qubit Oracle"
 *                                                       at phi = pi),
 *   D(vphi): c_i <- c_i - (1 - e^{i vphi}) <c>        (Algorithm "n-qubit
 *                                                       Inversion about Mean" at
 *                                                       vphi = pi, times -1),
 * with <c> = (1/N) sum_i c_i.  Iteration t = 0..K-1 applies D(vphi[t]) O(phi[t]).
 * The loss is L = -log P, P = sum over marked x of |c_x|^2 after the K
 * iterations.  Complex64 states only; the marked set must be a list of 1 to
 * 256 indices (grover_marked_from_list), else GROVER_EUNSUPPORTED.  Means are
 * exact sums of the FP32 amplitudes, rounded once; the per-iteration
 * constants are formed in FP64 (pass path) or in float-float arithmetic of
 * about 48 bits (on-chip path) and applied in FP32.  Where the state fits the SMs' shared
 * memory (GB300: n <= 22) and GROVER_OPT_RESIDENT is not 0, the whole sweep is
 * one cooperative launch with the state on chip (per-iteration sums exchanged
 * exactly through global memory, bounded waits: GROVER_ETIMEOUT at
 * grover_sync if one runs out); otherwise one pass over the state per
 * iteration plus one initial reduction.
 *
 *   phi, vphi  DEVICE arrays of K doubles (radians) on the state's device,
 *              read by the kernels when they run (stream order).
 *   stats      NULL or a DEVICE array of 2 doubles: receives P and L.
 *
 * Applies the K iterations to the handle's current state in place.  Returns
 * after enqueueing on the handle's stream.  P = 0 gives L = +inf. */
grover_status grover_phase_forward(grover_state *s, const grover_marked *mk, const double *phi,
                                   const double *vphi, uint64_t K, double *stats);

/* Adjoint of grover_phase_forward.  The handle's state must hold the output
 * psi_K of a forward call with the same mk, phi, vphi and K.  Each backward
 * pass recomputes psi_t from psi_{t+1} with the inverse iterators O(-phi[t])
 * D(-vphi[t]) (no stored intermediate states) and carries the adjoint
 * lambda_t = dL/d conj(psi_t) (Wirtinger derivative) through the same
 * operators, starting from lambda_K = -(marked part of psi_K) / P.  It writes
 *   grad_phi[t]  = dL/dphi[t]  = 2 Re(i sum_marked conj(lambda_t,x) psi_t,x),
 *   grad_vphi[t] = dL/dvphi[t] = 2 Re(i N conj(<lambda_{t+1}>) <psi_{t+1}>).
 *
 *   lam        DEVICE buffer of N complex64 (16-byte aligned, not overlapping
 *              the state), overwritten; holds lambda_0 on completion.
 *   grad_phi, grad_vphi  DEVICE arrays of K doubles, overwritten.
 *
 * On completion the handle's state holds psi_0 up to FP32 rounding (about K
 * units of roundoff).  On chip in one launch where the state and the adjoint
 * fit (GB300: n <= 21; the adjoint is carried as sqrt(P) lambda there, so its
 * sums stay in the fixed-point window), else K + 1 passes; enqueued on the
 * handle's stream. */
grover_status grover_phase_backward(grover_state *s, const grover_marked *mk, const double *phi,
                                    const double *vphi, uint64_t K, void *lam, double *grad_phi,
                                    double *grad_vphi);

/* ---- synchronisation and errors ----------------------------------------- */

/* Waits for the handle's stream and reads the device status word:
 * GROVER_ETIMEOUT if a bounded device-side wait gave up since the last call. */
grover_status grover_sync(grover_state *s);

/* Message for the last failure on s (s may be NULL: last failure on this host
 * thread).  The string is owned by the library. */
const char *grover_last_error(const grover_state *s);

/* Name of a status code. */
const char *grover_status_string(grover_status st);

#ifdef __cplusplus
}
#endif
#endif /* GROVER_H */
