/*
 * grover_oracle.h -- plain, slow FP64 CPU oracle for the Grover iterator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * timed CPU baseline of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA path and never calls it.
 *
 * Source: A. Chattopadhyay, V. Menon, "Fast simulation of Grover's quantum
 * search on classical computer" (arXiv 2005.04635).  Every function names the
 * section / algorithm / equation it follows.
 *
 * Conventions
 *   - A state psi of n qubits is N = 2^n complex amplitudes, stored as
 *     2N doubles interleaved (re_0, im_0, re_1, im_1, ...); index = basis state
 *     (section "Quantum State").
 *   - A marked set is a strictly increasing list of indices < N, or a bitmask of
 *     ceil(N/32) uint32 words (bit x%32 of word x/32 set <=> x marked).
 *   - Everything is computed in IEEE double precision, with no FMA contraction
 *     (built with -ffp-contract=off).
 */
#ifndef GROVER_ORACLE_H
#define GROVER_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- state preparation ------------------------------------------------- */
/* |0...0>: c_0 = 1, every other amplitude 0 (first step of both grover_search
 * algorithms). */
void or_init_zero(double *psi, int n);
/* c_i = 1/sqrt(N) for all i, i.e. H^{(x)n}|0> written out directly. */
void or_init_uniform(double *psi, int n);

/* ---- proposed method (section "Proposed Simulation Method") ------------ */
/* Algorithm "n-qubit Oracle": psi[k[i]] *= -1 for each listed solution. */
void or_oracle_list(double *psi, int n, const uint64_t *marked, size_t m);
/* Same operator, solutions given as a bitmask. */
void or_oracle_bitmask(double *psi, int n, const uint32_t *words);
/* Complex arithmetic mean <c> = (1/N) sum_i c_i, Re and Im summed separately in
 * index order with Neumaier's compensated summation (Algorithm "n-qubit
 * Inversion about Mean", first loop). */
void or_mean(const double *psi, int n, double *mu_re, double *mu_im);
/* Algorithm "n-qubit Inversion about Mean": c_i <- 2<c> - c_i for every i. */
void or_inversion_mean(double *psi, int n);
/* Proposed grover_search loop body repeated k times:
 * oracle then inversion about the mean. */
void or_grover_operator(double *psi, int n, const uint64_t *marked, size_t m,
                        uint64_t k);
void or_grover_operator_bitmask(double *psi, int n, const uint32_t *words,
                                uint64_t k);

/* ---- conventional circuit (section "Background") ----------------------- */
/* Eq. (unitary) / Algorithm "1-qubit Unitary Operation" with U = H on target
 * qubit q, as an out-of-place pair butterfly. */
void or_hadamard_qubit(double *psi, int n, int q);
/* H^{(x)n}: n single-qubit Hadamards. */
void or_hadamard_all(double *psi, int n);
/* Conditional phase shift 2|0><0| - I: keep c_0, negate all others. */
void or_phase_shift_zero(double *psi, int n);
/* Conventional grover_search loop body repeated k times:
 * oracle, H^{(x)n}, 2|0><0|-I, H^{(x)n}. */
void or_grover_gate(double *psi, int n, const uint64_t *marked, size_t m,
                    uint64_t k);

/* ---- the conventional circuit gate by gate (section "Background",
 *      Fig. oracle1; cost model O([f_o(n) + f_c(n) + 2n] N^{3/2})) ------- */
/* Pauli X on qubit q. */
void or_x_qubit(double *psi, int n, int q);
/* Multi-controlled Z on all n qubits (phase -1 on |1...1>): the action on the
 * register of Fig. oracle1's multi-controlled NOT onto an ancilla prepared in
 * (|0> - |1>)/sqrt(2) (phase kickback).  negate_all: also multiply the whole
 * state by -1.  One pass over all N amplitudes. */
void or_mcz(double *psi, int n, int negate_all);
/* k iterations, one gate (one pass) at a time: the oracle for each marked s
 * as X on every qubit where s has a 0, MCZ, the same X gates (f_o = sum over
 * marked s of 2 zeros(s) + 1); H^{(x)n} as n single-qubit Hadamards; the
 * phase shift 2|0><0| - I as X^{(x)n}, -MCZ, X^{(x)n} (f_c = 2n + 1); H^{(x)n}.
 * Returns the number of gates applied. */
uint64_t or_grover_circuit(double *psi, int n, const uint64_t *marked, size_t m, uint64_t k);

/* ---- iteration count, closed forms ------------------------------------- */
/* floor(pi/4 * sqrt(N/M)); 0 when m == 0. */
uint64_t or_optimal_iterations(int n, uint64_t m);
/* Uniform initial state, m marked indices, k iterations (textbook analysis of
 * G = (2|psi><psi| - I) O as a rotation by 2*theta, sin(theta) = sqrt(M/N)):
 * marked amplitude sin((2k+1)theta)/sqrt(M), unmarked cos((2k+1)theta)/sqrt(N-M).
 * A value whose group is empty is returned as 0. */
void or_closed_form_uniform(int n, uint64_t m, uint64_t k, double *a_marked,
                            double *a_unmarked);
/* Arbitrary initial state, in place: decomposes c into the marked mean alpha,
 * the unmarked mean beta and their zero-sum deviations d, e; k iterations
 * rotate (sqrt(M) alpha, sqrt(N-M) beta) by -2k*theta, keep d and multiply e by
 * (-1)^k. O(N) for any k. */
void or_closed_form_general(double *psi, int n, const uint64_t *marked,
                            size_t m, uint64_t k);

/* ---- measurement (section "Simulation Results", measurement outcome) --- */
void or_probs(const double *psi, int n, double *p);          /* |c_i|^2 */
double or_norm(const double *psi, int n);                    /* sum |c_i|^2 */
double or_success_prob(const double *psi, int n, const uint64_t *marked,
                       size_t m);
/* The m most probable basis states, ordered by (probability desc, index asc).
 * m <= N. */
void or_topm(const double *psi, int n, size_t m, uint64_t *idx, double *p);

/* ---- summation primitive ----------------------------------------------- */
/* Neumaier (1974) compensated sum of x[0], x[stride], ..., x[(count-1)*stride]
 * in that order. */
double or_neumaier_sum(const double *x, size_t count, size_t stride);

/* ---- generalised phase iterator (differentiation; not in the paper) ----- */
/* Oracle O(phi): c_x <- e^{i phi} c_x for marked x.  Diffusion D(vphi):
 * c_i <- c_i - (1 - e^{i vphi}) <c>.  At phi = vphi = pi, D(pi) O(pi) is -1
 * times the paper's Grover iterator G.  K iterations with per-iteration
 * phases phi[t], vphi[t] (t = 0..K-1), in place. */
void or_phase_grover(double *psi, int n, const uint64_t *marked, size_t m, const double *phi,
                     const double *vphi, uint64_t K);
/* Loss -log sum_marked |c_x|^2. */
double or_phase_loss(const double *psi, int n, const uint64_t *marked, size_t m);
/* The same iterator from the uniform state, reduced to the two amplitudes
 * alpha (every marked one) and beta (every unmarked one), which is exact for
 * a uniform start; returns the loss -log(M |alpha|^2), alpha and beta. */
double or_phase_reduced(int n, uint64_t m, const double *phi, const double *vphi, uint64_t K,
                        double *alpha_re, double *alpha_im, double *beta_re, double *beta_im);

/* ---- test hook ---------------------------------------------------------- */
/* Plants one known mistake (for tests that show the pins catch it):
 *   0 none; 1 inversion loops stop at N-1; 2 phase shift I-2|0><0|;
 *   3 update with <c> instead of 2<c>; 4 oracle flips index+1;
 *   5 imaginary part updated with the wrong sign; 6 butterfly outputs swapped;
 *   7 closed form rotates the wrong way; 8 mean divides by N-1.
 * Returns the previous value.  Never set outside tests. */
int or_set_mutation(int which);

#ifdef __cplusplus
}
#endif
#endif
