"""Worst-case error bounds for complex64 results of the operator iterator
(test infrastructure: host arithmetic on the bounds only, nothing of the
method itself).

One iteration from a stored complex64 state c, u = 2^-24:
  * y = O c is exact (sign flips).
  * The sum S = sum_i y_i: each thread adds the amplitudes of a tile pairwise
    in FP32 -- 8 per tile in the streaming pass, the cluster iterator and the
    one-CTA batches, 16 in the groups of CTAs and in the grid iterator's wide
    slices -- so the tile sum is within gamma_4 * sum_tile |y_i| of exact
    (at most four levels, gamma_j = j u / (1 - j u)), for the real and the
    imaginary part alike and hence in modulus, and the tile sums are added
    exactly as fixed point (truncation below 2^-100 per tile).  So
    |S_hat - S| <= gamma_4 sum_i |y_i| <= gamma_4 sqrt(N) ||c||
    (Cauchy-Schwarz).  2 mu = 2 S / N reaches the update as a float pair
    hi + lo within 2^-46 |2 mu|.  Every amplitude therefore sees 2 mu off by at
    most (2 gamma_4 + 2^-45) ||c|| / sqrt(N): an error vector of norm
    <= (2 gamma_4 + 2^-45) ||c||.
  * The update c'_i = fl(fl(hi - y_i) + lo) rounds twice per stored amplitude
    (relative u each, real and imaginary parts alike): an error vector of norm
    <= 2u (1 + 8u) ||c||.
  * Per iteration: rho = 2 gamma_4 + 2^-45 + 2u (1 + 8u) <= 10u + 64u^2 times
    the norm of the state that enters it (8u + 64u^2 where every tile has 8
    amplitudes).  With every amplitude summed exactly (GROVER_ACC_EXACT) the
    first term goes: rho <= 2u + 32u^2.
The exact iteration is unitary, so the error e_t after t iterations obeys
e_{t+1} <= e_t + rho (||psi|| + e_t): e_k <= ((1 + rho)^k (1 + e_0) - 1) ||psi||,
with e_0 <= u ||psi|| for a start rounded to complex64.

The generalised phase iterator D(vphi) O(phi) (one pass on a stored state c):
  * marked amplitudes take the FP32 phase factor (within u of e^{i phi}) times
    c_x, a complex product within sqrt(5) u |c_x| of exact (Brent, Percival
    and Zimmermann's bound; 2u with fused multiply-adds): (1 + sqrt(5)) u
    |c_x| + O(u^2) in all;
  * kappa = (1 - e^{i vphi}) <O c> comes from FP32 tile sums of 8 amplitudes
    (16 in the on-chip forward sweep's wide slices) added exactly (the marked
    correction in FP64), and |1 - e^{i vphi}| <= 2, so kappa's error, met by
    all N amplitudes, is an error vector of norm <= 2 gamma_4 ||c||; its float
    pair adds 2^-45 ||c||;
  * c - kappa_hi - kappa_lo rounds twice: 2u ||c'||.
  rho_phase <= (1 + sqrt(5) + 8 + 2) u + O(u^2) <= 14u + 64u^2.  The backward
  sweep applies the same operations (subtraction, then rotation) to the state
  and to the adjoint, each within the same rho per pass.

Where the state is known to hold one value on the M marked and one on the
N - M unmarked amplitudes (the bitwise group check of a uniform start), the
error vector holds M copies of one difference and N - M copies of another, so
each value is within the norm bound over sqrt(M) (resp. sqrt(N - M)).
"""
from __future__ import annotations

import math

U = 2.0 ** -24
RHO = {"default": 10 * U + 64 * U * U, "tile8": 8 * U + 64 * U * U, "exact": 2 * U + 32 * U * U,
       "phase": 14 * U + 64 * U * U}


def rho_fp64(n):
    """GROVER_ACC_FP64 (streaming pass, 8-amplitude tiles): the tile sums, then
    FP64 running sums and an FP64 tree, no chain of which is longer than the
    N / 8 tile sums: relative error <= 2^(n - 3) 2^-53 (1 + 4u) on
    sum |tile sums|, doubled in 2 mu."""
    return RHO["tile8"] + 2.0 ** (n - 55)


def norm_bound(k, norm=1.0, rho=RHO["default"], start=U):
    """Bound on the 2-norm of the error vector after k iterations (module
    docstring), plus 1e-12 for the fixed-point truncation (< 2^-66 per sum)."""
    return (math.pow(1.0 + rho, k) * (1.0 + start) - 1.0) * norm + 1e-12


def group_bounds(n, m, k, rho=RHO["default"]):
    """Per-value bounds on the marked and the unmarked value of a grouped state
    of norm 1: the norm bound over sqrt(M) and over sqrt(N - M)."""
    e = norm_bound(k, 1.0, rho)
    return e / math.sqrt(m), e / math.sqrt((1 << n) - m)


def p_bound(P, E):
    """|P_hat - P| for P = sum over marked |c_x|^2 when the state's error vector
    has norm <= E: sqrt(P_hat) is within E of sqrt(P) (triangle inequality on
    the marked part), so |P_hat - P| <= 2 sqrt(P) E + E^2."""
    return 2.0 * math.sqrt(P) * E + E * E


def loss_bound(P, E):
    """|log P_hat - log P| <= |dP| / (P - |dP|) (mean value theorem), for the
    loss -log P."""
    dP = p_bound(P, E)
    return dP / (P - dP) if dP < P else math.inf
