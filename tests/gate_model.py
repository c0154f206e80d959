"""Host model of the gate path's Walsh-Hadamard passes (test infrastructure).

grover_iterate_gate applies, per iteration, the oracle, then H^{(x)n} as
passes over index-bit groups [lo, lo + kb) (the first transform scaled by
2^-kb per pass, the phase shift 2|0><0| - I after its last pass), then the
unscaled transform.  This module restates that pass plan and gives

* ``error_bound``: a worst-case bound on the 2-norm of the complex64 gate
  path's error vector, computed from the state that enters each pass;
* ``emulate``: the same passes in FP64 with every input of a tensor-core pass
  replaced by the sum of its first S bf16 slices and every stored output
  rounded to FP32, so that one-, two- and three-slice kernels can be compared
  on the CPU without building any of them;
* ``exact_input``: a state on which a correct tensor-core kernel is exact in
  FP32 arithmetic while one dropping a slice is not.

Neither the oracle nor the library imports this module, and it imports
neither of them.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24  # unit roundoff of FP32


# ---- the pass plan of grover_iterate_gate ---------------------------------------------------
def tc_pass_supported(n, lo, kb):
    """Groups the tensor-core pass takes (the others run on CUDA cores)."""
    if lo == 0:
        return kb == 7 and n >= 13
    return 5 <= kb <= 7 and lo >= 13 - kb and lo + kb <= n


def groups(n, tensor_cores):
    """Index-bit group sizes of one H^{(x)n}: tensor cores take 7 bits from
    bit 0 and the rest in 7-bit groups, or in near-equal groups where that
    leaves fewer groups they cannot take; CUDA cores use ceil(n / 8) groups of
    balanced sizes."""
    if tensor_cores:
        greedy = [7] * (n // 7) + ([n % 7] if n % 7 else [])
        parts = len(greedy) - 1
        if n < 13 or parts < 1:
            return greedy
        rest = n - 7
        bal = [7] + [rest // parts + (1 if j < rest % parts else 0) for j in range(parts)]

        def fallbacks(gs):
            return sum(not tc_pass_supported(n, sum(gs[:i]), k) for i, k in enumerate(gs))
        return bal if fallbacks(bal) < fallbacks(greedy) else greedy
    g = (n + 7) // 8
    return [n // g + (1 if i < n % g else 0) for i in range(g)]


TC_AUTO_MIN_QUBITS = 26  # smallest n whose default gate path uses the tensor cores


def engine_groups(n, engine):
    """(group sizes, tensor cores used) of grover_iterate_gate for a complex64
    state: engine 0 CUDA cores, 1 tensor cores, -1 the default (CUDA cores
    below n = 26; from there the plan with fewer groups, ties to the 7-bit
    one, with the tensor cores on every group they take)."""
    if engine in (True, 1):
        return groups(n, True), True
    if engine in (False, 0) or n < TC_AUTO_MIN_QUBITS:
        return groups(n, False), False
    t, c = groups(n, True), groups(n, False)
    return (t if len(t) <= len(c) else c), True


def pass_plan(n, tensor_cores):
    """[(lo, kb, on_tensor_cores, scaled, phase_shift_after)] of one iteration;
    tensor_cores: True / 1, False / 0, or -1 for the default engine."""
    gs, tc = engine_groups(n, tensor_cores)
    los = [sum(gs[:i]) for i in range(len(gs))]
    plan = []
    for p in range(2 * len(gs)):
        gi = p % len(gs)
        lo, kb = los[gi], gs[gi]
        plan.append((lo, kb, bool(tc and tc_pass_supported(n, lo, kb)), p < len(gs), p == len(gs) - 1))
    return plan


# ---- arithmetic of one pass ---------------------------------------------------------------
def walsh(kb):
    """W[j, k] = (-1)^popcount(j & k), order 2^kb (float64, exact)."""
    K = 1 << kb
    j = np.arange(K)[:, None]
    k = np.arange(K)[None, :]
    x = j & k
    par = np.zeros_like(x)
    while np.any(x):
        par ^= x & 1
        x >>= 1
    return np.where(par == 1, -1.0, 1.0)


def fibres(x, n, lo, kb):
    """View of the state as [outer][2^kb][2^lo]: axis 1 runs over bits [lo, lo + kb)."""
    return x.reshape(1 << (n - lo - kb), 1 << kb, 1 << lo)


def apply_pass(x, n, lo, kb, scale):
    """scale * W_{2^kb} on index bits [lo, lo + kb) (FP64 matrix products over
    the interleaved re/im view; exact on the small-integer inputs of
    ``exact_input``, within a few FP64 roundings otherwise)."""
    K = 1 << kb
    W = _walsh_cached(kb) * scale
    r = np.ascontiguousarray(x, dtype=np.complex128).view(np.float64).reshape(1 << (n - lo - kb), K, 2 << lo)
    if lo == 0:
        t = np.ascontiguousarray(r.transpose(0, 2, 1)).reshape(-1, K)
        y = (t @ W).reshape(-1, 2, K).transpose(0, 2, 1)
    else:
        y = np.matmul(W, r)
    return np.ascontiguousarray(y).reshape(-1).view(np.complex128)


_WALSH = {}


def _walsh_cached(kb):
    if kb not in _WALSH:
        _WALSH[kb] = walsh(kb)
    return _WALSH[kb]


def flip(x, marked):
    y = x.copy()
    idx = np.asarray(marked, dtype=np.int64)
    y[idx] = -y[idx]
    return y


def phase_shift(x):
    """2|0><0| - I: negate every amplitude but index 0."""
    y = -x
    y[0] = x[0]
    return y


# ---- bf16 slices ----------------------------------------------------------------------------
def bf16_rn(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    bits = a.view(np.uint32)
    # finite inputs only: the sum stays below 2^32
    rounded = (bits + np.uint32(0x7FFF) + ((bits >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return rounded.view(np.float32)


def slices(a, count):
    """Sum (float64) of the first `count` of the three bf16 slices a = b0 + b1 + b2
    the tensor-core pass builds: b0 = bf16(a), b1 = bf16(a - b0), b2 = bf16(a - b0 - b1)."""
    r = np.asarray(a, dtype=np.float32)
    total = np.zeros(r.shape, dtype=np.float64)
    for _ in range(count):
        b = bf16_rn(r)
        total += b.astype(np.float64)
        r = (r - b).astype(np.float32)  # exact: b holds the leading bits of r
    return total


def split_parts(z, count):
    re = slices(z.real.astype(np.float32), count)
    im = slices(z.imag.astype(np.float32), count)
    return re + 1j * im


# ---- emulation of a (possibly faulty) complex64 gate path ----------------------------------
def emulate(psi0, n, marked, k, slice_count, tensor_cores=True):
    """The complex64 gate path with `slice_count` bf16 slices per tensor-core
    operand: FP64 passes on the sliced inputs, FP32 stores; CUDA-core passes
    exact then stored in FP32.  Returns complex128."""
    x = psi0.astype(np.complex64).astype(np.complex128)
    plan = pass_plan(n, tensor_cores)
    for _ in range(k):
        x = flip(x, marked)
        for lo, kb, tc, scaled, ph in plan:
            inp = split_parts(x, slice_count) if tc else x
            x = apply_pass(inp, n, lo, kb, 2.0 ** -kb if scaled else 1.0)
            if ph:
                x = phase_shift(x)
            x = x.astype(np.complex64).astype(np.complex128)
    return x


# ---- worst-case error bound of the complex64 gate path -------------------------------------
def error_bound(psi0, n, marked, k, tensor_cores=True):
    """Bound on ||gpu - exact||_2 after k iterations of the complex64 gate path
    from the FP32-rounded start psi0.

    Tensor-core pass over K = 2^kb mids, scale s: every real output sums K
    products of exact bf16 slices in an FP32 accumulator (K/16 MMA steps of 16
    products, each step rounded or truncated once, error <= 2u of the step's
    result), adds the two accumulators (one rounding) and scales exactly, so
    |error| <= (K/16 + 3) u s L1, L1 = sum_k |x_k| over the fibre and real
    component that feed the output (the state entering the pass).  The error
    vector of the pass then has norm <= (K/16 + 3) u s sqrt(K sum_fibres L1^2).
    CUDA-core pass of kb butterfly stages: each stage rounds every output once,
    so the error vector has norm <= (kb + 1) u ||output||.  A later pass
    multiplies an error vector's norm by s sqrt(K) (s W / sqrt(K) is
    orthogonal); sign flips and the phase shift preserve it."""
    x = psi0.astype(np.complex64).astype(np.complex128)
    plan = pass_plan(n, tensor_cores)
    E = 0.0
    for _ in range(k):
        x = flip(x, marked)
        for lo, kb, tc, scaled, ph in plan:
            K = 1 << kb
            s = 2.0 ** -kb if scaled else 1.0
            y = apply_pass(x, n, lo, kb, s)
            if tc:
                f = fibres(x, n, lo, kb)
                l1r = np.sum(np.abs(f.real), axis=1)
                l1i = np.sum(np.abs(f.imag), axis=1)
                new = (K / 16 + 3) * U32 * s * np.sqrt(K * (np.sum(l1r * l1r) + np.sum(l1i * l1i)))
            else:
                new = (kb + 1) * U32 * np.linalg.norm(y)
            E = E * s * np.sqrt(K) + new
            x = phase_shift(y) if ph else y
    return E


# ---- an input on which the tensor-core pass must be exact -------------------------------------
# 18 significant bits whose bf16 split needs all three slices:
# C = 2^17 + 511 -> b0 = 131072, b1 = 512, b2 = -1 (b0 + b1 = C + 1)
EXACT_C = 131583
EXACT_SCALE = 2.0 ** -40


def exact_factor(kb):
    """Vector over one group's 2^kb mids.  kb >= 4: a Walsh row of order 16
    (row 5, which sums to zero) on block 1 of 16 mids (block 0 if there is only
    one), zero elsewhere; kb < 4: the unit vector at mid 0."""
    K = 1 << kb
    f = np.zeros(K)
    if kb >= 4:
        b = 1 if K >= 32 else 0
        f[16 * b: 16 * b + 16] = walsh(4)[5]
    else:
        f[0] = 1.0
    return f


def exact_input(n, tensor_cores=True):
    """C 2^-40 (1 + i/2) times the tensor product over the engine's index-bit
    groups of ``exact_factor``.

    Every pass of one H^{(x)n} then sees, in each fibre, a power of two times
    C times either a Walsh row on one block of 16 mids (the factor) or its
    transform, one entry +-16 per block (first and second transform trade the
    two forms).  Each 16-wide MMA step therefore adds 16 products of one
    magnitude, or a single nonzero product, to an accumulator of at most seven
    such step sums: every step is exact even if the tensor core aligned its
    addends to the largest one and truncated everything beyond 24 bits
    (``tc_fibre`` checks this).  The state has zero mean and the oracle's
    marked index lies outside its support, so G x = -x exactly: after one
    iteration the gate path must return -x bit for bit.  A split keeping two
    slices sees C + 1 in place of C."""
    x = np.ones(1)
    for kb in engine_groups(n, tensor_cores)[0]:
        x = np.kron(exact_factor(kb), x)  # lower groups vary fastest
    return x * (EXACT_C * EXACT_SCALE) * (1.0 + 0.5j)


def exact_marked(n):
    """A marked index outside the support of exact_input (lowest mids 0..15 are zero)."""
    return np.array([1 << (n - 1)], dtype=np.uint64)


def _rz24(a):
    """Truncate float64 values to 24 significant bits (toward zero)."""
    m, e = np.frexp(a)
    return np.ldexp(np.trunc(np.ldexp(m, 24)), e - 24)


def _rn24(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def tc_fibre(v, kb, slice_count, guard_bits=0):
    """One fibre of a tensor-core pass under a pessimistic model of the FP32
    accumulator: per MMA step of 16 products, the accumulator and the products
    are aligned to the largest of them, everything below 24 + guard_bits bits
    of it is truncated, the sum is formed and truncated to 24 bits.  The b0
    products go to one accumulator, the b1 then b2 products to another, and
    the two are added with one rounding (as the kernel does; per chunk of 16
    mids the order is A0 += b0, A12 += b1, A12 += b2).  v: real values
    of the fibre (float32-representable); returns W v as the model computes it."""
    K = 1 << kb
    W = _walsh_cached(kb)
    r = np.asarray(v, dtype=np.float32)
    parts = []
    for _ in range(3):
        b = bf16_rn(r)
        parts.append(b.astype(np.float64))
        r = (r - b).astype(np.float32)
    parts = parts[:slice_count] + [np.zeros(K)] * (3 - slice_count)

    def step(acc, b, c):
        prods = W[:, c:c + 16] * b[None, c:c + 16]
        addends = np.concatenate([acc[:, None], prods], axis=1)
        big = np.max(np.abs(addends), axis=1)
        e = np.where(big > 0, np.floor(np.log2(np.where(big > 0, big, 1.0))), 0.0)
        q = np.ldexp(1.0, (e - 23 - guard_bits).astype(int))[:, None]
        t = np.trunc(addends / q) * q
        return _rz24(np.sum(t, axis=1))

    # per K chunk of 16: A0 += b0 products, A12 += b1 products, A12 += b2 products
    a0 = np.zeros(K)
    a12 = np.zeros(K)
    for c in range(0, K, 16):
        a0 = step(a0, parts[0], c)
        a12 = step(a12, parts[1], c)
        a12 = step(a12, parts[2], c)
    return _rn24(a0 + a12)
