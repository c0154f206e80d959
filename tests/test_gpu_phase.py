"""Generalised phase iterator and its adjoint (complex64) against the FP64 oracle.

The iterator D(vphi) O(phi) (oracle phase e^{i phi} on the marked amplitudes,
c <- c - (1 - e^{i vphi}) <c>) and the loss L = -log sum_marked |c_x|^2 are
checked through the C ABI:

* at phi = vphi = pi it is -1 times the paper's Grover iterator, so K steps
  equal (-1)^K grover_iterate;
* states and losses equal the oracle's FP64 iterator; for a uniform start the
  two-amplitude reduced model gives the exact FP64 loss at any n;
* gradients equal FP64 central differences of the oracle (h = 1e-6), and
  central differences of the GPU loss itself (h = 1e-4);
* lambda_0 (the adjoint of the initial state) reproduces directional
  derivatives of the oracle's loss; the backward sweep rewinds the state;
* 200 Adam steps through the torch.autograd.Function lower the loss and stay
  below Zalka's bound sin^2((2K+1) theta).

Tolerances.  Amplitudes are stored in FP32 after every pass; a pass rounds
the phase product (FP32 factor and product: <= 3 * 2^-24 relative) and the
subtraction of kappa (<= 2^-24 of |c - kappa|), so each pass adds at most
about 2^-22 * A, where A bounds the amplitudes, and unitary steps do not
amplify it: states within (K + 1) * 2^-21 * A.  The loss -log P moves by at
most 2 |dP| / P, giving |dL| <= 2 (K + 1) * 2^-20 for a state of unit norm.
Gradients: each is a product of means or of marked sums of the recomputed
state and adjoint, both carrying the state bound above; 2e-4 of the largest
component covers this with margin.  GPU finite differences with h = 1e-4
divide a loss rounding of about (K + 1) * 2^-23 by 2h: 2e-2 of the largest
component.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2005_04635_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_04635_gb300 import binding
    binding.lib()
    return binding


def dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda").contiguous()


PATHS = {"auto": -1, "pass": 0}


def run_forward(B, n, marked, phi, vphi, init=None, path="auto"):
    st = B.State(n, "c64")
    st.set_resident(PATHS[path])
    mk = B.Marked(n, marked)
    if init is None:
        st.init_uniform()
    else:
        st.init_state(np.asarray(init, dtype=np.complex64))
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    st.phase_forward(mk, dev(phi), dev(vphi), stats)
    torch.cuda.synchronize()
    return st, mk, stats.cpu().numpy()


def amps(st):
    torch.cuda.synchronize()
    return st.amps.cpu().numpy().astype(np.complex128)


def oracle_traj_max(n, marked, phi, vphi, psi0):
    """max |c| over the oracle's states psi_0 .. psi_K."""
    psi = psi0.astype(np.complex128).copy()
    a = float(np.max(np.abs(psi)))
    for t in range(len(phi)):
        oracle.phase_grover(psi, n, marked, phi[t:t + 1], vphi[t:t + 1])
        a = max(a, float(np.max(np.abs(psi))))
    return a


def state_tol(K, A):
    return (K + 1) * 2.0 ** -21 * A


def p_tol(K, A, P, M):
    """Bound on |dP| for P = sum over M marked |c_x|^2 when every amplitude is
    within d = state_tol(K, A): sum 2 |c_x| d + d^2 <= 2 d sqrt(M P) + M d^2."""
    d = state_tol(K, A)
    return 2 * d * math.sqrt(M * P) + M * d * d


def c64_start(n, seed):
    """Gaussian start rounded to complex64 (the GPU and the oracle start from
    the same values)."""
    return inputs.gaussian_state(n, seed).astype(np.complex64).astype(np.complex128)


# ---- forward ----------------------------------------------------------------------
@pytest.mark.parametrize("n,m,K", [(3, 1, 5), (12, 1, 50), (12, 4, 25), (17, 2, 40)])
@pytest.mark.parametrize("path", ["auto", "pass"])
def test_pi_is_minus_grover(B, n, m, K, path):
    marked = inputs.marked_indices(n, m, seed=700 + n)
    phi = np.full(K, np.pi)
    st, _, stats = run_forward(B, n, marked, phi, phi, path=path)
    got = amps(st)
    ref = oracle.init_uniform(n)
    oracle.grover_operator(ref, n, marked, K)
    ref *= (-1) ** K
    assert np.max(np.abs(got - ref)) <= state_tol(K, 1.0)
    p_ref = oracle.success_prob(ref, n, marked)
    assert abs(stats[0] - p_ref) <= p_tol(K, 1.0, p_ref, m)
    assert abs(stats[1] + math.log(p_ref)) <= p_tol(K, 1.0, p_ref, m) / p_ref


@pytest.mark.parametrize("n,m,K", [(1, 1, 3), (2, 1, 4), (3, 2, 7), (5, 32, 6), (9, 5, 10), (14, 3, 20),
                                   (14, 256, 8), (16, 1, 12)])
@pytest.mark.parametrize("path", ["auto", "pass"])
def test_forward_matches_oracle(B, n, m, K, path):
    marked = inputs.marked_indices(n, m, seed=710 + n + m)
    phi, vphi = inputs.uniform_phases(K, seed=720 + n)
    psi0 = c64_start(n, seed=730 + n)
    st, _, stats = run_forward(B, n, marked, phi, vphi, init=psi0, path=path)
    got = amps(st)
    ref = psi0.copy()
    oracle.phase_grover(ref, n, marked, phi, vphi)
    A = oracle_traj_max(n, marked, phi, vphi, psi0)
    err = np.max(np.abs(got - ref))
    assert err <= state_tol(K, A), (err, state_tol(K, A))
    L_ref = oracle.phase_loss(ref, n, marked)
    P_ref = math.exp(-L_ref)
    assert abs(stats[0] - P_ref) <= p_tol(K, A, P_ref, m)
    assert abs(stats[1] - L_ref) <= 1.01 * p_tol(K, A, P_ref, m) / P_ref


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_forward_k0_is_loss_of_start(B, path):
    n, K = 10, 0
    marked = inputs.marked_indices(n, 3, seed=740)
    psi0 = c64_start(n, seed=741)
    st, _, stats = run_forward(B, n, marked, [], [], init=psi0, path=path)
    assert np.array_equal(amps(st), psi0)
    p = float(np.sum(np.abs(psi0[marked.astype(np.int64)]) ** 2))
    assert abs(stats[0] - p) <= 1e-12 * max(p, 1.0)
    assert abs(stats[1] + math.log(p)) <= 1e-10


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_uniform_n20_matches_reduced_model(B, path):
    """Workload n = 20, M = 3, K = 32, phases U(0, 2 pi): loss and the two
    amplitudes against the exact FP64 reduced model."""
    n, m, K = 20, 3, 32
    marked = inputs.marked_indices(n, m, seed=750)
    phi, vphi = inputs.uniform_phases(K, seed=751)
    st, _, stats = run_forward(B, n, marked, phi, vphi, path=path)
    L_ref, alpha, beta = oracle.phase_reduced(n, m, phi, vphi)
    got = amps(st)
    mask = np.zeros(1 << n, dtype=bool)
    mask[marked.astype(np.int64)] = True
    A = 1.0 / math.sqrt(1 << n) + abs(alpha)
    assert np.max(np.abs(got[mask] - alpha)) <= state_tol(K, max(A, abs(alpha)))
    assert np.max(np.abs(got[~mask] - beta)) <= state_tol(K, max(A, abs(beta)))
    # relative error of P: amplitude error / |alpha|, twice
    rel = 2 * state_tol(K, max(A, abs(alpha))) / abs(alpha)
    assert abs(stats[1] - L_ref) <= rel * 1.01


# ---- backward ----------------------------------------------------------------------
def run_backward(B, st, mk, phi, vphi):
    n = st.n
    lam = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    gp = torch.full((len(phi),), float("nan"), dtype=torch.float64, device="cuda")
    gv = torch.full((len(phi),), float("nan"), dtype=torch.float64, device="cuda")
    st.phase_backward(mk, dev(phi), dev(vphi), lam, gp, gv)
    torch.cuda.synchronize()
    return gp.cpu().numpy(), gv.cpu().numpy(), lam.cpu().numpy().astype(np.complex128)


def oracle_loss_fn(n, marked, psi0):
    def f(phi, vphi):
        psi = psi0.copy()
        oracle.phase_grover(psi, n, marked, phi, vphi)
        return oracle.phase_loss(psi, n, marked)
    return f


@pytest.mark.parametrize("n,m,K", [(2, 1, 3), (6, 3, 8), (12, 2, 12), (13, 7, 10)])
@pytest.mark.parametrize("path", ["auto", "pass"])
def test_gradients_match_oracle_fd(B, n, m, K, path):
    marked = inputs.marked_indices(n, m, seed=760 + n)
    phi, vphi = inputs.uniform_phases(K, seed=761 + n)
    psi0 = c64_start(n, seed=762 + n)
    st, mk, _ = run_forward(B, n, marked, phi, vphi, init=psi0, path=path)
    gp, gv, _ = run_backward(B, st, mk, phi, vphi)
    fp, fv = oracle.phase_grad_fd(oracle_loss_fn(n, marked, psi0), phi, vphi, h=1e-6)
    scale = max(np.max(np.abs(fp)), np.max(np.abs(fv)))
    assert np.all(np.isfinite(gp)) and np.all(np.isfinite(gv))
    assert np.max(np.abs(gp - fp)) <= 2e-4 * scale, (gp, fp)
    assert np.max(np.abs(gv - fv)) <= 2e-4 * scale, (gv, fv)
    # the sweep rewinds the state to psi_0
    back = amps(st)
    A = oracle_traj_max(n, marked, phi, vphi, psi0)
    assert np.max(np.abs(back - psi0)) <= 2 * state_tol(K, A)


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_n20_gradients(B, path):
    """n = 20, M = 3, K = 32, uniform start: adjoint gradients against the FP64
    reduced model (central differences, h = 1e-6) and against central
    differences of the GPU loss (h = 1e-4)."""
    n, m, K = 20, 3, 32
    marked = inputs.marked_indices(n, m, seed=750)
    phi, vphi = inputs.uniform_phases(K, seed=751)
    st, mk, stats = run_forward(B, n, marked, phi, vphi, path=path)
    gp, gv, lam = run_backward(B, st, mk, phi, vphi)
    fp, fv = oracle.phase_grad_fd(lambda a, b: oracle.phase_reduced(n, m, a, b)[0], phi, vphi, h=1e-6)
    scale = max(np.max(np.abs(fp)), np.max(np.abs(fv)))
    assert np.max(np.abs(gp - fp)) <= 2e-4 * scale
    assert np.max(np.abs(gv - fv)) <= 2e-4 * scale
    # central differences of the GPU loss at a few components
    st2 = B.State(n, "c64")
    st2.set_resident(PATHS[path])
    stats2 = torch.zeros(2, dtype=torch.float64, device="cuda")

    def gpu_loss(a, b):
        st2.init_uniform()
        st2.phase_forward(mk, dev(a), dev(b), stats2)
        torch.cuda.synchronize()
        return float(stats2[1].item())

    h = 1e-4
    for t in (0, 7, K // 2, K - 1):
        for arr, g in ((phi, gp), (vphi, gv)):
            up, dn = arr.copy(), arr.copy()
            up[t] += h
            dn[t] -= h
            if arr is phi:
                d = (gpu_loss(up, vphi) - gpu_loss(dn, vphi)) / (2 * h)
            else:
                d = (gpu_loss(phi, up) - gpu_loss(phi, dn)) / (2 * h)
            assert abs(d - g[t]) <= 2e-2 * scale, (t, d, g[t])


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_lambda0_gives_directional_derivatives(B, path):
    """dL along a direction delta of the initial state is 2 Re <lambda_0, delta>."""
    n, m, K = 11, 4, 9
    marked = inputs.marked_indices(n, m, seed=770)
    phi, vphi = inputs.uniform_phases(K, seed=771)
    psi0 = c64_start(n, seed=772)
    st, mk, _ = run_forward(B, n, marked, phi, vphi, init=psi0, path=path)
    _, _, lam = run_backward(B, st, mk, phi, vphi)
    f = oracle_loss_fn(n, marked, psi0)
    for s in range(3):
        delta = inputs.gaussian_state(n, seed=773 + s)
        h = 1e-6

        def L_at(eps):
            psi = psi0 + eps * delta
            oracle.phase_grover(psi, n, marked, phi, vphi)
            return oracle.phase_loss(psi, n, marked)

        fd = (L_at(h) - L_at(-h)) / (2 * h)
        got = 2.0 * np.real(np.vdot(lam, delta))
        scale = 2.0 * np.linalg.norm(lam)
        assert abs(got - fd) <= 2e-4 * scale, (got, fd)
    assert f(phi, vphi) > 0


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_backward_k0(B, path):
    n = 9
    marked = inputs.marked_indices(n, 2, seed=780)
    psi0 = c64_start(n, seed=781)
    st, mk, _ = run_forward(B, n, marked, [], [], init=psi0, path=path)
    gp, gv, lam = run_backward(B, st, mk, [], [])
    assert gp.size == 0 and gv.size == 0
    idx = marked.astype(np.int64)
    p = float(np.sum(np.abs(psi0[idx]) ** 2))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[idx] = -psi0[idx] / p
    assert np.max(np.abs(lam - want)) <= 2.0 ** -23 * np.max(np.abs(want))
    assert np.array_equal(amps(st), psi0)


def test_rejects_unsupported(B):
    n, K = 8, 2
    phi = dev([1.0, 2.0])
    st = B.State(n, "c128")
    mk = B.Marked(n, [3])
    with pytest.raises(B.GroverError) as e:
        st.phase_forward(mk, phi, phi)
    assert e.value.status == 8
    s64 = B.State(n, "c64")
    empty = B.Marked(n, [])
    with pytest.raises(B.GroverError) as e:
        s64.phase_forward(empty, phi, phi)
    assert e.value.status == 8
    words = inputs.bitmask(n, [1, 2])
    bm = B.Marked(n, bitmask=words)
    with pytest.raises(B.GroverError) as e:
        s64.phase_forward(bm, phi, phi)
    assert e.value.status == 8
    s10 = B.State(10, "c64")
    big = B.Marked(10, np.arange(257, dtype=np.uint64))
    with pytest.raises(B.GroverError) as e:
        s10.phase_forward(big, phi, phi)
    assert e.value.status == 8
    # a lambda buffer that is the state itself
    with pytest.raises(B.GroverError) as e:
        s64.phase_backward(mk, phi, phi, s64.amps, phi.clone(), phi.clone())
    assert e.value.status == 1


# ---- autograd and training -------------------------------------------------------------
def test_autograd_function_and_adam(B):
    """Workload n = 20, M = 3, K = 32, phases U(0, 2 pi), 200 Adam steps."""
    from paper_2005_04635_gb300.autograd import phase_search_loss
    n, m, K = 20, 3, 32
    marked = inputs.marked_indices(n, m, seed=750)
    phi0, vphi0 = inputs.uniform_phases(K, seed=751)
    st = B.State(n, "c64")
    mk = B.Marked(n, marked)
    phi = dev(phi0).requires_grad_(True)
    vphi = dev(vphi0).requires_grad_(True)
    loss = phase_search_loss(phi, vphi, st, mk)
    loss.backward()
    fp, fv = oracle.phase_grad_fd(lambda a, b: oracle.phase_reduced(n, m, a, b)[0], phi0, vphi0, h=1e-6)
    scale = max(np.max(np.abs(fp)), np.max(np.abs(fv)))
    assert np.max(np.abs(phi.grad.cpu().numpy() - fp)) <= 2e-4 * scale
    assert np.max(np.abs(vphi.grad.cpu().numpy() - fv)) <= 2e-4 * scale
    opt = torch.optim.Adam([phi, vphi], lr=0.05)
    first = float(loss.item())
    losses = []
    for _ in range(200):
        opt.zero_grad()
        loss = phase_search_loss(phi, vphi, st, mk)
        loss.backward()
        opt.step()
        losses.append(float(loss.item()))
    final = float(phase_search_loss(phi.detach(), vphi.detach(), st, mk).item())
    L_ref = oracle.phase_reduced(n, m, phi.detach().cpu().numpy(), vphi.detach().cpu().numpy())[0]
    assert abs(final - L_ref) <= 1e-4
    theta = math.asin(math.sqrt(m / (1 << n)))
    bound = math.sin((2 * K + 1) * theta) ** 2
    assert math.exp(-L_ref) <= bound * (1 + 1e-9)
    # the FP64 reduced model under the same optimiser reaches 4.57 from 9.02
    assert final < first - 4.0, (first, final)


def test_onchip_sweep_wait_runs_out(B):
    """Failure detection without a GPU fault: CTA 0 of the on-chip forward
    sweep withholds its first contribution (test hook), every wait runs out,
    grover_sync reports GROVER_ETIMEOUT and the handle stays usable."""
    n, K = 16, 4
    marked = inputs.marked_indices(n, 2, seed=790)
    phi, vphi = inputs.uniform_phases(K, seed=791)
    st = B.State(n, "c64")
    mk = B.Marked(n, marked)
    st.set_resident(2)
    st.set_option(2, 20000)
    st.set_option(3, 1)
    st.init_uniform()
    st.phase_forward(mk, dev(phi), dev(vphi))
    with pytest.raises(B.GroverError) as ei:
        st.sync()
    assert ei.value.status == 4
    st.set_option(2, 1 << 22)
    st.init_uniform()
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    st.phase_forward(mk, dev(phi), dev(vphi), stats)
    st.sync()
    psi = oracle.init_uniform(n)
    oracle.phase_grover(psi, n, marked, phi, vphi)
    assert abs(float(stats[1]) - oracle.phase_loss(psi, n, marked)) <= 1e-4


@pytest.mark.parametrize("path", ["auto", "pass"])
def test_scaled_start_takes_side_sums(B, path):
    """A start scaled by 64 puts amplitudes outside the fixed-point window (the
    FP64 side sums of every reduction, and on chip the side slots of the grid
    exchange); the loss shifts by -log(64^2) and the gradients are unchanged."""
    n, m, K = 15, 3, 6
    marked = inputs.marked_indices(n, m, seed=795)
    phi, vphi = inputs.uniform_phases(K, seed=796)
    psi0 = c64_start(n, seed=797)
    psi0[int(marked[0])] = 0.9
    psi0 = psi0.astype(np.complex64).astype(np.complex128)
    scaled = (psi0 * 64.0).astype(np.complex64).astype(np.complex128)
    st, mk, stats = run_forward(B, n, marked, phi, vphi, init=scaled, path=path)
    ref = scaled.copy()
    oracle.phase_grover(ref, n, marked, phi, vphi)
    A = oracle_traj_max(n, marked, phi, vphi, scaled)
    assert np.max(np.abs(amps(st) - ref)) <= state_tol(K, A)
    L_ref = oracle.phase_loss(ref, n, marked)
    assert abs(stats[1] - L_ref) <= 1e-4
    gp, gv, _ = run_backward(B, st, mk, phi, vphi)
    fp, fv = oracle.phase_grad_fd(oracle_loss_fn(n, marked, psi0), phi, vphi, h=1e-6)
    # here P ~ 0.8 and the gradients are small (~1e-4), so the bound is absolute:
    # |dL/dphi| <= 2 and |dL/dvphi| <= 2 / sqrt(P) for a unit-norm start, and the
    # recomputed states carry (K + 1) 2^-20 of relative error
    tol = (K + 1) * 2.0 ** -20 * 2.0 / math.sqrt(math.exp(-L_ref) / 64.0 ** 2)
    assert np.max(np.abs(gp - fp)) <= tol and np.max(np.abs(gv - fv)) <= tol
