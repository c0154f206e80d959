"""torch.autograd wrapper of the generalised phase iterator (complex64).

``phase_search_loss(phi, vphi, state, marked)`` runs K iterations of
D(vphi[t]) O(phi[t]) (oracle phase e^{i phi} on the marked amplitudes,
c <- c - (1 - e^{i vphi}) <c>) from the uniform state, or from ``init``, and
returns L = -log sum_marked |c_x|^2 as a 0-d CUDA float64 tensor.  Its backward
is the library's adjoint sweep (grover_phase_backward): the states are
recomputed by the inverse iterators, so nothing but the phases is saved.  At
phi = vphi = pi every step is -1 times the paper's Grover iterator.

Plumbing only: the forward and adjoint passes are the library's kernels; torch
provides the buffers, the stream and the chain rule's scaling by the incoming
gradient.
"""
from __future__ import annotations

import torch

from .binding import Marked, State


class PhaseSearchLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, vphi, state: State, marked: Marked, init=None):
        if phi.shape != vphi.shape or phi.dim() != 1:
            raise ValueError("phi and vphi must be 1-d tensors of K phases")
        phi = phi.detach().contiguous()
        vphi = vphi.detach().contiguous()
        if init is None:
            state.init_uniform()
        else:
            state.init_state(init)
        stats = torch.empty(2, dtype=torch.float64, device=phi.device)
        state.phase_forward(marked, phi, vphi, stats)
        ctx.save_for_backward(phi, vphi)
        ctx.state, ctx.marked = state, marked
        ctx.p_success = stats[0]
        return stats[1]

    @staticmethod
    def backward(ctx, grad_loss):
        phi, vphi = ctx.saved_tensors
        state: State = ctx.state
        lam = torch.empty(1 << state.n, dtype=torch.complex64, device=phi.device)
        g_phi = torch.empty_like(phi)
        g_vphi = torch.empty_like(vphi)
        state.phase_backward(ctx.marked, phi, vphi, lam, g_phi, g_vphi)
        return grad_loss * g_phi, grad_loss * g_vphi, None, None, None


def phase_search_loss(phi, vphi, state: State, marked: Marked, init=None):
    """L = -log P after K phase iterations; differentiable in phi and vphi."""
    return PhaseSearchLoss.apply(phi, vphi, state, marked, init)
