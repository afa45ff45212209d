"""Differentiable far-field magnitudes over the library's JVP / JᵀVP kernels.

``far_field_magnitude(O, P, problem)`` returns zeta_k = (|F diag(P) S_k O|^2 + b)^(1/2) for
every scan position (Sec. 2, Eqs. exit_wave and expected_count; Sec. 4.1, Eq. magnitude)
as a torch tensor [K, m, m].  Its reverse-mode derivative is the library's J^T w and its
forward-mode derivative the library's J v (App. A; App. B Eq. jac_ampl), so any loss
written on zeta in torch can be differentiated through the CUDA kernels, e.g. the error
metrics of Eq. ell_magnitude.

Memory: the forward pass keeps the unit phasor psihat/zeta (8 K m^2 bytes) when that fits
``phasor_budget`` bytes, which lets the derivative kernels skip one 2D FFT per position;
otherwise the exit waves are recomputed from (O, P) in every derivative call.

Gradients follow torch's convention for complex inputs, which is the real-coordinate
gradient dRe + i dIm used throughout the library.
"""
from __future__ import annotations

import torch

from . import ptylm


class MagnitudeProblem:
    """Scan geometry for far_field_magnitude: a library context (object-only or joint)
    built from positions; no measurements are needed (y is a placeholder)."""

    def __init__(self, ny, nx, m, positions, background=1e-8, joint=False, phasor_budget=2 ** 30,
                 workspace_budget=0):
        self.ny, self.nx, self.m = int(ny), int(nx), int(m)
        self.K = int(positions.shape[0])
        self.joint = bool(joint)
        self.phasor_budget = int(phasor_budget)
        y = torch.zeros((self.K, self.m, self.m), dtype=torch.float32, device=positions.device)
        self.ctx = ptylm.lm_init(self.ny, self.nx, self.m, self.m, positions, y, ptylm.LOSS_GAUSSIAN,
                                 background, joint=int(self.joint), workspace_budget=workspace_budget)
        self._point = None  # identity of the (O, P) whose point the context currently holds

    @property
    def stores_phasor(self):
        return 8 * self.K * self.m * self.m <= self.phasor_budget

    def set_point(self, O, P):
        """Make (O, P) the point of the derivative kernels (recomputes zeta)."""
        zeta = torch.empty((self.K, self.m, self.m), dtype=torch.float32, device=O.device)
        ptylm.forward_magnitude(self.ctx, O, P, zeta, self.stores_phasor)
        self._point = self._key(O, P)
        return zeta

    @staticmethod
    def _key(O, P):
        return (O.data_ptr(), O._version, P.data_ptr(), P._version)

    def ensure_point(self, O, P):
        if self._point != self._key(O, P):
            self.set_point(O, P)


class _FarFieldMagnitude(torch.autograd.Function):
    @staticmethod
    def forward(O, P, problem):
        return problem.set_point(O, P)

    @staticmethod
    def setup_context(ctx, inputs, output):
        O, P, problem = inputs
        ctx.problem = problem
        ctx.save_for_backward(O, P)
        ctx.save_for_forward(O, P)

    @staticmethod
    def backward(ctx, grad_zeta):
        O, P = ctx.saved_tensors
        pb = ctx.problem
        pb.ensure_point(O, P)
        w = grad_zeta.contiguous().to(torch.float32)
        gO = torch.empty_like(O)
        want_p = pb.joint and ctx.needs_input_grad[1]
        gP = torch.empty_like(P) if want_p else None
        ptylm.jtvp(pb.ctx, w, gO, gP)
        return (gO if ctx.needs_input_grad[0] else None), gP, None

    @staticmethod
    def jvp(ctx, dO, dP, _):
        pb = ctx.problem
        O, P = ctx.saved_tensors
        pb.ensure_point(O, P)
        out = torch.empty((pb.K, pb.m, pb.m), dtype=torch.float32, device=O.device)
        dO = torch.zeros_like(O) if dO is None else dO.contiguous()
        vP = dP.contiguous() if (pb.joint and dP is not None) else None
        ptylm.jvp(pb.ctx, dO, out, vP=vP)
        return out


def far_field_magnitude(O, P, problem: MagnitudeProblem):
    """zeta [K, m, m] (float32) at (O, P); differentiable w.r.t. O (and P for joint problems)."""
    if O.dtype != torch.complex64 or P.dtype != torch.complex64:
        raise TypeError("O and P must be complex64 CUDA tensors")
    if not problem.joint and P.requires_grad:
        raise ValueError("probe gradients need a joint MagnitudeProblem")
    return _FarFieldMagnitude.apply(O.contiguous(), P.contiguous(), problem)
