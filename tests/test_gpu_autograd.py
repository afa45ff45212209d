"""Differentiable far-field magnitudes (paper_2103_01767_gb300.autograd) against the FP64
oracle and finite differences, with the phasor stored and with exit waves recomputed."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.fp32_eval import Fp32Model, evaluations
from tests.problems import make_case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import autograd, build
    build.build()
    return autograd


def c64(a, grad=False):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda().requires_grad_(grad)


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


@pytest.mark.parametrize("budget", [0, 2 ** 31])
@pytest.mark.parametrize("shape", [(96, 32, 37), (160, 64, 23), (288, 128, 11)])
def test_magnitude_forward_backward_and_jvp(ag, shape, budget):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=0, seed=70)
    pb = case.problem()
    problem = ag.MagnitudeProblem(n, n, m, torch.from_numpy(case.pos).cuda(), case.b, phasor_budget=budget)
    assert problem.stores_phasor == (budget > 0)
    O = case.O_true  # the truth: well-conditioned phases
    Od = c64(O, grad=True)
    zeta = ag.far_field_magnitude(Od, c64(case.P), problem)
    parity.check("zeta (autograd forward)", host(zeta), np.sqrt(oracle.intensity(pb, O)), TOL)
    parity.check("zeta (autograd forward)", host(zeta), np.sqrt(oracle.intensity(pb, O)), TOL, norm="max")
    w = synth.to_f32(synth.random_real((K, m, m), seed=71))
    (zeta * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    parity.check("J^T w (autograd backward)", host(Od.grad), oracle.jtvp(pb, O, w), TOL)
    parity.check("J^T w (autograd backward)", host(Od.grad), oracle.jtvp(pb, O, w), TOL, norm="max")
    # forward mode
    import torch.autograd.forward_ad as fwAD
    v = synth.to_c64(synth.random_complex((n, n), seed=72))
    with fwAD.dual_level():
        dual = fwAD.make_dual(c64(O), c64(v))
        out = ag.far_field_magnitude(dual, c64(case.P), problem)
        tangent = fwAD.unpack_dual(out).tangent
    jv_ref = oracle.jvp(pb, O, v)
    parity.check("J v (autograd forward mode)", host(tangent), jv_ref, TOL)
    parity.check_detector("J v (autograd forward mode)", host(tangent), jv_ref, oracle.intensity(pb, O) - case.b,
                          evaluations(Fp32Model((n, n), case.P, case.pos, case.y, 0, case.b), "jvp", O, v))


def test_joint_probe_gradient(ag):
    n, m, K = 160, 64, 23
    case = make_case(n, m, K=K, loss=0, seed=73)
    pb = case.problem()
    problem = ag.MagnitudeProblem(n, n, m, torch.from_numpy(case.pos).cuda(), case.b, joint=True)
    Od, Pd = c64(case.O_true, grad=True), c64(case.P, grad=True)
    w = synth.to_f32(synth.random_real((K, m, m), seed=74))
    (ag.far_field_magnitude(Od, Pd, problem) * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    rO, rP = oracle.jtvp(pb, case.O_true, w, probe_part=True)
    parity.check("joint J^T w object (autograd)", host(Od.grad), rO, TOL)
    parity.check("joint J^T w object (autograd)", host(Od.grad), rO, TOL, norm="max")
    parity.check("joint J^T w probe (autograd)", host(Pd.grad), rP, TOL)
    parity.check("joint J^T w probe (autograd)", host(Pd.grad), rP, TOL, norm="max")


def test_finite_differences(ag):
    """Directional derivative of L = sum w zeta (summed in FP64) by central differences of the
    CUDA forward model agrees with <grad, v> from the adjoint kernel.  zeta = (|psihat|^2+b)^(1/2)
    has kinks where psihat ~ 0, so w weights only pixels with zeta > 5% of its maximum, where a
    finite step cannot cross one (the oracle comparisons above cover every pixel exactly)."""
    n, m, K = 160, 64, 23
    case = make_case(n, m, K=K, loss=0, seed=75)
    problem = ag.MagnitudeProblem(n, n, m, torch.from_numpy(case.pos).cuda(), case.b)
    P = c64(case.P)
    zeta0 = np.sqrt(oracle.intensity(case.problem(), case.O_true))
    bright = (zeta0 > 0.05 * zeta0.max()).astype(np.float32)
    w = torch.from_numpy(synth.random_real((K, m, m), seed=76).astype(np.float32) * bright).cuda()
    O = c64(case.O_true, grad=True)
    L = (ag.far_field_magnitude(O, P, problem).double() * w.double()).sum()
    L.backward()
    v = c64(synth.random_complex((n, n), seed=77, scale=1.0))
    g = O.grad
    dd = float((torch.view_as_real(g).double() * torch.view_as_real(v).double()).sum())
    eps = 1e-3
    with torch.no_grad():
        Lp = (ag.far_field_magnitude(O + eps * v, P, problem).double() * w.double()).sum()
        Lm = (ag.far_field_magnitude(O - eps * v, P, problem).double() * w.double()).sum()
    fd = float(Lp - Lm) / (2 * eps)
    assert abs(fd - dd) <= 2e-3 * abs(dd), (fd, dd)


def test_torch_loss_gradient_matches_library_gradient(ag):
    """The Gaussian metric written in torch on top of far_field_magnitude differentiates to the
    library's fused gradient J^T grad_zeta l (App. A step 1)."""
    from paper_2103_01767_gb300 import ptylm
    n, m, K = 160, 64, 23
    case = make_case(n, m, K=K, loss=0, seed=78)
    pos = torch.from_numpy(case.pos).cuda()
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    O0 = synth.to_c64(case.O_true + synth.random_complex(case.O_true.shape, seed=79, scale=0.05))
    problem = ag.MagnitudeProblem(n, n, m, pos, case.b)
    O = c64(O0, grad=True)
    zeta = ag.far_field_magnitude(O, c64(case.P), problem)
    (0.5 * (zeta - y.sqrt()) ** 2).double().sum().backward()
    ctx = ptylm.lm_init(n, n, m, m, pos, y, ptylm.LOSS_GAUSSIAN, case.b)
    ptylm.forward_loss(ctx, c64(O0), c64(case.P), cache=1)
    g = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    ptylm.gradient(ctx, g)
    parity.check("grad f via torch-written metric", host(O.grad), host(g), TOL)
    parity.check("grad f via torch-written metric", host(O.grad), host(g), TOL, norm="max")
