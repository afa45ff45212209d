"""Parity at the full benchmark size (1024^2 object, 128^2 probe, 3600 jittered positions,
Poisson counts at 1e3 photons), with the context, grid and stream bench.py times.

The oracle cannot afford a full GGN product per test, so outputs are sampled: a 64 x 64
window of the object is touched only by the positions whose patches overlap it, and the
oracle run on just those positions gives the exact values of the full sums there.  The
error metric is compared over all 3600 positions.  Checks as in test_gpu_parity.py for
Poisson counts away from the truth: max(1e-5, 2 x the FP32 conditioning); at most twice the
error of the independent FP32 evaluation; and 1e-5 (2-norm and element-wise) on the
moderate-weight variant of the data.  Symmetry and positive semi-definiteness of the GGN
product are checked over the whole object.  Every achieved error is recorded."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.fp32_eval import Fp32Model, evaluations
from tests.problems import rel_err
from tests.test_gpu_parity import fp32_conditioning

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
WIN = (slice(480, 544), slice(480, 544))
_STATE = {}   # device positions of the benchmark context, set by the fixture


@pytest.fixture(scope="module")
def full(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    w = synth.LARGE
    dev = torch.device("cuda", 0)
    ctx, O0, P, y, pos, _ = bench.setup_workload(ptylm, torch, w, dev, torch.cuda.current_stream(dev))
    pos_np = pos.cpu().numpy()
    y_np = y.cpu().numpy().astype(np.float64)
    P_np = P.cpu().numpy().astype(np.complex128)
    # a point away from the flat start: the flat start plus a smooth phase texture
    O_np = O0.cpu().numpy().astype(np.complex128) * np.exp(0.3j * synth.object_texture(w.n, seed=9).imag)
    O_np = synth.to_c64(O_np)
    r, c = pos_np[:, 0], pos_np[:, 1]
    touch = (r < WIN[0].stop) & (r + w.m > WIN[0].start) & (c < WIN[1].stop) & (c + w.m > WIN[1].start)
    sub = oracle.Problem((w.n, w.n), P_np, pos_np[touch], y_np[touch], w.loss, 1e-8)
    whole = oracle.Problem((w.n, w.n), P_np, pos_np, y_np, w.loss, 1e-8)
    _STATE["pos"] = pos
    return ptylm, ctx, P, O_np, sub, whole, w


def dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def sub_fp32(sub, w):
    return Fp32Model((w.n, w.n), sub.P, sub.pos, sub.y, w.loss, 1e-8)


def test_full_size_error_metric(full):
    ptylm, ctx, P, O, sub, whole, w = full
    f, _ = ptylm.forward_loss(ctx, dev_c64(O), P, cache=0)
    f_ref = oracle.loss(whole, O)
    tol = max(TOL, 2.0 * fp32_conditioning(lambda A: oracle.loss(whole, A), w.m, O, trials=1))
    parity.check("f (all 3600 positions)", f, f_ref, tol, basis="2 x FP32 conditioning")


def test_full_size_gradient_window(full):
    ptylm, ctx, P, O, sub, whole, w = full
    assert sub.K > 100   # the window is covered by many overlapping patches
    ptylm.forward_loss(ctx, dev_c64(O), P, cache=1)
    g = torch.empty((w.n, w.n), dtype=torch.complex64, device="cuda")
    ptylm.gradient(ctx, g)
    ref = oracle.gradient(sub, O)[WIN]
    tol = max(TOL, 2.0 * fp32_conditioning(lambda A: oracle.gradient(sub, A)[WIN], w.m, O))
    got = host(g)[WIN]
    parity.check("grad f (64x64 window)", got, ref, tol, basis="2 x FP32 conditioning")
    parity.check_against_fp32("grad f (64x64 window)", got, ref,
                              [e[WIN] for e in evaluations(sub_fp32(sub, w), "gradient", O)])


def test_full_size_ggn_product_window(full):
    ptylm, ctx, P, O, sub, whole, w = full
    ptylm.forward_loss(ctx, dev_c64(O), P, cache=1)
    v = synth.to_c64(synth.random_complex((w.n, w.n), seed=21))
    out = torch.empty((w.n, w.n), dtype=torch.complex64, device="cuda")
    mdl = sub_fp32(sub, w)
    for lam in (0.0, 0.05):
        ptylm.ggn_matvec(ctx, dev_c64(v), out, lam)
        ref = oracle.ggn_matvec(sub, O, v, lam=lam)[WIN]
        tol = max(TOL, 2.0 * fp32_conditioning(lambda A, B: oracle.ggn_matvec(sub, A, B, lam=lam)[WIN], w.m, O, v))
        got = host(out)[WIN]
        parity.check(f"(G + {lam} I) v (64x64 window)", got, ref, tol, basis="2 x FP32 conditioning")
        parity.check_against_fp32(f"(G + {lam} I) v (64x64 window)", got, ref,
                                  [e[WIN] for e in evaluations(mdl, "ggn_matvec", O, v, lam=lam)])


def test_full_size_ggn_product_window_moderate_weights(full):
    """The benchmark's geometry with the measurements of the 1 % of detector pixels with the
    largest Poisson curvature weight replaced by the expected counts: 1e-5 on the window."""
    ptylm, ctx, P, O, sub, whole, w = full
    h = oracle.intensity(whole, O)
    d2l = 2.0 + 2.0 * whole.y / h
    y_mod = synth.to_f32(np.where(d2l > np.percentile(d2l, 99.0), h, whole.y))
    del h, d2l
    ctx2 = ptylm.lm_init(w.n, w.n, w.m, w.m, _STATE["pos"], torch.from_numpy(y_mod.astype(np.float32)).cuda(),
                         w.loss, 1e-8)
    ptylm.forward_loss(ctx2, dev_c64(O), P, cache=1)
    r, c = whole.pos[:, 0], whole.pos[:, 1]
    touch = (r < WIN[0].stop) & (r + w.m > WIN[0].start) & (c < WIN[1].stop) & (c + w.m > WIN[1].start)
    sub_mod = oracle.Problem((w.n, w.n), sub.P, whole.pos[touch], y_mod[touch], w.loss, 1e-8)
    v = synth.to_c64(synth.random_complex((w.n, w.n), seed=24))
    out = torch.empty((w.n, w.n), dtype=torch.complex64, device="cuda")
    ptylm.ggn_matvec(ctx2, dev_c64(v), out, 0.05)
    ref = oracle.ggn_matvec(sub_mod, O, v, lam=0.05)[WIN]
    parity.check("(G + 0.05 I) v (window, moderate weights)", host(out)[WIN], ref)
    parity.check("(G + 0.05 I) v (window, moderate weights)", host(out)[WIN], ref, norm="max")
    g = torch.empty_like(out)
    ptylm.gradient(ctx2, g)
    gref = oracle.gradient(sub_mod, O)[WIN]
    parity.check("grad f (window, moderate weights)", host(g)[WIN], gref)
    parity.check("grad f (window, moderate weights)", host(g)[WIN], gref, norm="max")
    ptylm.lm_destroy(ctx2)


def test_full_size_ggn_product_is_symmetric_psd(full):
    ptylm, ctx, P, O, sub, whole, w = full
    ptylm.forward_loss(ctx, dev_c64(O), P, cache=1)
    u = dev_c64(synth.random_complex((w.n, w.n), seed=22))
    v = dev_c64(synth.random_complex((w.n, w.n), seed=23))
    Gu, Gv = torch.empty_like(u), torch.empty_like(v)
    ptylm.ggn_matvec(ctx, u, Gu, 0.0)
    ptylm.ggn_matvec(ctx, v, Gv, 0.0)
    rdot = lambda a, b: float((a.real.double() * b.real.double() + a.imag.double() * b.imag.double()).sum())
    uGv, vGu = rdot(u, Gv), rdot(v, Gu)
    scale = np.sqrt(rdot(u, Gu) * rdot(v, Gv))
    assert abs(uGv - vGu) <= 1e-5 * scale
    assert rdot(u, Gu) > 0 and rdot(v, Gv) > 0
