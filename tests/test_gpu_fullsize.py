"""Parity at the full benchmark size (1024^2 object, 128^2 probe, 3600 jittered positions,
Poisson counts at 1e3 photons), with the context, grid and stream bench.py times.

The oracle cannot afford a full GGN product per test, so outputs are sampled: a 64 x 64
window of the object is touched only by the positions whose patches overlap it, and the
oracle run on just those positions gives the exact values of the full sums there.  The
error metric is compared over all 3600 positions.  Tolerance: max(1e-5, 2 x the FP32
conditioning) as in test_gpu_parity.py (Poisson counts away from the truth); symmetry and
positive semi-definiteness of the GGN product are checked over the whole object."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests.problems import rel_err
from tests.test_gpu_parity import fp32_conditioning

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
WIN = (slice(480, 544), slice(480, 544))


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
    return ptylm, ctx, P, O_np, sub, whole, w


def dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def test_full_size_error_metric(full):
    ptylm, ctx, P, O, sub, whole, w = full
    f, _ = ptylm.forward_loss(ctx, dev_c64(O), P, cache=0)
    f_ref = oracle.loss(whole, O)
    tol = max(TOL, 2.0 * fp32_conditioning(lambda A: oracle.loss(whole, A), w.m, O, trials=1))
    assert abs(f - f_ref) <= tol * abs(f_ref), (f, f_ref, tol)


def test_full_size_gradient_window(full):
    ptylm, ctx, P, O, sub, whole, w = full
    assert sub.K > 100   # the window is covered by many overlapping patches
    ptylm.forward_loss(ctx, dev_c64(O), P, cache=1)
    g = torch.empty((w.n, w.n), dtype=torch.complex64, device="cuda")
    ptylm.gradient(ctx, g)
    ref = oracle.gradient(sub, O)[WIN]
    tol = max(TOL, 2.0 * fp32_conditioning(lambda A: oracle.gradient(sub, A)[WIN], w.m, O))
    assert rel_err(host(g)[WIN], ref) <= tol, tol


def test_full_size_ggn_product_window(full):
    ptylm, ctx, P, O, sub, whole, w = full
    ptylm.forward_loss(ctx, dev_c64(O), P, cache=1)
    v = synth.to_c64(synth.random_complex((w.n, w.n), seed=21))
    out = torch.empty((w.n, w.n), dtype=torch.complex64, device="cuda")
    for lam in (0.0, 0.05):
        ptylm.ggn_matvec(ctx, dev_c64(v), out, lam)
        ref = oracle.ggn_matvec(sub, O, v, lam=lam)[WIN]
        tol = max(TOL, 2.0 * fp32_conditioning(lambda A, B: oracle.ggn_matvec(sub, A, B, lam=lam)[WIN], w.m, O, v))
        assert rel_err(host(out)[WIN], ref) <= tol, (lam, tol)


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
