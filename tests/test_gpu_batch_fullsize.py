"""Parity on the benchmark's 64-problem batch (objects 128-512, probes 32/64/128, 64-1024
positions, mixed losses), built exactly as bench.py builds it and run through one
persistent launch per operator.  For one problem of each probe side the oracle gives the
error metric over all of that problem's positions and the GGN product on a 32 x 32 window
(exact there from the positions whose patches overlap it).  Tolerances as in
test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests.problems import rel_err
from tests import parity
from tests.fp32_eval import Fp32Model, evaluations
from tests.test_gpu_parity import fp32_conditioning

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def batch64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    dev = torch.device("cuda", 0)
    members = synth.batch_members()
    probs, O0 = bench.setup_batch(ptylm, torch, dev, members)
    bt = ptylm.batch_init(probs, stream=torch.cuda.current_stream(dev))
    # a point away from the flat start
    O = torch.cat([(O0[bt.offsets[b]:bt.offsets[b + 1]].view(m.n, m.n) *
                    torch.from_numpy(np.exp(0.3j * synth.object_texture(m.n, seed=50 + b).imag).astype(np.complex64)).to(dev)
                    ).reshape(-1) for b, m in enumerate(members)])
    picks = [next(b for b, m in enumerate(members) if m.m == side) for side in (32, 64, 128)]
    return ptylm, bt, probs, members, O, picks


def problem(probs, members, b, positions=None):
    m = members[b]
    pos = probs[b]["positions"].cpu().numpy()
    y = probs[b]["y"].cpu().numpy().astype(np.float64)
    keep = np.ones(len(pos), bool) if positions is None else positions
    return oracle.Problem((m.n, m.n), probs[b]["probe"].cpu().numpy().astype(np.complex128), pos[keep], y[keep],
                          m.loss, 1e-8)


def tol_for(loss, fn, m, *arrays):
    return TOL if loss == 0 else max(TOL, 2.0 * fp32_conditioning(fn, m, *arrays, trials=1))


def test_batch64_error_metric(batch64):
    ptylm, bt, probs, members, O, picks = batch64
    f, _ = ptylm.batch_forward_loss(bt, O, cache=0)
    for b in picks:
        m = members[b]
        Ob = bt.views(O)[b].cpu().numpy().astype(np.complex128)
        pb = problem(probs, members, b)
        f_ref = oracle.loss(pb, Ob)
        tol = tol_for(m.loss, lambda A: oracle.loss(pb, A), m.m, Ob)
        parity.check(f"f[{b}] (probe {m.m}, all positions)", f[b], f_ref, tol,
                     basis="1e-5" if m.loss == 0 else "2 x FP32 conditioning")


def test_batch64_ggn_product_window(batch64):
    ptylm, bt, probs, members, O, picks = batch64
    ptylm.batch_forward_loss(bt, O, cache=1)
    v = torch.cat([torch.from_numpy(synth.to_c64(synth.random_complex((m.n, m.n), seed=60 + b)).astype(np.complex64))
                   .reshape(-1) for b, m in enumerate(members)]).cuda()
    out = torch.empty_like(v)
    ptylm.batch_ggn_matvec(bt, v, out, 0.01)
    for b in picks:
        m = members[b]
        c0 = m.n // 2 - 16
        win = (slice(c0, c0 + 32), slice(c0, c0 + 32))
        pos = probs[b]["positions"].cpu().numpy()
        touch = (pos[:, 0] < c0 + 32) & (pos[:, 0] + m.m > c0) & (pos[:, 1] < c0 + 32) & (pos[:, 1] + m.m > c0)
        pb = problem(probs, members, b, touch)
        Ob = bt.views(O)[b].cpu().numpy().astype(np.complex128)
        vb = bt.views(v)[b].cpu().numpy().astype(np.complex128)
        ref = oracle.ggn_matvec(pb, Ob, vb, lam=0.01)[win]
        tol = tol_for(m.loss, lambda A, B: oracle.ggn_matvec(pb, A, B, lam=0.01)[win], m.m, Ob, vb)
        got = bt.views(out)[b].cpu().numpy().astype(np.complex128)[win]
        assert touch.sum() > 0
        name = f"(G + 0.01 I) v[{b}] (probe {m.m}, 32x32 window)"
        if m.loss == 0:
            parity.check(name, got, ref)
            parity.check(name, got, ref, norm="max")
        else:
            parity.check(name, got, ref, tol, basis="2 x FP32 conditioning")
            mdl = Fp32Model((m.n, m.n), pb.P, pb.pos, pb.y, m.loss, 1e-8)
            parity.check_against_fp32(name, got, ref, [e[win] for e in evaluations(mdl, "ggn_matvec", Ob, vb,
                                                                                   lam=0.01)])
