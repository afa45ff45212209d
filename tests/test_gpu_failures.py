"""Failure detection through the C-ABI, with every failure made on the host: no test here
faults, traps or hangs the GPU.

* A bounded device wait that runs out: the single-launch CG iteration's grid-wide waits are
  given a limit of one poll (ptylm_lm_params.wait_polls), so they give up while the last CTA
  is still summing; every CTA still finishes its in-bounds work and exits, lm_solve returns
  PTYLM_ERR_TIMEOUT, and the same context then solves normally.
* Non-finite values: a NaN planted in the iterate on the host makes the error metric's FP64
  reduction non-finite (PTYLM_ERR_NAN).
* Invalid measurements (Sec. 2: y are photon counts, finite and >= 0): lm_init,
  ptylm_set_measurements and ptylm_batch_init reject negative, infinite and NaN entries with
  PTYLM_ERR_ARG, and a rejected ptylm_set_measurements leaves the context's data as it was."""
import math

import numpy as np
import pytest

from paper_2103_01767_gb300 import synth
from tests.problems import make_case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    return ptylm


def _c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def _setup(lib, n=192, m=64, K=60, loss=1, seed=41):
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=seed)
    pos = torch.from_numpy(case.pos).cuda()
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    ctx = lib.lm_init(n, n, m, m, pos, y, loss, case.b)
    return case, ctx, pos, y


def test_cg_wait_timeout_is_reported_and_the_context_recovers(lib):
    """On a tiled scan (patches side by side, no overlaps) every scatter adds one contribution
    per object pixel, so lm_solve is deterministic: after the timeout the same context must
    reproduce a fresh context's run bit for bit."""
    n, m = 256, 64
    case = make_case(n, m, loss=1, seed=44, grid=n // m, step=m, radius=0.3 * m, peak=1e4)
    assert case.pos.max() + m == n
    pos = torch.from_numpy(case.pos).cuda()
    y = torch.from_numpy(case.y.astype(np.float32)).cuda()
    ctx = lib.lm_init(n, n, m, m, pos, y, case.loss, case.b)
    P = _c64(case.P)
    O0 = _c64(synth.flat_object(n) * 0.9)
    O = O0.clone()
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_solve(ctx, O, P, max_outer=2, wait_polls=1)
    assert e.value.status == lib.PTYLM_ERR_TIMEOUT, e.value
    # the same context, default waits: the same result as a fresh context
    O1 = O0.clone()
    st1, info1 = lib.lm_solve(ctx, O1, P, hist_len=4, max_outer=3)
    ctx2 = lib.lm_init(n, n, m, m, pos, y, case.loss, case.b)
    O2 = O0.clone()
    st2, info2 = lib.lm_solve(ctx2, O2, P, hist_len=4, max_outer=3)
    assert st1 == st2 == lib.PTYLM_OK
    assert info1["n_outer"] == info2["n_outer"] == 3 and info1["cg_total"] == info2["cg_total"] > 0
    assert np.array_equal(info1["f"], info2["f"])
    assert torch.equal(O1, O2)
    lib.lm_destroy(ctx)
    lib.lm_destroy(ctx2)


def test_nan_in_the_iterate_is_reported(lib):
    case, ctx, _, _ = _setup(lib, loss=0, seed=42)
    P = _c64(case.P)
    O = synth.flat_object(case.n).astype(np.complex64)
    O[37, 101] = complex(math.nan, 0.0)
    with pytest.raises(lib.PtylmError) as e:
        lib.forward_loss(ctx, _c64(O), P, cache=0)
    assert e.value.status == lib.PTYLM_ERR_NAN
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_solve(ctx, _c64(O), P, max_outer=2)
    assert e.value.status == lib.PTYLM_ERR_NAN
    # a finite iterate afterwards evaluates normally
    f, _ = lib.forward_loss(ctx, _c64(synth.flat_object(case.n)), P, cache=0)
    assert math.isfinite(f)
    lib.lm_destroy(ctx)


@pytest.mark.parametrize("bad", [-1.0, math.inf, math.nan])
def test_invalid_measurements_are_rejected(lib, bad):
    case, ctx, pos, y = _setup(lib, seed=43)
    P = _c64(case.P)
    O = _c64(synth.flat_object(case.n))
    f_before, _ = lib.forward_loss(ctx, O, P, cache=0)
    y_bad = y.clone()
    y_bad.view(-1)[12345] = bad
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_init(case.n, case.n, case.m, case.m, pos, y_bad, case.loss, case.b)
    assert e.value.status == lib.PTYLM_ERR_ARG
    with pytest.raises(lib.PtylmError) as e:
        lib.ptylm_set_measurements(ctx, y_bad)
    assert e.value.status == lib.PTYLM_ERR_ARG
    f_after, _ = lib.forward_loss(ctx, O, P, cache=0)
    assert f_after == f_before          # the rejected data never reached the context
    with pytest.raises(lib.PtylmError) as e:
        lib.batch_init([dict(ny=case.n, nx=case.n, m=case.m, positions=pos, y=y_bad, probe=P, loss=case.loss,
                             background=case.b)])
    assert e.value.status == lib.PTYLM_ERR_ARG
    lib.lm_destroy(ctx)
