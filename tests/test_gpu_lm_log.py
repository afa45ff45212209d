"""The per-outer-iteration record of lm_solve (history arrays and the JSONL log written by the
binding): one line per outer iteration of Algorithm 1 with f, ||grad f||, mu, lambda, the
gain ratio, the CG count, whether the step was accepted, wall-clock seconds and the object
error; consistent with the solve's own summary."""
import json

import numpy as np
import pytest

from paper_2103_01767_gb300 import synth
from tests.problems import make_case

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


def test_lm_jsonl_log(lib, tmp_path):
    w = synth.SMALL
    case = make_case(w.n, w.m, loss=0, seed=0, grid=w.grid, step=w.step, radius=w.radius)
    ctx = lib.lm_init(w.n, w.n, w.m, w.m, torch.from_numpy(case.pos).cuda(),
                      torch.from_numpy(case.y.astype(np.float32)).cuda(), 0, case.b)
    mask = torch.from_numpy(synth.illumination_mask(w.n, case.P, case.pos, 0.1).astype(np.uint8)).cuda()
    O = torch.from_numpy(synth.flat_object(w.n).astype(np.complex64)).cuda()
    P = torch.from_numpy(case.P.astype(np.complex64)).cuda()
    ref = torch.from_numpy(case.O_true.astype(np.complex64)).cuda()
    path = str(tmp_path / "lm.jsonl")
    st, info = lib.lm_solve(ctx, O, P, hist_len=20, O_ref=ref, mask=mask, max_outer=8, log_path=path)
    rows = [json.loads(l) for l in open(path)]
    # on these noiseless data f reaches its FP32 floor after 7-8 outer iterations; the
    # scatter's float reductions round differently from run to run, so the damping may run
    # away (PTYLM_ERR_STALLED) one iteration early
    n = info["n_outer"]
    assert len(rows) == n and (n == 8 or (n == 7 and st == lib.PTYLM_ERR_STALLED)), (n, st)
    assert [r["t"] for r in rows] == list(range(n))
    assert sum(r["cg"] for r in rows) == info["cg_total"]
    secs = [r["seconds"] for r in rows]
    assert all(s > 0 for s in secs) and all(b > a for a, b in zip(secs, secs[1:]))
    assert abs(rows[-1]["f"] - info["f"][-1]) == 0.0 and rows[-1]["err"] == info["err"][-1]
    p = lib.default_lm_params(0)
    for r in rows:
        assert r["accepted"] == (r["rho"] > p.rho_min)
        assert r["lambda"] > 0 and r["grad_norm"] > 0 and p.mu_min <= r["mu"]
    # every outer iteration ends with an accepted step unless the damping ran away
    assert all(r["accepted"] for r in rows)
    assert np.allclose([r["rho"] for r in rows], info["rho"])
    lib.lm_destroy(ctx)
