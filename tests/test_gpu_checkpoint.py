"""Checkpoint / resume of Algorithm 1 on the GPU (lm_solve_resume): a run split in two, with
the iterate and the LM state (t, mu, delta) written to an .npz checkpoint and read back in
between, follows the uninterrupted run -- bit for bit on tiled scans, where no two patches
overlap and lm_solve is deterministic, and within tolerance on an overlapping scan, where the
scatter's float reductions round in a different order from run to run (the oracle's
bit-for-bit version is in test_oracle_pins.py).  Dropping the warm start or restarting the
surrogate schedule changes the continuation."""
import os

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


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _resume_split(lib, ctx, O0, P, tmp_path, n_first, n_second, **kw):
    """(uninterrupted run, split run with an .npz checkpoint between the parts)."""
    O_all = O0.clone()
    _, i_all = lib.lm_solve(ctx, O_all, P, hist_len=16, max_outer=n_first + n_second, **kw)
    O_a = O0.clone()
    st = lib.new_lm_state(ctx)
    _, i_a = lib.lm_solve(ctx, O_a, P, hist_len=16, max_outer=n_first, state=st, **kw)
    assert st["t"] == n_first and float(st["delta"].abs().max()) > 0
    path = os.path.join(str(tmp_path), "lm.npz")
    lib.save_lm_checkpoint(path, O_a, P, st)
    O_r, P_r, st_r = lib.load_lm_checkpoint(path)
    _, i_b = lib.lm_solve(ctx, O_r, P_r, hist_len=16, max_outer=n_second, state=st_r, **kw)
    assert st_r["t"] == n_first + n_second
    return (O_all, i_all), (O_a, i_a, st), (O_r, i_b)


def test_lm_resume_is_bit_identical_on_a_tiled_scan(lib, tmp_path):
    """On a tiled scan (no overlapping patches) lm_solve is deterministic, so the resumed run
    must equal the uninterrupted one bit for bit: iterate, error metric, damping and CG counts."""
    n, m = 256, 64
    case = make_case(n, m, loss=1, seed=63, grid=n // m, step=m, radius=0.3 * m, peak=1e4)
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(case.pos).cuda(),
                      torch.from_numpy(case.y.astype(np.float32)).cuda(), 1, case.b)
    P = _c64(case.P)
    O0 = _c64(synth.flat_object(n) * 0.9)
    (O_all, i_all), (O_a, i_a, st), (O_r, i_b) = _resume_split(lib, ctx, O0, P, tmp_path, 3, 4, beta=0.1)
    assert np.all(i_all["cg"] > 0)
    for k in ("f", "mu", "cg", "gnorm"):
        assert np.array_equal(np.concatenate([i_a[k], i_b[k]]), i_all[k]), k
    assert torch.equal(O_r, O_all)
    # control: the same continuation without the warm start lands elsewhere
    O_c = O_a.clone()
    lib.lm_solve(ctx, O_c, P, max_outer=4, state={"t": 3, "mu": st["mu"], "delta": None}, beta=0.1)
    assert not torch.equal(O_c, O_all)
    lib.lm_destroy(ctx)


def test_lm_resume_follows_the_uninterrupted_run_on_an_overlapping_scan(lib, tmp_path):
    """On an overlapping scan the scatter's float reductions round in a different order from run
    to run, and near a threshold of the damping update (rho = 0.25, 0.75) such a difference
    changes mu and with it every later step, so two runs of the same problem are not equal.  The
    resumed run must still start from the checkpoint exactly (its first error metric is that of
    the saved iterate) and stay on the uninterrupted run's path to within 1e-3 in f."""
    case = make_case(192, 64, K=60, loss=1, peak=1e3, seed=61)
    ctx = lib.lm_init(192, 192, 64, 64, torch.from_numpy(case.pos).cuda(),
                      torch.from_numpy(case.y.astype(np.float32)).cuda(), 1, case.b)
    P = _c64(case.P)
    O0 = _c64(synth.flat_object(192) * 0.9)
    (O_all, i_all), (O_a, i_a, st), (O_r, i_b) = _resume_split(lib, ctx, O0, P, tmp_path, 3, 4, fixed_cg=6)
    f_a, _ = lib.forward_loss(ctx, O_a, P, cache=0)
    assert abs(i_b["f"][0] - f_a) <= 1e-6 * abs(f_a)        # resumed at the checkpointed iterate
    f_split = np.concatenate([i_a["f"], i_b["f"]])
    assert np.all(np.abs(f_split - i_all["f"]) <= 1e-3 * np.abs(i_all["f"]))
    assert i_b["f"][-1] < i_b["f"][0]                          # and it keeps decreasing f
    lib.lm_destroy(ctx)


def test_joint_plm_s_resume_follows_the_surrogate_schedule(lib, tmp_path):
    """PLM-S on the joint state z = (O, P) across the end of a T = 4 surrogate schedule, tiled
    scan (deterministic): 2 + 3 outer iterations equal 5 uninterrupted ones bit for bit, and
    restarting the schedule at t = 0 does not."""
    import oracle
    n, m = 128, 32
    O_true = synth.to_c64(synth.object_texture(n, seed=4))
    P_true = synth.to_c64(synth.probe_disk_defocus(m, 10.0))
    pos, _ = synth.raster_positions(n, m, n // m, m, 0, seed=5)
    assert pos.max() + m == n
    pb = oracle.Problem((n, n), P_true, pos, None, 1, 1e-8)
    y = synth.to_f32(oracle.intensity(pb, O_true) * 50.0)
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(pos).cuda(), torch.from_numpy(y.astype(np.float32)).cuda(), 1,
                      1e-8, joint=1)
    P0 = _c64(synth.probe_disk_defocus(m, 10.0, phased=False) * np.sqrt(50.0))
    O0 = _c64(synth.flat_object(n) * 0.9)
    kw = dict(scaled=1, surrogate0=1.0, surrogate_end=1e-2, surrogate_T=4, beta=0.1)
    O_all, P_all = O0.clone(), P0.clone()
    _, i_all = lib.lm_solve(ctx, O_all, P_all, hist_len=6, max_outer=5, **kw)
    O_a, P_a = O0.clone(), P0.clone()
    st = lib.new_lm_state(ctx)
    assert st["delta"].numel() == n * n + m * m
    _, i_a = lib.lm_solve(ctx, O_a, P_a, hist_len=6, max_outer=2, state=st, **kw)
    path = os.path.join(str(tmp_path), "plm.npz")
    lib.save_lm_checkpoint(path, O_a, P_a, st)
    O_r, P_r, st_r = lib.load_lm_checkpoint(path)
    O_restart, P_restart = O_r.clone(), P_r.clone()
    st_restart = {"t": 0, "mu": st_r["mu"], "delta": st_r["delta"].clone()}
    _, i_b = lib.lm_solve(ctx, O_r, P_r, hist_len=6, max_outer=3, state=st_r, **kw)
    assert np.array_equal(np.concatenate([i_a["f"], i_b["f"]]), i_all["f"])
    assert torch.equal(O_r, O_all) and torch.equal(P_r, P_all)
    # restarting the surrogate schedule at t = 0 gives another trajectory
    lib.lm_solve(ctx, O_restart, P_restart, max_outer=3, state=st_restart, **kw)
    assert not torch.equal(O_restart, O_all)
    lib.lm_destroy(ctx)


def test_resume_argument_errors(lib):
    case = make_case(96, 32, K=5, loss=0, seed=62)
    ctx = lib.lm_init(96, 96, 32, 32, torch.from_numpy(case.pos).cuda(),
                      torch.from_numpy(case.y.astype(np.float32)).cuda(), 0, case.b)
    O, P = _c64(synth.flat_object(96)), _c64(case.P)
    for bad in ({"t": -1, "mu": 1e-5, "delta": None}, {"t": 0, "mu": 0.0, "delta": None},
                {"t": 0, "mu": float("nan"), "delta": None}):
        with pytest.raises(lib.PtylmError) as e:
            lib.lm_solve(ctx, O, P, max_outer=1, state=bad)
        assert e.value.status == lib.PTYLM_ERR_ARG
    lib.lm_destroy(ctx)
