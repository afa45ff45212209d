"""CUDA path (through the C-ABI) against the FP64 oracle on identical seeded inputs.

Tolerances: relative 1e-5 (2-norm) on f, grad f, J v, J^T w and (G + lambda I) v, the
FP32 bound stated for the method's hot path; the FP64 oracle's own error is ~1e-13."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests.problems import make_case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01767_gb300 import build, ptylm
    build.build()
    ptylm.load_library()
    return ptylm


def dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def dev_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


class GpuCase:
    def __init__(self, lib, case):
        self.lib, self.case = lib, case
        self.pos = dev_i32(case.pos)
        self.y = dev_f32(case.y)
        self.P = dev_c64(case.P)
        self.ctx = lib.lm_init(case.n, case.n, case.m, case.m, self.pos, self.y, case.loss, case.b)

    def point(self, seed=5, scale=0.05):
        O = synth.to_c64(self.case.O_true + synth.random_complex(self.case.O_true.shape, seed=seed, scale=scale))
        return O


# (object side, probe side, K) -- several tiles per side and ragged position counts; the last
# of each size makes the persistent CTAs loop over more than one position.
SHAPES = [(96, 32, 37), (160, 64, 23), (288, 128, 11), (256, 32, 3000), (512, 64, 1000), (640, 128, 400)]


@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_loss_and_gradient(lib, shape, loss):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=11)
    g = GpuCase(lib, case)
    O = g.point()
    Od = dev_c64(O)
    f, dl2 = lib.forward_loss(g.ctx, Od, g.P, cache=1)
    pb = case.problem()
    f_ref, dl2_ref = oracle.loss(pb, O, return_dl_norm2=True)
    assert abs(f - f_ref) <= TOL * abs(f_ref), (f, f_ref)
    assert abs(dl2 - dl2_ref) <= TOL * abs(dl2_ref), (dl2, dl2_ref)
    gd = torch.empty_like(Od)
    lib.gradient(g.ctx, gd)
    assert rel_err(host(gd), oracle.gradient(pb, O)) <= TOL
    # loss-only evaluation at another point leaves the linearisation intact
    f2, _ = lib.forward_loss(g.ctx, dev_c64(g.point(seed=6)), g.P, cache=0)
    assert abs(f2 - oracle.loss(pb, g.point(seed=6))) <= TOL * abs(f2)
    lib.gradient(g.ctx, gd)
    assert rel_err(host(gd), oracle.gradient(pb, O)) <= TOL


@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_ggn_matvec(lib, shape, loss):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=12)
    g = GpuCase(lib, case)
    O = g.point()
    lib.forward_loss(g.ctx, dev_c64(O), g.P, cache=1)
    v = synth.to_c64(synth.random_complex(O.shape, seed=13))
    vd = dev_c64(v)
    out = torch.empty_like(vd)
    pb = case.problem()
    for lam in (0.0, 0.37):
        lib.ggn_matvec(g.ctx, vd, out, lam)
        ref = oracle.ggn_matvec(pb, O, v, lam=lam)
        assert rel_err(host(out), ref) <= TOL, lam


@pytest.mark.parametrize("shape", SHAPES)
def test_jvp_and_jtvp(lib, shape):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=1, peak=1e3, seed=14)
    g = GpuCase(lib, case)
    O = g.point()
    lib.forward_loss(g.ctx, dev_c64(O), g.P, cache=1)
    pb = case.problem()
    v = synth.to_c64(synth.random_complex(O.shape, seed=15))
    out = torch.empty((K, m, m), dtype=torch.float32, device="cuda")
    lib.jvp(g.ctx, dev_c64(v), out)
    assert rel_err(host(out), oracle.jvp(pb, O, v)) <= TOL
    w = synth.to_f32(synth.random_real((K, m, m), seed=16))
    outO = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    lib.jtvp(g.ctx, dev_f32(w), outO)
    assert rel_err(host(outO), oracle.jtvp(pb, O, w)) <= TOL


def test_adjoint_identity_on_gpu(lib):
    """<J v, w> = <v, J^T w> for the CUDA operators themselves (FP32: relative 1e-5)."""
    case = make_case(160, 64, K=23, loss=0, seed=17)
    g = GpuCase(lib, case)
    O = g.point()
    lib.forward_loss(g.ctx, dev_c64(O), g.P, cache=1)
    v = dev_c64(synth.random_complex(O.shape, seed=18))
    w = dev_f32(synth.random_real((case.K, 64, 64), seed=19))
    jv = torch.empty((case.K, 64, 64), dtype=torch.float32, device="cuda")
    lib.jvp(g.ctx, v, jv)
    jtw = torch.empty_like(v)
    lib.jtvp(g.ctx, w, jtw)
    lhs = float((jv.double() * w.double()).sum())
    rhs = float((torch.view_as_real(v).double() * torch.view_as_real(jtw).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_host_pointer_matvec_matches_device(lib):
    case = make_case(96, 32, K=37, loss=0, seed=20)
    g = GpuCase(lib, case)
    O = g.point()
    lib.forward_loss(g.ctx, dev_c64(O), g.P, cache=1)
    v = np.ascontiguousarray(synth.random_complex(O.shape, seed=21), np.complex64)
    out_h = np.empty_like(v)
    lib.ggn_matvec(g.ctx, v, out_h, 0.1)
    out_d = torch.empty((96, 96), dtype=torch.complex64, device="cuda")
    lib.ggn_matvec(g.ctx, dev_c64(v), out_d, 0.1)
    assert rel_err(out_h, host(out_d)) <= 1e-6


def test_lm_small_workload_matches_oracle(lib):
    """Algorithm 1 on the 128^2 / 32^2 / 64-position noiseless amplitude workload: both reach
    1e-3 object error (after global-phase alignment) and end within 1e-3 of each other."""
    w = synth.SMALL
    case = make_case(w.n, w.m, loss=0, seed=0, grid=w.grid, step=w.step, radius=w.radius)
    g = GpuCase(lib, case)
    mask = synth.illumination_mask(w.n, case.P, case.pos, 0.1)
    O0 = synth.flat_object(w.n)
    _, info_ref = oracle.lm_solve(case.problem(), O0, O_ref=case.O_true, mask=mask, max_outer=60,
                                  target_err=1e-3)
    Od = dev_c64(O0)
    st, info = lib.lm_solve(g.ctx, Od, g.P, hist_len=60, O_ref=dev_c64(case.O_true),
                            mask=torch.from_numpy(mask.astype(np.uint8)).cuda(), max_outer=60,
                            target_err=1e-3)
    err_gpu = oracle.object_error(host(Od), case.O_true, mask)
    assert err_gpu <= 1e-3, info
    assert abs(err_gpu - info_ref["err"][-1]) <= 1e-3
    assert abs(info["err_final"] - err_gpu) <= 1e-5


def test_lm_host_buffers(lib):
    """lm_solve accepts host arrays for the iterate and the probe."""
    w = synth.SMALL
    case = make_case(w.n, w.m, loss=0, seed=0, grid=w.grid, step=w.step, radius=w.radius)
    g = GpuCase(lib, case)
    O = np.ascontiguousarray(synth.flat_object(w.n), np.complex64)
    P = np.ascontiguousarray(case.P, np.complex64)
    st, info = lib.lm_solve(g.ctx, O, P, max_outer=3)
    Od = dev_c64(synth.flat_object(w.n))
    st2, info2 = lib.lm_solve(g.ctx, Od, g.P, max_outer=3)
    assert rel_err(O, host(Od)) <= 1e-5
    assert info["cg_total"] == info2["cg_total"]


def test_zero_positions(lib):
    pos = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    y = torch.zeros((0, 32, 32), dtype=torch.float32, device="cuda")
    ctx = lib.lm_init(64, 64, 32, 32, pos, y, 0, 1e-8)
    O = dev_c64(synth.object_texture(64))
    P = dev_c64(synth.probe_disk_defocus(32, 10))
    f, dl2 = lib.forward_loss(ctx, O, P, cache=1)
    assert f == 0.0 and dl2 == 0.0
    out = torch.ones_like(O)
    lib.ggn_matvec(ctx, O, out, 0.5)
    assert torch.allclose(out, 0.5 * O)


def test_argument_errors(lib):
    case = make_case(96, 32, K=5, loss=0, seed=3)
    pos = dev_i32(case.pos)
    y = dev_f32(case.y)
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_init(96, 96, 48, 48, pos, y)
    assert e.value.status == lib.PTYLM_ERR_ARG
    bad = case.pos.copy()
    bad[2] = (96 - 32 + 1, 0)
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_init(96, 96, 32, 32, dev_i32(bad), y)
    assert e.value.status == lib.PTYLM_ERR_ARG
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_init(96, 96, 32, 32, pos, y, background=0.0)
    assert e.value.status == lib.PTYLM_ERR_ARG
    with pytest.raises(lib.PtylmError) as e:
        lib.lm_init(96, 96, 32, 32, pos, y, workspace_budget=1024)
    assert e.value.status == lib.PTYLM_ERR_NOMEM
    ctx = lib.lm_init(96, 96, 32, 32, pos, y)
    v = dev_c64(np.zeros((96, 96)))
    with pytest.raises(lib.PtylmError) as e:
        lib.ggn_matvec(ctx, v, torch.empty_like(v), 0.0)
    assert e.value.status == lib.PTYLM_ERR_STATE
