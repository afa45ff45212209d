"""Joint object+probe (blind) operators, the closed-form GGN diagonal and the scaled /
projected LM (PLM, PLM-J with Algorithm 2) of the CUDA path against the FP64 oracle.

Tolerances as in test_gpu_parity.py: relative 1e-5 for well-conditioned inputs (Gaussian
metric, Poisson at its noiseless truth); the Poisson diagonal at a perturbed point, whose
traces sum 2 y / h over dark pixels, uses max(1e-5, 2 x its FP32 conditioning)."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.problems import make_case, rel_err
from tests.test_gpu_parity import fp32_conditioning

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


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def setup(lib, shape, loss=0, seed=40, joint=1, at_truth=False):
    n, m, K = shape
    case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=seed, noisy=False)
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(case.pos).cuda(), f32(case.y), loss, case.b, joint=joint)
    if at_truth:
        O, P = case.O_true, case.P
    else:
        O = synth.to_c64(case.O_true + synth.random_complex(case.O_true.shape, seed=seed + 1, scale=0.05))
        P = synth.to_c64(case.P * 1.05 + synth.random_complex(case.P.shape, seed=seed + 2, scale=0.02))
    return case, ctx, O, P


SHAPES = [(96, 32, 37), (160, 64, 23), (288, 128, 11), (512, 64, 1000)]


@pytest.mark.parametrize("shape", SHAPES)
def test_joint_gradient(lib, shape):
    case, ctx, O, P = setup(lib, shape)
    f, _ = lib.forward_loss(ctx, c64(O), c64(P), cache=1)
    pb = case.problem()
    gO = torch.empty((shape[0], shape[0]), dtype=torch.complex64, device="cuda")
    gP = torch.empty((shape[1], shape[1]), dtype=torch.complex64, device="cuda")
    lib.gradient(ctx, gO, gP)
    rO, rP = oracle.gradient(pb, O, P, probe_part=True)
    parity.check("joint grad f, object block", host(gO), rO, TOL)
    parity.check("joint grad f, object block", host(gO), rO, TOL, norm="max")
    parity.check("joint grad f, probe block", host(gP), rP, TOL)
    parity.check("joint grad f, probe block", host(gP), rP, TOL, norm="max")
    assert abs(f - oracle.loss(pb, O, P)) <= TOL * abs(f)


@pytest.mark.parametrize("loss,at_truth", [(0, False), (1, True)])
@pytest.mark.parametrize("shape", SHAPES)
def test_joint_ggn_matvec(lib, shape, loss, at_truth):
    n, m, _ = shape
    case, ctx, O, P = setup(lib, shape, loss=loss, at_truth=at_truth)
    lib.forward_loss(ctx, c64(O), c64(P), cache=1)
    pb = case.problem()
    L = n * n + m * m
    v = synth.to_c64(synth.random_complex(L, seed=50))
    D = synth.to_f32(np.abs(synth.random_real(L, seed=51)) + 0.5)
    outO = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    outP = torch.empty((m, m), dtype=torch.complex64, device="cuda")
    for lam, Dv in ((0.0, None), (0.3, D)):
        lib.ggn_matvec(ctx, c64(v[:n * n].reshape(n, n)), outO, lam, None if Dv is None else f32(Dv),
                       vP=c64(v[n * n:].reshape(m, m)), outP=outP)
        ref = oracle.ggn_matvec_z(pb, O, v, lam=lam, D=Dv, P=P, joint=True)
        got = np.concatenate([host(outO).ravel(), host(outP).ravel()])
        parity.check(f"joint (G + {lam} D) v, whole z", got, ref, TOL)
        parity.check(f"joint (G + {lam} D) v, whole z", got, ref, TOL, norm="max")
        # the probe block alone, so a small block error cannot hide behind the object block
        parity.check(f"joint (G + {lam} D) v, probe block", host(outP).ravel(), ref[n * n:], TOL)
        parity.check(f"joint (G + {lam} D) v, probe block", host(outP).ravel(), ref[n * n:], TOL, norm="max")


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_joint_jvp_and_jtvp(lib, shape):
    n, m, K = shape
    case, ctx, O, P = setup(lib, shape)
    lib.forward_loss(ctx, c64(O), c64(P), cache=1)
    pb = case.problem()
    vO = synth.to_c64(synth.random_complex((n, n), seed=60))
    vP = synth.to_c64(synth.random_complex((m, m), seed=61))
    out = torch.empty((K, m, m), dtype=torch.float32, device="cuda")
    lib.jvp(ctx, c64(vO), out, vP=c64(vP))
    jv_ref = oracle.jvp(pb, O, vO, P=P, vP=vP)
    parity.check("joint J v", host(out), jv_ref, TOL)
    lit_pb = oracle.Problem((n, n), P, case.pos, None, case.loss, case.b)   # the probe of this point
    parity.check_detector("joint J v", host(out), jv_ref, oracle.intensity(lit_pb, O) - case.b)
    w = synth.to_f32(synth.random_real((K, m, m), seed=62))
    outO = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    outP = torch.empty((m, m), dtype=torch.complex64, device="cuda")
    lib.jtvp(ctx, f32(w), outO, outP)
    rO, rP = oracle.jtvp(pb, O, w, P=P, probe_part=True)
    parity.check("joint J^T w, object block", host(outO), rO, TOL)
    parity.check("joint J^T w, object block", host(outO), rO, TOL, norm="max")
    parity.check("joint J^T w, probe block", host(outP), rP, TOL)
    parity.check("joint J^T w, probe block", host(outP), rP, TOL, norm="max")


@pytest.mark.parametrize("joint", [0, 1])
@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_ggn_diag(lib, shape, loss, joint):
    """App. B closed form: GPU (FP32 sums, float atomics) vs oracle (FP64), with the floor."""
    n, m, _ = shape
    case, ctx, O, P = setup(lib, shape, loss=loss, joint=joint)
    if not joint:
        P = case.P
    lib.forward_loss(ctx, c64(O), c64(P), cache=1)
    pb = case.problem()
    L = n * n + (m * m if joint else 0)
    def diag_at(A, floor):
        rO, rP = oracle.ggn_diag(pb, A, P, floor_rel=floor)
        return np.concatenate([rO.ravel(), rP.ravel()]) if joint else rO.ravel()

    for floor in (0.0, 1e-6):
        D = torch.empty(L, dtype=torch.float32, device="cuda")
        lib.ggn_diag(ctx, D, floor)
        ref = diag_at(O, floor)
        tol = TOL if loss == 0 else max(TOL, 2.0 * fp32_conditioning(lambda A: diag_at(A, floor), m, O))
        basis = "1e-5" if loss == 0 else "2 x FP32 conditioning"
        parity.check(f"Dg(G) (floor {floor})", host(D), ref, tol, basis=basis)
        if joint:
            parity.check(f"Dg(G) probe block (floor {floor})", host(D)[n * n:], ref[n * n:], tol, basis=basis)


def test_plm_small_workload_matches_oracle(lib):
    """PLM (D = Dg(G), Jacobi PCG) on the 128^2 noiseless workload: both reach 1e-3 object error."""
    w = synth.SMALL
    case = make_case(w.n, w.m, loss=0, seed=0, grid=w.grid, step=w.step, radius=w.radius)
    ctx = lib.lm_init(w.n, w.n, w.m, w.m, torch.from_numpy(case.pos).cuda(), f32(case.y), 0, case.b)
    mask = synth.illumination_mask(w.n, case.P, case.pos, 0.1)
    O0 = synth.flat_object(w.n)
    _, _, info_ref = oracle.lm_solve2(case.problem(), O0, O_ref=case.O_true, mask=mask, max_outer=60,
                                      target_err=1e-3, scaled=1)
    Od = c64(O0)
    st, info = lib.lm_solve(ctx, Od, c64(case.P), hist_len=60, O_ref=c64(case.O_true),
                            mask=torch.from_numpy(mask.astype(np.uint8)).cuda(), max_outer=60, target_err=1e-3,
                            scaled=1)
    err = oracle.object_error(host(Od), case.O_true, mask)
    assert err <= 1e-3 and info_ref["err"][-1] <= 1e-3, (err, info, info_ref)
    assert abs(info["n_outer"] - info_ref["n_outer"]) <= 3, (info["n_outer"], info_ref["n_outer"])


def test_plm_joint_projected_blind_matches_oracle(lib):
    """PLM-J + Algorithm 2 on a small noiseless blind problem (flat object, unphased probe):
    the GPU and the oracle both reduce the blind-aligned object error twentyfold, keep |O| <= 1,
    and end within 1e-2 of each other in that error."""
    n, m = 96, 32
    O_true = synth.to_c64(synth.object_texture(n, seed=4))
    P_true = synth.to_c64(synth.probe_disk_defocus(m, 10.0))
    pos, _ = synth.raster_positions(n, m, 8, 8, 1, seed=5)
    pb = oracle.Problem((n, n), P_true, pos, None, 0, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true))
    mask = synth.illumination_mask(n, P_true, pos, 0.3)
    P0 = synth.to_c64(synth.probe_disk_defocus(m, 10.0, phased=False))
    O0 = synth.flat_object(n) * 0.9
    e0 = oracle.object_error_blind(O0, O_true, mask)
    O_ref_run, _, _ = oracle.lm_solve2(pb, O0, P0, max_outer=40, scaled=1, joint=1, projected=1)
    e_oracle = oracle.object_error_blind(O_ref_run, O_true, mask)
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(pos).cuda(), f32(pb.y), 0, 1e-8, joint=1)
    Od, Pd = c64(O0), c64(P0)
    st, info = lib.lm_solve(ctx, Od, Pd, hist_len=40, max_outer=40, scaled=1, projected=1)
    e_gpu = oracle.object_error_blind(host(Od), O_true, mask)
    assert np.abs(host(Od)).max() <= 1.0 + 1e-6
    assert e_gpu <= 0.05 * e0 and e_oracle <= 0.05 * e0, (e0, e_gpu, e_oracle)
    assert abs(e_gpu - e_oracle) <= 1e-2, (e_gpu, e_oracle)
    assert info["f"][-1] < 1e-3 * info["f"][0]


def test_joint_argument_errors(lib):
    case, ctx, O, P = setup(lib, (96, 32, 37), joint=0)
    lib.forward_loss(ctx, c64(O), c64(case.P), cache=1)
    g = torch.empty((96, 96), dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.PtylmError) as e:
        lib.gradient(ctx, g, torch.empty((32, 32), dtype=torch.complex64, device="cuda"))
    assert e.value.status == lib.PTYLM_ERR_ARG
    case, ctxj, O, P = setup(lib, (96, 32, 37), joint=1)
    lib.forward_loss(ctxj, c64(O), c64(P), cache=1)
    with pytest.raises(lib.PtylmError) as e:
        lib.ggn_matvec(ctxj, c64(O), g, 0.1)   # joint contexts need the probe blocks
    assert e.value.status == lib.PTYLM_ERR_ARG


def test_plm_surrogate_matches_oracle(lib):
    """PLM-S (App. E: s_t from 1 down to 1e-2 over T = 4 iterations, then the true Poisson
    metric) on a small noisy Poisson problem: at every iteration the GPU's f at its
    linearisation point agrees with the oracle's run to FP32 accuracy while the iterates
    coincide (the first iterations), and both runs end at the same true-metric value."""
    n, m = 96, 32
    case = make_case(n, m, loss=1, peak=1e3, seed=70, grid=8, step=8, jitter=1, radius=10.0, noisy=True)
    pb = case.problem()
    O0 = synth.flat_object(n)
    kw = dict(scaled=1, surrogate0=1.0, surrogate_end=1e-2, surrogate_T=4, max_outer=12)
    O_ref_run, _, info_ref = oracle.lm_solve2(pb, O0, **kw)
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(case.pos).cuda(), f32(case.y), 1, case.b)
    Od = c64(O0)
    st, info = lib.lm_solve(ctx, Od, c64(case.P), hist_len=12, **kw)
    assert info["n_outer"] == info_ref["n_outer"] == 12
    # t = 0: same point, surrogate background 1 + b
    assert abs(info["f"][0] - info_ref["f"][0]) <= 1e-5 * abs(info_ref["f"][0])
    f_gpu, f_orc = oracle.loss(pb, host(Od)), oracle.loss(pb, O_ref_run)
    f_min = oracle.poisson_f_min(pb.y)
    assert abs(f_gpu - f_orc) <= 1e-3 * abs(info_ref["f"][0] - f_min), (f_gpu, f_orc)
    # after T the recorded f is the true metric at the linearisation point
    assert info["f"][-1] >= f_min
