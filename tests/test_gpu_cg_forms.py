"""The single-launch CG iteration (one cooperative launch, two grid-wide FP64 reductions
inside it) against the three-launch form (p.q; x, r and r.z; p and q).  Both run on the
same grid, give each thread the same elements, sum them in the same order and reduce the
per-CTA partials in block order, so every CG iteration gives the same bits.

lm_solve as a whole is deterministic when no two patches overlap: the scatters of the
gradient and of the GGN product then add one contribution to each object pixel, so their
atomic adds cannot round differently from run to run.  On such scans (the object tiled
exactly by the patches) both forms must return the same iterate, probe and history bit for
bit -- plain LM on the Gaussian metric, PLM (Jacobi PCG, D = Dg(G)) on the Poisson metric, a
joint object + probe context, and a 512^2 object that gives the full vector grid with
several elements per thread.  On an overlapping scan the scatter order varies between runs,
and the error-metric history is compared to 1e-5."""
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


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).cuda()


def both_forms(lib, case, joint, **kw):
    n, m = case.n, case.m
    ctx = lib.lm_init(n, n, m, m, torch.from_numpy(case.pos).cuda(),
                      torch.from_numpy(np.ascontiguousarray(case.y, np.float32)).cuda(), case.loss, case.b,
                      joint=joint)
    P0 = case.P * (np.exp(0.2j) if joint else 1.0)
    runs = []
    for separate in (0, 1):
        O, P = c64(synth.flat_object(n)), c64(P0)
        lib.ptylm_profile(ctx, 1)
        st, info = lib.lm_solve(ctx, O, P, hist_len=8, separate_cg_kernels=separate, **kw)
        _, sections = lib.ptylm_profile_read(ctx, lib.KERNEL_CG_ITERATION)
        _, launches = lib.ptylm_profile_read(ctx, -1)
        lib.ptylm_profile(ctx, 0)
        runs.append(dict(st=st, info=info, O=O.cpu().numpy(), P=P.cpu().numpy(), sections=sections,
                         launches=launches))
    return runs


# (object side, probe side, loss, scaled, joint): raster of (n/m)^2 patches at step m
TILED = [(96, 32, 0, 0, 0), (96, 32, 1, 1, 0), (96, 32, 0, 1, 1), (512, 64, 1, 0, 0)]


@pytest.mark.parametrize("n,m,loss,scaled,joint", TILED)
def test_single_launch_cg_is_bit_identical_on_tiled_scans(lib, n, m, loss, scaled, joint):
    case = make_case(n, m, loss=loss, seed=3 + loss, grid=n // m, step=m, radius=0.3 * m,
                     peak=1e4 if loss else 0.0)
    assert case.pos.max() + m == n
    a, b = both_forms(lib, case, joint, max_outer=4, scaled=scaled)
    assert a["st"] == b["st"]
    cg = a["info"]["cg_total"]
    assert a["info"]["n_outer"] == b["info"]["n_outer"] >= 2 and b["info"]["cg_total"] == cg > 0
    assert a["sections"] == b["sections"] == cg                     # one timed section per CG iteration
    assert b["launches"] - a["launches"] == 2 * cg                  # three launches against one
    for key in ("f", "gnorm", "mu", "cg"):
        assert np.array_equal(a["info"][key], b["info"][key]), key
    assert np.array_equal(a["O"], b["O"])
    assert np.array_equal(a["P"], b["P"])


def test_single_launch_cg_on_overlapping_scan(lib):
    case = make_case(96, 32, loss=0, seed=3, grid=6, step=10, radius=9.6)
    a, b = both_forms(lib, case, 0, max_outer=4, fixed_cg=10)
    assert a["st"] == b["st"] == 0
    assert a["info"]["f"][0] == b["info"]["f"][0]                   # deterministic error metric
    assert rel_err(a["info"]["f"], b["info"]["f"]) <= 1e-5
