"""The single-launch CG iteration (one cooperative launch, two grid-wide FP64 reductions
inside it) against the three-launch form (p.q; x, r and r.z; p and q).  Both run on the
same grid, give each thread the same elements, sum them in the same order and reduce the
per-CTA partials in block order, so every CG iteration gives the same bits.  With the
adaptive stopping rule the single-launch form also takes the stopping test on the device
(the host queues several iterations and reads the count once per batch) where the
three-launch form reads r.r before every iteration: the iteration counts must agree.

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
    assert a["info"]["matvecs"] == b["info"]["matvecs"]
    assert b["sections"] == cg <= a["sections"]                     # queued iterations past the stop are no-ops
    for key in ("f", "gnorm", "mu", "cg"):
        assert np.array_equal(a["info"][key], b["info"][key]), key
    assert np.array_equal(a["O"], b["O"])
    assert np.array_equal(a["P"], b["P"])


def test_single_launch_cg_on_overlapping_scan(lib):
    case = make_case(96, 32, loss=0, seed=3, grid=6, step=10, radius=9.6)
    a, b = both_forms(lib, case, 0, max_outer=4, fixed_cg=10)
    assert a["st"] == b["st"] == 0
    cg = a["info"]["cg_total"]
    assert a["sections"] == b["sections"] == cg == b["info"]["cg_total"]   # one timed section per iteration
    assert b["launches"] - a["launches"] == 2 * cg                          # three launches against one
    assert a["info"]["f"][0] == b["info"]["f"][0]                   # deterministic error metric
    assert rel_err(a["info"]["f"], b["info"]["f"]) <= 1e-5


def lm_ctx(lib, case, budget=0):
    n, m = case.n, case.m
    return lib.lm_init(n, n, m, m, torch.from_numpy(case.pos).cuda(),
                       torch.from_numpy(np.ascontiguousarray(case.y, np.float32)).cuda(), case.loss, case.b,
                       workspace_budget=budget)


def test_lookahead_linearisation_and_its_fallback(lib):
    """Object-only lm_solve evaluates each trial point with the cached forward pass into a
    second cache set and starts the next outer iteration from it when the step is accepted.
    Under a workspace budget with no room for that set it runs the loss-only trial pass and
    its own linearisation instead; both runs give the same iterates (tiled scan: every
    scatter is deterministic), and the forward-launch counts show which path ran."""
    n, m = 96, 32
    case = make_case(n, m, loss=0, seed=11, grid=n // m, step=m, radius=0.3 * m)
    # smallest budget under which lm_solve runs at all (binary search over whole contexts)
    lo, hi = 1 << 16, 1 << 26
    while hi - lo > 4096:
        mid = (lo + hi) // 2
        try:
            ctx = lm_ctx(lib, case, mid)
            lib.lm_solve(ctx, c64(synth.flat_object(n)), c64(case.P), max_outer=1, fixed_cg=1)
            hi = mid
        except lib.PtylmError as e:
            assert e.status == lib.PTYLM_ERR_NOMEM
            lo = mid
    K, M, N = len(case.pos), m * m, n * n
    lookahead_bytes = 8 * K * M + 16 * N + K * M // 8 + 12 * N   # the set, plus room kept for PLM / projection
    runs = {}
    for name, budget in (("tight", hi + lookahead_bytes - 4096), ("unlimited", 0)):
        ctx = lm_ctx(lib, case, budget)
        O = c64(synth.flat_object(n))
        lib.ptylm_profile(ctx, 1)
        st, info = lib.lm_solve(ctx, O, c64(case.P), hist_len=8, max_outer=5, fixed_cg=8)
        n_cache = lib.ptylm_profile_read(ctx, lib.KERNEL_FORWARD_CACHE)[1]
        n_loss = lib.ptylm_profile_read(ctx, lib.KERNEL_FORWARD_LOSS)[1]
        lib.ptylm_profile(ctx, 0)
        assert st == 0 and info["n_outer"] == 5
        runs[name] = (info, O.cpu().numpy(), n_cache, n_loss, info["cg_total"] // 8)
    (i_t, O_t, c_t, l_t, trials_t), (i_u, O_u, c_u, l_u, trials_u) = runs["tight"], runs["unlimited"]
    assert (c_t, l_t) == (5, trials_t)                # a linearisation per iteration, loss-only trials
    assert c_u + l_u == 1 + trials_u and l_u < l_t    # trials double as the next linearisation
    assert rel_err(i_u["f"], i_t["f"]) <= 1e-6
    assert rel_err(O_u, O_t) <= 1e-5


def test_device_cg_stopping_at_the_iteration_limit(lib):
    """Adaptive CG capped by max_cg: the device-side stopping (single-launch form) and the
    host-side test (three-launch form) both stop every solve at the cap, report
    PTYLM_WARN_CG_MAXIT and return the same iterate (tiled scan: deterministic scatters)."""
    n, m = 96, 32
    case = make_case(n, m, loss=1, seed=5, grid=n // m, step=m, radius=0.3 * m, peak=1e4)
    a, b = both_forms(lib, case, 0, max_outer=3, max_cg=2)
    assert a["st"] == b["st"] == lib.PTYLM_WARN_CG_MAXIT
    cg = list(a["info"]["cg"])
    assert cg == list(b["info"]["cg"]) and all(c > 0 and c % 2 == 0 for c in cg)   # every solve stops at 2
    assert a["info"]["matvecs"] == b["info"]["matvecs"]
    assert np.array_equal(a["info"]["f"], b["info"]["f"])
    assert np.array_equal(a["O"], b["O"])
