"""Batches of independent reconstructions (one persistent launch per operator, CG under a
captured CUDA graph, schedule autotuner) against the FP64 oracle problem by problem.

Checks as in test_gpu_parity.py (`compare`): relative 1e-5, 2-norm and element-wise, for
the Gaussian metric; for the Poisson metric away from the truth the FP32 conditioning bound
and at most twice the error of the independent FP32 evaluation.  Every achieved error is
recorded."""
import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth
from tests import parity
from tests.problems import make_case, rel_err
from tests.fp32_eval import ORDERS, evaluations
from tests.test_gpu_parity import compare, fp32_conditioning, fp32_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5

# (object side, probe side, K, loss, noisy): uneven sizes, all three probe sides, ragged
# position counts (last work items partly empty), both losses
MEMBERS = [(96, 32, 37, 0, False), (160, 64, 23, 1, False), (288, 128, 11, 0, False), (128, 32, 100, 1, True),
           (256, 64, 50, 0, False), (256, 128, 5, 1, True)]


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
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def batch(lib):
    cases = []
    for i, (n, m, K, loss, noisy) in enumerate(MEMBERS):
        case = make_case(n, m, K=K, loss=loss, peak=1e3 if loss else 0.0, seed=80 + i, noisy=noisy)
        case.noisy = noisy
        case.at_truth = False
        cases.append(case)
    probs = [dict(ny=c.n, nx=c.n, m=c.m, positions=torch.from_numpy(c.pos).cuda(), y=f32(c.y), probe=c64(c.P),
                  loss=c.loss, background=c.b) for c in cases]
    bt = lib.batch_init(probs)
    points = [synth.to_c64(c.O_true + synth.random_complex(c.O_true.shape, seed=90 + i, scale=0.05))
              for i, c in enumerate(cases)]
    O = torch.cat([c64(p).reshape(-1) for p in points])
    return bt, cases, points, O


def test_offsets_concatenate_the_objects(lib, batch):
    bt, cases, _, _ = batch
    assert bt.offsets[0] == 0
    assert all(bt.offsets[i + 1] - bt.offsets[i] == c.n * c.n for i, c in enumerate(cases))


# schedule 0: every FFT tile with 32 values per thread; 18: the 32^2 and 64^2 problems with
# 16 values per thread (teams of 64 and 256 threads)
TILES = [0, 18]


@pytest.mark.parametrize("schedule", TILES)
def test_batch_forward_loss_and_gradient(lib, batch, schedule):
    bt, cases, points, O = batch
    lib.batch_set_schedule(bt, schedule)
    f, dl2 = lib.batch_forward_loss(bt, O, cache=1)
    g = torch.empty_like(O)
    lib.batch_gradient(bt, g)
    gv = bt.views(g)
    for b, (c, X) in enumerate(zip(cases, points)):
        pb = c.problem()
        mdl = fp32_model(c)
        f_ref, dl2_ref = oracle.loss(pb, X, return_dl_norm2=True)
        compare(f"f[{b}]", f[b], f_ref, c, lambda A: oracle.loss(pb, A), (X,),
                lambda: [mdl.loss_value(X, order=o)[0] for o in ORDERS])
        compare(f"||dl||^2[{b}]", dl2[b], dl2_ref, c, lambda A: oracle.loss(pb, A, return_dl_norm2=True)[1], (X,),
                lambda: [mdl.loss_value(X, order=o)[1] for o in ORDERS])
        g_ref = oracle.gradient(pb, X)
        compare(f"grad f[{b}]", host(gv[b]), g_ref, c, lambda A: oracle.gradient(pb, A), (X,),
                lambda: evaluations(mdl, "gradient", X))


def test_batch_loss_without_cache_matches(lib, batch):
    bt, cases, points, O = batch
    f1, _ = lib.batch_forward_loss(bt, O, cache=1)
    f0, _ = lib.batch_forward_loss(bt, O, cache=0)
    assert np.allclose(f0, f1, rtol=1e-6, atol=0)


@pytest.mark.parametrize("schedule", TILES)
def test_batch_ggn_matvec(lib, batch, schedule):
    bt, cases, points, O = batch
    lib.batch_set_schedule(bt, schedule)
    lib.batch_forward_loss(bt, O, cache=1)
    vs = [synth.to_c64(synth.random_complex((c.n, c.n), seed=100 + i)) for i, c in enumerate(cases)]
    v = torch.cat([c64(x).reshape(-1) for x in vs])
    out = torch.empty_like(v)
    lam = np.array([0.0, 0.3, 0.0, 1.7, 0.01, 0.5])
    lib.batch_ggn_matvec(bt, v, out, lam)
    ov = bt.views(out)
    for b, (c, X) in enumerate(zip(cases, points)):
        pb = c.problem()
        ref = oracle.ggn_matvec(pb, X, vs[b], lam=lam[b])
        mdl = fp32_model(c)
        compare(f"(G + lam I) v[{b}]", host(ov[b]), ref, c, lambda A, B: oracle.ggn_matvec(pb, A, B, lam=lam[b]),
                (X, vs[b]), lambda: evaluations(mdl, "ggn_matvec", X, vs[b], lam=lam[b]))


def test_every_schedule_gives_the_same_product(lib, batch):
    bt, cases, points, O = batch
    lib.batch_forward_loss(bt, O, cache=1)
    v = torch.cat([c64(synth.random_complex((c.n, c.n), seed=110 + i)).reshape(-1) for i, c in enumerate(cases)])
    choice, ms = lib.batch_tune(bt)
    # the batch has 32^2 and 64^2 problems, so every tile is timed
    assert 0 <= choice < lib.N_SCHEDULES and all(t > 0 for t in ms) and ms[choice] == min(ms)
    outs = []
    for s in range(lib.N_SCHEDULES):
        lib.batch_set_schedule(bt, s)   # a tile change relinearises at the same point
        out = torch.empty_like(v)
        lib.batch_ggn_matvec(bt, v, out, 0.2)
        outs.append(host(out))
    # within one FFT tile the schedules change only which CTA runs which positions (the order
    # of the scatter's float reductions); another tile rounds the FFT differently, so the
    # tiles are held against the oracle, problem by problem, with the checks of `compare`
    for s in range(lib.N_SCHEDULES):
        first = 6 * (s // 6)
        assert rel_err(outs[s], outs[first]) <= 2 * TOL, (s, lib.schedule_desc(s))
    views = [[o[bt.offsets[b]:bt.offsets[b + 1]].reshape(c.n, c.n) for b, c in enumerate(cases)] for o in outs]
    for b, (c, X) in enumerate(zip(cases, points)):
        pb = c.problem()
        vb = host(bt.views(v)[b])
        ref = oracle.ggn_matvec(pb, X, vb, lam=0.2)
        ev = evaluations(fp32_model(c), "ggn_matvec", X, vb, lam=0.2)
        for s in (0, 6, 12, 18):
            compare(f"(G + 0.2 I) v[{b}] schedule {s}", views[s][b], ref, c,
                    lambda A, B: oracle.ggn_matvec(pb, A, B, lam=0.2), (X, vb), lambda: ev)


@pytest.mark.parametrize("schedule", TILES)
def test_batch_ggn_diag(lib, batch, schedule):
    """App. B closed form per problem (FP32 sums and float atomics, per-problem floor) against
    the oracle's orc_ggn_diag, under both FFT tiles (the per-thread d2l sums follow the tile)."""
    bt, cases, points, O = batch
    lib.batch_set_schedule(bt, schedule)
    lib.batch_forward_loss(bt, O, cache=1)
    for floor in (0.0, 1e-6):
        D = torch.empty(bt.total, dtype=torch.float32, device="cuda")
        lib.batch_ggn_diag(bt, D, floor)
        Dh = D.cpu().numpy().astype(np.float64)
        for b, (c, X) in enumerate(zip(cases, points)):
            pb = c.problem()
            diag_at = lambda A: oracle.ggn_diag(pb, A, floor_rel=floor)[0].ravel()
            ref = diag_at(X)
            got = Dh[bt.offsets[b]:bt.offsets[b + 1]]
            if c.loss == 0:
                parity.check(f"batch Dg(G)[{b}] (floor {floor})", got, ref)
                parity.check(f"batch Dg(G)[{b}] (floor {floor})", got, ref, norm="max")
            else:
                tol = max(TOL, 2.0 * fp32_conditioning(diag_at, c.m, X))
                parity.check(f"batch Dg(G)[{b}] (floor {floor})", got, ref, tol, basis="2 x FP32 conditioning")


def test_batch_plm_reaches_accuracy_like_single_problem_plm(lib):
    """PLM (D = Dg(G), lambda = mu, Jacobi PCG) next to LM in one batch: the scaled problems
    reach 1e-3 object error in a number of outer iterations within 3 of the single-problem
    lm_solve(scaled=1) and of the oracle's PLM for the smallest; the LM problem of the same
    batch still matches its single-problem run."""
    specs = [(128, 32, 8, 8), (192, 64, 6, 16), (256, 128, 4, 32)]
    scaled = [1, 1, 0]
    cases, probs, O0, refs, masks = [], [], [], [], []
    for i, (n, m, grid, step) in enumerate(specs):
        c = make_case(n, m, loss=0, seed=140 + i, grid=grid, step=step, radius=0.3125 * m)
        cases.append(c)
        probs.append(dict(ny=n, nx=n, m=m, positions=torch.from_numpy(c.pos).cuda(), y=f32(c.y), probe=c64(c.P),
                          loss=0, background=c.b))
        O0.append(synth.flat_object(n))
        refs.append(c64(c.O_true))
        masks.append(torch.from_numpy(synth.illumination_mask(n, c.P, c.pos, 0.1).astype(np.uint8)).cuda())
    bt = lib.batch_init(probs)
    O = torch.cat([c64(o).reshape(-1) for o in O0])
    params = []
    for b in range(len(specs)):
        p = lib.default_lm_params(0)
        p.scaled = scaled[b]
        params.append(p)
    st, infos = lib.batch_lm_solve(bt, O, params, hist_len=80, O_refs=refs, masks=masks, max_outer=80,
                                   target_err=1e-3)
    ov = bt.views(O)
    for b, c in enumerate(cases):
        mask = synth.illumination_mask(c.n, c.P, c.pos, 0.1)
        assert oracle.object_error(host(ov[b]), c.O_true, mask) <= 1e-3, b
        ctx = lib.lm_init(c.n, c.n, c.m, c.m, torch.from_numpy(c.pos).cuda(), f32(c.y), 0, c.b)
        _, single = lib.lm_solve(ctx, c64(O0[b]), c64(c.P), hist_len=80, O_ref=refs[b], mask=masks[b], max_outer=80,
                                 target_err=1e-3, scaled=scaled[b])
        assert abs(infos[b]["n_outer"] - single["n_outer"]) <= 3, (b, infos[b]["n_outer"], single["n_outer"])
        assert infos[b]["err"][-1] <= 1e-3
    mask0 = synth.illumination_mask(128, cases[0].P, cases[0].pos, 0.1)
    _, _, info_ref = oracle.lm_solve2(cases[0].problem(), O0[0], O_ref=cases[0].O_true, mask=mask0, scaled=1,
                                      max_outer=80, target_err=1e-3)
    assert abs(infos[0]["n_outer"] - info_ref["n_outer"]) <= 3, (infos[0]["n_outer"], info_ref["n_outer"])


def test_batch_lm_reaches_accuracy_like_single_problem_lm(lib):
    """Noiseless amplitude problems of three probe sides: the batched LM reaches 1e-3 object
    error on each, in a number of outer iterations within 3 of the single-problem lm_solve
    (and of the oracle's run for the smallest)."""
    specs = [(128, 32, 8, 8), (192, 64, 6, 16), (256, 128, 4, 32)]
    cases, probs, O0, refs, masks = [], [], [], [], []
    for i, (n, m, grid, step) in enumerate(specs):
        c = make_case(n, m, loss=0, seed=120 + i, grid=grid, step=step, radius=0.3125 * m)
        cases.append(c)
        probs.append(dict(ny=n, nx=n, m=m, positions=torch.from_numpy(c.pos).cuda(), y=f32(c.y), probe=c64(c.P),
                          loss=0, background=c.b))
        O0.append(synth.flat_object(n))
        refs.append(c64(c.O_true))
        masks.append(torch.from_numpy(synth.illumination_mask(n, c.P, c.pos, 0.1).astype(np.uint8)).cuda())
    bt = lib.batch_init(probs)
    O = torch.cat([c64(o).reshape(-1) for o in O0])
    st, infos = lib.batch_lm_solve(bt, O, hist_len=80, O_refs=refs, masks=masks, max_outer=80, target_err=1e-3)
    ov = bt.views(O)
    for b, c in enumerate(cases):
        mask = synth.illumination_mask(c.n, c.P, c.pos, 0.1)
        assert oracle.object_error(host(ov[b]), c.O_true, mask) <= 1e-3, b
        ctx = lib.lm_init(c.n, c.n, c.m, c.m, torch.from_numpy(c.pos).cuda(), f32(c.y), 0, c.b)
        Od = c64(O0[b])
        _, single = lib.lm_solve(ctx, Od, c64(c.P), hist_len=80, O_ref=refs[b], mask=masks[b], max_outer=80,
                                 target_err=1e-3)
        assert abs(infos[b]["n_outer"] - single["n_outer"]) <= 3, (b, infos[b]["n_outer"], single["n_outer"])
        assert infos[b]["err"][-1] <= 1e-3
    _, info_ref = oracle.lm_solve(cases[0].problem(), O0[0], O_ref=cases[0].O_true,
                                  mask=synth.illumination_mask(128, cases[0].P, cases[0].pos, 0.1), max_outer=80,
                                  target_err=1e-3)
    assert abs(infos[0]["n_outer"] - info_ref["n_outer"]) <= 3
    assert lib.batch_launches(bt) > 0


def test_batch_lm_fixed_cg_counts(lib, batch):
    """fixed_cg runs exactly that many CG iterations per solve on every problem."""
    bt, cases, points, O = batch
    X = O.clone()
    st, infos = lib.batch_lm_solve(bt, X, hist_len=4, max_outer=2, fixed_cg=5)
    for info in infos:
        assert info["n_outer"] >= 1
        assert info["cg_total"] % 5 == 0 and info["cg_total"] >= 5
        assert np.all(info["cg"] % 5 == 0)


def test_batch_with_an_empty_member_and_a_border_scan(lib):
    """A member with no positions next to one whose patches all touch the object's border:
    the empty member's error metric and gradient are zero and its product is lambda v; the
    others match the oracle; the batched LM finishes the empty member at once and solves
    the others; the autotuner times only the tiles the batch uses (128^2 and 32^2 here)."""
    from tests.problems import Case
    n, m = 128, 32
    e = n - m
    pos = np.array([(0, 0), (0, e), (e, 0), (e, e), (0, 40), (40, e), (e, 17), (63, 0)], np.int32)
    O_true = synth.to_c64(synth.object_texture(n, seed=210))
    P = synth.to_c64(synth.probe_disk_defocus(m, 10.0))
    y = oracle.intensity(oracle.Problem((n, n), P, pos, None, 0, 1e-8), O_true)
    border = Case(n, m, pos, O_true, P, synth.to_f32(y), 0, 1e-8)
    big = make_case(160, 128, K=4, loss=0, seed=211)
    cases = [border, None, big]
    empty = dict(ny=64, nx=64, m=32, positions=torch.zeros((0, 2), dtype=torch.int32).cuda(),
                 y=torch.zeros((0, 32, 32), dtype=torch.float32).cuda(), probe=c64(P), loss=0, background=1e-8)
    probs = [dict(ny=c.n, nx=c.n, m=c.m, positions=torch.from_numpy(c.pos).cuda(), y=f32(c.y), probe=c64(c.P),
                  loss=0, background=c.b) if c is not None else empty for c in cases]
    bt = lib.batch_init(probs)
    assert [bt.offsets[i + 1] - bt.offsets[i] for i in range(3)] == [n * n, 64 * 64, 160 * 160]
    X = [synth.to_c64(border.O_true + synth.random_complex((n, n), seed=212, scale=0.05)),
         synth.to_c64(synth.random_complex((64, 64), seed=213)),
         synth.to_c64(big.O_true + synth.random_complex((160, 160), seed=214, scale=0.05))]
    O = torch.cat([c64(x).reshape(-1) for x in X])
    f, dl2 = lib.batch_forward_loss(bt, O, cache=1)
    g = torch.empty_like(O)
    lib.batch_gradient(bt, g)
    gv = bt.views(g)
    assert f[1] == 0.0 and dl2[1] == 0.0 and float(gv[1].abs().max()) == 0.0
    vs = [synth.to_c64(synth.random_complex(x.shape, seed=220 + i)) for i, x in enumerate(X)]
    v = torch.cat([c64(x).reshape(-1) for x in vs])
    out = torch.empty_like(v)
    lam = np.array([0.2, 0.7, 0.0])
    lib.batch_ggn_matvec(bt, v, out, lam)
    ov = bt.views(out)
    assert rel_err(host(ov[1]), 0.7 * vs[1]) <= 1e-6
    for b in (0, 2):
        c = cases[b]
        pb = c.problem()
        parity.check(f"edge batch f[{b}]", f[b], oracle.loss(pb, X[b]))
        parity.check(f"edge batch grad f[{b}]", host(gv[b]), oracle.gradient(pb, X[b]))
        parity.check(f"edge batch grad f[{b}]", host(gv[b]), oracle.gradient(pb, X[b]), norm="max")
        ref = oracle.ggn_matvec(pb, X[b], vs[b], lam=lam[b])
        parity.check(f"edge batch (G + lam I) v[{b}]", host(ov[b]), ref)
        parity.check(f"edge batch (G + lam I) v[{b}]", host(ov[b]), ref, norm="max")
    choice, ms = lib.batch_tune(bt)
    assert all(t > 0 for t in ms[:12]) and all(t == -1.0 for t in ms[12:]) and choice < 12
    st, infos = lib.batch_lm_solve(bt, O, hist_len=4, max_outer=3)
    assert infos[1]["n_outer"] == 0 and infos[0]["n_outer"] >= 1 and infos[2]["n_outer"] >= 1


def test_batch_argument_errors(lib):
    c = make_case(96, 32, K=10, loss=0, seed=1)
    good = dict(ny=96, nx=96, m=32, positions=torch.from_numpy(c.pos).cuda(), y=f32(c.y), probe=c64(c.P), loss=0)
    bad = dict(good)
    pos = c.pos.copy()
    pos[3] = (90, 0)   # 90 + 32 > 96
    bad["positions"] = torch.from_numpy(pos).cuda()
    with pytest.raises(lib.PtylmError) as e:
        lib.batch_init([good, bad])
    assert e.value.status == lib.PTYLM_ERR_ARG
    bt = lib.batch_init([good])
    v = torch.zeros(96 * 96, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.PtylmError) as e:
        lib.batch_ggn_matvec(bt, v, torch.empty_like(v))
    assert e.value.status == lib.PTYLM_ERR_STATE
