"""Pins for the FP64 oracle: each check is fixed by the paper or by mathematics, not by the
oracle's own formulas (closed forms, library special cases, invariants, finite
differences and dense brute force on tiny problems)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2103_01767_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_problem(loss=oracle.LOSS_GAUSSIAN, n=10, m=4, seed=0, noiseless=True, b=1e-8):
    """N = 10^2, M = 4^2, K = 6 positions (brute-force size)."""
    rng = np.random.default_rng(seed)
    O = synth.object_texture(n, seed=seed, sigma=1.0)
    P = synth.random_complex((m, m), seed=seed + 10, scale=0.7)
    pos = np.array([[0, 0], [0, 3], [0, 6], [3, 1], [6, 4], [5, 6]], np.int32)
    pb = oracle.Problem((n, n), P, pos, None, loss, b)
    h = oracle.intensity(pb, O)
    if noiseless:
        y = h.copy()
    else:
        y = rng.poisson(h * 50.0) / 50.0
    pb.y = np.ascontiguousarray(y, np.float64)
    return pb, O


def rdot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


# ----------------------------------------------------------------------------- transforms
def test_dft_closed_forms():
    """A delta transforms to the constant M^{-1/2}; a pure exponential to a scaled delta."""
    my, mx = 8, 4
    x = np.zeros((my, mx), complex)
    x[0, 0] = 1
    X = oracle.dft2(x)
    np.testing.assert_allclose(X, np.full((my, mx), 1 / math.sqrt(my * mx)), atol=1e-15)
    uy, ux = 3, 1
    yy, xx = np.mgrid[0:my, 0:mx]
    e = np.exp(2j * np.pi * (uy * yy / my + ux * xx / mx))
    X = oracle.dft2(e)  # forward sign -1 picks out frequency (uy, ux)
    ref = np.zeros((my, mx), complex)
    ref[uy, ux] = math.sqrt(my * mx)
    np.testing.assert_allclose(X, ref, atol=1e-12)
    # inverse undoes forward
    z = synth.random_complex((my, mx), seed=5)
    np.testing.assert_allclose(oracle.dft2(oracle.dft2(z), inverse=True), z, atol=1e-13)


@pytest.mark.parametrize("shape", [(32, 32), (16, 8), (64, 64), (128, 128)])
def test_fft_matches_direct_dft_and_numpy(shape):
    z = synth.random_complex(shape, seed=7)
    F = oracle.fft2(z)
    np.testing.assert_allclose(F, np.fft.fft2(z, norm="ortho"), atol=1e-11, rtol=0)
    if shape[0] * shape[1] <= 1024:
        np.testing.assert_allclose(F, oracle.dft2(z), atol=1e-11, rtol=0)
    np.testing.assert_allclose(oracle.fft2(F, inverse=True), z, atol=1e-12)
    # Parseval for the orthonormal transform
    assert abs(np.vdot(F, F).real - np.vdot(z, z).real) <= 1e-10 * np.vdot(z, z).real


# ----------------------------------------------------------------------------- forward model
def test_forward_matches_library_fft_and_parseval():
    n, m = 48, 16
    O = synth.object_texture(n, seed=0)
    P = synth.probe_disk_defocus(m, 5.0)
    pos, _ = synth.raster_positions(n, m, 4, 9, 1, seed=1)
    pb = oracle.Problem((n, n), P, pos, None, 0, 1e-8)
    ph, h = oracle.forward(pb, O)
    for k, (r, c) in enumerate(pos):
        psi = P * O[r:r + m, c:c + m]
        np.testing.assert_allclose(ph[k], np.fft.fft2(psi, norm="ortho"), atol=1e-12)
        # Parseval: sum_m h = ||psi||^2 + M b
        assert abs(h[k].sum() - (np.vdot(psi, psi).real + m * m * 1e-8)) < 1e-10 * h[k].sum()


def test_forward_translation_and_phase_invariance():
    n, m = 40, 8
    O = synth.object_texture(n, seed=3)
    P = synth.random_complex((m, m), seed=4)
    pos = np.array([[0, 0], [5, 7], [20, 3]], np.int32)
    pb = oracle.Problem((n, n), P, pos, None, 0, 1e-8)
    h = oracle.intensity(pb, O)
    # global phase leaves h unchanged (Sec. 2 ambiguity)
    np.testing.assert_allclose(oracle.intensity(pb, O * np.exp(0.7j)), h, rtol=1e-12)
    # shifting the object and the scan together leaves h unchanged
    O2 = np.roll(O, (4, 6), axis=(0, 1))
    pb2 = oracle.Problem((n, n), P, pos + np.array([4, 6], np.int32), None, 0, 1e-8)
    np.testing.assert_allclose(oracle.intensity(pb2, O2), h, rtol=1e-12)


# ----------------------------------------------------------------------------- error metric
@pytest.mark.parametrize("loss", [0, 1])
def test_ell_derivatives_by_finite_differences(loss):
    rng = np.random.default_rng(0)
    zeta = rng.uniform(0.3, 3.0, 50)
    y = rng.uniform(0.0, 5.0, 50)
    y[:5] = 0.0
    l, d1, d2 = oracle.ell_terms(loss, zeta, y)
    e = 1e-5
    lp, d1p, _ = oracle.ell_terms(loss, zeta + e, y)
    lm, d1m, _ = oracle.ell_terms(loss, zeta - e, y)
    np.testing.assert_allclose((lp - lm) / (2 * e), d1, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose((d1p - d1m) / (2 * e), d2, rtol=1e-7, atol=1e-9)
    # closed values of Eq. ell_magnitude at a few points
    if loss == 0:
        np.testing.assert_allclose(l, 0.5 * (zeta - np.sqrt(y)) ** 2, rtol=1e-14)
    else:
        np.testing.assert_allclose(l[:5], zeta[:5] ** 2, rtol=1e-14)  # 0 log 0 = 0


def test_noiseless_truth_zero_loss_and_gradient():
    """Gaussian metric: f = 0 and grad f = 0 at the truth of noiseless data (b included)."""
    pb, O = tiny_problem(0)
    f = oracle.loss(pb, O)
    assert abs(f) < 1e-20
    g = oracle.gradient(pb, O)
    assert np.abs(g).max() < 1e-12


def test_poisson_truth_value_and_stationarity():
    """Poisson metric at the truth with y = h: f = sum (y - y log y), grad f = 0."""
    pb, O = tiny_problem(1)
    y = pb.y
    f = oracle.loss(pb, O)
    ref = float(np.sum(y - np.where(y > 0, y * np.log(np.where(y > 0, y, 1)), 0)))
    assert abs(f - ref) <= 1e-12 * max(1.0, abs(ref))
    g = oracle.gradient(pb, O)
    assert np.abs(g).max() < 1e-9


# ----------------------------------------------------------------------------- derivatives
@pytest.mark.parametrize("loss", [0, 1])
def test_gradient_by_central_differences(loss):
    pb, O_true = tiny_problem(loss, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=11, scale=0.05)
    g = oracle.gradient(pb, O)
    v = synth.random_complex(O.shape, seed=12)
    e = 1e-6
    fd = (oracle.loss(pb, O + e * v) - oracle.loss(pb, O - e * v)) / (2 * e)
    assert abs(fd - rdot(g, v)) <= 1e-7 * abs(fd) + 1e-9


def test_probe_gradient_by_central_differences():
    pb, O_true = tiny_problem(1, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=13, scale=0.05)
    P = pb.P
    gO, gP = oracle.gradient(pb, O, probe_part=True)
    v = synth.random_complex(P.shape, seed=14)
    e = 1e-6
    fd = (oracle.loss(pb, O, P + e * v) - oracle.loss(pb, O, P - e * v)) / (2 * e)
    assert abs(fd - rdot(gP, v)) <= 1e-7 * abs(fd) + 1e-9


def zeta_of(pb, O, P=None):
    if P is not None:
        pb = oracle.Problem((pb.ny, pb.nx), P, pb.pos, pb.y, pb.loss, pb.b)
    return np.sqrt(oracle.intensity(pb, O))


def test_jvp_by_finite_differences_object_and_probe():
    pb, O = tiny_problem(0)
    vO = synth.random_complex(O.shape, seed=20)
    vP = synth.random_complex(pb.P.shape, seed=21)
    e = 1e-6
    fd = (zeta_of(pb, O + e * vO, pb.P + e * vP) - zeta_of(pb, O - e * vO, pb.P - e * vP)) / (2 * e)
    jv = oracle.jvp(pb, O, vO, vP=vP)
    np.testing.assert_allclose(jv, fd, rtol=1e-6, atol=1e-8)


def test_adjoint_identity():
    """<J v, w> = <v, J^T w> in real coordinates (object + probe), to 1e-12."""
    pb, O = tiny_problem(1, noiseless=False)
    vO = synth.random_complex(O.shape, seed=30)
    vP = synth.random_complex(pb.P.shape, seed=31)
    w = synth.random_real((pb.K, pb.my, pb.mx), seed=32)
    lhs = float(np.sum(oracle.jvp(pb, O, vO, vP=vP) * w))
    tO, tP = oracle.jtvp(pb, O, w, probe_part=True)
    rhs = rdot(vO, tO) + rdot(vP, tP)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def dense_jacobian(pb, O, e=1e-6):
    """Dense real-coordinate Jacobian of zeta (K*M x 2N) by central differences of the
    forward model, column by column (brute force)."""
    N = O.size
    cols = []
    for part in (1.0, 1j):
        for n in range(N):
            d = np.zeros(N, complex)
            d[n] = part * e
            d = d.reshape(O.shape)
            cols.append(((zeta_of(pb, O + d) - zeta_of(pb, O - d)) / (2 * e)).ravel())
    return np.stack(cols, axis=1)


def to_real(z):
    z = np.asarray(z).ravel()
    return np.concatenate([z.real, z.imag])


def from_real(x, shape):
    n = x.size // 2
    return (x[:n] + 1j * x[n:]).reshape(shape)


@pytest.mark.parametrize("loss", [0, 1])
def test_ggn_matvec_equals_dense_brute_force(loss):
    pb, O_true = tiny_problem(loss, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=40, scale=0.05)
    J = dense_jacobian(pb, O)
    zeta = zeta_of(pb, O).ravel()
    _, dl, d2l = oracle.ell_terms(loss, zeta, pb.y.ravel())
    G = J.T @ (d2l[:, None] * J)
    g_dense = J.T @ dl
    np.testing.assert_allclose(to_real(oracle.gradient(pb, O)), g_dense, rtol=1e-6, atol=1e-7)
    v = synth.random_complex(O.shape, seed=41)
    lam = 0.37
    out = oracle.ggn_matvec(pb, O, v, lam=lam)
    ref = G @ to_real(v) + lam * to_real(v)
    np.testing.assert_allclose(to_real(out), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_ggn_symmetric_psd_and_gauss_identity():
    pb, O_true = tiny_problem(0, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=50, scale=0.1)
    u = synth.random_complex(O.shape, seed=51)
    v = synth.random_complex(O.shape, seed=52)
    Gu = oracle.ggn_matvec(pb, O, u)
    Gv = oracle.ggn_matvec(pb, O, v)
    assert abs(rdot(u, Gv) - rdot(Gu, v)) <= 1e-12 * abs(rdot(u, Gv))
    assert rdot(v, Gv) >= 0
    jv = oracle.jvp(pb, O, v)
    assert abs(rdot(v, Gv) - float(np.sum(jv * jv))) <= 1e-12 * rdot(v, Gv)


def test_global_phase_null_direction():
    """J (i O) = 0 and G (i O) = 0: the global-phase ambiguity (Sec. 2)."""
    pb, O_true = tiny_problem(1, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=60, scale=0.05)
    Gv = oracle.ggn_matvec(pb, O, 1j * O)
    Gu = oracle.ggn_matvec(pb, O, synth.random_complex(O.shape, seed=61))
    assert np.abs(Gv).max() <= 1e-12 * np.abs(Gu).max()
    g1 = oracle.gradient(pb, O)
    g2 = oracle.gradient(pb, O * np.exp(0.4j))
    np.testing.assert_allclose(g2, g1 * np.exp(0.4j), atol=1e-12 * np.abs(g1).max())
    assert abs(oracle.loss(pb, O) - oracle.loss(pb, O * np.exp(0.4j))) < 1e-12 * abs(oracle.loss(pb, O))


def test_blind_scale_null_direction():
    """J (O, -P) = 0: the object/probe scale ambiguity of the blind problem (Sec. 2)."""
    pb, O = tiny_problem(0, noiseless=False)
    jv = oracle.jvp(pb, O, O, vP=-pb.P)
    assert np.abs(jv).max() < 1e-12 * np.abs(oracle.jvp(pb, O, O)).max()


def test_ggn_equals_hessian_at_noiseless_truth():
    """At the truth of noiseless Gaussian data the residual term of Eq. ggn_approximation
    vanishes, so G v equals the Hessian-vector product (central differences of grad f)."""
    pb, O = tiny_problem(0)
    v = synth.random_complex(O.shape, seed=70)
    e = 1e-5
    hv = (oracle.gradient(pb, O + e * v) - oracle.gradient(pb, O - e * v)) / (2 * e)
    gv = oracle.ggn_matvec(pb, O, v)
    np.testing.assert_allclose(gv, hv, rtol=1e-6, atol=1e-7 * np.abs(gv).max())


@pytest.mark.parametrize("loss", [0, 1])
def test_ggn_diag_closed_form_vs_dense(loss):
    """App. B: the closed-form diagonal equals the mean of the exact Re/Im diagonals of the
    dense G when tr_k uses the exact weights |psihat|^2/h (the printed form approximates
    h ~ |psihat|^2, a difference of order b)."""
    pb, O_true = tiny_problem(loss, noiseless=False, b=1e-12)
    O = O_true + synth.random_complex(O_true.shape, seed=80, scale=0.05)
    J = dense_jacobian(pb, O)
    zeta = zeta_of(pb, O).ravel()
    _, _, d2l = oracle.ell_terms(loss, zeta, pb.y.ravel())
    G = J.T @ (d2l[:, None] * J)
    N = O.size
    dg = np.diag(G)
    mean_diag = 0.5 * (dg[:N] + dg[N:])
    D_O, _ = oracle.ggn_diag(pb, O)
    np.testing.assert_allclose(D_O.ravel(), mean_diag, rtol=2e-6, atol=1e-9 * mean_diag.max())


def test_cg_matches_dense_solve():
    pb, O_true = tiny_problem(0, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=90, scale=0.05)
    g = oracle.gradient(pb, O)
    lam = 0.05
    J = dense_jacobian(pb, O)
    G = J.T @ J
    A = G + lam * np.eye(G.shape[0])
    x_ref = np.linalg.solve(A, -to_real(g))
    x, r, it, conv = oracle.cg(pb, O, g, lam, eta=1e-12, max_iter=400)
    assert conv
    np.testing.assert_allclose(to_real(x), x_ref, rtol=1e-5, atol=1e-7 * np.abs(x_ref).max())
    # residual returned is -g - A x
    np.testing.assert_allclose(to_real(r), -to_real(g) - A @ to_real(x), atol=1e-8)


@pytest.mark.parametrize("eta", [0.5, 0.1, 0.02])
def test_truncated_cg_stops_at_the_first_iterate_meeting_the_forcing_bound(eta):
    """Eq. lma_termination_magnitude: CG stops as soon as ||(G + lambda I) x + g|| <= eta ||g||,
    checked with the dense G: the returned iterate meets the bound, the one before it does
    not, and a warm start from the converged solution stops at once."""
    pb, O_true = tiny_problem(1, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=91, scale=0.05)
    g = oracle.gradient(pb, O)
    lam = 0.05
    J = dense_jacobian(pb, O)
    _, _, d2l = oracle.ell_terms(pb.loss, zeta_of(pb, O).ravel(), pb.y.ravel())
    A = J.T @ (d2l[:, None] * J) + lam * np.eye(2 * O.size)
    bound = eta * np.linalg.norm(to_real(g))
    residual = lambda x: np.linalg.norm(A @ to_real(x) + to_real(g))
    x, _, it, conv = oracle.cg(pb, O, g, lam, eta=eta, max_iter=400)
    assert conv and it >= 1
    assert residual(x) <= bound * (1 + 1e-9)
    x_prev, _, it_prev, conv_prev = oracle.cg(pb, O, g, lam, eta=eta, max_iter=it - 1)
    assert it_prev == it - 1 and not conv_prev and residual(x_prev) > bound
    _, _, it_warm, conv_warm = oracle.cg(pb, O, g, lam, eta=eta, max_iter=400, x0=x)
    assert conv_warm and it_warm == 0


@pytest.mark.parametrize("beta,scale,noiseless,root_branch",
                         [(0.9, 0.05, False, False), (0.9, 0.002, True, True), (1e-3, 0.05, False, False)])
def test_lm_forcing_term_is_min_of_beta_and_root_gradient_norm(beta, scale, noiseless, root_branch):
    """Reading C4: the first outer iteration of Algorithm 1 runs exactly as many CG
    iterations as a cold-started truncated CG with eta = min(beta, ||grad f||^(1/2)) and
    lambda = mu0 ||grad_zeta l|| (the truncated CG itself is pinned above)."""
    pb, O_true = tiny_problem(1, noiseless=noiseless)
    O0 = O_true + synth.random_complex(O_true.shape, seed=92, scale=scale)
    mu0 = 1e-2
    _, info = oracle.lm_solve(pb, O0, beta=beta, mu0=mu0, max_outer=1, max_cg=400)
    g = oracle.gradient(pb, O0)
    gnorm = np.linalg.norm(to_real(g))
    _, dl, _ = oracle.ell_terms(pb.loss, zeta_of(pb, O0).ravel(), pb.y.ravel())
    eta = min(beta, math.sqrt(gnorm))
    _, _, it, conv = oracle.cg(pb, O0, g, mu0 * np.linalg.norm(dl), eta=eta, max_iter=400)
    assert conv and info["mu"][0] <= mu0          # the first step was accepted (one CG solve)
    assert info["cg"][0] == it
    assert (math.sqrt(gnorm) < beta) == root_branch   # both branches of the minimum are exercised


def test_object_error_phase_invariance():
    O = synth.object_texture(32, seed=1)
    assert oracle.object_error(O * np.exp(1.3j), O) < 1e-14
    assert abs(oracle.object_error(1.1 * O, O) - 0.1) < 1e-12


def test_paper_lm_parameters_fixture():
    """The LM constants of Sec. 5 (tests/golden/lm_parameters.txt) are the oracle defaults."""
    vals = {}
    with open(os.path.join(GOLDEN, "lm_parameters.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    d = oracle.DEFAULT_LM
    for k in ("mu0", "mu_min", "nu", "rho_min", "kappa"):
        assert d[k] == vals[k]


def test_lm_converges_on_small_noiseless_workload():
    """Algorithm 1 on the 128^2 / 32^2 / 64-position noiseless workload from a flat start
    reaches 1e-3 object error against the truth (the solution is exact up to phase)."""
    w = synth.SMALL
    O_true = synth.to_c64(synth.object_texture(w.n, seed=0))
    P = synth.to_c64(synth.probe_disk_defocus(w.m, w.radius))
    pos, _ = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    pb = oracle.Problem((w.n, w.n), P, pos, None, 0, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true))
    mask = synth.illumination_mask(w.n, P, pos, 0.1)
    O, info = oracle.lm_solve(pb, synth.flat_object(w.n), O_ref=O_true, mask=mask,
                              max_outer=60, target_err=1e-3)
    assert info["status"] == 0
    assert info["err"][-1] <= 1e-3, info
    assert info["n_outer"] < 60


# ----------------------------------------------------------------------------- joint / PLM
def dense_jacobian_joint(pb, O, P, e=1e-6):
    """Dense real-coordinate Jacobian of zeta w.r.t. z = [O; P] (K*M x 2(N+M)) by central
    differences of the forward model: columns ordered Re O, Re P, Im O, Im P."""
    N, M = O.size, P.size

    def zeta_at(Ov, Pv):
        return zeta_of(pb, Ov, Pv).ravel()

    cols = []
    for part in (1.0, 1j):
        for n in range(N):
            d = np.zeros(N, complex)
            d[n] = part * e
            d = d.reshape(O.shape)
            cols.append((zeta_at(O + d, P) - zeta_at(O - d, P)) / (2 * e))
        for m in range(M):
            d = np.zeros(M, complex)
            d[m] = part * e
            d = d.reshape(P.shape)
            cols.append((zeta_at(O, P + d) - zeta_at(O, P - d)) / (2 * e))
    return np.stack(cols, axis=1)


def z_real(z):
    return np.concatenate([z.real, z.imag])


@pytest.mark.parametrize("loss", [0, 1])
def test_joint_ggn_matvec_and_diag_vs_dense(loss):
    pb, O_true = tiny_problem(loss, noiseless=False, b=1e-12)
    O = O_true + synth.random_complex(O_true.shape, seed=100, scale=0.05)
    P = pb.P * 1.1 + synth.random_complex(pb.P.shape, seed=101, scale=0.05)
    J = dense_jacobian_joint(pb, O, P)
    zeta = zeta_of(pb, O, P).ravel()
    _, _, d2l = oracle.ell_terms(loss, zeta, pb.y.ravel())
    G = J.T @ (d2l[:, None] * J)
    L = O.size + P.size
    v = synth.random_complex(L, seed=102)
    D = np.abs(synth.random_real(L, seed=103)) + 0.5
    lam = 0.3
    out = oracle.ggn_matvec_z(pb, O, v, lam=lam, D=D, P=P, joint=True)
    ref = G @ z_real(v) + lam * np.concatenate([D, D]) * z_real(v)
    np.testing.assert_allclose(z_real(out), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    # closed-form diagonal of both blocks (App. B, Eq. ggn_joint_diag) = mean of Re/Im diagonals
    D_O, D_P = oracle.ggn_diag(pb, O, P)
    dg = np.diag(G)
    mean_diag = 0.5 * (dg[:L] + dg[L:])
    np.testing.assert_allclose(np.concatenate([D_O.ravel(), D_P.ravel()]), mean_diag, rtol=2e-6,
                               atol=1e-9 * mean_diag.max())


def test_jacobi_pcg_matches_dense_solve_joint():
    pb, O_true = tiny_problem(0, noiseless=False)
    O = O_true + synth.random_complex(O_true.shape, seed=110, scale=0.05)
    P = pb.P
    gO, gP = oracle.gradient(pb, O, P, probe_part=True)
    g = np.concatenate([gO.ravel(), gP.ravel()])
    D_O, D_P = oracle.ggn_diag(pb, O, P, floor_rel=1e-6)
    D = np.concatenate([D_O.ravel(), D_P.ravel()])
    lam = 0.05
    J = dense_jacobian_joint(pb, O, P)
    A = J.T @ J + lam * np.diag(np.concatenate([D, D]))
    x_ref = np.linalg.solve(A, -z_real(g))
    x, r, it, conv = oracle.pcg(pb, O, g, lam, D, eta=1e-12, max_iter=800, P=P, joint=True)
    assert conv
    np.testing.assert_allclose(z_real(x), x_ref, rtol=1e-5, atol=1e-7 * np.abs(x_ref).max())
    # the preconditioned solve needs far fewer iterations than plain CG on the same system
    _, _, it_plain, _ = oracle.pcg(pb, O, g, lam, None, eta=1e-6, max_iter=800, P=P, joint=True)
    _, _, it_pcg, _ = oracle.pcg(pb, O, g, lam, D, eta=1e-6, max_iter=800, P=P, joint=True)
    assert it_pcg <= it_plain


def test_projection_is_the_nearest_feasible_point():
    v = synth.random_complex(500, seed=120, scale=2.0)
    p = oracle.project(v, 1.0)
    assert np.abs(p).max() <= 1.0 + 1e-15
    np.testing.assert_allclose(oracle.project(p, 1.0), p)           # idempotent
    inside = np.abs(v) <= 1.0
    np.testing.assert_allclose(p[inside], v[inside])                # feasible points unchanged
    # no feasible point is closer: compare with random points of the unit disk
    rng = np.random.default_rng(121)
    q = np.sqrt(rng.uniform(0, 1, (200, 500))) * np.exp(2j * np.pi * rng.uniform(0, 1, (200, 500)))
    assert np.all(np.abs(v - p)[None, :] <= np.abs(v[None, :] - q) + 1e-12)


def test_plm_scaled_converges_on_small_workload():
    """PLM (D = Dg(G), lambda = mu, Jacobi PCG) on the 128^2 noiseless workload reaches 1e-3."""
    w = synth.SMALL
    O_true = synth.to_c64(synth.object_texture(w.n, seed=0))
    P = synth.to_c64(synth.probe_disk_defocus(w.m, w.radius))
    pos, _ = synth.raster_positions(w.n, w.m, w.grid, w.step, w.jitter, seed=1)
    pb = oracle.Problem((w.n, w.n), P, pos, None, 0, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true))
    mask = synth.illumination_mask(w.n, P, pos, 0.1)
    O, _, info = oracle.lm_solve2(pb, synth.flat_object(w.n), O_ref=O_true, mask=mask, max_outer=60,
                                  target_err=1e-3, scaled=1)
    assert info["status"] == 0 and info["err"][-1] <= 1e-3, info


def test_plm_joint_projected_blind_reconstruction_improves():
    """PLM-J with Algorithm 2 on a small noiseless blind problem: the object error falls by an
    order of magnitude from a flat start with a wrong (unphased) probe, and the iterate
    satisfies the constraints |O| <= 1 (Eq. constraints)."""
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
    O, P, info = oracle.lm_solve2(pb, O0, P0, max_outer=40, scaled=1, joint=1, projected=1)
    assert info["status"] == 0
    assert np.abs(O).max() <= 1.0 + 1e-12
    e = oracle.object_error_blind(O, O_true, mask)
    assert e <= 0.05 * e0, (e0, e)
    assert info["f"][-1] < 1e-3 * info["f"][0]


def test_blind_error_metric_invariances():
    """The blind-problem error is zero under a complex scale and a linear phase ramp of the
    reference (the ambiguities of Sec. 2) and positive otherwise."""
    O = synth.object_texture(48, seed=9)
    yy, xx = np.mgrid[0:48, 0:48]
    Ot = (0.7 - 0.4j) * O * np.exp(1j * (0.3 + 0.05 * yy - 0.02 * xx))
    assert oracle.object_error_blind(Ot, O) < 1e-10
    assert oracle.object_error_blind(O + 0.1 * synth.random_complex(O.shape, seed=8), O) > 0.05


# ------------------------------------------------------------------- App. E surrogate metric
def test_surrogate_schedule_shape():
    """App. E: s_t starts at s_0, falls monotonically on an evenly spaced logarithmic grid
    (constant ratio between iterations), and is exactly 0 from t = T on; T = 0 is off."""
    s0, s_end, T = 1.0, 1e-4, 9
    s = np.array([oracle.surrogate_at(t, s0, s_end, T) for t in range(T + 3)])
    assert s[0] == s0 and abs(s[T - 1] - s_end) <= 1e-15
    assert np.all(np.diff(s[:T]) < 0)
    ratios = s[1:T] / s[:T - 1]
    assert np.allclose(ratios, ratios[0], rtol=1e-12, atol=0)
    assert np.allclose(np.log10(s[:T]), np.linspace(0.0, -4.0, T), atol=1e-12)
    assert np.all(s[T:] == 0.0)
    assert oracle.surrogate_at(0, s0, s_end, 0) == 0.0
    assert oracle.surrogate_at(0, s0, s_end, 1) == s0 and oracle.surrogate_at(1, s0, s_end, 1) == 0.0


def small_poisson_problem(seed=30, b=1e-8):
    n, m = 48, 16
    O_true = synth.to_c64(synth.object_texture(n, seed=seed))
    P = synth.to_c64(synth.probe_disk_defocus(m, 5.0))
    pos, _ = synth.raster_positions(n, m, 6, 6, 1, seed=seed + 1)
    pb = oracle.Problem((n, n), P, pos, None, oracle.LOSS_POISSON, b)
    h = oracle.intensity(pb, O_true)
    P = synth.to_c64(P * np.sqrt(300.0 / h.max()))
    pb = oracle.Problem((n, n), P, pos, None, oracle.LOSS_POISSON, b)
    pb.y = synth.poisson_counts(oracle.intensity(pb, O_true), seed=seed + 2)
    return pb, O_true


def test_surrogate_is_a_shifted_background():
    """Eq. expected_count_surrogate only adds s_t to the background: a constant schedule
    (s_0 = s_end = s) gives the same iterates as the plain method on b + s."""
    pb, O_true = small_poisson_problem()
    s = 0.37
    O0 = synth.flat_object(pb.nx)
    Oa, _, ia = oracle.lm_solve2(pb, O0, max_outer=3, scaled=1, surrogate0=s, surrogate_end=s, surrogate_T=50)
    pb_b = oracle.Problem((pb.ny, pb.nx), pb.P, pb.pos, pb.y, pb.loss, pb.b + s)
    Ob, _, ib = oracle.lm_solve2(pb_b, O0, max_outer=3, scaled=1)
    assert np.array_equal(Oa, Ob)
    assert np.array_equal(ia["f"], ib["f"])


def test_surrogate_reverts_to_the_true_metric():
    """From t = T on the method optimises the Poisson metric itself: the f recorded at
    iteration T is the true metric at the iterate the first T iterations produced, while the
    entries before T are the surrogate's (larger background), not the true metric's."""
    pb, _ = small_poisson_problem()
    kw = dict(scaled=1, surrogate0=1.0, surrogate_end=1e-2, surrogate_T=3)
    O0 = synth.flat_object(pb.nx)
    O3, _, _ = oracle.lm_solve2(pb, O0, max_outer=3, **kw)
    O5, _, i5 = oracle.lm_solve2(pb, O0, max_outer=5, **kw)
    assert abs(i5["f"][3] - oracle.loss(pb, O3)) <= 1e-12 * abs(i5["f"][3])
    # the surrogate iterations really used a larger background: their f differ from the truth
    O1, _, _ = oracle.lm_solve2(pb, O0, max_outer=1, **kw)
    assert abs(i5["f"][1] - oracle.loss(pb, O1)) > 1e-6 * abs(i5["f"][1])
    assert np.isfinite(i5["f"]).all() and i5["f"][4] <= i5["f"][3]


# ----------------------------------------------------------------------- Algorithm 1, densely
def dense_lm(pb, O0, mu0, n_outer, kappa=4.0, nu=1.0, rho_min=1e-4, mu_min=1e-8):
    """Algorithm 1 (D = I) on a tiny problem with every linear-algebra step done densely:
    J by central differences of the forward model, g = J^T dl and G = J^T diag(d2l) J from
    the pinned metric derivatives, the step by a direct solve of (G + lambda I) d = -g, the
    predicted reduction from its definition -(g.d + d.G.d / 2), lambda = mu ||dl||^nu.
    Returns the iterate, the error metric at each linearisation, mu after each outer
    iteration, the gain ratio of the step that ended it, and the smallest distance of a
    gain ratio to the mu thresholds 1/4 and 3/4."""
    O, mu = O0.copy(), mu0
    hist_f, hist_mu, hist_rho, margin = [], [], [], np.inf
    for _ in range(n_outer):
        J = dense_jacobian(pb, O)
        l, dl, d2l = oracle.ell_terms(pb.loss, zeta_of(pb, O).ravel(), pb.y.ravel())
        f = float(l.sum())
        g = J.T @ dl
        G = J.T @ (d2l[:, None] * J)
        hist_f.append(f)
        while True:
            lam = mu * np.linalg.norm(dl) ** nu
            d = np.linalg.solve(G + lam * np.eye(G.shape[0]), -g)
            O_try = O + from_real(d, O.shape)
            pred = -(g @ d + 0.5 * d @ (G @ d))
            rho = (f - oracle.loss(pb, O_try)) / pred if pred > 0 else -1.0
            margin = min(margin, abs(rho - 0.25), abs(rho - 0.75))
            if rho > 0.75:
                mu = max(mu / kappa, mu_min)
            elif rho <= 0.25:
                mu = kappa * mu
            if rho > rho_min:
                O = O_try
                break
        hist_mu.append(mu)
        hist_rho.append(rho)
    return O, np.array(hist_f), np.array(hist_mu), np.array(hist_rho), margin


def dense_plm(pb, O0, mu0, n_outer, floor=1e-6, kappa=4.0, rho_min=1e-4, mu_min=1e-8):
    """PLM (Sec. 3.3): Algorithm 1 with D = Dg(G) (the closed form, pinned against the dense
    diagonal above) and lambda = mu, every step solved densely; returns as dense_lm."""
    O, mu = O0.copy(), mu0
    hist_f, hist_mu, hist_rho, margin = [], [], [], np.inf
    for _ in range(n_outer):
        J = dense_jacobian(pb, O)
        l, dl, d2l = oracle.ell_terms(pb.loss, zeta_of(pb, O).ravel(), pb.y.ravel())
        f = float(l.sum())
        g = J.T @ dl
        G = J.T @ (d2l[:, None] * J)
        D_O, _ = oracle.ggn_diag(pb, O, floor_rel=floor)
        D = np.concatenate([D_O.ravel(), D_O.ravel()])   # the same scale on Re and Im
        hist_f.append(f)
        while True:
            d = np.linalg.solve(G + mu * np.diag(D), -g)
            O_try = O + from_real(d, O.shape)
            pred = -(g @ d + 0.5 * d @ (G @ d))
            rho = (f - oracle.loss(pb, O_try)) / pred if pred > 0 else -1.0
            margin = min(margin, abs(rho - 0.25), abs(rho - 0.75))
            if rho > 0.75:
                mu = max(mu / kappa, mu_min)
            elif rho <= 0.25:
                mu = kappa * mu
            if rho > rho_min:
                O = O_try
                break
        hist_mu.append(mu)
        hist_rho.append(rho)
    return O, np.array(hist_f), np.array(hist_mu), np.array(hist_rho), margin


@pytest.mark.parametrize("loss,mu0", [(0, 1e-1), (1, 1.0)])
def test_plm_trajectory_equals_dense_algorithm(loss, mu0):
    """The oracle's PLM (Jacobi PCG run to a 1e-10 relative residual, D = Dg(G) floored at
    1e-6 of its maximum, lambda = mu) follows the dense restatement step for step."""
    pb, O_true = tiny_problem(loss, noiseless=False)
    O0 = O_true + synth.random_complex(O_true.shape, seed=80 + loss, scale=0.08)
    n_outer = 5
    O_d, f_d, mu_d, rho_d, margin = dense_plm(pb, O0, mu0, n_outer)
    assert margin > 1e-3
    O_o, _, info = oracle.lm_solve2(pb, O0, beta=1e-10, mu0=mu0, max_outer=n_outer, max_cg=1000, scaled=1)
    assert info["n_outer"] == n_outer
    np.testing.assert_allclose(info["f"], f_d, rtol=1e-6)
    np.testing.assert_array_equal(info["mu"], mu_d)
    np.testing.assert_allclose(info["rho"], rho_d, rtol=1e-4)
    assert np.linalg.norm(O_o - O_d) <= 1e-5 * np.linalg.norm(O_d)
    assert f_d[-1] < f_d[0]


@pytest.mark.parametrize("loss,mu0", [(0, 1e-2), (1, 1e-1)])
def test_lm_trajectory_equals_dense_algorithm(loss, mu0):
    """The oracle's matrix-free Algorithm 1 (truncated CG run to a 1e-10 relative residual,
    the predicted reduction from the CG residual, lambda from ||grad_zeta l||) follows the
    dense restatement step for step: same error metric at every linearisation, same gain
    ratio (the predicted reduction from its definition against the oracle's residual form),
    same mu after every outer iteration (no gain ratio within 1e-3 of a mu threshold), same
    iterate."""
    pb, O_true = tiny_problem(loss, noiseless=False)
    O0 = O_true + synth.random_complex(O_true.shape, seed=70 + loss, scale=0.08)
    n_outer = 5
    O_d, f_d, mu_d, rho_d, margin = dense_lm(pb, O0, mu0, n_outer)
    assert margin > 1e-3
    O_o, info = oracle.lm_solve(pb, O0, beta=1e-10, mu0=mu0, max_outer=n_outer, max_cg=1000)
    assert info["n_outer"] == n_outer
    np.testing.assert_allclose(info["f"], f_d, rtol=1e-6)
    np.testing.assert_array_equal(info["mu"], mu_d)
    np.testing.assert_allclose(info["rho"], rho_d, rtol=1e-4)
    assert np.linalg.norm(O_o - O_d) <= 1e-5 * np.linalg.norm(O_d)
    assert f_d[-1] < f_d[0]


@pytest.mark.parametrize("loss,mu0", [(0, 1e-1), (1, 1.0)])
def test_joint_plm_trajectory_equals_dense_algorithm(loss, mu0):
    """PLM on the joint state z = (O, P) (BPR, Sec. 3.3 with the joint diagonal): the oracle
    (Jacobi PCG to a 1e-10 relative residual) follows a dense restatement -- joint J by
    central differences, D = Dg(G) from the pinned joint closed form (each block floored at
    1e-6 of its maximum), direct solves of (G + mu D) d = -g -- step for step."""
    pb, O_true = tiny_problem(loss, noiseless=False, b=1e-12)
    O0 = O_true + synth.random_complex(O_true.shape, seed=110 + loss, scale=0.06)
    P0 = pb.P * (1.0 + synth.random_complex(pb.P.shape, seed=120 + loss, scale=0.05))
    N, M = O0.size, P0.size
    O, P, mu = O0.copy(), P0.copy(), mu0
    f_d, mu_d, rho_d, margin = [], [], [], np.inf
    for _ in range(4):
        J = dense_jacobian_joint(pb, O, P)
        l, dl, d2l = oracle.ell_terms(pb.loss, zeta_of(pb, O, P).ravel(), pb.y.ravel())
        f = float(l.sum())
        g = J.T @ dl
        G = J.T @ (d2l[:, None] * J)
        D_O, D_P = oracle.ggn_diag(pb, O, P=P, floor_rel=1e-6)
        Dz = np.concatenate([D_O.ravel(), D_P.ravel()])
        D = np.concatenate([Dz, Dz])                     # Re O, Re P, Im O, Im P
        f_d.append(f)
        while True:
            d = np.linalg.solve(G + mu * np.diag(D), -g)
            dz = d[:N + M] + 1j * d[N + M:]
            O_try, P_try = O + dz[:N].reshape(O.shape), P + dz[N:].reshape(P.shape)
            pred = -(g @ d + 0.5 * d @ (G @ d))
            rho = (f - oracle.loss(pb, O_try, P_try)) / pred if pred > 0 else -1.0
            margin = min(margin, abs(rho - 0.25), abs(rho - 0.75))
            if rho > 0.75:
                mu = max(mu / 4.0, 1e-8)
            elif rho <= 0.25:
                mu = 4.0 * mu
            if rho > 1e-4:
                O, P = O_try, P_try
                break
        mu_d.append(mu)
        rho_d.append(rho)
    assert margin > 1e-3
    O_o, P_o, info = oracle.lm_solve2(pb, O0, P0, beta=1e-10, mu0=mu0, max_outer=4, max_cg=4000,
                                      scaled=1, joint=1)
    assert info["n_outer"] == 4
    np.testing.assert_allclose(info["f"], f_d, rtol=1e-6)
    np.testing.assert_array_equal(info["mu"], mu_d)
    np.testing.assert_allclose(info["rho"], rho_d, rtol=1e-4)
    assert np.linalg.norm(O_o - O) <= 1e-5 * np.linalg.norm(O)
    assert np.linalg.norm(P_o - P) <= 1e-5 * np.linalg.norm(P)
    assert f_d[-1] < f_d[0]


def radial_projection(v, radius):
    a = np.abs(v)
    return np.where(a > radius, v * (radius / np.maximum(a, 1e-300)), v)


@pytest.mark.parametrize("loss,sigma", [(0, 0.3), (1, 1.5)])
def test_projected_joint_plm_trajectory_equals_dense_algorithm(loss, sigma):
    """Algorithm 2 on top of joint PLM (Sec. 4.3, reading C9): after an accepted step the
    iterate is projected onto |O| <= 1, kept if f(Pi) - f_min < gamma (f - f_min), else an
    Armijo search along s = Pi(z + d) - z (or -g when s is no descent direction) with
    projection at every trial; gain ratio and mu use the unprojected step.  The oracle matches
    a dense restatement step for step (the object's amplitudes reach 1, so the projection and
    the line search are both exercised; a strict sufficient-decrease constant sigma makes the
    search halve its step)."""
    gamma, tau_s, p_s, max_ls, rO, rP = 1e-6, 1e-8, 2.1, 30, 1.0, 1e8
    pb, O_true = tiny_problem(loss, noiseless=False, b=1e-12)
    y = pb.y.ravel()
    f_min = float(np.sum(y - np.where(y > 0, y * np.log(np.where(y > 0, y, 1.0)), 0.0))) if loss else 0.0
    O0 = O_true + synth.random_complex(O_true.shape, seed=130 + loss, scale=0.06)
    P0 = pb.P * (1.0 + synth.random_complex(pb.P.shape, seed=140 + loss, scale=0.05))
    N, M = O0.size, P0.size
    proj = lambda z: np.concatenate([radial_projection(z[:N], rO), radial_projection(z[N:], rP)])
    fz = lambda z: oracle.loss(pb, z[:N].reshape(O0.shape), z[N:].reshape(P0.shape))
    z, mu = np.concatenate([O0.ravel(), P0.ravel()]), 1.0
    f_d, mu_d, rho_d, margin, searched, projected, halved = [], [], [], np.inf, 0, 0, 0
    for _ in range(4):
        O, P = z[:N].reshape(O0.shape), z[N:].reshape(P0.shape)
        J = dense_jacobian_joint(pb, O, P)
        l, dl, d2l = oracle.ell_terms(pb.loss, zeta_of(pb, O, P).ravel(), y)
        f = float(l.sum())
        g = J.T @ dl
        G = J.T @ (d2l[:, None] * J)
        D_O, D_P = oracle.ggn_diag(pb, O, P=P, floor_rel=1e-6)
        Dz = np.concatenate([D_O.ravel(), D_P.ravel()])
        D = np.concatenate([Dz, Dz])
        g_c = g[:N + M] + 1j * g[N + M:]
        f_d.append(f)
        while True:
            d = np.linalg.solve(G + mu * np.diag(D), -g)
            trial = z + d[:N + M] + 1j * d[N + M:]
            pred = -(g @ d + 0.5 * d @ (G @ d))
            rho = (f - fz(trial)) / pred if pred > 0 else -1.0
            margin = min(margin, abs(rho - 0.25), abs(rho - 0.75))
            if rho > 0.75:
                mu = max(mu / 4.0, 1e-8)
            elif rho <= 0.25:
                mu = 4.0 * mu
            if rho > 1e-4:
                tp = proj(trial)
                projected += int(np.any(np.abs(trial[:N]) > rO))
                if fz(tp) - f_min < gamma * (f - f_min):
                    z = tp
                else:
                    searched += 1
                    s = tp - z
                    ss = float(np.sum(np.abs(s) ** 2))
                    if not (float(np.sum((g_c.conj() * s).real)) <= -tau_s * ss ** (p_s / 2)):
                        s = -g_c
                    sn2 = float(np.sum(np.abs(s) ** 2))
                    alpha = 1.0
                    for _ls in range(max_ls):
                        t_ = proj(z + alpha * s)
                        if fz(t_) <= f - sigma * alpha * sn2:
                            z = t_
                            break
                        alpha *= 0.5
                        halved += 1
                break
        mu_d.append(mu)
        rho_d.append(rho)
    assert margin > 1e-3 and projected > 0 and searched > 0 and halved > 0
    O_o, P_o, info = oracle.lm_solve2(pb, O0, P0, beta=1e-10, mu0=1.0, max_outer=4, max_cg=4000,
                                      scaled=1, joint=1, projected=1, sigma=sigma)
    assert info["n_outer"] == 4
    np.testing.assert_allclose(info["f"], f_d, rtol=1e-6)
    np.testing.assert_array_equal(info["mu"], mu_d)
    np.testing.assert_allclose(info["rho"], rho_d, rtol=1e-4)
    assert np.linalg.norm(O_o.ravel() - z[:N]) <= 1e-5 * np.linalg.norm(z[:N])
    assert np.linalg.norm(P_o.ravel() - z[N:]) <= 1e-5 * np.linalg.norm(z[N:])


# ------------------------------------------------------------------- checkpoint / resume
def _npz_roundtrip(tmp_path, name, O, P, state):
    """Save (z, mu, t, delta) to .npz and read it back, as a checkpoint on disk."""
    path = os.path.join(str(tmp_path), name)
    np.savez(path, O=O, P=P, t=state["t"], mu=state["mu"], delta=state["delta"])
    d = np.load(path)
    return d["O"], d["P"], {"t": int(d["t"]), "mu": float(d["mu"]), "delta": d["delta"]}


def test_lm_resume_reproduces_the_uninterrupted_run_bit_for_bit(tmp_path):
    """Algorithm 1 carries (z, mu, t, delta) from one outer iteration to the next (Sec. 4.2;
    delta warm-starts the next CG solve): 7 outer iterations in one run equal 3 + 4 with the
    state checkpointed to disk in between, bit for bit (iterate, f, mu, CG counts)."""
    pb, _ = small_poisson_problem()
    O0 = synth.flat_object(pb.nx)
    O_all, info_all = oracle.lm_solve(pb, O0, max_outer=7)
    O_a, info_a = oracle.lm_solve(pb, O0, max_outer=3)
    O_r, _, st = _npz_roundtrip(tmp_path, "lm.npz", O_a, pb.P, info_a["state"])
    assert st["t"] == 3 and np.any(st["delta"] != 0)
    O_b, info_b = oracle.lm_solve(pb, O_r, max_outer=4, state=st)
    assert np.array_equal(O_b, O_all)
    for k in ("f", "mu", "cg", "gnorm"):
        assert np.array_equal(np.concatenate([info_a[k], info_b[k]]), info_all[k]), k
    assert info_b["state"]["t"] == 7 and info_b["state"]["mu"] == info_all["state"]["mu"]
    # without the warm start the continuation differs: the state matters
    O_c, _ = oracle.lm_solve(pb, O_r, max_outer=4, state=dict(st, delta=np.zeros_like(st["delta"])))
    assert not np.array_equal(O_c, O_all)


def test_plm_s_joint_resume_follows_the_surrogate_schedule_bit_for_bit(tmp_path):
    """The same for PLM-S on the joint state z = (O, P) (Sec. 3.3, App. E): the resumed run
    picks up the surrogate level s_t at t = state.t, so 2 + 3 iterations across the end of a
    T = 4 schedule equal 5 uninterrupted ones bit for bit; restarting the schedule (t = 0)
    does not."""
    n, m = 96, 32
    O_true = synth.to_c64(synth.object_texture(n, seed=4))
    P_true = synth.to_c64(synth.probe_disk_defocus(m, 10.0))
    pos, _ = synth.raster_positions(n, m, 8, 8, 1, seed=5)
    pb = oracle.Problem((n, n), P_true, pos, None, 1, 1e-8)
    pb.y = synth.to_f32(oracle.intensity(pb, O_true) * 50.0)
    P0 = synth.to_c64(synth.probe_disk_defocus(m, 10.0, phased=False) * np.sqrt(50.0))
    O0 = synth.flat_object(n) * 0.9
    # beta = 0.1: with Poisson's 0.9 the warm start alone meets the forcing bound after the
    # first solve and no CG iteration would run (the state would then hardly matter)
    kw = dict(scaled=1, joint=1, surrogate0=1.0, surrogate_end=1e-2, surrogate_T=4, beta=0.1)
    O_all, P_all, i_all = oracle.lm_solve2(pb, O0, P0, max_outer=5, **kw)
    assert np.all(i_all["cg"] > 0)
    O_a, P_a, i_a = oracle.lm_solve2(pb, O0, P0, max_outer=2, **kw)
    O_r, P_r, st = _npz_roundtrip(tmp_path, "plm.npz", O_a, P_a, i_a["state"])
    assert st["delta"].size == n * n + m * m
    O_b, P_b, i_b = oracle.lm_solve2(pb, O_r, P_r, max_outer=3, state=st, **kw)
    assert np.array_equal(O_b, O_all) and np.array_equal(P_b, P_all)
    assert np.array_equal(np.concatenate([i_a["f"], i_b["f"]]), i_all["f"])
    O_c, _, _ = oracle.lm_solve2(pb, O_r, P_r, max_outer=3, state=dict(st, t=0), **kw)
    assert not np.array_equal(O_c, O_all)
