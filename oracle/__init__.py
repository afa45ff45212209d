"""FP64 CPU oracle for the matrix-free Levenberg-Marquardt ptychography method
(arXiv 2103.01767).

TEST INFRASTRUCTURE ONLY: this package is the plain, slow reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` import it.  It shares no code with the CUDA path.

The arithmetic lives in ``ptylm_oracle.c`` (plain C99, double precision); this module
compiles it with gcc and wraps it with ctypes.  Complex arrays are numpy ``complex128``,
real arrays ``float64``, positions ``int32`` [K, 2] holding the (row, col) of each patch's
top-left corner.

Paper passages each wrapper follows (section / equation):
  forward        Sec. 2, Eqs. exit_wave and expected_count
  loss           Sec. 4.1, Eqs. error_metric_magnitude and ell_magnitude
  jvp / jtvp     App. B, Eq. jac_ampl (real-coordinate form)
  gradient       App. A step 1 (grad f = J^T grad_zeta l)
  ggn_matvec     App. A steps 2-4, Eq. ggn_magnitude_appendix_2
  ggn_diag       App. B, Eqs. ggn_diag_mat and ggn_joint_diag
  cg / lm_solve  Algorithm 1 with Eqs. lma_termination_magnitude and lma_termination_eta
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptylm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libptylm_oracle.so")
_lock = threading.Lock()
_lib = None

LOSS_GAUSSIAN = 0
LOSS_POISSON = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP).  Returns its path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("my", ctypes.c_int),
                ("mx", ctypes.c_int), ("K", ctypes.c_int), ("loss", ctypes.c_int),
                ("b", ctypes.c_double)]


class _LMParams(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("kappa", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("beta", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("target_err", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_loss.restype = ctypes.c_double
            _lib.orc_object_error.restype = ctypes.c_double
            _lib.orc_cg.restype = ctypes.c_int
            _lib.orc_lm_solve.restype = ctypes.c_int
            _lib.orc_fft2.restype = ctypes.c_int
            _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _r(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pos(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    assert a.ndim == 2 and a.shape[1] == 2
    return a


class Problem:
    """Geometry + data of one reconstruction: object shape, probe, positions, y, b, loss."""

    def __init__(self, obj_shape, probe, positions, y=None, loss=LOSS_GAUSSIAN, b=1e-8):
        self.ny, self.nx = int(obj_shape[0]), int(obj_shape[1])
        self.P = _c(probe)
        self.my, self.mx = self.P.shape
        self.pos = _pos(positions)
        self.K = self.pos.shape[0]
        if self.K:
            assert self.pos[:, 0].min() >= 0 and self.pos[:, 1].min() >= 0
            assert self.pos[:, 0].max() + self.my <= self.ny
            assert self.pos[:, 1].max() + self.mx <= self.nx
        self.y = None if y is None else _r(y).reshape(self.K, self.my, self.mx)
        self.loss = int(loss)
        self.b = float(b)

    @property
    def M(self):
        return self.my * self.mx

    def geom(self):
        return _Geom(self.ny, self.nx, self.my, self.mx, self.K, self.loss, self.b)

    def subset(self, idx):
        """The same problem restricted to the positions ``idx`` (sums over k split)."""
        idx = np.asarray(idx)
        return Problem((self.ny, self.nx), self.P, self.pos[idx],
                       None if self.y is None else self.y[idx], self.loss, self.b)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def dft2(x, inverse=False):
    """Direct orthonormal 2D DFT (definition).  sign -1 forward, +1 inverse."""
    x = _c(x)
    out = np.empty_like(x)
    _load().orc_dft2(_p(x), _p(out), x.shape[0], x.shape[1], 1 if inverse else -1)
    return out


def fft2(x, inverse=False):
    """The oracle's own radix-2 orthonormal 2D FFT."""
    x = _c(x).copy()
    rc = _load().orc_fft2(_p(x), x.shape[0], x.shape[1], 1 if inverse else -1)
    if rc:
        raise ValueError("fft2 needs power-of-two sides")
    return x


def forward(pb: Problem, O):
    """(psihat [K,my,mx] complex128, h [K,my,mx] float64)."""
    O = _c(O)
    ph = np.empty((pb.K, pb.my, pb.mx), np.complex128)
    h = np.empty((pb.K, pb.my, pb.mx), np.float64)
    g = pb.geom()
    _load().orc_forward(ctypes.byref(g), _p(O), _p(pb.P), _p(pb.pos), _p(ph), _p(h))
    return ph, h


def intensity(pb: Problem, O):
    return forward(pb, O)[1]


def loss(pb: Problem, O, P=None, return_dl_norm2=False):
    """f = sum l(zeta, y); optionally also ||grad_zeta l||^2."""
    O = _c(O)
    P = pb.P if P is None else _c(P)
    g = pb.geom()
    n2 = ctypes.c_double(0.0)
    f = _load().orc_loss(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(pb.y), ctypes.byref(n2))
    return (f, n2.value) if return_dl_norm2 else f


def ell_terms(loss_kind, zeta, y):
    """Per-element (l, dl/dzeta, d2l/dzeta2) of Eq. ell_magnitude."""
    zeta, y = _r(zeta), _r(y)
    n = zeta.size
    l, d1, d2 = np.empty(n), np.empty(n), np.empty(n)
    _load().orc_ell_terms(int(loss_kind), ctypes.c_long(n), _p(zeta), _p(y), _p(l), _p(d1), _p(d2))
    return l.reshape(zeta.shape), d1.reshape(zeta.shape), d2.reshape(zeta.shape)


def jvp(pb: Problem, O, vO, P=None, vP=None):
    O, vO = _c(O), _c(vO)
    P = pb.P if P is None else _c(P)
    vP = None if vP is None else _c(vP)
    out = np.empty((pb.K, pb.my, pb.mx), np.float64)
    g = pb.geom()
    _load().orc_jvp(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(vO), _p(vP), _p(out))
    return out


def jtvp(pb: Problem, O, w, P=None, probe_part=False):
    O, w = _c(O), _r(w)
    P = pb.P if P is None else _c(P)
    outO = np.empty((pb.ny, pb.nx), np.complex128)
    outP = np.empty((pb.my, pb.mx), np.complex128) if probe_part else None
    g = pb.geom()
    _load().orc_jtvp(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(w), _p(outO), _p(outP))
    return (outO, outP) if probe_part else outO


def gradient(pb: Problem, O, P=None, probe_part=False):
    O = _c(O)
    P = pb.P if P is None else _c(P)
    gO = np.empty((pb.ny, pb.nx), np.complex128)
    gP = np.empty((pb.my, pb.mx), np.complex128) if probe_part else None
    g = pb.geom()
    _load().orc_gradient(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(pb.y), _p(gO), _p(gP))
    return (gO, gP) if probe_part else gO


def ggn_matvec(pb: Problem, O, vO, lam=0.0, D_O=None, P=None, vP=None, D_P=None):
    """(G + lambda D) v.  Returns outO, or (outO, outP) when vP is given."""
    O, vO = _c(O), _c(vO)
    P = pb.P if P is None else _c(P)
    vP = None if vP is None else _c(vP)
    D_O = None if D_O is None else _r(D_O)
    D_P = None if D_P is None else _r(D_P)
    outO = np.empty((pb.ny, pb.nx), np.complex128)
    outP = np.empty((pb.my, pb.mx), np.complex128) if vP is not None else None
    g = pb.geom()
    _load().orc_ggn_matvec(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(pb.y), _p(vO), _p(vP),
                           ctypes.c_double(lam), _p(D_O), _p(D_P), _p(outO), _p(outP))
    return outO if vP is None else (outO, outP)


def ggn_diag(pb: Problem, O, P=None, floor_rel=0.0):
    O = _c(O)
    P = pb.P if P is None else _c(P)
    D_O = np.empty((pb.ny, pb.nx), np.float64)
    D_P = np.empty((pb.my, pb.mx), np.float64)
    g = pb.geom()
    _load().orc_ggn_diag(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(pb.y),
                         ctypes.c_double(floor_rel), _p(D_O), _p(D_P))
    return D_O, D_P


def cg(pb: Problem, O, grad, lam, eta, max_iter, x0=None):
    """Truncated CG for (G + lambda I) x = -grad; returns (x, r, iterations, converged)."""
    O, grad = _c(O), _c(grad)
    x = np.zeros((pb.ny, pb.nx), np.complex128) if x0 is None else _c(x0).copy()
    r = np.empty_like(x)
    conv = ctypes.c_int(0)
    g = pb.geom()
    it = _load().orc_cg(ctypes.byref(g), _p(O), _p(pb.P), _p(pb.pos), _p(pb.y), _p(grad),
                        ctypes.c_double(lam), ctypes.c_double(eta), int(max_iter), _p(x), _p(r),
                        ctypes.byref(conv))
    return x, r, it, bool(conv.value)


def object_error(O, O_ref, mask=None):
    """min over a global phase of ||e^{i phi} O - O_ref|| / ||O_ref|| on ``mask``."""
    O, O_ref = _c(O), _c(O_ref)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    return float(_load().orc_object_error(ctypes.c_long(O.size), _p(O), _p(O_ref), _p(m)))


DEFAULT_LM = dict(mu0=1e-5, mu_min=1e-8, kappa=4.0, nu=1.0, rho_min=1e-4, mu_max=1e16,
                  max_outer=50, max_cg=100, target_err=0.0)


class _LMState(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("mu", ctypes.c_double), ("delta", ctypes.c_void_p)]


def _state_in(state, mu0, L):
    """(ctypes state, delta buffer) from a state dict {t, mu, delta} or a fresh start."""
    if state is None:
        state = {"t": 0, "mu": mu0, "delta": np.zeros(L, np.complex128)}
    delta = np.ascontiguousarray(np.asarray(state["delta"], np.complex128).reshape(-1)).copy()
    assert delta.size == L
    return _LMState(int(state["t"]), float(state["mu"]), delta.ctypes.data), delta


def lm_solve(pb: Problem, O0, O_ref=None, mask=None, beta=None, state=None, **kw):
    """Algorithm 1 (object-only, D = I).  Returns (O, info dict with the history).
    state: None (fresh start) or a dict {t, mu, delta} from an earlier info["state"]; the run
    continues from it, and info["state"] is the state after its last outer iteration."""
    prm = dict(DEFAULT_LM)
    prm.update(kw)
    if beta is None:
        beta = 0.1 if pb.loss == LOSS_GAUSSIAN else 0.9
    p = _LMParams(prm["mu0"], prm["mu_min"], prm["kappa"], prm["nu"], prm["rho_min"], beta,
                  prm["mu_max"], int(prm["max_outer"]), int(prm["max_cg"]), prm["target_err"])
    O = _c(O0).copy()
    L = int(prm["max_outer"])
    hf, hg, hmu, herr, hrho = (np.full(L, np.nan) for _ in range(5))
    hcg = np.zeros(L, np.int32)
    n_outer, cg_total = ctypes.c_int(0), ctypes.c_int(0)
    Oref = None if O_ref is None else _c(O_ref)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    g = pb.geom()
    cst, delta = _state_in(state, prm["mu0"], O.size)
    st = _load().orc_lm_solve(ctypes.byref(g), _p(O), _p(pb.P), _p(pb.pos), _p(pb.y),
                              ctypes.byref(p), _p(Oref), _p(m), ctypes.byref(n_outer),
                              ctypes.byref(cg_total), _p(hf), _p(hg), _p(hmu), _p(hcg),
                              _p(herr), _p(hrho), L, ctypes.byref(cst))
    n = n_outer.value
    return O, dict(status=st, n_outer=n, cg_total=cg_total.value, f=hf[:n], gnorm=hg[:n],
                   mu=hmu[:n], cg=hcg[:n], err=herr[:n], rho=hrho[:n],
                   state={"t": cst.t, "mu": cst.mu, "delta": delta.reshape(O.shape)})


# ---------------------------------------------------------------------------------------
# Scaled / joint / projected LM (PLM, PLM-J with Algorithm 2)
# ---------------------------------------------------------------------------------------
class _LM2Params(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("kappa", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("beta", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("target_err", ctypes.c_double),
                ("scaled", ctypes.c_int), ("joint", ctypes.c_int), ("projected", ctypes.c_int),
                ("radius_O", ctypes.c_double), ("radius_P", ctypes.c_double),
                ("gamma", ctypes.c_double), ("tau_s", ctypes.c_double), ("p_s", ctypes.c_double),
                ("sigma", ctypes.c_double), ("max_ls", ctypes.c_int), ("diag_floor", ctypes.c_double),
                ("f_min", ctypes.c_double), ("surrogate0", ctypes.c_double),
                ("surrogate_end", ctypes.c_double), ("surrogate_T", ctypes.c_int)]


def _z(pb, O, P=None):
    O = _c(O)
    return O if P is None else np.concatenate([O.ravel(), _c(P).ravel()])


def ggn_matvec_z(pb: Problem, O, v, lam=0.0, D=None, P=None, joint=False):
    """(G + lambda D) v on the z = [O; P] vector (joint) or O alone; v, D flat of length N(+M)."""
    z = _z(pb, O, P if joint else None)
    v = _c(v).ravel()
    out = np.empty_like(v)
    Pf = pb.P if P is None else _c(P)
    D = None if D is None else _r(D).ravel()
    g = pb.geom()
    _load().orc_ggn_matvec_z(ctypes.byref(g), _p(z), _p(Pf), _p(pb.pos), _p(pb.y), int(joint), _p(v),
                             ctypes.c_double(lam), _p(D), _p(out))
    return out


def pcg(pb: Problem, O, grad, lam, D, eta, max_iter, P=None, joint=False, x0=None):
    """Truncated PCG for (G + lambda D) x = -grad with the Jacobi preconditioner (1+lambda) D
    (D None: plain CG, D = I).  Vectors flat over z.  Returns (x, r, iterations, converged)."""
    z = _z(pb, O, P if joint else None)
    grad = _c(grad).ravel()
    x = np.zeros_like(grad) if x0 is None else _c(x0).ravel().copy()
    r = np.empty_like(x)
    D = None if D is None else _r(D).ravel()
    conv = ctypes.c_int(0)
    Pf = pb.P if P is None else _c(P)
    g = pb.geom()
    lib = _load()
    lib.orc_pcg.restype = ctypes.c_int
    it = lib.orc_pcg(ctypes.byref(g), _p(z), _p(Pf), _p(pb.pos), _p(pb.y), int(joint), _p(grad),
                     ctypes.c_double(lam), _p(D), ctypes.c_double(eta), int(max_iter), _p(x), _p(r),
                     ctypes.byref(conv))
    return x, r, it, bool(conv.value)


def project(v, radius):
    """Radial projection onto {|v_i| <= radius} (Eq. constraints)."""
    v = _c(v).copy()
    _load().orc_project(ctypes.c_long(v.size), _p(v), ctypes.c_double(radius))
    return v


def surrogate_at(t, surrogate0=1.0, surrogate_end=1e-4, surrogate_T=0):
    """s_t of the App. E surrogate schedule (0 when off or once t >= T)."""
    p = _LM2Params()
    p.surrogate0, p.surrogate_end, p.surrogate_T = surrogate0, surrogate_end, int(surrogate_T)
    lib = _load()
    lib.orc_surrogate_at.restype = ctypes.c_double
    return float(lib.orc_surrogate_at(ctypes.byref(p), int(t)))


def poisson_f_min(y):
    """sum(y - y log y): the Poisson metric's value at h = y (its minimum over h)."""
    y = np.asarray(y, np.float64)
    return float(np.sum(y - np.where(y > 0, y * np.log(np.where(y > 0, y, 1.0)), 0.0)))


DEFAULT_LM2 = dict(DEFAULT_LM, scaled=1, joint=0, projected=0, radius_O=1.0, radius_P=1e8, gamma=1e-6,
                   tau_s=1e-8, p_s=2.1, sigma=1e-4, max_ls=30, diag_floor=1e-6,
                   surrogate0=1.0, surrogate_end=1e-4, surrogate_T=0)


def lm_solve2(pb: Problem, O0, P0=None, O_ref=None, mask=None, beta=None, state=None, **kw):
    """Algorithm 1 with D = Dg(G) and Jacobi PCG (scaled), the joint state (joint) and the
    Algorithm 2 plug-in (projected).  Returns (O, P, info).  state as in lm_solve (delta over
    the whole state z: [ny*nx] or [ny*nx + my*mx] for joint problems)."""
    prm = dict(DEFAULT_LM2)
    prm.update(kw)
    if beta is None:
        beta = 0.1 if pb.loss == LOSS_GAUSSIAN else 0.9
    f_min = poisson_f_min(pb.y) if pb.loss == LOSS_POISSON else 0.0
    p = _LM2Params(prm["mu0"], prm["mu_min"], prm["kappa"], prm["nu"], prm["rho_min"], beta, prm["mu_max"],
                   int(prm["max_outer"]), int(prm["max_cg"]), prm["target_err"], int(prm["scaled"]),
                   int(prm["joint"]), int(prm["projected"]), prm["radius_O"], prm["radius_P"], prm["gamma"],
                   prm["tau_s"], prm["p_s"], prm["sigma"], int(prm["max_ls"]), prm["diag_floor"], f_min,
                   prm["surrogate0"], prm["surrogate_end"], int(prm["surrogate_T"]))
    O = _c(O0).copy()
    P = (pb.P if P0 is None else _c(P0)).copy()
    L = int(prm["max_outer"])
    hf, hg, hmu, herr, hrho = (np.full(L, np.nan) for _ in range(5))
    hcg = np.zeros(L, np.int32)
    n_outer, cg_total = ctypes.c_int(0), ctypes.c_int(0)
    Oref = None if O_ref is None else _c(O_ref)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    g = pb.geom()
    lib = _load()
    lib.orc_lm_solve2.restype = ctypes.c_int
    Lz = O.size + (P.size if int(prm["joint"]) else 0)
    cst, delta = _state_in(state, prm["mu0"], Lz)
    st = lib.orc_lm_solve2(ctypes.byref(g), _p(O), _p(P), _p(pb.pos), _p(pb.y), ctypes.byref(p), _p(Oref),
                           _p(m), ctypes.byref(n_outer), ctypes.byref(cg_total), _p(hf), _p(hg), _p(hmu),
                           _p(hcg), _p(herr), _p(hrho), L, ctypes.byref(cst))
    n = n_outer.value
    return O, P, dict(status=st, n_outer=n, cg_total=cg_total.value, f=hf[:n], gnorm=hg[:n], mu=hmu[:n],
                      cg=hcg[:n], err=herr[:n], rho=hrho[:n],
                      state={"t": cst.t, "mu": cst.mu, "delta": delta})


def object_error_blind(O, O_ref, mask=None, ramp_iterations=3):
    """Object error for the blind problem (Sec. 2: its solutions are unique only up to a
    complex scale and a linear phase ramp): min over c in C and a ramp exp(i(a0 + a1 y + a2 x))
    of ||c e^{i ramp} O - O_ref|| / ||O_ref|| on the mask.  The ramp is fitted by weighted
    least squares on the phase difference, repeated so that wrapped phases settle; then the
    closed-form c = <O', O_ref>/||O'||^2."""
    O = np.asarray(O, np.complex128)
    R = np.asarray(O_ref, np.complex128)
    mk = np.ones(O.shape, bool) if mask is None else np.asarray(mask, bool)
    yy, xx = np.nonzero(mk)
    o, r = O[mk], R[mk]
    A = np.stack([np.ones_like(yy), yy, xx], axis=1).astype(np.float64)
    for _ in range(ramp_iterations):
        w = np.abs(o) * np.abs(r)
        ph = np.angle(r * np.conj(o))
        coef, *_ = np.linalg.lstsq(A * w[:, None], ph * w, rcond=None)
        o = o * np.exp(1j * (A @ coef))
    c = np.vdot(o, r) / np.vdot(o, o)
    return float(np.linalg.norm(c * o - r) / np.linalg.norm(r))
