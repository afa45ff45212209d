"""Thin ctypes binding over the C-ABI of libptylm.so (include/ptylm.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  Arrays may be CUDA torch tensors (device pointers) or, where the C-ABI accepts
host memory, numpy arrays / CPU tensors.  The binding raises if the shared library is
missing; there is no fallback implementation.

Names follow the C-ABI: lm_init, forward_loss, gradient, jvp, jtvp, ggn_matvec, lm_solve,
lm_destroy, ptylm_strerror.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libptylm.so")

PTYLM_OK = 0
PTYLM_ERR_ARG = 1
PTYLM_ERR_NOMEM = 2
PTYLM_ERR_CUDA = 3
PTYLM_ERR_NAN = 4
PTYLM_ERR_TIMEOUT = 5
PTYLM_ERR_STALLED = 6
PTYLM_ERR_STATE = 7
PTYLM_WARN_CG_MAXIT = 16

LOSS_GAUSSIAN = 0
LOSS_POISSON = 1


class PtylmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("my", ctypes.c_int),
                ("mx", ctypes.c_int), ("K", ctypes.c_int), ("loss", ctypes.c_int),
                ("background", ctypes.c_float), ("joint", ctypes.c_int),
                ("workspace_budget", ctypes.c_size_t), ("values_per_thread", ctypes.c_int)]


class LMParams(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("kappa", ctypes.c_double), ("nu", ctypes.c_double),
                ("rho_min", ctypes.c_double), ("beta", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("fixed_cg", ctypes.c_int),
                ("target_err", ctypes.c_double), ("O_ref", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("scaled", ctypes.c_int), ("projected", ctypes.c_int),
                ("radius_O", ctypes.c_double), ("radius_P", ctypes.c_double),
                ("gamma", ctypes.c_double), ("tau_s", ctypes.c_double), ("p_s", ctypes.c_double),
                ("sigma", ctypes.c_double), ("max_ls", ctypes.c_int), ("diag_floor", ctypes.c_double),
                ("surrogate0", ctypes.c_double), ("surrogate_end", ctypes.c_double),
                ("surrogate_T", ctypes.c_int), ("separate_cg_kernels", ctypes.c_int),
                ("wait_polls", ctypes.c_int)]


class LMState(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("mu", ctypes.c_double), ("delta", ctypes.c_void_p)]


class LMStats(ctypes.Structure):
    _fields_ = [("n_outer", ctypes.c_int), ("cg_total", ctypes.c_int),
                ("matvecs_total", ctypes.c_int), ("f_final", ctypes.c_double),
                ("err_final", ctypes.c_double), ("hist_len", ctypes.c_int),
                ("hist_f", ctypes.c_void_p), ("hist_gnorm", ctypes.c_void_p),
                ("hist_mu", ctypes.c_void_p), ("hist_cg", ctypes.c_void_p),
                ("hist_err", ctypes.c_void_p), ("hist_rho", ctypes.c_void_p),
                ("hist_lambda", ctypes.c_void_p), ("hist_time", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def load_library():
    """Load libptylm.so (it must have been built: paper_2103_01767_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2103_01767_gb300/build.py)")
            lib = ctypes.CDLL(LIB_PATH)
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.lm_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Desc), vp, vp, vp]
            lib.forward_loss.argtypes = [vp, vp, vp, ctypes.POINTER(d), ctypes.POINTER(d), i]
            lib.gradient.argtypes = [vp, vp, vp]
            lib.jvp.argtypes = [vp, vp, vp, vp]
            lib.jtvp.argtypes = [vp, vp, vp, vp]
            lib.ggn_matvec.argtypes = [vp, vp, vp, d, vp, vp, vp]
            lib.lm_solve.argtypes = [vp, vp, vp, ctypes.POINTER(LMParams), ctypes.POINTER(LMStats)]
            lib.lm_solve_resume.argtypes = [vp, vp, vp, ctypes.POINTER(LMParams), ctypes.POINTER(LMState),
                                            ctypes.POINTER(LMStats)]
            lib.lm_destroy.argtypes = [vp]
            lib.forward_intensity.argtypes = [vp, vp, vp, vp]
            lib.ptylm_set_measurements.argtypes = [vp, vp]
            lib.ggn_diag.argtypes = [vp, vp, d]
            lib.forward_magnitude.argtypes = [vp, vp, vp, vp, i]
            lib.ptylm_forward_loss_noalloc.argtypes = [i, i, i, i, i, ctypes.c_float, vp, vp, vp, vp, vp, vp]
            lib.ptylm_profile.argtypes = [vp, i]
            lib.ptylm_fp32_peak.argtypes = [i, i, ctypes.POINTER(d), ctypes.POINTER(d), vp]
            lib.ptylm_profile_select.argtypes = [vp, ctypes.c_uint]
            lib.ptylm_profile_read.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
            lib.ptylm_strerror.argtypes = [i]
            lib.ptylm_strerror.restype = ctypes.c_char_p
            lib.ptylm_last_error.restype = ctypes.c_char_p
            lib.ptylm_default_lm_params.argtypes = [ctypes.POINTER(LMParams), i]
            P = ctypes.POINTER
            lib.ptylm_batch_init.argtypes = [P(vp), i, P(Desc), P(vp), P(vp), P(vp), vp]
            lib.ptylm_batch_offset.argtypes = [vp, i]
            lib.ptylm_batch_offset.restype = ctypes.c_long
            lib.ptylm_batch_forward_loss.argtypes = [vp, vp, P(d), P(d), i]
            lib.ptylm_batch_gradient.argtypes = [vp, vp]
            lib.ptylm_batch_ggn_matvec.argtypes = [vp, vp, vp, P(d)]
            lib.ptylm_batch_lm_solve.argtypes = [vp, vp, P(LMParams), P(LMStats)]
            lib.ptylm_batch_tune.argtypes = [vp, P(i), P(ctypes.c_float), i]
            lib.ptylm_batch_set_schedule.argtypes = [vp, i]
            lib.ptylm_batch_ggn_diag.argtypes = [vp, vp, d]
            lib.ptylm_batch_profile_read.argtypes = [vp, P(ctypes.c_longlong)]
            lib.ptylm_batch_destroy.argtypes = [vp]
            u64 = ctypes.c_uint64
            lib.ptylm_net_create.argtypes = [P(vp), i, P(i), i, u64, vp]
            lib.ptylm_net_num_params.argtypes = [vp]
            lib.ptylm_net_num_params.restype = ctypes.c_long
            lib.ptylm_net_set_params.argtypes = [vp, vp]
            lib.ptylm_net_get_params.argtypes = [vp, vp, vp]
            lib.ptylm_net_forward.argtypes = [vp, vp, i, vp]
            lib.ptylm_net_activation.argtypes = [vp, i, i, vp]
            lib.ptylm_net_loss_grad.argtypes = [vp, vp, vp, vp, i, P(d)]
            lib.ptylm_net_pairs.argtypes = [vp, vp, i, vp, i, vp, vp, vp]
            lib.ptylm_net_train.argtypes = [vp, vp, i, i, vp, i, i, d, u64, vp]
            lib.ptylm_learned_inputs.argtypes = [vp, vp, vp, vp, i, vp]
            lib.ptylm_learned_init.argtypes = [vp, vp, vp, vp, i, vp]
            lib.ptylm_net_destroy.argtypes = [vp]
            for name in ("ptylm_net_create", "ptylm_net_set_params", "ptylm_net_get_params", "ptylm_net_forward",
                         "ptylm_net_loss_grad", "ptylm_net_pairs", "ptylm_net_train", "ptylm_learned_inputs",
                         "ptylm_learned_init", "ptylm_net_destroy", "ptylm_net_activation"):
                getattr(lib, name).restype = i
            for name in ("ptylm_batch_init", "ptylm_batch_forward_loss", "ptylm_batch_gradient",
                         "ptylm_batch_ggn_matvec", "ptylm_batch_lm_solve", "ptylm_batch_tune",
                         "ptylm_batch_set_schedule", "ptylm_batch_profile_read", "ptylm_batch_destroy",
                         "ptylm_batch_ggn_diag"):
                getattr(lib, name).restype = i
            for name in ("lm_init", "forward_loss", "gradient", "jvp", "jtvp", "ggn_matvec",
                         "lm_solve", "lm_destroy", "forward_intensity", "ptylm_set_measurements",
                         "ptylm_forward_loss_noalloc", "ggn_diag", "forward_magnitude",
                         "ptylm_profile", "ptylm_profile_select",
                         "ptylm_profile_read"):
                getattr(lib, name).restype = i
            _lib = lib
    return _lib


def ptylm_strerror(status: int) -> str:
    return load_library().ptylm_strerror(int(status)).decode()


def _check(status, allow=()):
    if status != PTYLM_OK and status not in allow:
        lib = load_library()
        raise PtylmError(status, f"{lib.ptylm_strerror(status).decode()}: "
                                 f"{lib.ptylm_last_error().decode()}")
    return status


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported array type {type(x)!r}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Context:
    """Owns one C context (lm_init ... lm_destroy); positions and y are copied by the C side."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc

    def close(self):
        if self.handle:
            lm_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lm_init(ny, nx, my, mx, positions, y, loss=LOSS_GAUSSIAN, background=1e-8, joint=0,
            workspace_budget=0, stream=None, values_per_thread=0) -> Context:
    """positions: device int32 [K, 2]; y: device float32 [K, my, mx] (copied).
    values_per_thread: FFT tile (0 automatic, 32, or 16 for probe sides 32 and 64)."""
    lib = load_library()
    K = 0 if positions is None else int(positions.shape[0])
    desc = Desc(int(ny), int(nx), int(my), int(mx), K, int(loss), float(background), int(joint),
                int(workspace_budget), int(values_per_thread))
    h = ctypes.c_void_p()
    _check(lib.lm_init(ctypes.byref(h), ctypes.byref(desc), _ptr(positions), _ptr(y),
                       _stream_ptr(stream)))
    return Context(h.value, desc)


def lm_destroy(ctx: Context) -> None:
    if ctx.handle:
        _check(load_library().lm_destroy(ctx.handle))
        ctx.handle = None


def forward_loss(ctx: Context, O, P, cache: int = 0):
    """Returns (f, ||grad_zeta l||^2) as Python floats."""
    f, n2 = ctypes.c_double(), ctypes.c_double()
    _check(load_library().forward_loss(ctx.handle, _ptr(O), _ptr(P), ctypes.byref(f),
                                       ctypes.byref(n2), int(cache)))
    return f.value, n2.value


def gradient(ctx: Context, gO, gP=None) -> None:
    _check(load_library().gradient(ctx.handle, _ptr(gO), _ptr(gP)))


def jvp(ctx: Context, vO, out, vP=None) -> None:
    _check(load_library().jvp(ctx.handle, _ptr(vO), _ptr(vP), _ptr(out)))


def jtvp(ctx: Context, w, outO, outP=None) -> None:
    _check(load_library().jtvp(ctx.handle, _ptr(w), _ptr(outO), _ptr(outP)))


def ggn_matvec(ctx: Context, vO, outO, lam: float = 0.0, D=None, vP=None, outP=None) -> None:
    _check(load_library().ggn_matvec(ctx.handle, _ptr(vO), _ptr(vP), ctypes.c_double(lam), _ptr(D),
                                     _ptr(outO), _ptr(outP)))


def ptylm_set_measurements(ctx: Context, y) -> None:
    _check(load_library().ptylm_set_measurements(ctx.handle, _ptr(y)))


def _require_tensor(x, name, dtype, numel=None, min_numel=None, shape=None):
    """Check one argument of the context-free entry point, which has no context holding
    sizes or types: a contiguous torch tensor of `dtype` with the given element count or
    shape (device placement is checked afterwards)."""
    import torch
    if not isinstance(x, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor on the GPU, got {type(x).__name__}")
    if x.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")
    if numel is not None and x.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {x.numel()}")
    if min_numel is not None and x.numel() < min_numel:
        raise ValueError(f"{name} must have at least {min_numel} elements, got {x.numel()}")


def ptylm_forward_loss_noalloc(ny, nx, m, positions, y, O, P, out, loss=LOSS_GAUSSIAN,
                               background=1e-8, stream=None) -> None:
    """Context-free, allocation-free (f, ||grad_zeta l||^2) into device double[2] `out`.

    The library trusts every pointer it is given, so the types, sizes and device of the
    arguments are checked here first (ValueError): O complex64 [ny, nx], P complex64
    [m, m], positions int32 [K, 2], y float32 with K*m*m elements, out float64 with at least
    two elements, all CUDA tensors on the current device."""
    import torch
    ny, nx, m = int(ny), int(nx), int(m)
    _require_tensor(positions, "positions", torch.int32)
    if positions.dim() != 2 or positions.shape[1] != 2:
        raise ValueError(f"positions must have shape [K, 2], got {tuple(positions.shape)}")
    K = int(positions.shape[0])
    _require_tensor(O, "O", torch.complex64, numel=ny * nx)
    _require_tensor(P, "P", torch.complex64, numel=m * m)
    _require_tensor(y, "y", torch.float32, numel=K * m * m)
    _require_tensor(out, "out", torch.float64, min_numel=2)
    args = {"O": O, "P": P, "positions": positions, "y": y, "out": out}
    for name, t in args.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor (host memory is not accepted here)")
    dev = torch.cuda.current_device()
    for name, t in args.items():
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    _check(load_library().ptylm_forward_loss_noalloc(ny, nx, m, K, int(loss), float(background),
                                                     _ptr(O), _ptr(P), _ptr(positions), _ptr(y), _ptr(out),
                                                     _stream_ptr(stream)))


def ptylm_fp32_peak(launches=5, iters=40000, stream=None):
    """(TFLOP/s, ms) of the median timed launch of the library's FFMA loop on the current device."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ptylm_fp32_peak(int(launches), int(iters), ctypes.byref(tf), ctypes.byref(ms),
                                          _stream_ptr(stream)))
    return tf.value, ms.value


def forward_intensity(ctx: Context, O, P, h_out) -> None:
    _check(load_library().forward_intensity(ctx.handle, _ptr(O), _ptr(P), _ptr(h_out)))


KERNEL_FORWARD_LOSS = 0
KERNEL_FORWARD_CACHE = 1
KERNEL_GGN_MATVEC = 2
KERNEL_JTVP = 3
KERNEL_JVP = 4
KERNEL_FORWARD_INTENSITY = 5
KERNEL_FORWARD_CACHE_JOINT = 6
KERNEL_GGN_MATVEC_JOINT = 7
KERNEL_JTVP_JOINT = 8
KERNEL_JVP_JOINT = 9
KERNEL_CG_ITERATION = 15   # the vector work of one CG iteration of lm_solve


def ptylm_profile(ctx: Context, enable: bool) -> None:
    _check(load_library().ptylm_profile(ctx.handle, int(bool(enable))))


def ptylm_profile_select(ctx: Context, kernels) -> None:
    """Time only the launches of the given kernel ids (empty: stop)."""
    mask = 0
    for k in kernels:
        mask |= 1 << int(k)
    _check(load_library().ptylm_profile_select(ctx.handle, mask))


def ptylm_profile_read(ctx: Context, kernel: int):
    """(total device ms, launches) for one kernel id; kernel=-1 -> (0, all launches)."""
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load_library().ptylm_profile_read(ctx.handle, int(kernel), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def forward_magnitude(ctx: Context, O, P, zeta_out, store_phasor: bool = False) -> None:
    _check(load_library().forward_magnitude(ctx.handle, _ptr(O), _ptr(P), _ptr(zeta_out), int(bool(store_phasor))))


def ggn_diag(ctx: Context, D_out, floor_rel: float = 0.0) -> None:
    """Closed-form Dg(G) over z (object, then probe for joint contexts) into D_out."""
    _check(load_library().ggn_diag(ctx.handle, _ptr(D_out), ctypes.c_double(floor_rel)))


def default_lm_params(loss: int) -> LMParams:
    p = LMParams()
    load_library().ptylm_default_lm_params(ctypes.byref(p), int(loss))
    return p


def lm_solve(ctx: Context, O, P, params: LMParams | None = None, hist_len: int = 0,
             O_ref=None, mask=None, state=None, log_path=None, **overrides):
    """Run Algorithm 1 in place on O.  Returns (status, stats dict).  PTYLM_WARN_CG_MAXIT and
    PTYLM_ERR_STALLED (the damping ran away: no step decreases f any more at FP32 resolution)
    are returned rather than raised; O, P and the history then hold the last iterate.
    state: None (fresh start) or a dict {t, mu, delta} (delta a contiguous complex64 tensor or
    array of the state's length, updated in place); the run continues from it through
    lm_solve_resume and the dict is updated to the state after the run (also stats["state"]).
    log_path: append one JSON line per outer iteration (t, f, ||grad f||, mu, lambda, gain
    ratio, CG iterations, accepted, seconds, object error) to this file (needs hist_len)."""
    p = default_lm_params(ctx.desc.loss) if params is None else params
    for k, v in overrides.items():
        setattr(p, k, v)
    if O_ref is not None:
        p.O_ref = _ptr(O_ref)
    if mask is not None:
        p.mask = _ptr(mask)
    L = int(hist_len)
    hf, hg, hmu, herr, hrho, hlam, htime = (np.full(max(L, 1), math.nan) for _ in range(7))
    hcg = np.zeros(max(L, 1), np.int32)
    st = LMStats(0, 0, 0, 0.0, 0.0, L, hf.ctypes.data, hg.ctypes.data, hmu.ctypes.data,
                 hcg.ctypes.data, herr.ctypes.data, hrho.ctypes.data, hlam.ctypes.data, htime.ctypes.data)
    lib = load_library()
    if state is None:
        status = _check(lib.lm_solve(ctx.handle, _ptr(O), _ptr(P), ctypes.byref(p), ctypes.byref(st)),
                        allow=(PTYLM_WARN_CG_MAXIT, PTYLM_ERR_STALLED))
    else:
        cs = LMState(int(state["t"]), float(state["mu"]), _ptr(state.get("delta")))
        status = _check(lib.lm_solve_resume(ctx.handle, _ptr(O), _ptr(P), ctypes.byref(p), ctypes.byref(cs),
                                            ctypes.byref(st)), allow=(PTYLM_WARN_CG_MAXIT, PTYLM_ERR_STALLED))
        state["t"], state["mu"] = cs.t, cs.mu
    n = min(st.n_outer, L)
    out = dict(n_outer=st.n_outer, cg_total=st.cg_total, matvecs=st.matvecs_total,
               f_final=st.f_final, err_final=st.err_final, f=hf[:n].copy(),
               gnorm=hg[:n].copy(), mu=hmu[:n].copy(), cg=hcg[:n].copy(),
               err=herr[:n].copy(), rho=hrho[:n].copy(), lam=hlam[:n].copy(), seconds=htime[:n].copy(),
               state=state)
    if log_path is not None:
        write_lm_log(log_path, out, p)
    return status, out


def write_lm_log(path, info, params) -> None:
    """One JSON line per outer iteration of an lm_solve history (appended to `path`)."""
    import json
    t0 = int(info["state"]["t"]) - int(info["n_outer"]) if info.get("state") else 0
    with open(path, "a") as fh:
        for i in range(len(info["f"])):
            def num(a):
                return float(a[i]) if math.isfinite(float(a[i])) else None
            fh.write(json.dumps({"t": t0 + i, "f": num(info["f"]), "grad_norm": num(info["gnorm"]),
                                 "mu": num(info["mu"]), "lambda": num(info["lam"]), "rho": num(info["rho"]),
                                 "cg": int(info["cg"][i]), "accepted": bool(info["rho"][i] > params.rho_min),
                                 "seconds": num(info["seconds"]), "err": num(info["err"])}) + "\n")


def new_lm_state(ctx: Context, mu0: float | None = None, device=None):
    """A fresh resumable state {t: 0, mu: mu0 (the Sec. 5 default), delta: zeros} for ctx;
    delta is a complex64 CUDA tensor of the state's length."""
    import torch
    L = ctx.desc.ny * ctx.desc.nx + (ctx.desc.my * ctx.desc.mx if ctx.desc.joint else 0)
    mu = default_lm_params(ctx.desc.loss).mu0 if mu0 is None else float(mu0)
    return {"t": 0, "mu": mu, "delta": torch.zeros(L, dtype=torch.complex64, device=device or "cuda")}


def save_lm_checkpoint(path, O, P, state) -> None:
    """Write the iterate (O, P) and the LM state (t, mu, delta) to an .npz file."""
    def host(a):
        return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    np.savez(path, O=host(O), P=host(P), t=int(state["t"]), mu=float(state["mu"]), delta=host(state["delta"]))


def load_lm_checkpoint(path, device="cuda"):
    """(O, P, state) from save_lm_checkpoint's file, as complex64 CUDA tensors."""
    import torch
    d = np.load(path)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(device)
    return t(d["O"]), t(d["P"]), {"t": int(d["t"]), "mu": float(d["mu"]), "delta": t(d["delta"])}


# ---------------------------------------------------------------------------------------
# Batches of independent reconstructions
# ---------------------------------------------------------------------------------------
N_SCHEDULES = 24


def schedule_desc(choice: int) -> dict:
    """What batch schedule `choice` (0 .. N_SCHEDULES - 1) sets: the work-item order
    (0: largest patches first, 1: round robin), the positions each team handles per item,
    and the FFT tile of the 32^2 and 64^2 problems as values per thread (teams of
    S^2 / values threads)."""
    sched, tile = choice % 6, choice // 6
    order, per_team = ((0, 1), (0, 2), (0, 4), (1, 1), (1, 2), (1, 4))[sched]
    return {"order": order, "positions_per_team": per_team,
            "values_per_thread_32": 16 if tile & 1 else 32, "values_per_thread_64": 16 if tile & 2 else 32}


class Batch:
    """Owns one C batch (ptylm_batch_init ... ptylm_batch_destroy)."""

    def __init__(self, handle, descs, offsets):
        self.handle = handle
        self.descs = descs
        self.offsets = offsets          # [B + 1] element offsets of the problems
        self.B = len(descs)

    @property
    def total(self):
        return self.offsets[-1]

    def views(self, vec):
        """Per-problem [ny, nx] views of a flat batch vector (torch tensor)."""
        return [vec[self.offsets[b]:self.offsets[b + 1]].view(d.ny, d.nx) for b, d in enumerate(self.descs)]

    def close(self):
        if self.handle:
            _check(load_library().ptylm_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_init(problems, stream=None) -> Batch:
    """problems: list of dicts with ny, nx, m, positions (device int32 [K, 2]), y (device
    float32 [K, m, m]), probe (device complex64 [m, m]), loss, background."""
    lib = load_library()
    B = len(problems)
    descs = (Desc * B)()
    pos = (ctypes.c_void_p * B)()
    ys = (ctypes.c_void_p * B)()
    probes = (ctypes.c_void_p * B)()
    for b, pr in enumerate(problems):
        K = int(pr["positions"].shape[0])
        descs[b] = Desc(int(pr["ny"]), int(pr["nx"]), int(pr["m"]), int(pr["m"]), K, int(pr.get("loss", 0)),
                        float(pr.get("background", 1e-8)), 0, 0)
        pos[b] = _ptr(pr["positions"])
        ys[b] = _ptr(pr["y"])
        probes[b] = _ptr(pr["probe"])
    h = ctypes.c_void_p()
    _check(lib.ptylm_batch_init(ctypes.byref(h), B, descs, pos, ys, probes, _stream_ptr(stream)))
    offsets = [int(lib.ptylm_batch_offset(h, b)) for b in range(B + 1)]
    return Batch(h, [descs[b] for b in range(B)], offsets)


def batch_forward_loss(batch: Batch, O, cache: int = 0):
    """Returns (f[B], ||grad_zeta l||^2[B]) as numpy arrays."""
    f = np.zeros(batch.B)
    n2 = np.zeros(batch.B)
    _check(load_library().ptylm_batch_forward_loss(
        batch.handle, _ptr(O), f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        n2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(cache)))
    return f, n2


def batch_gradient(batch: Batch, g) -> None:
    _check(load_library().ptylm_batch_gradient(batch.handle, _ptr(g)))


def batch_ggn_matvec(batch: Batch, v, out, lam=None) -> None:
    lp = None
    if lam is not None:
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (batch.B,)))
        lp = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(load_library().ptylm_batch_ggn_matvec(batch.handle, _ptr(v), _ptr(out), lp))


def batch_tune(batch: Batch):
    """Returns (chosen schedule, measured ms per schedule); a schedule whose FFT tile no
    problem of the batch uses is not timed and reads -1."""
    choice = ctypes.c_int(-1)
    ms = (ctypes.c_float * N_SCHEDULES)()
    _check(load_library().ptylm_batch_tune(batch.handle, ctypes.byref(choice), ms, N_SCHEDULES))
    return choice.value, list(ms)


def batch_ggn_diag(batch: Batch, D_out, floor_rel: float = 0.0) -> None:
    """Closed-form GGN diagonal of every problem at the batch's linearisation point into the
    float32 vector D_out (batch layout, total elements)."""
    import torch
    if not isinstance(D_out, torch.Tensor) or D_out.dtype != torch.float32 or D_out.numel() < batch.total:
        raise ValueError("D_out must be a float32 tensor of at least batch.total elements")
    _check(load_library().ptylm_batch_ggn_diag(batch.handle, _ptr(D_out), float(floor_rel)))


def batch_set_schedule(batch: Batch, choice: int) -> None:
    _check(load_library().ptylm_batch_set_schedule(batch.handle, int(choice)))


def batch_launches(batch: Batch) -> int:
    n = ctypes.c_longlong()
    _check(load_library().ptylm_batch_profile_read(batch.handle, ctypes.byref(n)))
    return n.value


def batch_lm_solve(batch: Batch, O, params=None, hist_len: int = 0, O_refs=None, masks=None, **overrides):
    """Algorithm 1 on every problem, in place on the flat batch vector O.  params: one
    LMParams (copied per problem, loss-specific defaults otherwise) or a list of B.  Returns
    (status, [stats dict per problem]); PTYLM_ERR_STALLED and PTYLM_WARN_CG_MAXIT are
    returned, not raised."""
    lib = load_library()
    B = batch.B
    prm = (LMParams * B)()
    for b in range(B):
        if params is None:
            p = default_lm_params(batch.descs[b].loss)
        elif isinstance(params, (list, tuple)):
            p = params[b]
        else:
            p = params
        ctypes.memmove(ctypes.byref(prm[b]), ctypes.byref(p), ctypes.sizeof(LMParams))
        for k, v in overrides.items():
            setattr(prm[b], k, v)
        if O_refs is not None and O_refs[b] is not None:
            prm[b].O_ref = _ptr(O_refs[b])
        if masks is not None and masks[b] is not None:
            prm[b].mask = _ptr(masks[b])
    L = int(hist_len)
    hists = []
    stats = (LMStats * B)()
    for b in range(B):
        hf, hg, hmu, herr = (np.full(max(L, 1), math.nan) for _ in range(4))
        hcg = np.zeros(max(L, 1), np.int32)
        hists.append((hf, hg, hmu, hcg, herr))
        stats[b] = LMStats(0, 0, 0, 0.0, 0.0, L, hf.ctypes.data, hg.ctypes.data, hmu.ctypes.data,
                           hcg.ctypes.data, herr.ctypes.data, None, None, None)
    status = _check(lib.ptylm_batch_lm_solve(batch.handle, _ptr(O), prm, stats),
                    allow=(PTYLM_WARN_CG_MAXIT, PTYLM_ERR_STALLED))
    out = []
    for b in range(B):
        st = stats[b]
        n = min(st.n_outer, L)
        hf, hg, hmu, hcg, herr = hists[b]
        out.append(dict(n_outer=st.n_outer, cg_total=st.cg_total, matvecs=st.matvecs_total, f_final=st.f_final,
                        err_final=st.err_final, f=hf[:n].copy(), gnorm=hg[:n].copy(), mu=hmu[:n].copy(),
                        cg=hcg[:n].copy(), err=herr[:n].copy()))
    return status, out


# ---------------------------------------------------------------------------------------
# Learned initialisation (128 x 128 patterns)
# ---------------------------------------------------------------------------------------
class Net:
    """Owns one C network (ptylm_net_create ... ptylm_net_destroy)."""

    def __init__(self, handle, widths, max_batch, m=128):
        self.handle = handle
        self.widths = tuple(widths)
        self.max_batch = max_batch
        self.m = m

    @property
    def num_params(self):
        return int(load_library().ptylm_net_num_params(self.handle))

    def close(self):
        if self.handle:
            _check(load_library().ptylm_net_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_create(widths=(64, 128, 256), max_batch=64, seed=0, m=128, stream=None) -> Net:
    w = (ctypes.c_int * 3)(*[int(x) for x in widths])
    h = ctypes.c_void_p()
    _check(load_library().ptylm_net_create(ctypes.byref(h), int(m), w, int(max_batch), int(seed), _stream_ptr(stream)))
    return Net(h, widths, max_batch, int(m))


def net_set_params(net: Net, params) -> None:
    p = np.ascontiguousarray(params, np.float32)
    if p.size != net.num_params:
        raise ValueError(f"expected {net.num_params} parameters, got {p.size}")
    _check(load_library().ptylm_net_set_params(net.handle, p.ctypes.data))


def net_get_params(net: Net):
    """(params, grads of the last loss_grad / training step) as float32 numpy arrays."""
    p = np.empty(net.num_params, np.float32)
    g = np.empty(net.num_params, np.float32)
    _check(load_library().ptylm_net_get_params(net.handle, p.ctypes.data, g.ctypes.data))
    return p, g


def net_forward(net: Net, X, out, N=None) -> None:
    N = int(X.shape[0]) if N is None else int(N)
    _check(load_library().ptylm_net_forward(net.handle, _ptr(X), N, _ptr(out)))


def net_activation(net: Net, layer: int, N: int):
    """Output of hidden layer `layer` (1..5) of the first N images of the last forward pass,
    as a float32 CUDA tensor [N, C, H, H]."""
    import torch
    m = net.m
    c1, c2, c3 = net.widths
    C = (c1, c2, c3, c2, c1)[layer - 1]
    H = (m // 2, m // 4, m // 8, m // 4, m // 2)[layer - 1]
    out = torch.empty((N, C, H, H), dtype=torch.float32, device="cuda")
    _check(load_library().ptylm_net_activation(net.handle, int(layer), int(N), _ptr(out)))
    return out


def net_loss_grad(net: Net, X, T, mask, N=None) -> float:
    N = int(X.shape[0]) if N is None else int(N)
    loss = ctypes.c_double()
    _check(load_library().ptylm_net_loss_grad(net.handle, _ptr(X), _ptr(T), _ptr(mask), N, ctypes.byref(loss)))
    return loss.value


def net_pairs(net: Net, pool, side, samples, P, X, T) -> None:
    _check(load_library().ptylm_net_pairs(net.handle, _ptr(pool), int(side), _ptr(samples), int(samples.shape[0]),
                                          _ptr(P), _ptr(X), _ptr(T)))


def net_train(net: Net, pool, n_obj, side, P, steps, batch, lr=1e-3, seed=0):
    """Returns the per-step loss history (numpy)."""
    hist = np.zeros(max(1, int(steps)))
    _check(load_library().ptylm_net_train(net.handle, _ptr(pool), int(n_obj), int(side), _ptr(P), int(steps),
                                          int(batch), float(lr), int(seed), hist.ctypes.data))
    return hist[:int(steps)]


def learned_inputs(ctx: Context, net: Net, P, idx, X) -> None:
    _check(load_library().ptylm_learned_inputs(ctx.handle, net.handle, _ptr(P), _ptr(idx), int(idx.shape[0]), _ptr(X)))


def learned_init(ctx: Context, net: Net, P, idx, O0) -> None:
    _check(load_library().ptylm_learned_init(ctx.handle, net.handle, _ptr(P), _ptr(idx), int(idx.shape[0]), _ptr(O0)))
