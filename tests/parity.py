"""Parity bookkeeping shared by the GPU tests.

Every comparison of the CUDA path with the FP64 oracle goes through `check`, which
computes the error it reached, records it next to its bound, and asserts.  Two norms:

  rel2   ||gpu - ref||_2 / ||ref||_2           (whole-vector relative error)
  max    max |gpu - ref| / max |ref|            (element-wise: a wrong value at a few border
                                                 or dark pixels cannot hide under bright ones)

At the end of the session conftest.py writes the records as JSON lines to the file named by
the environment variable PTYLM_PARITY_LOG (if set); tests/parity_table.py turns such a log
into the table of achieved errors kept in the design notes.
"""
from __future__ import annotations

import os

import numpy as np

TOL = 1e-5          # the relative bound of the hot path in FP32
RECORDS: list[dict] = []


def rel2(a, b) -> float:
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 0:
        return float(abs(a - b) / max(abs(b), 1e-300))
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def max_rel(a, b) -> float:
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


NORMS = {"rel2": rel2, "max": max_rel}


def _test_id() -> str:
    tid = os.environ.get("PYTEST_CURRENT_TEST", "?")
    return tid.rsplit(" ", 1)[0]


def record(quantity: str, err: float, tol: float, norm: str = "rel2", basis: str = "1e-5", **extra) -> float:
    RECORDS.append(dict(test=_test_id(), quantity=quantity, norm=norm, err=float(err), tol=float(tol),
                        basis=basis, **{k: (float(v) if isinstance(v, (float, np.floating)) else v)
                                        for k, v in extra.items()}))
    return err


def check(quantity: str, gpu, ref, tol: float = TOL, norm: str = "rel2", basis: str = "1e-5", **extra) -> float:
    """Error of `gpu` against `ref` in `norm`; recorded, then asserted <= tol."""
    err = NORMS[norm](gpu, ref)
    record(quantity, err, tol, norm, basis, **extra)
    assert err <= tol, f"{quantity}: {norm} error {err:.3e} > {tol:.3e} ({basis})"
    return err


def check_against_fp32(quantity: str, gpu, ref, fp32_evals, factor: float = 2.0, norm: str = "rel2") -> float:
    """The CUDA path's error against the oracle is no worse than `factor` times the worst
    error of independent single-precision evaluations of the same quantity (fp32_evals, each
    an array computed in FP32 with no code shared with the CUDA path), or 1e-5.  Where an
    input makes every single-precision evaluation miss 1e-5, this shows the miss comes from
    the arithmetic, not from the kernel."""
    err = NORMS[norm](gpu, ref)
    e32 = max(NORMS[norm](f, ref) for f in fp32_evals)
    tol = max(TOL, factor * e32)
    record(quantity, err, tol, norm, basis=f"{factor:g} x independent FP32 evaluation", fp32_err=e32)
    assert err <= tol, f"{quantity}: {norm} error {err:.3e} > {factor:g} x FP32 evaluation error {e32:.3e}"
    return err


# Detector pixels whose expected intensity |psihat|^2 is at least LIT_REL times the largest
# one are "lit".  At darker pixels the unit phasor psihat / zeta that J v = Re(conj(psihat /
# zeta) dpsihat) projects onto is set by the FFT's absolute rounding error, so single
# precision cannot resolve J v there element by element (any FP32 evaluation misses 1e-5 of
# max |J v| at some of them, also at the noiseless truth); on lit pixels it can.
LIT_REL = 1e-5


def check_detector(quantity: str, gpu, ref, intensity, fp32_evals=None) -> float:
    """An output per detector pixel (J v): element-wise 1e-5 of max |ref| on the lit pixels of
    `intensity` (|psihat|^2, same shape); over all pixels element-wise no worse than twice the
    worst independent FP32 evaluation (when given)."""
    gpu, ref, intensity = np.asarray(gpu), np.asarray(ref), np.asarray(intensity)
    lit = intensity >= LIT_REL * intensity.max()
    err = float(np.max(np.abs(gpu - ref)[lit]) / max(float(np.max(np.abs(ref))), 1e-300))
    record(quantity, err, TOL, "max (lit pixels)", lit_fraction=float(lit.mean()))
    assert err <= TOL, f"{quantity}: element-wise error on lit pixels {err:.3e} > {TOL:.3e}"
    if fp32_evals is not None:
        check_against_fp32(quantity, gpu, ref, fp32_evals, norm="max")
    return err


def write_log(path: str) -> None:
    import json
    with open(path, "a") as fh:
        for r in RECORDS:
            fh.write(json.dumps(r) + "\n")
