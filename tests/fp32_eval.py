"""An independent single-precision evaluation of the model and its derivatives, for the
parity tests only.

It restates Sec. 2 (Eqs. exit_wave, expected_count), Sec. 4.1 (Eqs. magnitude,
ell_magnitude) and App. A / App. B (Eq. jac_ampl) in numpy/scipy complex64 arithmetic:
the patches, the orthonormal 2D FFTs (scipy.fft keeps single precision), the per-pixel
metric terms and the overlap scatter-add are all FP32; only the error metric's final sum is
FP64, as on the CUDA path.  It shares no code with the CUDA kernels or with the FP64 oracle.
Its use: where an input makes the FP64 oracle's answer sensitive at the level of FP32
rounding, the CUDA path's error is compared with the worst error of four roundings of this
evaluation (two FFT implementations -- scipy's pocketfft and a radix-2 transform written
here -- each taking the two axes in either order), all measured against the oracle.

Conventions as in the library: positions (row, col) of each patch's top-left corner,
real-coordinate gradients (d/dRe + i d/dIm), y in natural DFT order.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

F32 = np.float32
C64 = np.complex64


def _radix2(x, inverse):
    """Radix-2 decimation-in-time DFT over the last axis (a power of two) in complex64, the
    twiddles exp(-+2 pi i k / n) computed in FP64 and rounded once; orthonormal."""
    n = x.shape[-1]
    if n == 1:
        return x
    even, odd = _radix2(x[..., 0::2], inverse), _radix2(x[..., 1::2], inverse)
    sign = 1.0 if inverse else -1.0
    w = np.exp(sign * 2j * np.pi * np.arange(n // 2) / n).astype(C64)
    t = w * odd
    out = np.concatenate([even + t, even - t], axis=-1) * F32(1.0 / np.sqrt(2.0))
    return out.astype(C64)


def _fft2(x, order, inverse=False):
    """Four single-precision roundings of the orthonormal 2D DFT: scipy's (pocketfft) 2D
    transform (order 0), scipy's 1D transforms columns first (1), the radix-2 transform rows
    first (2) and columns first (3)."""
    if order == 0:
        out = (sfft.ifft2 if inverse else sfft.fft2)(x, axes=(-2, -1), norm="ortho")
    elif order == 1:
        f = sfft.ifft if inverse else sfft.fft
        out = f(f(x, axis=-2, norm="ortho"), axis=-1, norm="ortho")
    elif order == 2:
        out = np.swapaxes(_radix2(np.swapaxes(_radix2(x, inverse), -1, -2), inverse), -1, -2)
    else:
        out = _radix2(np.swapaxes(_radix2(np.swapaxes(x, -1, -2), inverse), -1, -2), inverse)
    out = np.ascontiguousarray(out)
    assert out.dtype == C64
    return out


def _ifft2(x, order):
    return _fft2(x, order, inverse=True)


ORDERS = (0, 1, 2, 3)


class Fp32Model:
    def __init__(self, shape, P, pos, y, loss, b):
        self.ny, self.nx = shape
        self.P = np.asarray(P, C64)
        self.m = self.P.shape[0]
        self.pos = np.asarray(pos, np.int64)
        self.y = np.asarray(y, F32)
        self.loss = int(loss)
        self.b = F32(b)

    def patches(self, A):
        A = np.asarray(A, C64)
        m = self.m
        return np.stack([A[r:r + m, c:c + m] for r, c in self.pos]) if len(self.pos) else np.zeros((0, m, m), C64)

    def scatter(self, chi):
        out = np.zeros((self.ny, self.nx), C64)
        m = self.m
        for k, (r, c) in enumerate(self.pos):
            out[r:r + m, c:c + m] += chi[k]
        return out

    def far_field(self, O, order):
        return _fft2(self.P[None] * self.patches(O), order)

    def terms(self, psihat):
        """h, zeta, dl and d2l per pixel (FP32)."""
        h = (psihat.real * psihat.real + psihat.imag * psihat.imag + self.b).astype(F32)
        zeta = np.sqrt(h)
        y = self.y
        if self.loss == 0:
            dl = zeta - np.sqrt(y)
            d2l = np.ones_like(zeta)
        else:
            dl = F32(2) * zeta - F32(2) * y / zeta
            d2l = F32(2) + F32(2) * y / h
        return h, zeta, dl, d2l

    def loss_value(self, O, order=0):
        h, zeta, dl, _ = self.terms(self.far_field(O, order))
        y = self.y
        if self.loss == 0:
            d = zeta - np.sqrt(y)
            l = F32(0.5) * d * d
        else:
            ylog = np.where(y > 0, y * np.log(h), F32(0))
            l = h - ylog
        return float(np.sum(l, dtype=np.float64)), float(np.sum(dl.astype(np.float64) ** 2))

    def jtvp(self, O, w, order=0):
        psihat = self.far_field(O, order)
        _, zeta, _, _ = self.terms(psihat)
        chi = _ifft2(psihat * (np.asarray(w, F32) / zeta), order)
        return self.scatter(np.conj(self.P)[None] * chi)

    def gradient(self, O, order=0):
        psihat = self.far_field(O, order)
        _, zeta, dl, _ = self.terms(psihat)
        chi = _ifft2(psihat * (dl / zeta), order)
        return self.scatter(np.conj(self.P)[None] * chi)

    def jvp(self, O, v, order=0):
        psihat = self.far_field(O, order)
        _, zeta, _, _ = self.terms(psihat)
        dpsihat = _fft2(self.P[None] * self.patches(v), order)
        return ((np.conj(psihat) * dpsihat).real / zeta).astype(F32)

    def ggn_matvec(self, O, v, lam=0.0, order=0):
        psihat = self.far_field(O, order)
        _, zeta, _, d2l = self.terms(psihat)
        u = psihat / zeta
        t = (np.conj(u) * _fft2(self.P[None] * self.patches(v), order)).real.astype(F32) * d2l
        chi = _ifft2(u * t, order)
        return self.scatter(np.conj(self.P)[None] * chi) + F32(lam) * np.asarray(v, C64)


def evaluations(model: Fp32Model, method: str, *args, **kw):
    """The quantity under the four FFT roundings of _fft2 (independent FP32 evaluations)."""
    return [getattr(model, method)(*args, order=o, **kw) for o in ORDERS]
