"""Plain PyTorch FP32 (complex64, CPU) reference of the model's operators.

Used only to measure the rounding error that any FP32 FFT-based evaluation of these
operators has on a given input, so that parity tolerances for ill-conditioned inputs (the
Poisson metric at dark pixels with counts, where the weights 2y/zeta^2 amplify the FFT's
absolute rounding error) are derived from FP32 arithmetic rather than guessed.  It follows
the same equations as the oracle (Sec. 2 Eqs. exit_wave / expected_count, Sec. 4.1
Eq. ell_magnitude, App. A steps 2-4) with torch.fft in single precision.
"""
import numpy as np
import torch


def _index(pos, m):
    pos = torch.as_tensor(np.asarray(pos), dtype=torch.long)
    ar = torch.arange(m)
    r = pos[:, 0, None, None] + ar[None, :, None]
    c = pos[:, 1, None, None] + ar[None, None, :]
    return r.expand(-1, m, m), c.expand(-1, m, m)


def _c64(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.complex64))


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32))


class Ref32:
    def __init__(self, case):
        self.m = case.m
        self.n = case.n
        self.P = _c64(case.P)
        self.y = _f32(case.y)
        self.b = float(case.b)
        self.loss = case.loss
        self.r, self.c = _index(case.pos, case.m)

    def _fft(self, A):
        return torch.fft.fft2(self.P * _c64(A)[self.r, self.c], norm="ortho")

    def _scatter(self, chi):
        out = torch.zeros((self.n, self.n), dtype=torch.complex64)
        out.index_put_((self.r, self.c), torch.conj(self.P) * chi, accumulate=True)
        return out

    def _terms(self, ps):
        h = ps.real ** 2 + ps.imag ** 2 + self.b
        z = torch.sqrt(h)
        y = self.y
        if self.loss == 0:
            d = z - torch.sqrt(y)
            return h, z, 0.5 * d * d, d, torch.ones_like(z)
        l = h - torch.where(y > 0, y * torch.log(h), torch.zeros_like(h))
        return h, z, l, 2 * z - 2 * y / z, 2 + 2 * y / h

    def loss_and_dl2(self, O):
        _, _, l, dl, _ = self._terms(self._fft(O))
        return float(l.double().sum()), float((dl.double() ** 2).sum())

    def gradient(self, O):
        ps = self._fft(O)
        _, z, _, dl, _ = self._terms(ps)
        return self._scatter(torch.fft.ifft2(ps * (dl / z), norm="ortho")).numpy()

    def ggn_matvec(self, O, v, lam=0.0):
        ps = self._fft(O)
        _, z, _, _, d2 = self._terms(ps)
        a = ps * (torch.sqrt(d2) / z)
        dps = self._fft(v)
        t = a.real * dps.real + a.imag * dps.imag
        return (self._scatter(torch.fft.ifft2(a * t, norm="ortho")) + lam * _c64(v)).numpy()

    def jvp(self, O, v):
        ps = self._fft(O)
        _, z, _, _, _ = self._terms(ps)
        dps = self._fft(v)
        return ((ps.real * dps.real + ps.imag * dps.imag) / z).numpy()

    def jtvp(self, O, w):
        ps = self._fft(O)
        _, z, _, _, _ = self._terms(ps)
        return self._scatter(torch.fft.ifft2(ps * (_f32(w) / z), norm="ortho")).numpy()
