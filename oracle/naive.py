"""'Method 1' of Sec. IV-A: autodiff through a table-interpolated NUFFT (test infrastructure only).

Sec. II-B and Sec. IV-A describe the baseline the paper compares against: the
NUFFT's interpolator lookup table is read with linear interpolation so that
autodiff can run through it, and the derivatives of the floor / ceiling
operations inside the lookup are taken as zero.  Per dimension the kernel value
at offset u is read from a table of psi sampled at L points per grid unit,
    psi_lin(u) = (1 - a) tab[l] + a tab[l + 1],  |u| L = l + a,  l = floor(|u| L),
so the 2-D weight psi_lin(u_1) psi_lin(u_2) is bilinear in the table.  The
autodiff derivative w.r.t. omega^[d] differentiates only the 'a' term:
    d psi_lin / du = sign(u) L (tab[l + 1] - tab[l]),  du / d omega^[d] = K_d / (2 pi),
with the window offset floor(t) held constant.  A second variant uses the
analytic psi' in place of the table difference.  Neither is ever used as truth;
they reproduce the accuracy comparison of Sec. IV-A.
"""
import math

import numpy as np

from .nufft import KBNufft, kb_kernel, kb_kernel_deriv


class TableNufft(KBNufft):
    """KBNufft whose interpolation weights come from a linearly interpolated table."""

    def __init__(self, shape, omega, L=512, analytic_derivative=False, **kw):
        super().__init__(shape, omega, **kw)
        self.L = int(L)
        self.analytic = bool(analytic_derivative)
        nt = self.L * self.J // 2
        self.table = kb_kernel(np.arange(nt + 2) / self.L, self.J, self.beta)
        self.table[nt:] = 0.0          # psi(J/2) = 0 (open support)
        self.dtaps = []
        new_taps = []
        for d in range(self.D):
            idx, _, u = self.taps[d]
            au = np.abs(u) * self.L
            l = np.floor(au).astype(np.int64)
            a = au - l
            l = np.minimum(l, nt)
            w = (1 - a) * self.table[l] + a * self.table[l + 1]
            if self.analytic:
                dw = kb_kernel_deriv(u, self.J, self.beta)
            else:
                dw = np.sign(u) * self.L * (self.table[l + 1] - self.table[l])
            new_taps.append((idx, w, u))
            self.dtaps.append(dw * self.K[d] / (2.0 * math.pi))
        self.taps = new_taps

    def forward_and_jac(self, x):
        """y = A_lin x and the autodiff diagonals dy/d omega^[d]; shapes (M,), (D, M)."""
        x = np.asarray(x, dtype=np.complex128)
        xs = self._scale_image(x)
        grid = np.zeros(self.K, dtype=np.complex128)
        grid[np.ix_(*self.place)] = xs
        G = np.fft.fftn(grid)
        M = self.omega.shape[1]
        y = np.zeros(M, dtype=np.complex128)
        jac = np.zeros((self.D, M), dtype=np.complex128)
        for js in np.ndindex(*([self.J] * self.D)):
            idx = tuple(self.taps[d][0][:, js[d]] for d in range(self.D))
            g = G[idx]
            ws = [self.taps[d][1][:, js[d]] for d in range(self.D)]
            y += np.prod(ws, axis=0) * g
            for d in range(self.D):
                prod = self.dtaps[d][:, js[d]].copy()
                for e in range(self.D):
                    if e != d:
                        prod = prod * ws[e]
                jac[d] += prod * g
        return y, jac


def naive_vjp_omega(shape, omega, x, v, smaps=None, L=512, analytic_derivative=False, **kw):
    """grad_omega (D, M) by method 1: sum_c Re{conj(v_c) . d y_c / d omega}."""
    op = TableNufft(shape, omega, L=L, analytic_derivative=analytic_derivative, **kw)
    x = np.asarray(x, dtype=np.complex128)
    xc = x[None] if smaps is None and x.ndim == len(shape) else (
        x if smaps is None else np.asarray(smaps, dtype=np.complex128) * x[None])
    v = np.asarray(v, dtype=np.complex128)
    out = np.zeros(op.omega.shape)
    for c in range(xc.shape[0]):
        _, jac = op.forward_and_jac(xc[c])
        out += np.real(np.conj(v[c])[None] * jac)
    return out
