"""Same-kernel NUFFT in FP64, step by step as in the Appendix (test infrastructure only).

The Appendix writes the NUFFT entries as
    a~_mn = sum_{j=1..J} u_j^*(omega_m) s_n exp(-i gamma (k_m + j) n),  gamma = 2 pi / K,
i.e. three steps: (1) scale the signal by s_n, (2) take a K-point FFT of the
zero-padded, scaled signal (K >= N), (3) interpolate the K uniform frequencies
onto the M sample locations with J-tap coefficients u_j at offsets k_m.

Readings where the paper is silent (each is listed with the design notes):
  * Interpolator: Kaiser-Bessel, psi(u) = I0(beta sqrt(1 - (2u/J)^2)) for
    |u| < J/2 and 0 otherwise (open support), with Beatty et al.'s
    beta = pi sqrt((J/sigma)^2 (sigma - 1/2)^2 - 0.8).
  * Scaling: s_n = prod_d 1 / psi_hat(r_n^[d] / K_d), psi_hat the continuous
    Fourier transform of psi in closed form.
  * Placement: voxel n_d (centre r = n_d - N_d//2) goes to grid index
    r mod K_d; sample t = omega K / (2 pi) uses the J integers k with
    |t - k| < J/2, i.e. k = floor(t - J/2) + 1 .. floor(t - J/2) + J
    (for even J: floor(t) - J/2 + 1 .. floor(t) + J/2), grid index k mod K.
  * Grid size: K_d = the smallest even integer >= sigma N_d whose only prime
    factors are 2, 3 and 5.
  * The FFT is unnormalised with exp(-i ...); the adjoint is the exact
    conjugate transpose of the three steps (spread, K * ifft, crop, scale).

D-dimensional arrays: image (N_1..N_D), grid (K_1..K_D), omega (D, M).
An optional leading channel axis is carried through every step.
"""
import math

import numpy as np
from scipy.special import i0

from .nudft import voxel_centres


def kb_beta(J, sigma):
    """Beatty et al.'s Kaiser-Bessel shape parameter for width J, oversampling sigma."""
    return math.pi * math.sqrt((J / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def kb_kernel(u, J, beta):
    """psi(u) = I0(beta sqrt(1 - (2u/J)^2)) on |u| < J/2, zero elsewhere."""
    u = np.asarray(u, dtype=np.float64)
    z = 1.0 - (2.0 * u / J) ** 2
    inside = np.abs(u) < J / 2.0
    return np.where(inside, i0(beta * np.sqrt(np.where(inside, z, 0.0))), 0.0)


def kb_kernel_deriv(u, J, beta):
    """d psi / du on |u| < J/2 (analytic; I0' = I1), zero elsewhere."""
    from scipy.special import i1
    u = np.asarray(u, dtype=np.float64)
    inside = np.abs(u) < J / 2.0
    z = np.where(inside, 1.0 - (2.0 * u / J) ** 2, 1.0)
    s = np.sqrt(z)
    dz = -8.0 * u / (J * J)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(s > 0, i1(beta * s) * beta * dz / (2.0 * s), 0.0)
    return np.where(inside, d, 0.0)


def kb_fourier(f, J, beta):
    """Continuous Fourier transform of psi: int psi(u) exp(-2 pi i f u) du.

    Closed form J sinh(sqrt(a)) / sqrt(a) with a = beta^2 - (pi J f)^2
    (J sin(sqrt(-a)) / sqrt(-a) when a < 0)."""
    f = np.asarray(f, dtype=np.float64)
    a = beta ** 2 - (math.pi * J * f) ** 2
    out = np.empty_like(a)
    pos, neg = a > 0, a < 0
    sa = np.sqrt(np.abs(a))
    out[pos] = J * np.sinh(sa[pos]) / sa[pos]
    out[neg] = J * np.sin(sa[neg]) / sa[neg]
    out[~(pos | neg)] = J
    return out


def grid_size(N, sigma):
    """Smallest even 2,3,5-smooth integer >= sigma * N."""
    K = int(math.ceil(sigma * N - 1e-9))
    while True:
        if K % 2 == 0:
            q = K
            for p in (2, 3, 5):
                while q % p == 0:
                    q //= p
            if q == 1:
                return K
        K += 1


class KBNufft:
    """FP64 NUFFT with a Kaiser-Bessel interpolator (Appendix, three steps)."""

    def __init__(self, shape, omega, J=6, sigma=2.0, beta=None, K=None):
        self.shape = tuple(int(n) for n in shape)
        self.D = len(self.shape)
        self.J = int(J)
        self.sigma = float(sigma)
        self.beta = kb_beta(self.J, self.sigma) if beta is None else float(beta)
        self.K = tuple(grid_size(n, self.sigma) for n in self.shape) if K is None else tuple(K)
        self.omega = np.asarray(omega, dtype=np.float64)
        assert self.omega.shape[0] == self.D
        r = voxel_centres(self.shape)
        # step (1): scaling factors s_n, one factor per dimension
        self.scale = [1.0 / kb_fourier(r[d] / self.K[d], self.J, self.beta) for d in range(self.D)]
        # grid index of each voxel centre: r mod K
        self.place = [np.mod(r[d].astype(np.int64), self.K[d]) for d in range(self.D)]
        # step (3) geometry: t = omega K / (2 pi), window k = floor(t - J/2) + 1 + (0 .. J-1)
        self.taps = []
        for d in range(self.D):
            t = self.omega[d] * self.K[d] / (2.0 * math.pi)
            k = (np.floor(t - self.J / 2.0) + 1.0)[:, None] + np.arange(self.J)[None, :]
            u = t[:, None] - k                         # offsets, in (-J/2, J/2]
            self.taps.append((np.mod(k.astype(np.int64), self.K[d]), kb_kernel(u, self.J, self.beta), u))

    # -- helpers -----------------------------------------------------------
    def _scale_image(self, x):
        s = np.ones(self.shape)
        for d in range(self.D):
            sh = [1] * self.D
            sh[d] = self.shape[d]
            s = s * self.scale[d].reshape(sh)
        return x * s

    def _tap_iter(self):
        """Yield (grid index tuple, weight) for every one of the J^D taps."""
        for js in np.ndindex(*([self.J] * self.D)):
            idx = tuple(self.taps[d][0][:, js[d]] for d in range(self.D))
            w = np.ones(self.omega.shape[1])
            for d in range(self.D):
                w = w * self.taps[d][1][:, js[d]]
            yield idx, w

    # -- operators ---------------------------------------------------------
    def forward(self, x):
        """y = interp(FFT_K(pad(s . x))).  x: (..., N_1..N_D) -> (..., M)."""
        x = np.asarray(x, dtype=np.complex128)
        lead = x.shape[: x.ndim - self.D]
        xs = self._scale_image(x)
        grid = np.zeros(lead + self.K, dtype=np.complex128)
        grid[(Ellipsis,) + np.ix_(*self.place)] = xs
        G = np.fft.fftn(grid, axes=tuple(range(len(lead), len(lead) + self.D)))
        y = np.zeros(lead + (self.omega.shape[1],), dtype=np.complex128)
        for idx, w in self._tap_iter():
            y += w * G[(Ellipsis,) + idx]
        return y

    def adjoint(self, y):
        """x = s . crop(K * IFFT_K(spread(y))): the conjugate transpose of forward."""
        y = np.asarray(y, dtype=np.complex128)
        lead = y.shape[:-1]
        Ktot = int(np.prod(self.K))
        flat_lead = int(np.prod(lead, dtype=np.int64))
        yl = y.reshape(flat_lead, -1)
        G = np.zeros((flat_lead, Ktot), dtype=np.complex128)
        for idx, w in self._tap_iter():
            lin = np.ravel_multi_index(idx, self.K)
            for c in range(flat_lead):
                v = w * yl[c]
                G[c] += np.bincount(lin, weights=v.real, minlength=Ktot) \
                    + 1j * np.bincount(lin, weights=v.imag, minlength=Ktot)
        G = G.reshape(lead + self.K)
        g = np.fft.ifftn(G, axes=tuple(range(len(lead), len(lead) + self.D))) * Ktot
        x = g[(Ellipsis,) + np.ix_(*self.place)]
        return self._scale_image(x)
