"""Exact NUDFT and its analytic Jacobians in FP64 (test infrastructure only).

System model of Sec. II-B, Eq. (e,ndft): for sample locations omega_i in R^D
(radians per voxel) and voxel centres r_j on a Cartesian grid,

    [A(omega)]_ij = exp(-i omega_i . r_j),   y = A x.

Voxel centres: r_j^[d] = n_d - N_d // 2 for n_d = 0 .. N_d - 1 (integer voxel
units, so A is 2*pi-periodic in every omega^[d]).

The products are evaluated with separable phasors: exp(-i omega_i . r_j) is
the product over d of exp(-i omega_i^[d] r_j^[d]), so y_i is a chain of small
contractions instead of an M x N matrix.  That is a reordering of the same
sum, nothing more.

Array conventions: an image x has shape (N_1, ..., N_D) (C order, last axis
fastest); omega has shape (D, M), one row per coordinate omega^[d].
"""
import numpy as np

_CHUNK = 2048  # sample points per contraction block (bounds host memory)


def voxel_centres(shape):
    """Return [r^[1], ..., r^[D]], r^[d]_n = n - N_d // 2 (Sec. II-B)."""
    return [np.arange(n, dtype=np.float64) - (n // 2) for n in shape]


def _as_omega(omega, D):
    om = np.asarray(omega, dtype=np.float64)
    if om.ndim != 2 or om.shape[0] != D:
        raise ValueError("omega must have shape (D, M) with D = image dims")
    return om


def _trailing_outer(phasors):
    """Row-wise Kronecker product of the per-dim phasor blocks for d >= 2.

    phasors: list of (m, N_d) arrays; returns (m, N_2 * ... * N_D)."""
    m = phasors[0].shape[0]
    P = np.ones((m, 1), dtype=np.complex128)
    for E in phasors[1:]:
        P = (P[:, :, None] * E[:, None, :]).reshape(m, -1)
    return P


def nudft_forward(x, omega):
    """y_i = sum_j x_j exp(-i omega_i . r_j)  (Eq. (e,ndft)).  Returns (M,)."""
    x = np.asarray(x, dtype=np.complex128)
    D = x.ndim
    om = _as_omega(omega, D)
    r = voxel_centres(x.shape)
    M = om.shape[1]
    X = x.reshape(x.shape[0], -1)
    y = np.empty(M, dtype=np.complex128)
    for s in range(0, M, _CHUNK):
        sl = slice(s, min(s + _CHUNK, M))
        E = [np.exp(-1j * np.outer(om[d, sl], r[d])) for d in range(D)]
        T = E[0] @ X                              # sum over n_1
        y[sl] = np.sum(T * _trailing_outer(E), axis=1)  # sum over n_2..n_D
    return y


def nudft_adjoint(y, omega, shape):
    """x_j = sum_i y_i exp(+i omega_i . r_j): the conjugate transpose A' y."""
    y = np.asarray(y, dtype=np.complex128)
    D = len(shape)
    om = _as_omega(omega, D)
    r = voxel_centres(shape)
    M = om.shape[1]
    X = np.zeros((shape[0], int(np.prod(shape[1:], dtype=np.int64))), dtype=np.complex128)
    for s in range(0, M, _CHUNK):
        sl = slice(s, min(s + _CHUNK, M))
        E = [np.exp(+1j * np.outer(om[d, sl], r[d])) for d in range(D)]
        X += E[0].T @ (y[sl, None] * _trailing_outer(E))
    return X.reshape(shape)


def nudft_jac_omega(x, omega):
    """Diagonals of d(Ax)/d omega^[d], d = 1..D  (Sec. II-C).

    Differentiating y_i = sum_j x_j exp(-i omega_i . r_j) term by term w.r.t.
    omega_i^[d] gives sum_j x_j (-i r_j^[d]) exp(-i omega_i . r_j); the
    off-diagonal entries (i != l) vanish.  Returns a (D, M) complex array."""
    x = np.asarray(x, dtype=np.complex128)
    D = x.ndim
    r = voxel_centres(x.shape)
    out = []
    for d in range(D):
        shape = [1] * D
        shape[d] = x.shape[d]
        out.append(nudft_forward(x * (-1j) * r[d].reshape(shape), omega))
    return np.stack(out)


def nudft_matrix(shape, omega):
    """Dense A(omega) built entry by entry (brute force, tiny sizes only)."""
    D = len(shape)
    om = _as_omega(omega, D)
    r = voxel_centres(shape)
    grids = np.meshgrid(*r, indexing="ij")
    R = np.stack([g.ravel() for g in grids])          # (D, N)
    M, N = om.shape[1], R.shape[1]
    A = np.empty((M, N), dtype=np.complex128)
    for i in range(M):
        for j in range(N):
            phase = 0.0
            for d in range(D):
                phase += om[d, i] * R[d, j]
            A[i, j] = np.cos(phase) - 1j * np.sin(phase)
    return A


class NUDFT:
    """Operator pair (forward, adjoint) of the exact NUDFT for one image shape."""

    def __init__(self, shape, omega):
        self.shape = tuple(int(n) for n in shape)
        self.omega = _as_omega(omega, len(self.shape))

    def forward(self, x):
        return nudft_forward(x, self.omega)

    def adjoint(self, y):
        return nudft_adjoint(y, self.omega, self.shape)
