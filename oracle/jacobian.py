"""Multi-coil operators and Jacobian-vector products (test infrastructure only).

Generic over an operator object ``op`` exposing ``shape``, ``omega`` (D, M),
``forward(x)`` and ``adjoint(y)`` (single coil, leading channel axes allowed):
the exact ``nudft.NUDFT`` or the same-kernel ``nufft.KBNufft``.

Sensitivity model (Sec. II-G): E = (I_Nc kron A) S with S_c = diag(s_c), so
[E x]_c = A (s_c . x) and E' y = sum_c conj(s_c) . A' y_c.  Without maps
(smaps is None) each channel carries its own image: y_c = A x_c.

Jacobians:
  * d(Ax)/d omega^[d] = -i diag{A (x . r^[d])}            (Sec. II-C, Eq. (e,Ax))
  * with maps, A(s_c . x . r^[d]) per coil                  (Sec. II-G)
  * VJP for a real loss L with v = dL/dRe(y) + i dL/dIm(y): grad_omega^[d] =
    sum_c Re{ conj(v_c) . (-i) A(s_c . x . r^[d]) }         (Sec. III, Eq. (e,jac,Ax,v))
    and grad_x = E' v (the Jacobian w.r.t. x is E itself, Sec. II-C).
    Eq. (e,jac,Ax,v) is written with v = dL/d(Ax)^*; the convention here is
    twice that, which removes the factor 2 of the real-valued chain rule.
  * JVP for a perturbation delta omega: dy_c = sum_d delta omega^[d] . (-i) A(s_c . x . r^[d]).
"""
import numpy as np

from .nudft import voxel_centres


def _r_weight(shape, d):
    r = voxel_centres(shape)[d]
    sh = [1] * len(shape)
    sh[d] = shape[d]
    return r.reshape(sh)


def _coil_images(x, smaps):
    x = np.asarray(x, dtype=np.complex128)
    if smaps is None:
        return x
    return np.asarray(smaps, dtype=np.complex128) * x[None]


def sense_forward(op, x, smaps=None):
    """y = E x, shape (C, M)."""
    xc = _coil_images(x, smaps)
    if xc.ndim == len(op.shape):
        xc = xc[None]
    return np.stack([op.forward(xc[c]) for c in range(xc.shape[0])])


def sense_adjoint(op, y, smaps=None):
    """x = E' y.  With maps: sum_c conj(s_c) A' y_c, shape (N...); without: (C, N...)."""
    y = np.asarray(y, dtype=np.complex128)
    xc = np.stack([op.adjoint(y[c]) for c in range(y.shape[0])])
    if smaps is None:
        return xc
    return np.sum(np.conj(np.asarray(smaps, dtype=np.complex128)) * xc, axis=0)


def omega_channels(op, x, smaps=None):
    """g[c, d] = A(s_c . x . r^[d]), the D extra NUFFT channels of Eq. (e,Ax); shape (C, D, M)."""
    xc = _coil_images(x, smaps)
    if xc.ndim == len(op.shape):
        xc = xc[None]
    D = len(op.shape)
    return np.stack([np.stack([op.forward(xc[c] * _r_weight(op.shape, d)) for d in range(D)])
                     for c in range(xc.shape[0])])


def vjp_omega_x(op, x, v, smaps=None):
    """(grad_omega (D, M), grad_x) for incoming gradient v (C, M), Eq. (e,jac,Ax,v)."""
    g = omega_channels(op, x, smaps)
    v = np.asarray(v, dtype=np.complex128)
    grad_omega = np.sum(np.real(np.conj(v)[:, None, :] * (-1j) * g), axis=0)
    grad_x = sense_adjoint(op, v, smaps)
    return grad_omega, grad_x


def jvp_omega(op, x, domega, smaps=None):
    """dy (C, M) = sum_d domega^[d] . (-i) A(s_c . x . r^[d])  (Eq. (e,Ax))."""
    g = omega_channels(op, x, smaps)
    dom = np.asarray(domega, dtype=np.float64)
    return np.sum(dom[None] * (-1j) * g, axis=1)


def adjoint_vjp_omega(op, g, y, smaps=None):
    """d/d omega of Re<g, E'(omega) y> for the adjoint output x^ = E' y (Eq. (e,A'y)).

    Eq. (e,A'y): [d(A'y)/d omega^[d]]_jl = i r_j^[d] exp(+i omega_l . r_j) y_l.
    Contracting with an incoming image gradient g (same convention as v):
      grad[d, l] = sum_c Re{ sum_j conj(g_j) conj(s_cj) i r_j^[d] exp(+i omega_l . r_j) y_cl }
                 = sum_c Re{ i y_cl conj([A(s_c . g . r^[d])]_l) }.
    Without maps g has one image per channel.  Returns (D, M)."""
    y = np.asarray(y, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    D = len(op.shape)
    out = np.zeros((D, op.omega.shape[1]))
    for c in range(y.shape[0]):
        gc = g[c] if smaps is None else g * np.asarray(smaps, dtype=np.complex128)[c]
        for d in range(D):
            t = np.conj(op.forward(gc * _r_weight(op.shape, d)))   # sum_j conj(w_j) e^{+i omega.r_j}
            out[d] += np.real(1j * y[c] * t)
    return out


def gram_vjp_omega(op, x, g, smaps=None):
    """d/d omega of Re<g, E' E x>, from the Gram Jacobian of Sec. II-E, Eq. (e,A'A,x,omd).

    [dE'E/d omega_1 ... dE'E/d omega_M] x = -i E' diag{E(x . r^[d])} + i diag{r^[d]} E' diag{E x}
    (A -> E by Sec. II-G).  Column (c, l) of E' diag{w} contracted with g^H is
    conj([E g]_cl) w_cl, and of diag{r} E' diag{w} is conj([E(g . r)]_cl) w_cl;
    omega_l enters every coil's column l, so coils are summed.  Returns (D, M)."""
    D = len(op.shape)
    Ex = sense_forward(op, x, smaps)
    Eg = sense_forward(op, g, smaps)
    out = np.zeros((D, op.omega.shape[1]))
    for d in range(D):
        rw = _r_weight(op.shape, d)
        Exr = sense_forward(op, np.asarray(x) * rw, smaps)
        Egr = sense_forward(op, np.asarray(g) * rw, smaps)
        term = -1j * np.conj(Eg) * Exr + 1j * np.conj(Egr) * Ex
        out[d] = np.sum(np.real(term), axis=0)
    return out


def dense_sense_matrix(op_matrix, smaps):
    """Stack [A diag(s_1); ...; A diag(s_C)] for a dense single-coil A (tiny sizes)."""
    S = np.asarray(smaps, dtype=np.complex128).reshape(len(smaps), -1)
    return np.concatenate([op_matrix * S[c][None, :] for c in range(S.shape[0])], axis=0)


def psd_inverse_vjp(op, E_dense, b, g, smaps=None, lam=1e-2):
    """z = F^-1 b, F = E'E + lam I, and the VJPs of Re<g, z> (Sec. II-F, Eq. (e,inv,omd)).

    Eq. (e,inv,omd): D_omega F^-1 b = -F^-1 (D_omega F z), z = F^-1 b, so with
    u = F^-1 g (F Hermitian): grad_b = u and grad_omega = -gram_vjp(x = z, g = u).
    F is solved densely here (tiny sizes).  Returns (z, grad_b, grad_omega)."""
    shape = op.shape
    N = int(np.prod(shape))
    F = E_dense.conj().T @ E_dense + lam * np.eye(N)
    z = np.linalg.solve(F, np.asarray(b, dtype=np.complex128).ravel()).reshape(shape)
    u = np.linalg.solve(F, np.asarray(g, dtype=np.complex128).ravel()).reshape(shape)
    return z, u, -gram_vjp_omega(op, z, u, smaps)
