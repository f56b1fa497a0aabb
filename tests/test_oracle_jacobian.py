"""Pins of the Jacobian products (Eq. (e,Ax), (e,A'y), (e,jac,Ax,v), Sec. II-G) by finite differences."""
import numpy as np
import pytest

from oracle import jacobian as jb
from oracle.nudft import NUDFT
from oracle.nufft import KBNufft
from paper_2111_02912_gb300.workloads import gaussian_bump_maps


def _case(shape=(6, 8), M=9, C=3, seed=20):
    g = np.random.default_rng(seed)
    om = g.uniform(-np.pi, np.pi, (len(shape), M))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    S = gaussian_bump_maps(shape, C).astype(np.complex128)
    v = g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))
    return g, om, x, S, v


def _loss(om, x, S, v, shape):
    """L = Re(v' E(omega) x): its gradient w.r.t. (Re y, Im y) is v."""
    return np.real(np.vdot(v, jb.sense_forward(NUDFT(shape, om), x, S)))


def test_vjp_omega_matches_finite_differences():
    shape = (6, 8)
    g, om, x, S, v = _case(shape)
    grad, _ = jb.vjp_omega_x(NUDFT(shape, om), x, v, S)
    h = 1e-6
    for d in range(2):
        for i in range(om.shape[1]):
            e = np.zeros_like(om)
            e[d, i] = h
            fd = (_loss(om + e, x, S, v, shape) - _loss(om - e, x, S, v, shape)) / (2 * h)
            assert abs(fd - grad[d, i]) <= 1e-7 * max(1.0, np.abs(grad).max())


def test_vjp_x_matches_finite_differences():
    shape = (4, 6)
    g, om, x, S, v = _case(shape, M=7)
    _, gx = jb.vjp_omega_x(NUDFT(shape, om), x, v, S)
    h = 1e-6
    for j in np.ndindex(*shape):
        e = np.zeros(shape, complex)
        e[j] = h
        dre = (_loss(om, x + e, S, v, shape) - _loss(om, x - e, S, v, shape)) / (2 * h)
        dim = (_loss(om, x + 1j * e, S, v, shape) - _loss(om, x - 1j * e, S, v, shape)) / (2 * h)
        assert abs((dre + 1j * dim) - gx[j]) < 1e-7 * np.abs(gx).max()


def test_jvp_omega_matches_finite_differences():
    shape = (6, 8)
    g, om, x, S, _ = _case(shape)
    dom = g.standard_normal(om.shape)
    dy = jb.jvp_omega(NUDFT(shape, om), x, dom, S)
    h = 1e-6
    fd = (jb.sense_forward(NUDFT(shape, om + h * dom), x, S)
          - jb.sense_forward(NUDFT(shape, om - h * dom), x, S)) / (2 * h)
    assert np.allclose(dy, fd, atol=1e-7 * np.abs(dy).max())


def test_adjoint_vjp_equals_forward_vjp_with_roles_swapped():
    """d/d omega Re<g, E' y> (Eq. (e,A'y)) equals vjp_omega_x(x=g, v=y), and matches FD."""
    shape = (6, 8)
    g, om, x, S, v = _case(shape)
    gimg = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    a = jb.adjoint_vjp_omega(NUDFT(shape, om), gimg, v, S)
    b, _ = jb.vjp_omega_x(NUDFT(shape, om), gimg, v, S)
    assert np.allclose(a, b, atol=1e-10 * np.abs(b).max())
    h = 1e-6

    def f(o):
        return np.real(np.vdot(gimg, jb.sense_adjoint(NUDFT(shape, o), v, S)))
    for d in range(2):
        for i in range(om.shape[1]):
            e = np.zeros_like(om)
            e[d, i] = h
            assert abs((f(om + e) - f(om - e)) / (2 * h) - a[d, i]) < 1e-7 * np.abs(a).max()


def test_no_map_channels_are_independent():
    shape = (6, 8)
    g, om, x, S, v = _case(shape)
    xc = S * x[None]
    op = NUDFT(shape, om)
    assert np.allclose(jb.sense_forward(op, xc, None), jb.sense_forward(op, x, S))
    gs, _ = jb.vjp_omega_x(op, x, v, S)
    gn, _ = jb.vjp_omega_x(op, xc, v, None)
    assert np.allclose(gs, gn)


@pytest.mark.parametrize("shape", [(16, 20), (8, 8, 10)])
def test_nufft_jacobians_close_to_exact(shape):
    g = np.random.default_rng(21)
    M, C = 300, 2
    om = g.uniform(-np.pi, np.pi, (len(shape), M))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    S = gaussian_bump_maps(shape, C).astype(np.complex128)
    v = g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))
    ge, gxe = jb.vjp_omega_x(NUDFT(shape, om), x, v, S)
    gn, gxn = jb.vjp_omega_x(KBNufft(shape, om), x, v, S)
    assert np.linalg.norm(gn - ge) / np.linalg.norm(ge) < 1e-4
    assert np.linalg.norm(gxn - gxe) / np.linalg.norm(gxe) < 1e-4


def test_gram_vjp_matches_finite_differences():
    """Eq. (e,A'A,x,omd) contracted with g equals d/d omega Re<g, E'E x> (SENSE, exact NUDFT)."""
    shape = (6, 8)
    g, om, x, S, _ = _case(shape, M=7, C=2)
    gimg = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    a = jb.gram_vjp_omega(NUDFT(shape, om), x, gimg, S)

    def f(o):
        op = NUDFT(shape, o)
        return np.real(np.vdot(gimg, jb.sense_adjoint(op, jb.sense_forward(op, x, S), S)))
    h = 1e-6
    for d in range(2):
        for i in range(om.shape[1]):
            e = np.zeros_like(om)
            e[d, i] = h
            assert abs((f(om + e) - f(om - e)) / (2 * h) - a[d, i]) < 1e-7 * np.abs(a).max()


def test_psd_inverse_vjp_matches_finite_differences():
    """Eq. (e,inv,omd): gradients of Re<g, (E'E + lam I)^-1 b> w.r.t. omega and b (dense solves)."""
    from oracle.nudft import nudft_matrix
    shape, lam = (4, 6), 0.3
    g, om, x, S, _ = _case(shape, M=9, C=2)
    b = x
    gimg = g.standard_normal(shape) + 1j * g.standard_normal(shape)

    def solve(o):
        E = jb.dense_sense_matrix(nudft_matrix(shape, o), S)
        F = E.conj().T @ E + lam * np.eye(E.shape[1])
        return np.linalg.solve(F, b.ravel()).reshape(shape)

    E = jb.dense_sense_matrix(nudft_matrix(shape, om), S)
    z, gb, go = jb.psd_inverse_vjp(NUDFT(shape, om), E, b, gimg, S, lam)
    assert np.allclose(z, solve(om), atol=1e-12)
    h = 1e-6
    for d in range(2):
        for i in range(om.shape[1]):
            e = np.zeros_like(om)
            e[d, i] = h
            fd = (np.real(np.vdot(gimg, solve(om + e))) - np.real(np.vdot(gimg, solve(om - e)))) / (2 * h)
            assert abs(fd - go[d, i]) < 1e-6 * max(1.0, np.abs(go).max())
    # grad_b: L = Re<g, F^-1 b> is linear in b with gradient F^-1 g (F Hermitian)
    for j in [(0, 0), (2, 3)]:
        e = np.zeros(shape, complex)
        e[j] = h
        F = E.conj().T @ E + lam * np.eye(E.shape[1])
        f = lambda bb: np.real(np.vdot(gimg, np.linalg.solve(F, bb.ravel())))
        dre = (f(b + e) - f(b - e)) / (2 * h)
        dim = (f(b + 1j * e) - f(b - 1j * e)) / (2 * h)
        assert abs((dre + 1j * dim) - gb[j]) < 1e-7 * np.abs(gb).max()
