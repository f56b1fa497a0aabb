"""Pins of the exact NUDFT oracle against brute force, hand closed forms and the FFT."""
import json
import math
import os

import numpy as np
import pytest

from oracle.nudft import nudft_adjoint, nudft_forward, nudft_jac_omega, nudft_matrix, voxel_centres

HERE = os.path.dirname(__file__)


def _c(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("shape", [(7,), (4, 6), (2, 4, 6)])
def test_forward_adjoint_match_brute_force_matrix(shape):
    g = np.random.default_rng(1)
    D, M = len(shape), 11
    om = g.uniform(-4, 4, (D, M))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    y = g.standard_normal(M) + 1j * g.standard_normal(M)
    A = nudft_matrix(shape, om)
    assert np.allclose(nudft_forward(x, om), A @ x.ravel(), rtol=0, atol=1e-12)
    assert np.allclose(nudft_adjoint(y, om, shape).ravel(), A.conj().T @ y, rtol=0, atol=1e-12)


def test_hand_closed_forms():
    gold = json.load(open(os.path.join(HERE, "golden", "nudft_hand.json")))
    for key in ("one_d", "two_d"):
        case = gold[key]
        shape = tuple(case["shape"])
        x = _c(case["x"])
        om = np.array(case["omega"])
        assert np.allclose(nudft_forward(x, om), _c(case["y"]), atol=1e-14)
        assert np.allclose(nudft_jac_omega(x, om), _c(case["jac"]), atol=1e-14)
    c1 = gold["one_d"]
    om = np.array(c1["omega"])
    xa = nudft_adjoint(np.ones(om.shape[1]), om, (2,))
    assert np.allclose(xa, _c(c1["adjoint_of_ones"]), atol=1e-14)


@pytest.mark.parametrize("shape", [(16,), (8, 12), (4, 6, 8)])
def test_cartesian_sampling_is_a_phase_modulated_fft(shape):
    """omega^[d] = 2 pi k / N_d on the full grid: y_k = (-1)^{sum k} fftn(x)[k mod N]."""
    g = np.random.default_rng(2)
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    ks = [np.arange(-n // 2, n // 2) for n in shape]
    K = np.meshgrid(*ks, indexing="ij")
    om = np.stack([2 * np.pi * K[d].ravel() / shape[d] for d in range(len(shape))])
    y = nudft_forward(x, om)
    F = np.fft.fftn(x)
    idx = tuple(np.mod(K[d].ravel(), shape[d]) for d in range(len(shape)))
    sign = (-1.0) ** np.sum([K[d].ravel() for d in range(len(shape))], axis=0)
    assert np.allclose(y, sign * F[idx], atol=1e-10 * np.abs(F).max())
    N = x.size
    assert math.isclose(np.vdot(y, y).real, N * np.vdot(x, x).real, rel_tol=1e-12)  # Parseval
    assert np.allclose(nudft_adjoint(y, om, shape), N * x, atol=1e-9)                # A'A = N I


def test_single_voxel():
    g = np.random.default_rng(3)
    shape = (6, 10)
    x = np.zeros(shape, complex)
    x[1, 7] = 1.0
    r0 = np.array([1 - 3, 7 - 5], float)
    om = g.uniform(-np.pi, np.pi, (2, 9))
    y = nudft_forward(x, om)
    assert np.allclose(y, np.exp(-1j * (r0 @ om)), atol=1e-14)
    jac = nudft_jac_omega(x, om)
    assert np.allclose(jac, -1j * r0[:, None] * y[None], atol=1e-13)


def test_jacobian_matches_central_differences():
    g = np.random.default_rng(4)
    shape = (6, 8)
    om = g.uniform(-np.pi, np.pi, (2, 5))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    jac = nudft_jac_omega(x, om)
    h = 1e-6
    for d in range(2):
        e = np.zeros_like(om)
        e[d] = h
        fd = (nudft_forward(x, om + e) - nudft_forward(x, om - e)) / (2 * h)
        assert np.allclose(jac[d], fd, rtol=1e-7, atol=1e-7 * np.abs(jac).max())


def test_periodic_in_omega():
    g = np.random.default_rng(5)
    shape = (8, 6)
    om = g.uniform(-np.pi, np.pi, (2, 7))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    shift = np.array([[2 * np.pi], [-4 * np.pi]])
    assert np.allclose(nudft_forward(x, om + shift), nudft_forward(x, om), atol=1e-11)


def test_adjoint_identity():
    g = np.random.default_rng(6)
    shape = (10, 12)
    om = g.uniform(-np.pi, np.pi, (2, 300))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    y = g.standard_normal(300) + 1j * g.standard_normal(300)
    lhs = np.vdot(y, nudft_forward(x, om))
    rhs = np.vdot(nudft_adjoint(y, om, shape), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_voxel_centres_half_fov():
    r = voxel_centres((8, 6))
    assert r[0][0] == -4 and r[0][-1] == 3 and r[1][0] == -3 and np.max(np.abs(r[0])) == 4
