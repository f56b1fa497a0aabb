"""Pins of the FP64 same-kernel NUFFT oracle (Appendix) against quadrature, the exact NUDFT and its error bound."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import roots_legendre

from oracle.nudft import NUDFT, nudft_adjoint, nudft_forward, voxel_centres
from oracle.nufft import KBNufft, grid_size, kb_beta, kb_fourier, kb_kernel, kb_kernel_deriv

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("J,sigma", [(6, 2.0), (5, 1.25), (4, 2.0)])
def test_kernel_transform_closed_form_vs_quadrature(J, sigma):
    beta = kb_beta(J, sigma)
    xg, wg = roots_legendre(200)
    u = xg * J / 2.0
    for f in np.linspace(0, 0.5 * (1 - 1 / (2 * sigma)) + 0.1, 9):
        quad = np.sum(wg * kb_kernel(u, J, beta) * np.cos(2 * np.pi * f * u)) * J / 2.0
        assert math.isclose(kb_fourier(np.array([f]), J, beta)[0], quad, rel_tol=1e-12)


def test_kernel_shape():
    J, beta = 6, kb_beta(6, 2.0)
    assert kb_kernel(np.array([3.0, -3.0, 3.5]), J, beta).tolist() == [0.0, 0.0, 0.0]  # open support
    u = np.linspace(-2.9, 2.9, 41)
    k = kb_kernel(u, J, beta)
    assert np.allclose(k, k[::-1]) and np.argmax(k) == 20                              # even, peak at 0


def test_beta_matches_hand_evaluated_values():
    """Beatty's beta at the paper's settings (Sec. IV-C), evaluated by hand in the golden file."""
    gold = json.load(open(os.path.join(GOLDEN, "kb_beta_hand.json")))
    for c in gold["cases"]:
        assert math.isclose(kb_beta(c["J"], c["sigma"]), c["beta"], rel_tol=1e-9)


@pytest.mark.parametrize("J,sigma", [(6, 2.0), (5, 1.25), (8, 2.0)])
def test_kernel_derivative_matches_central_differences(J, sigma):
    """d psi / du (used by the analytic-derivative autodiff variant of Sec. IV-A) against central
    differences of psi itself, inside the support and away from its edges; odd symmetry; zero outside."""
    beta = kb_beta(J, sigma)
    u = np.linspace(-0.49 * J, 0.49 * J, 97)
    h = 1e-5
    fd = (kb_kernel(u + h, J, beta) - kb_kernel(u - h, J, beta)) / (2 * h)
    d = kb_kernel_deriv(u, J, beta)
    scale = np.max(np.abs(d))
    assert np.max(np.abs(d - fd)) < 1e-7 * scale
    assert np.allclose(d, -d[::-1], rtol=0, atol=1e-12 * scale)
    assert kb_kernel_deriv(np.array([0.0]), J, beta)[0] == 0.0
    assert kb_kernel_deriv(np.array([J / 2.0, -J / 2.0, J]), J, beta).tolist() == [0.0, 0.0, 0.0]


def test_grid_size_rule():
    assert [grid_size(n, 2.0) for n in (64, 320, 96, 128)] == [128, 640, 192, 256]
    assert [grid_size(n, 1.25) for n in (64, 320, 40)] == [80, 400, 50]
    assert grid_size(7, 2.0) == 16  # 14 = 2*7 is not 5-smooth


@pytest.mark.parametrize("shape,M", [((32,), 500), ((16, 24), 700), ((8, 10, 12), 400)])
def test_nufft_close_to_exact_nudft(shape, M):
    g = np.random.default_rng(7)
    om = g.uniform(-np.pi, np.pi, (len(shape), M))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    op = KBNufft(shape, om)
    ye = nudft_forward(x, om)
    err = np.linalg.norm(op.forward(x) - ye) / np.linalg.norm(ye)
    assert err < 5e-5
    y = g.standard_normal(M) + 1j * g.standard_normal(M)
    xe = nudft_adjoint(y, om, shape)
    assert np.linalg.norm(op.adjoint(y) - xe) / np.linalg.norm(xe) < 5e-5


def test_low_accuracy_setting_is_less_accurate():
    """Sec. IV-C: grid 1.25x with J=5 trades accuracy for speed."""
    g = np.random.default_rng(8)
    shape, M = (32, 32), 900
    om = g.uniform(-np.pi, np.pi, (2, M))
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    ye = nudft_forward(x, om)
    hi = np.linalg.norm(KBNufft(shape, om).forward(x) - ye)
    lo = np.linalg.norm(KBNufft(shape, om, J=5, sigma=1.25).forward(x) - ye)
    assert lo > 3 * hi and lo / np.linalg.norm(ye) < 1e-2


def test_nufft_adjoint_identity():
    g = np.random.default_rng(9)
    shape, M = (12, 20), 333
    om = g.uniform(-7, 7, (2, M))
    op = KBNufft(shape, om)
    x = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    y = g.standard_normal(M) + 1j * g.standard_normal(M)
    lhs = np.vdot(y, op.forward(x))
    assert abs(lhs - np.vdot(op.adjoint(y), x)) <= 1e-12 * abs(lhs)


def test_nufft_dense_matrix_matches_appendix_entry_formula():
    """a~_mn = sum_j u_j(omega_m) s_n exp(-i gamma (k_m + j) n): build it entry by entry (1-D)."""
    g = np.random.default_rng(10)
    N, M, J = 6, 5, 6
    om = g.uniform(-np.pi, np.pi, (1, M))
    op = KBNufft((N,), om, J=J)
    K, beta = op.K[0], op.beta
    r = voxel_centres((N,))[0]
    s = 1.0 / kb_fourier(r / K, J, beta)
    A = np.zeros((M, N), complex)
    for m in range(M):
        t = om[0, m] * K / (2 * np.pi)
        km = math.floor(t - J / 2)
        for n in range(N):
            for j in range(1, J + 1):
                u = t - (km + j)
                A[m, n] += kb_kernel(np.array([u]), J, beta)[0] * s[n] * np.exp(-1j * 2 * np.pi / K * (km + j) * r[n])
    X = np.eye(N)
    dense = np.stack([op.forward(X[:, n]) for n in range(N)], axis=1)
    assert np.allclose(dense, A, atol=1e-12 * np.abs(A).max())


def test_jvp_error_within_appendix_bound():
    """E1 <= eps_p ||r||_inf with eps_p = max_m ||row_m(A~ - A)||_2 (the l2 -> l_inf norm)."""
    g = np.random.default_rng(11)
    N, M = 24, 200
    om = g.uniform(-np.pi, np.pi, (1, M))
    op = KBNufft((N,), om)
    I = np.eye(N)
    E = np.stack([op.forward(I[:, n]) - nudft_forward(I[:, n], om) for n in range(N)], axis=1)
    eps_p = np.max(np.linalg.norm(E, axis=1))
    r = voxel_centres((N,))[0]
    for _ in range(20):
        x = g.standard_normal(N) + 1j * g.standard_normal(N)
        E1 = np.max(np.abs(op.forward(x * r) - nudft_forward(x * r, om))) / np.linalg.norm(x)
        assert E1 <= eps_p * np.max(np.abs(r)) * (1 + 1e-9)


def test_nufft_is_exact_on_a_single_frequency_sample_at_origin():
    """omega = 0: y = sum_n x_n for the NUDFT; the NUFFT agrees to its error level."""
    g = np.random.default_rng(12)
    x = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
    op = KBNufft((16, 16), np.zeros((2, 1)))
    assert abs(op.forward(x)[0] - x.sum()) < 1e-5 * abs(x).sum()


@pytest.mark.parametrize("J,bound", [(5, 2e-4), (7, 5e-6), (3, 5e-2)])
def test_odd_width_window_covers_the_whole_support(J, bound):
    """Odd J: the window must hold every integer k with |t - k| < J/2 (a dropped tap shows as a large error)."""
    g = np.random.default_rng(13)
    om = g.uniform(-np.pi, np.pi, (2, 800))
    x = g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))
    ye = nudft_forward(x, om)
    op = KBNufft((32, 32), om, J=J)
    assert np.linalg.norm(op.forward(x) - ye) / np.linalg.norm(ye) < bound
    t = om[0] * op.K[0] / (2 * np.pi)
    k = np.floor(t - J / 2) + 1
    assert np.all(np.abs(t - k) < J / 2) and np.all(np.abs(t - (k - 1)) >= J / 2)
    assert np.all(np.abs(t - (k + J - 1)) < J / 2) and np.all(np.abs(t - (k + J)) >= J / 2)
