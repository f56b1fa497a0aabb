"""Method 1 (table autodiff) vs the proposed Jacobian: the accuracy comparison of Sec. IV-A."""
import numpy as np

from oracle import jacobian as jb
from oracle.naive import TableNufft, naive_vjp_omega
from oracle.nudft import NUDFT
from oracle.nufft import KBNufft
from paper_2111_02912_gb300.workloads import workload


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_table_forward_matches_kb_forward():
    g = np.random.default_rng(30)
    om = g.uniform(-np.pi, np.pi, (2, 200))
    x = g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))
    yk = KBNufft((16, 16), om).forward(x)
    yt, _ = TableNufft((16, 16), om, L=4096).forward_and_jac(x)
    assert _rel(yt, yk) < 1e-6


def test_table_jacobian_is_the_derivative_of_the_piecewise_linear_model():
    """Away from table knots the autodiff slope is the exact derivative of the table model."""
    g = np.random.default_rng(31)
    om = g.uniform(-np.pi, np.pi, (1, 50))
    x = g.standard_normal(16) + 1j * g.standard_normal(16)
    op = TableNufft((16,), om, L=64)
    _, jac = op.forward_and_jac(x)
    h = 1e-9
    yp, _ = TableNufft((16,), om + h, L=64).forward_and_jac(x)
    ym, _ = TableNufft((16,), om - h, L=64).forward_and_jac(x)
    fd = (yp - ym) / (2 * h)
    close = np.abs(fd - jac[0]) <= 1e-4 * np.abs(jac).max()
    assert close.mean() > 0.9


def test_proposed_more_accurate_than_autodiff_on_spoke_case():
    """Sec. IV-A: one radial spoke, 40x40, 8 coils, L = ||E x||^2 (v = 2 E x)."""
    w = workload("spoke40")
    sh, om, x, S = w["shape"], w["omega"], w["x"], w["smaps"]
    ex = NUDFT(sh, om)
    v = 2 * jb.sense_forward(ex, x, S)
    ge, _ = jb.vjp_omega_x(ex, x, v, S)
    gp, _ = jb.vjp_omega_x(KBNufft(sh, om), x, v, S)
    e_prop = _rel(gp, ge)
    assert e_prop < 1e-4
    for L in (64, 512):
        assert _rel(naive_vjp_omega(sh, om, x, v, S, L=L), ge) > 50 * e_prop
    assert _rel(naive_vjp_omega(sh, om, x, v, S, L=512, analytic_derivative=True), ge) > 5 * e_prop
