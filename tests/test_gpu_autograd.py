"""torch.autograd layer over the C ABI: gradients against the FP64 oracle (Sec. II-C..F)."""
import numpy as np
import pytest

from gpu_helpers import host, make_case, rel, to_dev
from oracle import jacobian as jb
from oracle.nufft import KBNufft

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup(shape=(24, 20), M=800, C=3, seed=51):
    import torch

    from paper_2111_02912_gb300.autograd import NufftOperator
    case = make_case(shape, M, C, True, seed=seed)
    om = to_dev(case["omega"]).requires_grad_(True)
    op = NufftOperator(shape, om, smaps=to_dev(case["smaps"]))
    return case, om, op, KBNufft(shape, case["omega"]), torch


def test_forward_function_gradients():
    from paper_2111_02912_gb300.autograd import nufft
    case, om, op, ref, torch = _setup()
    x = to_dev(case["x"]).requires_grad_(True)
    y = nufft(x, om, op)
    y.backward(to_dev(case["v"]))
    go, gx = jb.vjp_omega_x(ref, case["x"], case["v"], case["smaps"])
    assert rel(host(y), jb.sense_forward(ref, case["x"], case["smaps"])) < TOL
    assert rel(host(om.grad), go) < TOL and rel(host(x.grad), gx) < TOL


def test_adjoint_function_gradients():
    from paper_2111_02912_gb300.autograd import nufft_adjoint
    case, om, op, ref, torch = _setup(seed=52)
    y = to_dev(case["y"]).requires_grad_(True)
    g = np.random.default_rng(3).standard_normal(case["shape"]) + 1j * np.random.default_rng(4).standard_normal(case["shape"])
    x = nufft_adjoint(y, om, op)
    x.backward(to_dev(g.astype(np.complex64)))
    assert rel(host(x), jb.sense_adjoint(ref, case["y"], case["smaps"])) < TOL
    assert rel(host(y.grad), jb.sense_forward(ref, g, case["smaps"])) < TOL                    # d(E'y)/dy = E'
    assert rel(host(om.grad), jb.adjoint_vjp_omega(ref, g, case["y"], case["smaps"])) < TOL    # Eq. (e,A'y)


def test_gram_function_gradients():
    from paper_2111_02912_gb300.autograd import gram
    case, om, op, ref, torch = _setup(seed=53)
    lam = 0.7
    x = to_dev(case["x"]).requires_grad_(True)
    g = (np.random.default_rng(5).standard_normal(case["shape"]) * (1 + 1j)).astype(np.complex64)
    z = gram(x, om, op, lam)
    z.backward(to_dev(g))
    S = case["smaps"]
    gram_ref = lambda v: jb.sense_adjoint(ref, jb.sense_forward(ref, v, S), S) + lam * v
    assert rel(host(z), gram_ref(case["x"])) < TOL
    assert rel(host(x.grad), gram_ref(g.astype(np.complex128))) < TOL
    assert rel(host(om.grad), jb.gram_vjp_omega(ref, case["x"], g, S)) < TOL            # Eq. (e,A'A,x,omd)


def test_psd_inverse_function_gradients():
    from paper_2111_02912_gb300.autograd import psd_inverse
    shape, M, C = (12, 10), 400, 2
    case, om, op, ref, torch = _setup(shape, M, C, seed=54)
    S = case["smaps"]
    N = int(np.prod(shape))
    I = np.eye(N).reshape((N,) + shape)
    E = np.concatenate([np.stack([ref.forward(S[c] * I[n]) for n in range(N)], axis=1) for c in range(C)])
    lam = 0.05 * np.linalg.norm(E, 2) ** 2          # well conditioned: CG converges in a few dozen steps
    b = to_dev(case["x"]).requires_grad_(True)
    g = (np.random.default_rng(6).standard_normal(shape) * (1 - 1j)).astype(np.complex64)
    z = psd_inverse(b, om, op, lam, 60)
    z.backward(to_dev(g))
    z_ref, gb_ref, go_ref = jb.psd_inverse_vjp(ref, E, case["x"], g, S, lam)
    assert rel(host(z), z_ref) < 1e-4
    assert rel(host(b.grad), gb_ref) < 1e-4
    assert rel(host(om.grad), go_ref) < 1e-4                                             # Eq. (e,inv,omd)


def test_unrolled_cg_recompute_matches_stored_and_converges_to_implicit_gradient():
    from paper_2111_02912_gb300.autograd import cg_sense_unrolled, nufft, psd_inverse
    case, om, op, ref, torch = _setup((16, 16), 600, 2, seed=55)
    S = case["smaps"]
    x_true = to_dev(case["x"])
    y = nufft(x_true, om, op).detach()
    lam = 2.0
    grads = []
    for recompute in (True, False):
        om.grad = None
        xk = cg_sense_unrolled(y, om, op, lam, 8, recompute=recompute)
        loss = torch.sum(torch.abs(xk - x_true) ** 2)
        loss.backward()
        grads.append(host(om.grad).copy())
    assert rel(grads[0], grads[1]) < 1e-5
    # many iterations: the unrolled gradient approaches the implicit one of Eq. (e,inv,omd)
    om.grad = None
    xk = cg_sense_unrolled(y, om, op, lam, 40, recompute=True)
    torch.sum(torch.abs(xk - x_true) ** 2).backward()
    g_unrolled = host(om.grad).copy()
    from paper_2111_02912_gb300.autograd import nufft_adjoint
    om.grad = None
    z = psd_inverse(nufft_adjoint(y, om, op), om, op, lam, 60)
    torch.sum(torch.abs(z - x_true) ** 2).backward()
    assert rel(g_unrolled, host(om.grad)) < 2e-3
