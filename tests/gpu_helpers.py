"""Shared helpers of the GPU parity tests (seeded inputs; the oracle is the judge)."""
import numpy as np

from paper_2111_02912_gb300.workloads import gaussian_bump_maps, random_image, random_omega, rng


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_case(shape, M, C, maps, seed, omega=None):
    g = rng(100 + seed)
    D = len(shape)
    om = random_omega(g, D, M) if omega is None else omega
    S = gaussian_bump_maps(shape, C) if maps else None
    x = random_image(g, shape) if maps else np.stack([random_image(g, shape) for _ in range(C)])
    v = (g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))).astype(np.complex64)
    y = (g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))).astype(np.complex64)
    dom = g.standard_normal((D, M)).astype(np.float32)
    return dict(shape=tuple(shape), omega=om, x=x, smaps=S, v=v, y=y, domega=dom, C=C)


def to_dev(a):
    import torch
    if a is None:
        return None
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return None if t is None else t.detach().cpu().numpy()


def max_rel(a, b):
    """Largest element error over the largest reference magnitude (catches a few wrong cells)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
