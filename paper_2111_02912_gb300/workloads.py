"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds geometry and random numbers only (no NUFFT arithmetic); the
CUDA path and the oracle both draw their inputs from it.  Every generator
returns numpy arrays: images complex64 (N_1..N_D), maps complex64 (C, N...),
sample locations float32 (D, M) in radians per voxel.

The paper trains on fastMRI brain data and tests on one radial spoke
(Sec. IV-A, IV-B); neither the data nor its coil maps are available, so these
stand in: i.i.d. Gaussian or random-ellipsoid images, smooth Gaussian-bump
coil maps, golden-angle 2-D radial and perturbed 3-D radial trajectories.
"""
import math

import numpy as np

SEED = 2111_02912
GOLDEN_ANGLE_DEG = 111.246117975  # 180 / golden ratio, the 2-D golden-angle increment


def rng(index):
    return np.random.default_rng(SEED + int(index))


def random_image(g, shape):
    """Real and imaginary parts i.i.d. N(0, 1)."""
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


def random_omega(g, D, M):
    """omega i.i.d. uniform on [-pi, pi)^D."""
    return g.uniform(-math.pi, math.pi, size=(D, M)).astype(np.float32)


def radial_2d(n_spokes, n_read, golden=True, g=None):
    """Spokes through the k-space centre: omega = pi (2m/n_read - 1) (cos th, sin th)."""
    if golden:
        th = np.deg2rad(GOLDEN_ANGLE_DEG) * np.arange(n_spokes)
    else:
        th = g.uniform(0, math.pi, n_spokes)
    kr = math.pi * (2.0 * np.arange(n_read) / n_read - 1.0)
    om = np.stack([np.outer(np.cos(th), kr).ravel(), np.outer(np.sin(th), kr).ravel()])
    return om.astype(np.float32)


def fibonacci_directions(n):
    """Near-uniform unit vectors on the sphere (golden-section spiral)."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z])


def radial_3d(g, n_spokes, n_read, walk_sigma=2e-3 * math.pi):
    """3-D radial readouts with a per-sample random-walk perturbation, wrapped to [-pi, pi)."""
    dirs = fibonacci_directions(n_spokes)                        # (3, S)
    kr = math.pi * (2.0 * np.arange(n_read) / n_read - 1.0)       # (R,)
    om = dirs[:, :, None] * kr[None, None, :]                     # (3, S, R)
    walk = np.cumsum(g.normal(0.0, walk_sigma, size=om.shape), axis=2)
    om = om + walk
    om = np.mod(om + math.pi, 2.0 * math.pi) - math.pi
    return om.reshape(3, -1).astype(np.float32)


def gaussian_bump_maps(shape, C, width=0.35, radius=0.4):
    """s_c(r) = exp(-|r - c_c|^2 / (2 (width N)^2)) exp(i 2 pi c / C), centres at radius*N."""
    D = len(shape)
    Nref = float(max(shape))
    grids = np.meshgrid(*[np.arange(n) - n // 2 for n in shape], indexing="ij")
    if D == 2:
        ang = 2 * math.pi * np.arange(C) / C
        centres = radius * Nref * np.stack([np.cos(ang), np.sin(ang)])
    elif D == 3:
        centres = radius * Nref * fibonacci_directions(C)
    else:
        centres = radius * Nref * np.where(np.arange(C) % 2 == 0, 1.0, -1.0)[None]
    out = np.empty((C,) + tuple(shape), dtype=np.complex64)
    for c in range(C):
        d2 = sum((grids[d] - centres[d, c]) ** 2 for d in range(D))
        out[c] = np.exp(-d2 / (2 * (width * Nref) ** 2)) * np.exp(2j * math.pi * c / C)
    return out


def ellipsoid_phantom(g, shape, n_ellipsoids=12, noise=0.01):
    """Sum of random ellipsoids (random centres, axes, intensities) plus complex N(0, noise) noise."""
    D = len(shape)
    grids = np.meshgrid(*[(np.arange(n) - n // 2) / (n / 2) for n in shape], indexing="ij")
    img = np.zeros(shape, dtype=np.float64)
    for _ in range(n_ellipsoids):
        c = g.uniform(-0.5, 0.5, D)
        a = g.uniform(0.1, 0.5, D)
        v = g.uniform(0.1, 1.0)
        inside = sum(((grids[d] - c[d]) / a[d]) ** 2 for d in range(D)) <= 1.0
        img[inside] += v
    sd = math.sqrt(noise)
    img = img + sd * g.standard_normal(shape) + 1j * sd * g.standard_normal(shape)
    return img.astype(np.complex64)


# ---- named workloads ---------------------------------------------------------

def workload(name, scale=1.0):
    """Return dict(shape, x, smaps (or None), omega, C) for a named workload.

    small64   : 64x64 i.i.d. image, 1 coil, M=4096 uniform omega (2-D)
    radial320 : 320x320 image, 16 Gaussian-bump coils, 80 golden-angle spokes x 640
    radial3d  : 128x128x96 ellipsoid phantom, 8 coils, 8000 perturbed 3-D spokes x 250
    radial3d_small : the same at half the side (64x64x48, 2000 spokes x 125: the same points per
                grid cell), for profiling the 3-D kernels on a few hundred MB
    spoke40   : 40x40 image with random phase, 8 coils, one 80-point spoke through the centre
    """
    if name == "small64":
        g = rng(0)
        shape = (64, 64)
        return dict(shape=shape, x=random_image(g, shape), smaps=None,
                    omega=random_omega(g, 2, 4096), C=1)
    if name == "radial320":
        g = rng(1)
        shape = (320, 320)
        return dict(shape=shape, x=random_image(g, shape), smaps=gaussian_bump_maps(shape, 16),
                    omega=radial_2d(80, 640), C=16)
    if name == "radial3d":
        g = rng(2)
        shape = (128, 128, 96)
        n_spokes = max(1, int(round(8000 * scale)))
        return dict(shape=shape, x=ellipsoid_phantom(g, shape), smaps=gaussian_bump_maps(shape, 8),
                    omega=radial_3d(g, n_spokes, 250), C=8)
    if name == "radial3d_small":
        g = rng(5)
        shape = (64, 64, 48)
        n_spokes = max(1, int(round(2000 * scale)))
        return dict(shape=shape, x=ellipsoid_phantom(g, shape), smaps=gaussian_bump_maps(shape, 8),
                    omega=radial_3d(g, n_spokes, 125), C=8)
    if name == "spoke40":
        g = rng(3)
        shape = (40, 40)
        mag = ellipsoid_phantom(g, shape, n_ellipsoids=6, noise=0.0).real
        x = (mag * np.exp(1j * g.uniform(-math.pi, math.pi, shape))).astype(np.complex64)
        th = g.uniform(0, math.pi)
        kr = math.pi * (2.0 * np.arange(80) / 80 - 1.0)
        om = np.stack([kr * math.cos(th), kr * math.sin(th)]).astype(np.float32)
        return dict(shape=shape, x=x, smaps=gaussian_bump_maps(shape, 8), omega=om, C=8)
    raise KeyError(name)


def batched_problems(n=64, seed_index=4, sides=(64, 128, 192, 256, 320, 384), m_range=(4000, 200000),
                     coil_range=(1, 32)):
    """n independent 2-D problems of uneven size: side uniform over `sides`, M uniform over
    m_range, random-angle radial spokes of 2N samples (the last one truncated), coils uniform
    over coil_range; images i.i.d. N(0,1), Gaussian-bump maps, incoming gradients v i.i.d."""
    g = rng(seed_index)
    out = []
    for _ in range(n):
        N = int(g.choice(sides))
        M = int(g.integers(m_range[0], m_range[1] + 1))
        C = int(g.integers(coil_range[0], coil_range[1] + 1))
        n_read = 2 * N
        n_spokes = -(-M // n_read)
        om = radial_2d(n_spokes, n_read, golden=False, g=g)[:, :M]
        shape = (N, N)
        v = ((g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))) / math.sqrt(2)).astype(np.complex64)
        out.append(dict(shape=shape, x=random_image(g, shape), smaps=gaussian_bump_maps(shape, C),
                        omega=np.ascontiguousarray(om), v=v, C=C))
    return out
