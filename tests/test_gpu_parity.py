"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: rel-L2 1e-5 against the same-kernel FP64 NUFFT, 5e-4 against the
exact NUDFT, 1e-3 for grad_omega against the exact Jacobian.
"""
import numpy as np
import pytest

from gpu_helpers import host, make_case, max_rel, rel, to_dev
from oracle import jacobian as jb
from oracle.nudft import NUDFT
from oracle.naive import TableNufft
from oracle.nufft import KBNufft

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-5
TOL_EXACT = 5e-4
TOL_GRAD_EXACT = 1e-3

CASES = [
    # name, shape, M, C, maps, opts
    ("1d", (64,), 700, 1, False, {}),
    ("2d_maps", (32, 40), 1500, 3, True, {}),
    ("2d_multi_image", (24, 18), 900, 5, False, {}),
    ("2d_small64", (64, 64), 4096, 1, False, {}),
    ("2d_many_coils", (16, 16), 600, 40, True, {}),
    ("2d_low_accuracy", (40, 48), 1200, 2, True, dict(J=5, sigma=1.25)),
    ("2d_ragged", (30, 22), 37, 2, True, {}),
    ("3d_maps", (16, 20, 12), 2000, 2, True, {}),
    ("3d_multi_image", (12, 10, 14), 800, 3, False, {}),
    ("2d_narrow_last_bin", (26, 30), 1500, 3, True, dict(bin_size=(16, 16))),      # K = 52, 60
    ("3d_narrow_last_bin", (10, 14, 12), 900, 2, True, dict(bin_size=(8, 12, 8))),  # K = 20, 28, 24
    ("2d_J4", (20, 24), 700, 2, True, dict(J=4)),
    ("2d_J8", (20, 24), 700, 2, True, dict(J=8)),
    ("2d_J7", (20, 24), 700, 2, True, dict(J=7)),
    # one tile per axis: the general (atomic) spread kernel instead of the cell-owner one
    ("2d_general_spread", (20, 24), 900, 3, True, dict(bin_size=(40, 48))),
    ("3d_general_spread", (8, 10, 6), 500, 2, True, dict(bin_size=(16, 20, 12))),
    ("2d_coils_6", (24, 24), 800, 6, True, {}),
    ("2d_tiny_grid_J8", (8, 10), 300, 3, True, dict(J=8)),   # K = 16, 20: tiles wrap more than once
    ("2d_coils_40_jvp", (16, 20), 500, 40, True, {}),        # several coil chunks in every kernel
    # grid sizes with a register-resident two-phase FFT kernel (64, 80, 96 = 8x8, 8x10, 8x12)
    ("2d_fft2_multi_image", (32, 40), 900, 3, False, {}),    # no coil sum in the last inverse pass
    ("2d_fft2_coils_40", (32, 32), 600, 40, True, {}),       # three coil chunks of up to sixteen
    # 9..16 coils: the last inverse pass adds two coil chunks into the image the pass before cleared
    ("2d_fft2_pair_c9", (32, 40), 1200, 9, True, {}),         # chunks of 8 and 1
    ("2d_fft2_pair_c12", (40, 32), 1200, 12, True, {}),       # chunks of 8 and 4
    ("2d_fft2_pair_c16_low_accuracy", (64, 64), 1500, 16, True, dict(J=5, sigma=1.25)),   # K = 80
    ("3d_fft2_pair_c16", (32, 40, 48), 1500, 16, True, {}),   # cleared by the second of two middle passes
    ("2d_fft2_low_accuracy", (64, 64), 1500, 2, True, dict(J=5, sigma=1.25)),   # K = 80
    ("3d_fft2_maps", (32, 40, 48), 2000, 2, True, {}),
    ("1d_fft2", (256,), 900, 3, True, {}),
    # two-phase sizes K = 768 (24 x 32) and 384 (16 x 24)
    ("2d_fft2_split_768", (384, 64), 1500, 2, True, {}),
    ("2d_fft2_split_384", (192, 40), 1200, 3, False, {}),
]


def _plan(case, **opts):
    from paper_2111_02912_gb300 import Plan
    return Plan(case["shape"], to_dev(case["omega"]), max_coils=case["C"], **opts)


def _clustered(shape, M, seed):
    """Samples packed near the k-space centre: many work items per spread tile."""
    g = np.random.default_rng(seed)
    return np.clip(g.normal(0.0, 0.15, (len(shape), M)), -np.pi, np.pi).astype(np.float32)


CASES += [
    ("2d_clustered", (32, 32), 20000, 4, True, {}),
    ("3d_clustered", (12, 12, 12), 8000, 2, True, {}),
]


@pytest.mark.parametrize("name,shape,M,C,maps,opts", CASES, ids=[c[0] for c in CASES])
def test_all_products_match_same_kernel_oracle(name, shape, M, C, maps, opts):
    import torch
    seed = sum(map(ord, name))
    om = _clustered(shape, M, seed) if "clustered" in name else None
    case = make_case(shape, M, C, maps, seed=seed, omega=om)
    plan = _plan(case, **opts)
    X, S, V, Y, DOM = (to_dev(case[k]) for k in ("x", "smaps", "v", "y", "domega"))
    y = plan.forward(X, S)
    xa = plan.adjoint(Y, S)
    dy, y2 = plan.jvp_omega(X, DOM, S, want_y=True)
    dy_only = plan.jvp_omega(X, DOM, S)
    go, gx = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    op = KBNufft(shape, case["omega"], **{k: v for k, v in opts.items() if k != "bin_size"})
    s = case["smaps"]
    y_ref = jb.sense_forward(op, case["x"], s)
    assert rel(host(y), y_ref) < TOL_SAME
    assert rel(host(y2), y_ref) < TOL_SAME
    xa_ref = jb.sense_adjoint(op, case["y"], s)
    assert rel(host(xa), xa_ref) < TOL_SAME
    assert max_rel(host(xa), xa_ref) < TOL_SAME       # element by element, not only in the norm
    dy_ref = jb.jvp_omega(op, case["x"], case["domega"], s)
    assert rel(host(dy), dy_ref) < TOL_SAME
    assert rel(host(dy_only), dy_ref) < TOL_SAME
    go_ref, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], s)
    assert rel(host(go), go_ref) < TOL_SAME
    assert rel(host(gx), gx_ref) < TOL_SAME
    assert max_rel(host(gx), gx_ref) < TOL_SAME


# The strip spread: every coils-per-warp width (64 / NSL coils for NSL rows), J 4..8, grids
# just wide enough for it (K1 = 16 + J - 1 columns, K0 = NSL + J - 1 rows: windows wrap around both
# axes), several coil groups, and the two other spread kernels on the same problem.
STRIP_CASES = [
    # name, shape, M, C, maps, opts
    ("strip_c1", (48, 40), 2500, 1, False, {}),
    ("strip_c2", (40, 48), 2500, 2, True, {}),
    ("strip_c3", (36, 20), 1500, 3, False, {}),
    ("strip_c5", (24, 32), 1500, 5, True, {}),
    ("strip_c12", (32, 24), 1200, 12, True, {}),
    ("strip_c20_two_groups", (24, 40), 1500, 20, True, {}),
    ("strip_c33_three_groups", (20, 24), 800, 33, True, {}),
    ("strip_narrow_J4", (20, 10), 900, 4, True, dict(J=4)),          # K = 40 x 20, K1 = 16 + J
    ("strip_narrow_J6", (12, 12), 600, 16, True, {}),                # K = 24 x 24: K1 = 16 + J + 2
    ("strip_narrow_J8", (20, 12), 700, 2, True, dict(J=8)),          # K1 = 24 = 16 + J
    ("strip_J5_odd_width", (30, 26), 1200, 6, True, dict(J=5)),
    ("strip_J7_ragged_tile", (34, 22), 1100, 8, True, dict(J=7)),    # K1 = 44: last column tile 12 wide
    ("strip_sigma125", (64, 48), 2000, 4, True, dict(sigma=1.25)),   # K = 80 x 60
    ("strip_variant_tiles", (32, 40), 1500, 3, True, dict(spread="tiles")),
    ("strip_variant_general", (32, 40), 1500, 3, True, dict(spread="general")),
    ("strip_variant_strips", (32, 40), 1500, 3, True, dict(spread="strips")),
    # 3-D strips: units of R0 x R1 rows (k0, k1) by 16 cells of the last axis, every coils-per-warp
    # width (R0 x R1 = 4 x 8, 2 x 4, 4 x 4, 2 x 2), grids just wide enough, ragged row groups and
    # column tiles, two coil groups, and the cell-owner kernel on the same kind of problem
    ("strip3d_c2", (16, 20, 24), 3000, 2, True, {}),
    ("strip3d_c5", (12, 16, 20), 2000, 5, True, {}),
    ("strip3d_c8", (16, 12, 16), 2500, 8, True, {}),
    ("strip3d_c16_J4", (10, 12, 14), 1500, 16, True, dict(J=4)),
    ("strip3d_narrow_J8", (8, 8, 12), 800, 3, True, dict(J=8)),          # K = 16 x 16 x 24
    ("strip3d_J5_ragged_tile", (10, 14, 18), 1500, 6, True, dict(J=5)),  # last column tile 4 wide
    ("strip3d_J7", (14, 10, 12), 1200, 4, True, dict(J=7)),
    ("strip3d_sigma125_ragged_rows", (24, 16, 20), 2000, 3, True, dict(sigma=1.25)),   # K = 30 x 20 x 30
    ("strip3d_two_coil_groups", (12, 12, 16), 1000, 20, True, {}),
    ("strip3d_variant_tiles", (16, 20, 24), 2000, 3, True, dict(spread="tiles")),
]


@pytest.mark.parametrize("name,shape,M,C,maps,opts", STRIP_CASES, ids=[c[0] for c in STRIP_CASES])
def test_strip_spread_adjoint_and_vjp(name, shape, M, C, maps, opts):
    import torch
    seed = sum(map(ord, name))
    case = make_case(shape, M, C, maps, seed=seed)
    plan = _plan(case, **opts)
    X, S, V, Y = (to_dev(case[k]) for k in ("x", "smaps", "v", "y"))
    xa = plan.adjoint(Y, S)
    go, gx = plan.vjp_omega_x(X, V, S)
    gx_only = plan.vjp_omega_x(X, V, S, need_omega=False)[1]
    torch.cuda.synchronize()
    op = KBNufft(shape, case["omega"], **{k: v for k, v in opts.items() if k in ("J", "sigma")})
    s = case["smaps"]
    xa_ref = jb.sense_adjoint(op, case["y"], s)
    assert rel(host(xa), xa_ref) < TOL_SAME and max_rel(host(xa), xa_ref) < TOL_SAME
    go_ref, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], s)
    assert rel(host(go), go_ref) < TOL_SAME
    assert rel(host(gx), gx_ref) < TOL_SAME and max_rel(host(gx), gx_ref) < TOL_SAME
    assert rel(host(gx_only), gx_ref) < TOL_SAME


def test_strip_variant_refused_where_it_does_not_apply():
    from paper_2111_02912_gb300 import _abi
    case = make_case((8, 10), 100, 2, True, seed=1)            # K1 = 20 < 16 + J - 1
    with pytest.raises(_abi.NufftError) as e:
        _plan(case, spread="strips")
    assert e.value.status == _abi.NUFFT_ERR_UNSUPPORTED


def test_small64_against_exact_nudft_and_jacobian():
    """64x64, M = 4096 uniform omega: the method's own accuracy (Appendix bounds) at FP32."""
    import torch
    case = make_case((64, 64), 4096, 1, False, seed=7)
    plan = _plan(case)
    X, V = to_dev(case["x"]), to_dev(case["v"])
    y = plan.forward(X)
    go, gx = plan.vjp_omega_x(X, V)
    torch.cuda.synchronize()
    ex = NUDFT((64, 64), case["omega"])
    assert rel(host(y), jb.sense_forward(ex, case["x"])) < TOL_EXACT
    go_ref, gx_ref = jb.vjp_omega_x(ex, case["x"], case["v"])
    assert rel(host(go), go_ref) < TOL_GRAD_EXACT
    assert rel(host(gx), gx_ref) < TOL_EXACT


def test_radial320_full_size_parity():
    """The 320x320, 16-coil, 80 golden-angle spokes x 640 workload, full size, every output."""
    import torch

    from paper_2111_02912_gb300 import Plan
    from paper_2111_02912_gb300.workloads import workload
    w = workload("radial320")
    g = np.random.default_rng(5)
    C, M = w["C"], w["omega"].shape[1]
    v = (g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))).astype(np.complex64)
    plan = Plan(w["shape"], to_dev(w["omega"]), max_coils=C)
    X, S, V = to_dev(w["x"]), to_dev(w["smaps"]), to_dev(v)
    y = plan.forward(X, S)
    go, gx = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    op = KBNufft(w["shape"], w["omega"])
    assert rel(host(y), jb.sense_forward(op, w["x"], w["smaps"])) < TOL_SAME
    go_ref, gx_ref = jb.vjp_omega_x(op, w["x"], v, w["smaps"])
    assert rel(host(go), go_ref) < TOL_SAME
    assert rel(host(gx), gx_ref) < TOL_SAME
    # exact NUDFT on a point subset (the exact sum is O(MN) per coil)
    sub = np.arange(0, M, 25)
    ex = NUDFT(w["shape"], w["omega"][:, sub])
    assert rel(host(y)[:, sub], jb.sense_forward(ex, w["x"], w["smaps"])) < TOL_EXACT
    ge, _ = jb.vjp_omega_x(ex, w["x"], v[:, sub], w["smaps"])
    assert rel(host(go)[:, sub], ge) < TOL_GRAD_EXACT


def test_empty_and_single_point():
    import torch
    case = make_case((16, 16), 0, 2, True, seed=3)
    plan = _plan(case)
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    y = plan.forward(X, S)
    xa = plan.adjoint(to_dev(np.zeros((2, 0), np.complex64)), S)
    torch.cuda.synchronize()
    assert y.shape == (2, 0) and float(xa.abs().max()) == 0.0
    one = make_case((16, 16), 1, 2, True, seed=4)
    plan.set_points(to_dev(one["omega"]))
    y1 = plan.forward(X, S)
    torch.cuda.synchronize()
    assert rel(host(y1), jb.sense_forward(KBNufft((16, 16), one["omega"]), case["x"], case["smaps"])) < TOL_SAME
    # no points with 16 coils on two-phase grid sizes: the last inverse pass adds two coil chunks
    # into an image that must still come out zero (output buffers start as garbage)
    big = make_case((32, 40), 0, 16, True, seed=5)
    plan16 = _plan(big)
    X16, S16 = to_dev(big["x"]), to_dev(big["smaps"])
    out = torch.full((32, 40), float("nan"), dtype=torch.complex64, device="cuda")
    xa16 = plan16.adjoint(to_dev(np.zeros((16, 0), np.complex64)), S16, out=out)
    go16 = torch.empty((2, 0), dtype=torch.float32, device="cuda")
    gx16 = torch.full((32, 40), float("nan"), dtype=torch.complex64, device="cuda")
    plan16.vjp_omega_x(X16, to_dev(np.zeros((16, 0), np.complex64)), S16, out=(go16, gx16))
    torch.cuda.synchronize()
    assert float(xa16.abs().max()) == 0.0 and float(gx16.abs().max()) == 0.0 and go16.shape == (2, 0)


def test_periodic_omega_and_boundary_values():
    """omega shifted by multiples of 2 pi, and omega exactly at -pi / on grid points."""
    import torch
    g = np.random.default_rng(11)
    M = 1000
    om = g.uniform(-np.pi, np.pi, (2, M)).astype(np.float32)
    om[:, :10] = -np.float32(np.pi)
    om[:, 10:20] = (2 * np.pi * g.integers(-32, 32, (2, 10)) / 64).astype(np.float32)
    case = make_case((32, 32), M, 2, True, seed=5, omega=om)
    plan = _plan(case)
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    y = host(plan.forward(X, S))
    shifted = (om + np.float32(2 * np.pi) * g.integers(-3, 4, om.shape).astype(np.float32)).astype(np.float32)
    plan.set_points(to_dev(shifted))
    y_s = host(plan.forward(X, S))
    torch.cuda.synchronize()
    ref = jb.sense_forward(KBNufft((32, 32), om), case["x"], case["smaps"])
    assert rel(y, ref) < TOL_SAME
    ref_s = jb.sense_forward(KBNufft((32, 32), shifted), case["x"], case["smaps"])
    assert rel(y_s, ref_s) < TOL_SAME


def test_adjoint_identity_in_fp32():
    import torch
    case = make_case((48, 40), 3000, 4, True, seed=6)
    plan = _plan(case)
    X, S, Y = to_dev(case["x"]), to_dev(case["smaps"]), to_dev(case["y"])
    lhs = torch.vdot(Y.flatten(), plan.forward(X, S).flatten())
    rhs = torch.vdot(plan.adjoint(Y, S).flatten(), X.flatten())
    assert abs(complex(lhs) - complex(rhs)) < 1e-5 * abs(complex(lhs))


def test_gather_is_deterministic_and_resort_is_consistent():
    import torch
    case = make_case((40, 40), 5000, 3, True, seed=8)
    plan = _plan(case)
    X, S, V = to_dev(case["x"]), to_dev(case["smaps"]), to_dev(case["v"])
    a = plan.forward(X, S).clone()
    plan.set_points(to_dev(case["omega"]))
    b = plan.forward(X, S).clone()
    g1, x1 = plan.vjp_omega_x(X, V, S)
    g2, x2 = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(g1, g2)
    assert rel(host(x1), host(x2)) < 1e-6        # spread: the hit lists' fill order changes rounding only


def test_launch_counter_and_profile_hooks():
    import torch

    from paper_2111_02912_gb300 import nufft_launch_count
    case = make_case((32, 32), 2000, 2, True, seed=9)
    plan = _plan(case)
    X, S, V = to_dev(case["x"]), to_dev(case["smaps"]), to_dev(case["v"])
    plan.profile_enable(True)
    n0 = nufft_launch_count()
    plan.forward(X, S)
    plan.vjp_omega_x(X, V, S)
    n1 = nufft_launch_count()
    torch.cuda.synchronize()
    prof = plan.profile_read()
    assert n1 - n0 == sum(v[0] for v in prof.values())
    assert {"fft_fwd_first", "fft_fwd_mid", "gather_fwd", "gather_vjp", "spread", "fft_inv_last"} <= set(prof)
    assert all(ms > 0 for _, ms in prof.values())


def test_radial3d_full_size_sampled_against_exact_nudft():
    """128x128x96, 8 coils, 2,000,000 perturbed 3-D radial points: y and grad_omega on a point sample
    (each depends on its own point only, so the exact NUDFT of a sample is an exact check), and
    grad_x (the 3-D adjoint spread, heavy tiles included) on a voxel sample against the exact sum."""
    import torch

    from paper_2111_02912_gb300 import Plan
    from paper_2111_02912_gb300.workloads import workload
    w = workload("radial3d")
    C, M = w["C"], w["omega"].shape[1]
    g = np.random.default_rng(9)
    v = (g.standard_normal((C, M)) + 1j * g.standard_normal((C, M))).astype(np.complex64)
    plan = Plan(w["shape"], to_dev(w["omega"]), max_coils=C)
    X, S, V = to_dev(w["x"]), to_dev(w["smaps"]), to_dev(v)
    y = host(plan.forward(X, S))
    go, gx = plan.vjp_omega_x(X, V, S)
    go, gx = host(go), host(gx)
    torch.cuda.synchronize()
    sub = np.sort(g.choice(M, 300, replace=False))
    ex = NUDFT(w["shape"], w["omega"][:, sub])
    assert rel(y[:, sub], jb.sense_forward(ex, w["x"], w["smaps"])) < TOL_EXACT
    ge, _ = jb.vjp_omega_x(ex, w["x"], v[:, sub], w["smaps"])
    assert rel(go[:, sub], ge) < TOL_GRAD_EXACT
    # grad_x = E'v, Sec. II-D with the maps of Sec. II-G, depends on all 2 M points: the exact sum
    # sum_c conj(s_c,j) sum_i v_ci exp(+i omega_i . r_j) on 200 sampled voxels, in FP64, point chunks
    from oracle.nudft import voxel_centres
    r = np.stack([c.ravel() for c in np.meshgrid(*voxel_centres(w["shape"]), indexing="ij")])   # (3, N)
    vox = np.sort(g.choice(r.shape[1], 200, replace=False))
    rs = r[:, vox].astype(np.float64)
    om64 = w["omega"].astype(np.float64)
    acc = np.zeros((C, vox.size), np.complex128)
    for i0 in range(0, M, 100_000):
        ph = np.exp(1j * (om64[:, i0:i0 + 100_000].T @ rs))                 # (chunk, 200)
        acc += v[:, i0:i0 + 100_000].astype(np.complex128) @ ph
    gx_exact = np.sum(np.conj(w["smaps"].reshape(C, -1)[:, vox].astype(np.complex128)) * acc, axis=0)
    gx_s = gx.reshape(-1)[vox]
    assert rel(gx_s, gx_exact) < TOL_EXACT
    assert max_rel(gx_s, gx_exact) < TOL_EXACT


@pytest.mark.parametrize("name,shape,M,C,clustered", [
    ("det_radial_like", (48, 40), 3000, 16, False),
    ("det_clustered_split_units", (32, 32), 20000, 4, True),   # units split into parts: ordered combine
    ("det_two_coil_groups", (24, 40), 1500, 20, False),
    ("det_3d", (16, 20, 24), 3000, 8, False),
    ("det_3d_clustered_split_units", (12, 12, 16), 12000, 2, True),
])
def test_deterministic_adjoint_is_bitwise_reproducible(name, shape, M, C, clustered):
    """deterministic=1: repeated calls, and a re-sort of the same omega, give bitwise equal results."""
    import torch
    seed = sum(map(ord, name))
    om = _clustered(shape, M, seed) if clustered else None
    case = make_case(shape, M, C, True, seed=seed, omega=om)
    plan = _plan(case, deterministic=True)
    X, S, V, Y = (to_dev(case[k]) for k in ("x", "smaps", "v", "y"))
    xa1 = plan.adjoint(Y, S).clone()
    xa2 = plan.adjoint(Y, S).clone()
    g1, gx1 = plan.vjp_omega_x(X, V, S)
    g1, gx1 = g1.clone(), gx1.clone()
    plan.set_points(to_dev(case["omega"]))                      # a fresh sort of the same points
    xa3 = plan.adjoint(Y, S).clone()
    g3, gx3 = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    assert torch.equal(xa1, xa2) and torch.equal(xa1, xa3)
    assert torch.equal(gx1, gx3) and torch.equal(g1, g3)
    op = KBNufft(shape, case["omega"])
    xa_ref = jb.sense_adjoint(op, case["y"], case["smaps"])
    assert rel(host(xa1), xa_ref) < TOL_SAME and max_rel(host(xa1), xa_ref) < TOL_SAME
    _, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], case["smaps"])
    assert rel(host(gx1), gx_ref) < TOL_SAME


def test_deterministic_refused_without_the_strip_spread():
    from paper_2111_02912_gb300 import _abi
    case = make_case((8, 10, 6), 100, 2, True, seed=2)
    with pytest.raises(_abi.NufftError) as e:
        _plan(case, deterministic=True)
    assert e.value.status == _abi.NUFFT_ERR_UNSUPPORTED


# Interpolation weights read from a linearly interpolated table of psi (nufft_opts.kernel_mode =
# NUFFT_KERNEL_TABLE): every product against the oracle's table NUFFT of the same density.
TABLE_CASES = [
    # name, shape, M, C, maps, opts, L
    ("table_1d", (64,), 700, 2, True, {}, 512),
    ("table_2d_strips", (32, 40), 1500, 3, True, {}, 512),
    ("table_2d_strips_L64", (32, 40), 1500, 3, True, {}, 64),
    ("table_2d_tiles", (32, 40), 1500, 3, True, dict(spread="tiles"), 256),
    ("table_2d_low_accuracy", (40, 48), 1200, 2, True, dict(J=5, sigma=1.25), 1024),
    ("table_3d", (16, 20, 12), 2000, 2, True, {}, 512),
]


@pytest.mark.parametrize("name,shape,M,C,maps,opts,L", TABLE_CASES, ids=[c[0] for c in TABLE_CASES])
def test_table_kernel_mode_matches_oracle_table_nufft(name, shape, M, C, maps, opts, L):
    import torch
    seed = sum(map(ord, name))
    case = make_case(shape, M, C, maps, seed=seed)
    plan = _plan(case, kernel_mode="table", table_density=L, **opts)
    X, S, V, Y, DOM = (to_dev(case[k]) for k in ("x", "smaps", "v", "y", "domega"))
    y = plan.forward(X, S)
    xa = plan.adjoint(Y, S)
    dy = plan.jvp_omega(X, DOM, S)
    go, gx = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    kw = {k: v for k, v in opts.items() if k in ("J", "sigma")}
    op = TableNufft(shape, case["omega"], L=L, **kw)
    s = case["smaps"]
    y_ref = jb.sense_forward(op, case["x"], s)
    assert rel(host(y), y_ref) < TOL_SAME
    xa_ref = jb.sense_adjoint(op, case["y"], s)
    assert rel(host(xa), xa_ref) < TOL_SAME and max_rel(host(xa), xa_ref) < TOL_SAME
    assert rel(host(dy), jb.jvp_omega(op, case["x"], case["domega"], s)) < TOL_SAME
    go_ref, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], s)
    assert rel(host(go), go_ref) < TOL_SAME
    assert rel(host(gx), gx_ref) < TOL_SAME and max_rel(host(gx), gx_ref) < TOL_SAME
    # the table differs from the kernel itself by its interpolation error (O(1 / L^2) inside the
    # support, plus the ramp over the last 1 / L to the zero beyond |u| = J / 2)
    y_direct = jb.sense_forward(KBNufft(shape, case["omega"], **kw), case["x"], s)
    assert 0.0 < rel(y_ref, y_direct) < 1e-4


def test_kernel_mode_refused_by_the_allocation_free_forward():
    from paper_2111_02912_gb300 import _abi
    case = make_case((16, 16), 100, 1, False, seed=3)
    o = _abi.nufft_default_opts(2, (16, 16))
    o.kernel_mode = _abi.NUFFT_KERNEL_TABLE
    om, x = to_dev(case["omega"]), to_dev(case["x"])
    import torch
    y = torch.empty((1, 100), dtype=torch.complex64, device="cuda")
    with pytest.raises(_abi.NufftError) as e:
        _abi.nufft_forward_noalloc(o, 100, om.data_ptr(), 1, x.data_ptr(), 0, y.data_ptr(), 0)
    assert e.value.status == _abi.NUFFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("name,shape,M,C,maps", [
    ("dual_16_coils", (48, 40), 3000, 16, True),     # grad_x on the plan's second stream
    ("dual_multi_image", (32, 24), 2000, 5, False),
    ("single_stream_20_coils", (24, 40), 1500, 20, True),   # more than 16 coils with maps: one stream
])
def test_vjp_with_both_outputs_equals_each_output_alone(name, shape, M, C, maps):
    """The VJP with both outputs (two streams on 2-D strip plans) gives bitwise the grad_omega of the
    omega-only call and the grad_x of the x-only call (deterministic plan: one summation order)."""
    import torch
    seed = sum(map(ord, name))
    case = make_case(shape, M, C, maps, seed=seed)
    plan = _plan(case, deterministic=True)
    X, S, V = (to_dev(case[k]) for k in ("x", "smaps", "v"))
    go, gx = plan.vjp_omega_x(X, V, S)
    go, gx = go.clone(), gx.clone()
    go1 = plan.vjp_omega_x(X, V, S, need_x=False)[0].clone()
    gx1 = plan.vjp_omega_x(X, V, S, need_omega=False)[1].clone()
    torch.cuda.synchronize()
    assert torch.equal(go, go1) and torch.equal(gx, gx1)
    op = KBNufft(shape, case["omega"])
    go_ref, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], case["smaps"])
    assert rel(host(go), go_ref) < TOL_SAME and rel(host(gx), gx_ref) < TOL_SAME


def test_sort_points_on_another_stream_then_calls_on_the_main_stream():
    """nufft_sort_points sorts now on the caller's stream; later calls ordered after it (an event)
    need no sort of their own and give the same results; a second sort_points does nothing."""
    import torch
    case = make_case((32, 40), 2000, 4, True, seed=91)
    plan = _plan(case)
    X, S, V = (to_dev(case[k]) for k in ("x", "smaps", "v"))
    y0 = plan.forward(X, S).clone()
    go0, gx0 = (t.clone() for t in plan.vjp_omega_x(X, V, S))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.set_points(to_dev(case["omega"]))
        plan.sort_points()
        plan.sort_points()
        ev = torch.cuda.Event()
        ev.record(side)
    torch.cuda.current_stream().wait_event(ev)
    y1 = plan.forward(X, S)
    go1, gx1 = plan.vjp_omega_x(X, V, S)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1) and torch.equal(go0, go1)
    assert rel(host(gx1), host(gx0)) < 1e-6


@pytest.mark.parametrize("shape,M,C,gather", [
    ((32, 40), 1500, 8, "quads"), ((32, 40), 1500, 12, "quads"), ((32, 40), 1500, 16, "pairs"),
    ((32, 40), 1500, 24, "auto"), ((16, 20, 12), 1500, 8, "quads"), ((64,), 700, 8, "quads"),
])
def test_forward_gather_variants_match_the_oracle(shape, M, C, gather):
    """nufft_opts.gather_variant: coil pairs or quads in the forward gather give the same operator."""
    import torch
    seed = sum(map(ord, gather)) + C
    case = make_case(shape, M, C, True, seed=seed)
    plan = _plan(case, gather=gather)
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    y = plan.forward(X, S)
    torch.cuda.synchronize()
    y_ref = jb.sense_forward(KBNufft(shape, case["omega"]), case["x"], case["smaps"])
    assert rel(host(y), y_ref) < TOL_SAME and max_rel(host(y), y_ref) < TOL_SAME


@pytest.mark.parametrize("shape,M,opts", [
    ((64,), 700, {}), ((32, 40), 1500, {}), ((20, 24), 900, dict(J=5)), ((20, 24), 900, dict(J=7)),
    ((20, 24), 900, dict(J=8)), ((8, 10), 400, dict(J=8)), ((16, 20, 12), 1500, {}),
    ((10, 12, 14), 1200, dict(J=8)), ((12, 10, 14), 1000, dict(J=5)), ((24, 16, 20), 1500, dict(sigma=1.25)),
])
def test_eight_coil_gathers_match_the_oracle(shape, M, opts):
    """8 coils (a cell's channel block is half a 128-byte line): the forward and VJP gathers in 1-D,
    2-D and 3-D, windows wrapping the last axis, J = 5..8, and sigma = 1.25."""
    import torch
    C = 8
    seed = sum(shape) + M
    case = make_case(shape, M, C, True, seed=seed)
    plan = _plan(case, **opts)
    X, S, V = to_dev(case["x"]), to_dev(case["smaps"]), to_dev(case["v"])
    y = plan.forward(X, S)
    go, gx = plan.vjp_omega_x(X, V, S)
    go_only, _ = plan.vjp_omega_x(X, V, S, need_omega=True, need_x=False)
    torch.cuda.synchronize()
    op = KBNufft(shape, case["omega"], **opts)
    assert rel(host(y), jb.sense_forward(op, case["x"], case["smaps"])) < TOL_SAME
    assert max_rel(host(y), jb.sense_forward(op, case["x"], case["smaps"])) < TOL_SAME
    go_ref, gx_ref = jb.vjp_omega_x(op, case["x"], case["v"], case["smaps"])
    assert rel(host(go), go_ref) < TOL_SAME and rel(host(go_only), go_ref) < TOL_SAME
    assert rel(host(gx), gx_ref) < TOL_SAME
