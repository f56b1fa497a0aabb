"""GPU test of nufft_forward_noalloc, the allocation-free forward entry point.

Some callers cannot allocate device memory: their device memory is owned by
another allocator (a framework's caching allocator, a service with a fixed
memory budget) or they must not allocate while they run.  For them the
library offers one plan-free forward NUFFT whose scratch lives in a static
device array.  This test calls it through the C ABI twice in a row, on two
different problems, and checks each result against the plan-based
nufft_forward within the parity tolerance of the other GPU tests; it also
checks that a problem too large for the array is refused.  The file is named
so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import host, make_case, rel, to_dev

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-5


def _opts(abi, shape, C):
    o = abi.nufft_default_opts(len(shape), shape)
    o.max_coils = C
    return o


def _noalloc_forward(abi, case):
    import torch
    shape, C, M = case["shape"], case["C"], case["omega"].shape[1]
    om, X, S = to_dev(case["omega"]), to_dev(case["x"]), to_dev(case["smaps"])
    y = torch.full((C, M), float("nan"), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    abi.nufft_forward_noalloc(_opts(abi, shape, C), M, om.data_ptr(), C, X.data_ptr(),
                              S.data_ptr() if S is not None else None, y.data_ptr(), stream)
    torch.cuda.synchronize()
    return host(y)


def _plan_forward(case):
    import torch

    from paper_2111_02912_gb300 import Plan
    plan = Plan(case["shape"], to_dev(case["omega"]), max_coils=case["C"])
    y = plan.forward(to_dev(case["x"]), to_dev(case["smaps"]))
    torch.cuda.synchronize()
    return host(y)


def test_noalloc_forward_matches_plan_forward_on_two_calls_in_a_row():
    from paper_2111_02912_gb300 import _abi
    first = make_case((48, 40), 3000, 3, True, seed=41)
    second = make_case((64, 64), 4096, 1, False, seed=42)
    for case in (first, second):
        y_static = _noalloc_forward(_abi, case)
        y_plan = _plan_forward(case)
        assert np.isfinite(y_static).all()
        assert rel(y_static, y_plan) < TOL_SAME


def test_noalloc_forward_in_1d_and_3d_and_smaller_after_larger():
    """The array keeps the last call's contents: a small problem after a larger one (1-D and 3-D
    layouts of the scratch) must not see them."""
    from paper_2111_02912_gb300 import _abi
    cases = [make_case((12, 10, 14), 2500, 2, True, seed=43),   # 3-D
             make_case((96, 80), 6000, 4, True, seed=44),       # the largest of the sequence
             make_case((64,), 700, 3, False, seed=45),          # 1-D, far smaller
             make_case((8, 10, 6), 300, 1, False, seed=46)]     # 3-D again, smaller still
    for case in cases:
        y_static = _noalloc_forward(_abi, case)
        y_plan = _plan_forward(case)
        assert np.isfinite(y_static).all()
        assert rel(y_static, y_plan) < TOL_SAME


def test_noalloc_forward_refuses_problems_beyond_its_scratch():
    import torch

    from paper_2111_02912_gb300 import _abi
    o = _opts(_abi, (1024, 1024), 16)       # grid 2048^2 x 16 coils: far past the static array
    dummy = torch.zeros(16, dtype=torch.complex64, device="cuda")   # never read: refused before any work
    p = dummy.data_ptr()
    status = _abi.lib().nufft_forward_noalloc(ctypes.byref(o), 1000, p, 16, p, p, p, None)
    assert status == _abi.NUFFT_ERR_UNSUPPORTED
    assert b"limited to" in _abi.lib().nufft_last_error()
