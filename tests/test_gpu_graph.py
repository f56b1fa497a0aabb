"""A whole step (bin sort, forward, VJP) captured in a CUDA graph and replayed gives the eager results.

The benchmark times the step that way; the replay reads the same device buffers, so a changed
omega (re-sorted inside the graph) must give the new results too.
"""
import numpy as np
import pytest

from gpu_helpers import host, make_case, rel, to_dev

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_step_and_follows_new_omega():
    import torch

    from paper_2111_02912_gb300 import Plan
    shape, M, C = (48, 40), 3000, 4
    case = make_case(shape, M, C, True, seed=61)
    om = to_dev(case["omega"])
    X, S, V = to_dev(case["x"]), to_dev(case["smaps"]), to_dev(case["v"])
    plan = Plan(shape, om, max_coils=C)
    y = torch.empty((C, M), dtype=torch.complex64, device=om.device)
    go = torch.empty((2, M), dtype=torch.float32, device=om.device)
    gx = torch.empty(shape, dtype=torch.complex64, device=om.device)

    def step():
        plan.set_points(om)
        plan.forward(X, S, out=y)
        plan.vjp_omega_x(X, V, S, out=(go, gx))

    def eager():
        step()
        torch.cuda.synchronize()
        return host(y).copy(), host(go).copy(), host(gx).copy()

    ref = eager()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        y.zero_(), go.zero_(), gx.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(y), ref[0]) and np.array_equal(host(go), ref[1])
        assert rel(host(gx), ref[2]) < 1e-6          # the adjoint spread sums in arrival order

    # new sample locations in the same buffer: the replay re-sorts them
    g = np.random.default_rng(62)
    om.copy_(torch.from_numpy(g.uniform(-np.pi, np.pi, (2, M)).astype(np.float32)))
    graph.replay()
    torch.cuda.synchronize()
    replayed = host(y).copy(), host(go).copy(), host(gx).copy()
    fresh = eager()
    assert np.array_equal(replayed[0], fresh[0]) and np.array_equal(replayed[1], fresh[1])
    assert rel(replayed[2], fresh[2]) < 1e-6
    assert rel(fresh[0], ref[0]) > 0.1                 # the locations did change the result


def test_forward_captured_alone_after_eager_set_points_replays_correctly():
    """Only the forward is captured: the sort it completes must stay outside the graph."""
    import torch

    from paper_2111_02912_gb300 import Plan
    shape, M, C = (40, 32), 2500, 3
    case = make_case(shape, M, C, True, seed=63)
    om = to_dev(case["omega"])
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    plan = Plan(shape, om, max_coils=C)
    y = torch.empty((C, M), dtype=torch.complex64, device=om.device)
    plan.forward(X, S, out=y)
    torch.cuda.synchronize()
    ref = host(y).copy()
    plan.set_points(om)                              # eager; the rest of the sort is still pending
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forward(X, S, out=y)                    # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    plan.set_points(om)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forward(X, S, out=y)
    for _ in range(3):
        y.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(y), ref)


def test_set_points_twice_before_use():
    """A histogram that was never scanned is cleared by the next set_points."""
    import torch

    from paper_2111_02912_gb300 import Plan
    shape, M, C = (32, 32), 2000, 2
    case = make_case(shape, M, C, True, seed=64)
    om = to_dev(case["omega"])
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    plan = Plan(shape, om, max_coils=C)
    ref = host(plan.forward(X, S)).copy()
    other = torch.from_numpy(np.random.default_rng(65).uniform(-np.pi, np.pi, (2, M)).astype(np.float32)).to(om.device)
    plan.set_points(other)
    plan.set_points(om)
    y = host(plan.forward(X, S))
    torch.cuda.synchronize()
    assert np.array_equal(y, ref)


def test_set_points_keeps_its_own_copy_of_omega():
    """The caller may overwrite omega on the stream right after set_points: the sort reads the copy."""
    import torch

    from paper_2111_02912_gb300 import Plan
    shape, M, C = (48, 32), 3000, 2
    case = make_case(shape, M, C, True, seed=66)
    om = to_dev(case["omega"])
    X, S = to_dev(case["x"]), to_dev(case["smaps"])
    ref = host(Plan(shape, om, max_coils=C).forward(X, S)).copy()
    plan = Plan(shape, om, max_coils=C)
    buf = om.clone()
    plan.forward(X, S)                               # the plan's first sort is done
    plan.set_points(buf)
    buf.copy_(torch.from_numpy(np.random.default_rng(67).uniform(-np.pi, np.pi, (2, M)).astype(np.float32)))
    y = host(plan.forward(X, S))
    torch.cuda.synchronize()
    assert np.array_equal(y, ref)
