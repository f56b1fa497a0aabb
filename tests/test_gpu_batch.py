"""Batched uneven problems: CUDA-graph replay equals the plain per-call path and the oracle."""
import numpy as np
import pytest

from gpu_helpers import host, rel
from oracle import jacobian as jb
from oracle.nufft import KBNufft

pytestmark = pytest.mark.gpu


def _problems():
    from paper_2111_02912_gb300.workloads import batched_problems
    return batched_problems(n=6, seed_index=40, sides=(32, 48, 64), m_range=(500, 4000), coil_range=(1, 6))


def test_graph_replay_matches_plain_calls_and_oracle():
    import torch

    from paper_2111_02912_gb300.batch import BatchedJacobian
    probs = _problems()
    bj = BatchedJacobian(probs, streams=3, autotune=True)
    bj.run_plain()
    torch.cuda.synchronize()
    plain = [tuple(host(t).copy() for t in o) for o in bj.outputs()]
    for it in bj.items:
        it.y.zero_(); it.go.zero_(); it.gx.zero_()
    bj.capture()
    for _ in range(2):                       # replays are repeatable
        bj.replay()
    torch.cuda.synchronize()
    for (y0, g0, x0), (y1, g1, x1) in zip(plain, [tuple(host(t) for t in o) for o in bj.outputs()]):
        assert np.array_equal(y0, y1) and np.array_equal(g0, g1)      # gather: deterministic
        assert rel(x1, x0) < 1e-6                                       # spread: rounding order only
    for p, (y, go, gx) in zip(probs, bj.outputs()):
        op = KBNufft(p["shape"], p["omega"])
        assert rel(host(y), jb.sense_forward(op, p["x"], p["smaps"])) < 1e-5
        go_ref, gx_ref = jb.vjp_omega_x(op, p["x"], p["v"], p["smaps"])
        assert rel(host(go), go_ref) < 1e-5 and rel(host(gx), gx_ref) < 1e-5


def test_every_configuration_the_autotuner_can_pick_matches_the_oracle():
    """Spread kernel x bin shape x strip part: each candidate computes the same operators."""
    import torch

    from paper_2111_02912_gb300.batch import CONFIG_CANDIDATES_2D, _Item, _step, plan_for
    p = _problems()[2]
    it = _Item(p, torch.device("cuda"))
    op = KBNufft(p["shape"], p["omega"])
    y_ref = jb.sense_forward(op, p["x"], p["smaps"])
    go_ref, gx_ref = jb.vjp_omega_x(op, p["x"], p["v"], p["smaps"])
    ran = 0
    for cfg in CONFIG_CANDIDATES_2D:
        plan = plan_for(it, cfg)
        _step(plan, it)
        torch.cuda.synchronize()
        assert rel(host(it.y), y_ref) < 1e-5, cfg
        assert rel(host(it.go), go_ref) < 1e-5 and rel(host(it.gx), gx_ref) < 1e-5, cfg
        ran += 1
    assert ran == len(CONFIG_CANDIDATES_2D)


def test_autotuner_picks_a_candidate_and_caches_it():
    from paper_2111_02912_gb300.batch import CONFIG_CANDIDATES_2D, Autotuner, BatchedJacobian
    tuner = Autotuner()
    probs = _problems()[:2]
    bj = BatchedJacobian(probs, autotune=True, tuner=tuner)
    for it in bj.items:
        assert it.config in CONFIG_CANDIDATES_2D
    assert len(tuner.cache) >= 1
    n = len(tuner.cache)
    BatchedJacobian(probs, autotune=True, tuner=tuner)    # same classes: no new timing runs
    assert len(tuner.cache) == n
