"""The ASL loop's schedule and coupling on the GPU: VEM noise from the
device step counter (sg_vem_eps) against the oracle, bit-exact, also when a
captured graph advances it; TPS held at rho = N * TPS / B (Eq. 2) by the
two-stream loop, and the time-feedback report (Eq. 1-4)."""

import numpy as np
import pytest
import torch

from oracle.vem import vem_eps
from tests._helpers import bits
from workloads.configs import DR_RANGES, base_params
from workloads.maps import make_map

pytestmark = pytest.mark.gpu


def _sim(n=64, seed=3):
    from paper_2305_04180_gb300 import Sim

    p = base_params(**DR_RANGES, seed=seed)
    maps = [make_map(s) for s in range(1, 5)]
    s = Sim(p, maps, (np.arange(n) % 4).astype(np.int32))
    s.reset()
    return s


@pytest.mark.parametrize("n,or_final,decay", [(64, 12.0, 20_000), (16, 3.0, 500_000), (1000, 2.0, 123_457)])
def test_vem_eps_matches_oracle_along_the_schedule(n, or_final, decay):
    s = _sim(n)
    sched = dict(e_min=0.01, e_max=0.8, or_start=float(n), or_final=or_final, decay_steps=decay)
    t = 0
    for K in (0, 7, 50, 400):
        if K:
            s.rollout(K)
            t += K
        e = s.vem_eps(**sched)
        torch.cuda.synchronize()
        assert np.array_equal(bits(e.cpu().numpy()), bits(vem_eps(n, t, **sched))), (n, t)
    # far past the decay: set the step counter directly
    f, u = s.get_state()
    u[2, :] = 10**6
    s.set_state(f, u)
    e = s.vem_eps(**sched)
    assert np.array_equal(bits(e.cpu().numpy()), bits(vem_eps(n, 10**6, **sched)))


def test_vem_eps_rejects_bad_schedules():
    from paper_2305_04180_gb300._lib import SgError

    s = _sim(16)
    for bad in (dict(or_final=1.0), dict(or_start=17.0), dict(decay_steps=0.0)):
        with pytest.raises(SgError):
            s.vem_eps(**bad)


def test_graph_replays_advance_the_vem_schedule():
    from paper_2305_04180_gb300.trainer import ColorTrainer

    s = _sim(64, seed=5)
    vem = dict(e_min=0.01, e_max=0.8, or_start=64.0, or_final=12.0, decay_steps=5_000)
    tr = ColorTrainer(s, batch=64, slots=32, tps=8, learn_start=0, two_streams=True, vem=vem, seed=1)
    s.rollout(8, policy="eps_q", qnet=tr.actor, eps=tr.eps, replay=tr.replay)
    g = tr.capture_iteration(8, 2, concurrent=False)
    for rep in range(4):
        g.launch(tr.s_actor)
        torch.cuda.synchronize()
        # the graph's VEM kernel ran at t = 8 + 8 rep, before that replay's rollout
        ref = vem_eps(64, 8 + 8 * rep, **vem)
        assert np.array_equal(bits(tr.eps.cpu().numpy()), bits(ref)), rep


def test_two_stream_loop_holds_tps_and_reports_the_feedback_periods():
    from paper_2305_04180_gb300.trainer import ColorTrainer

    s = _sim(128, seed=7)
    tr = ColorTrainer(s, batch=64, slots=64, tps=4, learn_start=2048, two_streams=True, seed=3)
    rho = tr.steps_per_vec_step()
    assert rho == 128 * 4 / 64
    tr.run(200, rollout_k=8)
    # Eq. 2 by count from the first chunk that reaches learn_start (the
    # second: 2 x 8 steps x 128 envs = 2048 transitions) on: 192 steps x rho
    assert tr.updates == rho * (200 - 8)
    rep = tr.tfm_report()
    assert rep["chunks"] == 25 and rep["v_period_ms"] > 0 and rep["b_period_ms"] > 0
    assert abs(rep["xi_ms"] - (rho * rep["b_period_ms"] - rep["v_period_ms"])) < 1e-9
    assert abs(rep["tps"] - 64 * tr.updates / (200 * 128)) < 1e-12
    th = tr.learner.get_params()
    assert np.isfinite(th).all()
    assert tr.replay.steps_recorded() == 200
