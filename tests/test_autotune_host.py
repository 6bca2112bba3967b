"""Host-side logic of the autotuner (no GPU): candidate sweep, choice of the
fastest, state restored, JSON cache reuse."""

import numpy as np

from paper_2305_04180_gb300.autotune import CANDIDATES, autotune_rollout


class FakeSim:
    def __init__(self):
        self.device = 0
        self.n, self.obs_dim, self.n_maps = 10, 37, 2
        self.env_beams = np.full(10, 32, np.int32)
        self.map_shapes = [(366, 366), (128, 128)]
        self.env_map_host = np.arange(10, dtype=np.int32) % 2
        self.launch = None
        self.state = ("s0",)
        self.set_calls = 0

    def set_launch(self, **kw):
        self.launch = kw

    def get_state(self):
        return self.state

    def set_state(self, *s):
        self.set_calls += 1


def test_sweep_picks_fastest_and_caches(tmp_path):
    sim = FakeSim()
    key = lambda c: tuple(sorted(c.items()))  # noqa: E731
    fake_ms = {key(c): 10.0 + i for i, c in enumerate(CANDIDATES)}
    best = CANDIDATES[7]
    fake_ms[key(best)] = 1.0

    def timer(s, cfg, K, reps, state):
        return fake_ms[key(cfg)]

    path = str(tmp_path / "c.json")
    r = autotune_rollout(sim, K=16, cache_path=path, timer=timer)
    assert r["config"] == best
    assert sim.launch == best and sim.set_calls >= 1
    r2 = autotune_rollout(sim, K=16, cache_path=path, timer=lambda *a: 1 / 0)
    assert r2["cached"] and r2["config"] == r["config"]
    # another rollout length is another cache entry
    r3 = autotune_rollout(sim, K=32, cache_path=path, timer=timer)
    assert not r3["cached"]
