"""Task2Task driver (Grey vs Color): the two training setups are what the
paper describes, and the arrival-rate evaluation accounts for every env's
first episode.  A short training run only; the comparison itself is an
experiment (numbers in the design notes), not a test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_setups_differ_as_described():
    from paper_2305_04180_gb300.task2task import COLOR_RANGES, make_setup

    g = make_setup("grey", 16, seed=1)
    c = make_setup("color", 16, seed=1)
    fg, _ = g.get_state()
    fc, _ = c.get_state()
    # rows 5..8: dt, K, cap, sigma
    assert np.all(fg[5] == np.float32(0.1)) and np.all(fg[6] == np.float32(0.6))
    assert np.all(fg[7] == 1.0) and np.all(fg[8] == 0.0)
    assert g.n_maps == 1 and np.all(np.asarray(g.env_map_host) == 0)
    assert c.n_maps == 16 and len(set(np.asarray(c.env_map_host).tolist())) == 16
    assert np.ptp(fc[5]) > 0 and np.ptp(fc[6]) > 0 and np.ptp(fc[7]) > 0 and np.ptp(fc[8]) > 0
    assert fc[5].min() >= COLOR_RANGES["dt_lo"] and fc[5].max() <= COLOR_RANGES["dt_hi"]


@pytest.mark.parametrize("arch,beams", [("dueling", 32), ("paper", 27)])
def test_short_training_and_evaluation_account_for_every_episode(arch, beams):
    """Also with the paper's robot and network: 27 beams (a 32-entry state)
    and the [32, 256, 128, 5] Q-network."""
    from paper_2305_04180_gb300.task2task import train_and_evaluate

    r = train_and_evaluate("color", 40_000, n_envs=16, seed=2, eval_envs_per_map=2, arch=arch, beams=beams)
    # 2,500 vectorized steps in chunks of 8; learning starts with the chunk
    # that reaches 30,000 transitions (the 235th, 128 transitions each), so
    # 2,500 - 8 x 234 = 628 steps train at rho = 16 x 256 / 256 = 16
    assert r["transitions"] == 40_000 and r["updates"] == 628 * 16
    for part in ("train_maps", "test_maps"):
        e = r[part]
        assert e["episodes"] == e["maps"] * 2
        assert e["arrive"] + e["collide"] + e["truncate"] == e["episodes"]
        assert 0.0 <= e["arrival_rate"] <= 1.0
    assert r["tfm"]["tps"] > 0 and r["tfm"]["v_period_ms"] > 0
