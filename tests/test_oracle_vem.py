"""Pins of the VEM exploration-noise oracle (oracle/vem.py) against what the
paper fixes: E_min for the first copy and E_min + E_max for the N-th while
the exploring interval spans all copies (Sec. 3.1.1), the exploiting interval
at E_min, the Sparrow schedule of the hyper-parameter table (N = 16, OR 16 ->
3 over 500K interacting steps, E_min 0.01, E_max 0.8), linear interpolation
inside the exploring interval."""

import numpy as np

from oracle.vem import or_at, vem_eps

SPARROW = dict(e_min=0.01, e_max=0.8, or_start=16, or_final=3, decay_steps=500_000)


def test_full_exploring_interval_is_the_linear_ramp():
    e = vem_eps(16, 0, **SPARROW)
    ref = np.linspace(0.01, 0.81, 16)
    assert np.allclose(e, ref, rtol=0, atol=2e-7)
    assert e[0] == np.float32(0.01) and e[-1] == np.float32(0.01 + 0.8)


def test_after_the_decay_three_copies_explore():
    # OR = 3: copies 13, 14, 15 ramp over E_min, E_min + E_max / 2, E_min + E_max
    for T in (500_000 // 16, 10**7):
        e = vem_eps(16, T, **SPARROW)
        assert np.all(e[:13] == np.float32(0.01))
        assert np.allclose(e[13:], [0.01, 0.41, 0.81], rtol=0, atol=2e-7)


def test_halfway_the_interval_is_half_shrunk():
    # 250K interacting steps: OR = 9.5, exploring interval starts at 6.5
    assert or_at(250_000, 16, 3, 500_000) == 9.5
    e = vem_eps(16, 250_000 // 16, **SPARROW)
    assert np.all(e[:7] == np.float32(0.01))
    for i in range(7, 16):
        assert abs(e[i] - (0.01 + 0.8 * (i - 6.5) / 8.5)) <= 2e-7
    assert e[-1] == np.float32(0.81)


def test_monotone_in_env_index_and_in_time():
    prev = None
    for T in range(0, 40_000, 997):
        e = vem_eps(64, T, 0.01, 0.8, 64, 12, 100_000)
        assert np.all(np.diff(e) >= 0) and e.min() >= np.float32(0.01) and e.max() <= np.float32(0.81)
        if prev is not None:
            assert np.all(e <= prev)  # the exploring interval only shrinks
        prev = e
