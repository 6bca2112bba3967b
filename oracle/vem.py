"""Float64 oracle of the VEM exploration-noise schedule.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU legs use it.

Passage followed: Sec. 3.1.1 (vectorized data collection, the VEM figure and
its description) and the framework hyper-parameter table (E_min 0.01, E_max
0.8, OR 16 -> 3 over 500K interacting steps for Sparrow): the vectorized envs
split into an exploiting interval, whose envs use E_min, and an exploring
interval OR at the end of the index range, whose noise grows linearly from
E_min to E_min + E_max; OR shrinks linearly with the interacting steps.

Readings where the paper is silent (its figure is missing): OR is a real
number of envs, OR(T) = OR_start + (OR_final - OR_start) min(1, T / decay);
env i is in the exploring interval when i >= N - OR and then gets
E_min + E_max (i - (N - OR)) / (OR - 1), so with OR = N env 0 has E_min and
env N - 1 has E_min + E_max; T = N x (vectorized steps taken).
"""

from __future__ import annotations

import numpy as np


def or_at(T, or_start, or_final, decay_steps):
    """Size of the exploring interval after T interacting steps."""
    frac = min(1.0, float(T) / float(decay_steps))
    return float(or_start) + (float(or_final) - float(or_start)) * frac


def vem_eps(n, vec_steps, e_min, e_max, or_start, or_final, decay_steps):
    """Per-env exploration noise (float32) after vec_steps vectorized steps."""
    OR = or_at(float(n) * float(vec_steps), or_start, or_final, decay_steps)
    first = float(n) - OR
    out = np.empty(n, np.float32)
    for i in range(n):
        e = float(np.float32(e_min))
        if i >= first:
            e = float(np.float32(e_min)) + float(np.float32(e_max)) * ((i - first) / (OR - 1.0))
        out[i] = np.float32(e)
    return out
