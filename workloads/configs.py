"""The five synthetic workloads of the vectorized Sparrow step.

Each workload is a plain description: env count, which seeded map each env
uses, beams per env, the randomisation ranges of the per-episode parameters
(Sec. 3.2.4 "vectorized diversity"; nominal values from the paper's simulation
parameter table), rollout length and policy.  The numbers for the nominal
robot come from the paper: K = 0.6, control interval 0.1 s, maximal linear
velocity 18 cm/s, maximal angular velocity 1 rad/s (simulation-parameter
table), and the 5-action table of Sec. 4.3.1.  One cell is read as 1 cm.

Nothing here computes any part of the step: these are inputs.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .maps import make_map

# Target (linear cm/s, angular rad/s) per discrete action, Sec. 4.3.1.
ACTION_TABLE = (
    (0.36, 1.0),   # turn left
    (18.0, 1.0),   # go straight and turn left
    (18.0, 0.0),   # go straight
    (18.0, -1.0),  # go straight and turn right
    (0.36, -1.0),  # turn right
)


def base_params(**overrides) -> dict:
    """Simulation parameters shared by the oracle and the CUDA path.

    All lengths are in cells (1 cell = 1 cm), angles in radians, times in
    seconds.  ``*_lo``/``*_hi`` are the uniform ranges re-drawn at every
    episode start; lo == hi disables that randomisation.
    """
    p = dict(
        n_beams=32,
        fov=float(np.float32(1.5 * math.pi)),  # 270 degree fan
        range_max=100.0,
        march_step=1.0,
        robot_radius=10.0,
        goal_radius=20.0,
        near_dist=30.0,          # r_d = -1 below this obstacle distance
        t_max=2000,
        start_offset=30.0,
        start_jitter=5.0,
        dt_lo=0.1, dt_hi=0.1,
        k_lo=0.6, k_hi=0.6,
        cap_lo=1.0, cap_hi=1.0,
        sigma_lo=0.0, sigma_hi=0.0,
        delay_lo=0, delay_hi=0,
        v_nom=18.0,
        w_nom=1.0,
        actions=ACTION_TABLE,
        seed=42,
    )
    p.update(overrides)
    return p


# Domain randomisation of the "Color" setup (Sec. 4.3.2): control interval,
# control delay, velocity range, K and sensor-noise magnitude per episode.
DR_RANGES = dict(
    dt_lo=0.05, dt_hi=0.2,
    delay_lo=0, delay_hi=2,
    k_lo=0.6, k_hi=1.0,
    cap_lo=0.5, cap_hi=1.5,
    sigma_lo=0.0, sigma_hi=2.0,
)


# Moving obstacles (the extension the paper's Sec. 5 names as future work):
# four discs of radius 8 cm per env, 4..30 cm/s (the robot's nominal top
# speed is 18 cm/s), none starting within 60 cm of S or G.
DYN_RANGES = dict(n_dyn=4, dyn_radius=8.0, dyn_speed_lo=4.0, dyn_speed_hi=30.0, dyn_keepout=60.0)


@dataclass
class Workload:
    name: str
    n_envs: int
    map_specs: list            # list of (seed, side)
    env_map: np.ndarray        # int32 [n_envs]
    env_beams: np.ndarray | None  # int32 [n_envs] or None (all n_beams)
    params: dict
    steps: int
    policy: str                # "random" or "eps_q"
    eps: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    def maps(self):
        return [make_map(s, side) for (s, side) in self.map_specs]


def _eps_linear(n, lo, hi):
    """VEM exploration noise linearly spaced over env index (Sec. 3.1.1)."""
    if n == 1:
        return np.array([lo], dtype=np.float32)
    i = np.arange(n, dtype=np.float64)
    return (lo + (hi - lo) * i / (n - 1)).astype(np.float32)


def workload(name: str, n_envs: int | None = None, steps: int | None = None) -> Workload:
    """Build a workload by name, optionally shrinking env count / steps.

    Shrinking keeps every other property (map recipe, randomisation, beams)
    so that a small case exercises the same code paths as the full one.
    """
    if name == "plain16":
        n = n_envs or 16
        return Workload(
            name="plain sim, 16 envs, one 366x366 map, 32 beams, 1000 steps",
            n_envs=n, map_specs=[(1, 366)],
            env_map=np.zeros(n, np.int32), env_beams=None,
            params=base_params(), steps=steps or 1000, policy="random")
    if name == "dr1024":
        n = n_envs or 1024
        n_maps = min(32, n)
        return Workload(
            name="domain-randomized sim, 1024 envs over 32 maps 366x366, 32 beams, 10000 steps",
            n_envs=n, map_specs=[(1 + m, 366) for m in range(n_maps)],
            env_map=(np.arange(n) % n_maps).astype(np.int32), env_beams=None,
            params=base_params(**DR_RANGES), steps=steps or 10000, policy="random")
    if name == "dyn1024":
        n = n_envs or 1024
        n_maps = min(32, n)
        return Workload(
            name="domain-randomized sim with 4 moving obstacles per env, 1024 envs over 32 maps 366x366, 32 beams",
            n_envs=n, map_specs=[(1 + m, 366) for m in range(n_maps)],
            env_map=(np.arange(n) % n_maps).astype(np.int32), env_beams=None,
            params=base_params(**DR_RANGES, **DYN_RANGES), steps=steps or 10000, policy="random")
    if name == "uneven8192":
        n = n_envs or 8192
        rng = np.random.default_rng(3)
        sides = rng.choice([128, 256, 366, 512, 1024], size=n)
        beams = rng.choice([16, 32, 64], size=n).astype(np.int32)
        return Workload(
            name="uneven batching, 8192 envs, one map per env side in {128..1024}, beams in {16,32,64}, 64-step rollouts",
            n_envs=n, map_specs=[(1000 + i, int(sides[i])) for i in range(n)],
            env_map=np.arange(n, dtype=np.int32), env_beams=beams,
            params=base_params(n_beams=64), steps=steps or 64, policy="random")
    if name == "qnet4096":
        n = n_envs or 4096
        n_maps = min(32, n)
        return Workload(
            name="fused Q-net rollout, 4096 envs over 32 maps 366x366, 32 beams, eps-greedy",
            n_envs=n, map_specs=[(1 + m, 366) for m in range(n_maps)],
            env_map=(np.arange(n) % n_maps).astype(np.int32), env_beams=None,
            params=base_params(), steps=steps or 128, policy="eps_q",
            eps=_eps_linear(n, 0.01, 0.3),
            extra=dict(batch=256, ring=1 << 20, gamma=0.98, lr=1e-4, target_every=200))
    if name == "full65536":
        n = n_envs or 65536
        n_maps = min(1024, n)
        rng = np.random.default_rng(5)
        sides = rng.choice([256, 366, 512, 1024], size=n_maps)
        beams = rng.choice([16, 32, 64], size=n).astype(np.int32)
        return Workload(
            name="full learned loop, 65536 envs over 1024 maps, beams 16..64, DR, 128-step fused rollouts",
            n_envs=n, map_specs=[(5000 + m, int(sides[m])) for m in range(n_maps)],
            env_map=(np.arange(n) % n_maps).astype(np.int32), env_beams=beams,
            params=base_params(n_beams=64, **DR_RANGES), steps=steps or 128, policy="eps_q",
            eps=_eps_linear(n, 0.01, 0.3),
            extra=dict(batch=4096, ring=1 << 22, gamma=0.98, lr=1e-4, target_every=200))
    raise KeyError(name)


WORKLOADS = ("plain16", "dr1024", "uneven8192", "qnet4096", "full65536", "dyn1024")
