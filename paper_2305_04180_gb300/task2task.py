"""Task2Task generalisation (Sec. 4.3.2, "Task2Task generalization"): Grey
against Color, both trained with the ASL loop, evaluated by the target-area
arrival rate on held-out maps.

* Grey: every env uses the nominal simulation parameters (K 0.6, control
  interval 0.1 s, no delay, nominal velocity range, no sensor noise) and the
  same training map (Map0 x N).
* Color: control interval, control delay, velocity range, K and sensor-noise
  magnitude are re-drawn from intervals around the nominal values at every
  episode start, and the N envs spread over N training maps (Map0..Map15 for
  N = 16).
* Evaluation: greedy policy (no exploration), nominal parameters, a number
  of envs per held-out map (Map16..Map31 in the paper; here seeded synthetic
  maps that no training env sees); each env's first episode counts:
  arrival rate = arrived episodes / episodes (collision and truncation end
  the others).

The maps are the seeded synthetic grids of ``workloads.maps``; the network is
this library's dueling MLP or (``--arch paper --beams 27``) the paper's own
[32, 256, 128, 5] network on a 27-beam robot.  Run as a script for a JSON line
per setup: ``python -m paper_2305_04180_gb300.task2task --transitions 500000``.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from .sim import Sim
from .trainer import ColorTrainer

# Uniform intervals of the Color setup around the nominal values (the
# paper's "moderate interval around the initial values")
COLOR_RANGES = dict(dt_lo=0.05, dt_hi=0.2, delay_lo=0, delay_hi=2, k_lo=0.6, k_hi=1.0, cap_lo=0.5, cap_hi=1.5,
                    sigma_lo=0.0, sigma_hi=2.0)
TRAIN_SEEDS = tuple(range(1, 17))      # Map0..Map15
TEST_SEEDS = tuple(range(1001, 1017))  # held-out maps


def _maps(seeds):
    from workloads.maps import make_map

    return [make_map(s) for s in seeds]


def _params(**overrides):
    from workloads.configs import base_params

    return base_params(**overrides)


def make_setup(kind: str, n_envs: int = 16, seed: int = 0, beams: int = 32) -> Sim:
    """The training simulator of the Grey or the Color setup (beams: LiDAR
    beams; the paper's robot has 27, a 32-entry state)."""
    if kind == "grey":
        maps = _maps(TRAIN_SEEDS[:1])
        env_map = np.zeros(n_envs, np.int32)
        p = _params(seed=seed, n_beams=beams)
    elif kind == "color":
        maps = _maps(TRAIN_SEEDS)
        env_map = (np.arange(n_envs) % len(maps)).astype(np.int32)
        p = _params(seed=seed, n_beams=beams, **COLOR_RANGES)
    else:
        raise ValueError(f"unknown setup {kind!r}")
    sim = Sim(p, maps, env_map)
    sim.reset()
    return sim


def evaluate(qnet, seeds=TEST_SEEDS, envs_per_map: int = 8, max_steps: int = 2000, seed: int = 12345,
             chunk: int = 250, beams: int = 32) -> dict:
    """Greedy arrival rate of qnet on the maps of `seeds` with nominal
    parameters: envs_per_map envs per map, each env's first episode."""
    maps = _maps(seeds)
    n = len(maps) * envs_per_map
    sim = Sim(_params(seed=seed, n_beams=beams), maps, (np.arange(n) % len(maps)).astype(np.int32))
    sim.reset()
    eps = torch.zeros(n, device=sim.device)
    done = torch.empty((chunk, n), dtype=torch.uint8, device=sim.device)
    outcome = np.zeros(n, np.uint8)
    steps = 0
    while steps < max_steps + 1 and not outcome.all():
        k = min(chunk, max_steps + 1 - steps)
        sim.rollout(k, policy="eps_q", qnet=qnet, eps=eps, done_seq=done[:k])
        d = done[:k].cpu().numpy()
        for i in np.flatnonzero(outcome == 0):
            hit = np.flatnonzero(d[:, i])
            if hit.size:
                outcome[i] = d[hit[0], i]
        steps += k
    col = (outcome & 1) != 0
    arr = ((outcome & 2) != 0) & ~col  # a collision in the arrival step counts as a collision
    trn = ((outcome & 4) != 0) & ~col & ~arr
    episodes = int((outcome != 0).sum())
    return dict(maps=len(maps), episodes=episodes, arrive=int(arr.sum()), collide=int(col.sum()),
                truncate=int(trn.sum()), arrival_rate=float(arr.sum()) / max(1, episodes))


def train_and_evaluate(kind: str, transitions: int, n_envs: int = 16, seed: int = 0, tps: int = 256,
                       batch: int = 256, rollout_k: int = 8, eval_envs_per_map: int = 8, arch: str = "dueling",
                       beams: int = 32) -> dict:
    """Train one setup with the ASL loop (the paper's Sparrow hyper-parameters:
    TPS 256, batch 256, learning start 30K transitions, lr 1e-4, gamma 0.98,
    target update 200, upload every 50, VEM with OR N -> 3N/16 over 500K)
    for `transitions` interacting steps; evaluate on the training maps and
    on the held-out maps."""
    sim = make_setup(kind, n_envs, seed, beams)
    tr = ColorTrainer(sim, batch=batch, slots=max(64, 1_000_000 // n_envs), tps=tps, learn_start=30_000, lr=1e-4,
                      gamma=0.98, target_every=200, upload_every=50, seed=seed, two_streams=True,
                      max_rollout_k=rollout_k, arch=arch)
    t0 = time.perf_counter()
    tr.run(max(1, transitions // n_envs), rollout_k=rollout_k)
    train_s = time.perf_counter() - t0
    train_seeds = TRAIN_SEEDS[:1] if kind == "grey" else TRAIN_SEEDS
    return dict(setup=kind, seed=seed, n_envs=n_envs, arch=arch, beams=beams, transitions=tr.transitions,
                updates=tr.updates, train_seconds=train_s, tfm=tr.tfm_report(),
                train_maps=evaluate(tr.learner, train_seeds, eval_envs_per_map, beams=beams),
                test_maps=evaluate(tr.learner, TEST_SEEDS, eval_envs_per_map, beams=beams))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--transitions", type=int, default=500_000)
    ap.add_argument("--seeds", type=int, default=1)
    ap.add_argument("--envs", type=int, default=16)
    ap.add_argument("--arch", default="dueling", choices=["dueling", "paper"],
                    help="Q-network: dueling 256-256, or the paper's [32, 256, 128, 5]")
    ap.add_argument("--beams", type=int, default=32, help="LiDAR beams (the paper's robot: 27)")
    a = ap.parse_args(argv)
    for seed in range(a.seeds):
        for kind in ("grey", "color"):
            print(json.dumps(train_and_evaluate(kind, a.transitions, a.envs, seed, arch=a.arch, beams=a.beams)),
                  flush=True)


if __name__ == "__main__":
    main()
