"""Autotuner of the network-free rollout's launch configuration.

For a given simulator it times every candidate (kernel variant: one warp
per env, persistent work-list grid, warps sharing an env, pose/observation
pipelines with and without time slicing; envs per CTA and warps per env) on
rollouts of the requested length, restoring the env state after each trial,
and applies the fastest.
Results are cached as JSON per (device, workload signature, rollout length),
so later runs of the same workload reuse them without timing.  The choice
never changes the results, only their speed.
"""

from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

def _cand(kernel, **kw):
    d = dict(kernel=kernel, warps_per_block=4, warps_per_env=1, obs_warps=0, blocks_per_sm=0, order="index",
             segment=0)
    d.update(kw)
    return d


CANDIDATES = ([_cand("grid", warps_per_block=w) for w in (2, 4, 8)]
              + [_cand("queue", warps_per_block=w, order=o) for w in (2, 4, 8) for o in ("index", "cost")]
              + [_cand("split", warps_per_block=8, warps_per_env=W) for W in (2, 3, 4)]
              + [_cand("pipe", warps_per_block=b, obs_warps=P, order=o)
                 for P, b, o in ((7, 8, "map"), (7, 16, "map"), (7, 16, "index"), (3, 8, "map"), (3, 4, "map"),
                                 (5, 12, "map"), (15, 16, "map"))]
              + [_cand("pipe", warps_per_block=8, obs_warps=7, order="map", segment=S) for S in (256, 512, 1024, 2048)]
              + [_cand("pipe", warps_per_block=16, obs_warps=7, order="map", segment=S) for S in (512, 1024, 2048)])
KEYS = ("kernel", "warps_per_block", "warps_per_env", "obs_warps", "blocks_per_sm", "order", "segment")
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _device_name(sim) -> str:
    try:
        return torch.cuda.get_device_name(sim.device)
    except Exception:
        return "unknown"


def signature(sim, K: int) -> str:
    """Cache key: device name, env count, per-env beams, map sizes, env->map, K."""
    h = hashlib.sha1()
    h.update(_device_name(sim).encode())
    h.update(str((sim.n, sim.obs_dim, sim.n_maps, int(K))).encode())
    h.update(np.asarray(sim.env_beams if sim.env_beams is not None else [], np.int32).tobytes())
    h.update(np.asarray(sim.map_shapes, np.int32).tobytes())
    h.update(np.asarray(sim.env_map_host, np.int32).tobytes())
    if getattr(sim, "n_dyn", 0):
        h.update(f"dyn{sim.n_dyn}".encode())
    return h.hexdigest()


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _apply(sim, cfg):
    sim.set_launch(**{k: cfg[k] for k in KEYS})


def _time_config(sim, cfg, K, reps, state):
    _apply(sim, cfg)
    times = []
    for _ in range(reps + 1):
        sim.set_state(*state)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.rollout(K)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times[1:]))


def autotune_rollout(sim, K: int = 32, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
                     candidates=None, timer=None) -> dict:
    """Pick and apply the fastest launch configuration for sim.rollout(K).

    Returns {"config": ..., "ms": ..., "table": [...], "cached": bool}.
    `timer(sim, cfg, K, reps, state) -> ms` may replace the CUDA-event timer.
    """
    candidates = list(candidates or CANDIDATES)
    if getattr(sim, "n_dyn", 0):
        # the split launch replays the pose chain per warp without the discs
        candidates = [c for c in candidates if c["kernel"] != "split"]
    key = signature(sim, K)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        cfg = cache[key]["config"]
        _apply(sim, cfg)
        return dict(cache[key], cached=True)
    state = sim.get_state()
    timer = timer or _time_config
    table = []
    for cfg in candidates:
        ms = timer(sim, cfg, K, reps, state)
        table.append(dict(cfg, ms=ms))
    sim.set_state(*state)
    best = min(table, key=lambda r: r["ms"])
    cfg = {k: best[k] for k in KEYS}
    _apply(sim, cfg)
    result = {"config": cfg, "ms": best["ms"], "table": table}
    if cache_path:
        cache[key] = result
        save_cache(cache_path, cache)
    return dict(result, cached=False)
