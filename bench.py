#!/usr/bin/env python
"""Throughput of the vectorized Sparrow step on GB300: env-steps/s.

Default workload: 1,024 envs over 32 seeded 366x366 maps with every
per-episode randomisation on (control interval, delay, K, velocity cap, LiDAR
noise), 32 beams, uniformly random actions; one bench step is one
``sg_sim_rollout`` of 10,000 vectorized steps (10.24 M env-steps).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
this host's cores instead (the reference arm of this build).

Timing: W untimed warm-up steps, then K timed steps, each bracketed by CUDA
events on the launching stream; a 256 MiB buffer is written between timed
steps (outside the events) to flush the 126 MiB L2.  Barrier + synchronize
on both sides of the timed loop; the max over ranks is reported.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "env-steps/s on 1 GB300 (plain sim vs fused Q-net rollout); % of L2/HBM roofline"
UNIT = "env-steps/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dr1024")
    ap.add_argument("--rollout-steps", type=int, default=None, help="vectorized steps per bench step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------ CPU oracle
def _oracle_shard(args):
    """Worker: run envs [i0, i1) of the workload on the CPU oracle."""
    name, i0, i1, K, t0 = args
    from oracle.sim import OracleSim
    from workloads import workload

    w = workload(name)
    o = OracleSim(w.params, w.maps(), w.env_map, w.env_beams, prec="f32")
    for i in range(i0, i1):
        o.reset_env(i, 0)
    o.L.orc_reset_march_samples()
    t = time.perf_counter()
    o.rollout_random_range(i0, i1, K, t0)
    dt = time.perf_counter() - t
    return (i1 - i0) * K, dt, int(o.L.orc_march_samples())


def oracle_pool(cores):
    import multiprocessing as mp

    return mp.get_context("spawn").Pool(cores)


def time_oracle(pool, cores, name, n_envs, K):
    """Env-steps/s of the oracle over all n_envs envs for K steps, sharded by
    env over `cores` processes (envs are independent).  Wall time of the
    slowest shard counts."""
    per = math.ceil(n_envs / cores)
    jobs = [(name, i, min(n_envs, i + per), K, 0) for i in range(0, n_envs, per)]
    t = time.perf_counter()
    res = pool.map(_oracle_shard, jobs)
    wall = time.perf_counter() - t
    steps = sum(r[0] for r in res)
    samples = sum(r[2] for r in res)
    busy = max(r[1] for r in res)
    return steps, wall, busy, samples


# ------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ our arm
def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2305_04180_gb300 import Sim
    from workloads import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and not a.no_cpu_baseline:
        pool = oracle_pool(cores)  # spawned before the first GPU call
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = workload(a.workload)
    K = a.rollout_steps or w.steps
    maps = w.maps()
    sim = Sim(w.params, maps, w.env_map, w.env_beams)
    n = sim.n
    sim.reset(seed=w.params["seed"] + 7919 * rank)
    obs = sim.new_obs()
    obs_seq = torch.empty((K, n, sim.obs_dim), dtype=torch.float32, device="cuda")
    rew_seq = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done_seq = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step():
        sim.rollout(K, obs=obs, obs_seq=obs_seq, rew_seq=rew_seq, done_seq=done_seq, stream=stream)

    for _ in range(a.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.25)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall0 = time.perf_counter()
    for i in range(a.steps):
        flush.zero_()
        ev[i][0].record(stream)
        one_step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    tot_ms = sum(ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    env_steps = n * K * a.steps * world
    value = env_steps / (tot_ms / 1e3)
    ms_per_step = tot_ms / a.steps
    st = sim.status()

    # ---- end to end through the public API with host buffers ---------------
    # per step: upload the start state from pinned host memory (sg_sim_set_state),
    # roll out K steps, read the per-step rewards and done flags back to pinned
    # host memory.
    f0, u0 = sim.get_state()
    rew_h = torch.empty((K, n), dtype=torch.float32, pin_memory=True)
    done_h = torch.empty((K, n), dtype=torch.uint8, pin_memory=True)
    e2e_steps = max(2, min(a.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(f0, u0)
        one_step()
        rew_h.copy_(rew_seq, non_blocking=True)
        done_h.copy_(done_seq, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = int(f0.nbytes + u0.nbytes)
    d2h = int(rew_h.numel() * 4 + done_h.numel())

    out = None
    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": a.steps,
            "warmup": a.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded maps: border + 20 rectangles + 10 discs per map)",
            "config": {
                "workload": w.name,
                "n_envs": n,
                "maps": len(maps),
                "rollout_steps_per_bench_step": K,
                "env_steps_per_bench_step": n * K,
                "policy": "random (on-device counter RNG)",
                "outputs_per_env_step": "observation (obs_dim floats), reward, done flags",
                "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                "parallelism": "replicas" if world > 1 else "single GPU",
            },
            "e2e": {"value": n * K * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": a.steps,
            "clocks": clk,
            "wall_s": wall,
            "device_status": st,
            "step_ms": ms,
        }
    return out, pool, (w, n, K, ms_per_step, clk)


def roofline_alu(samples_per_env_step, n, K, ms_per_step, clk):
    """March samples of the step definition per second against the lane-issue
    bound of the SMs (see DESIGN: 152 SMs x 128 lanes x SM clock / 8 lane
    instructions per sample)."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = 152 * 128 * mhz * 1e6 / 8.0 / 1e9  # Gsample/s
    achieved = samples_per_env_step * n * K / (ms_per_step / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gsample/s",
            "frac": achieved / peak, "traffic": None,
            "peak_basis": f"152 SM x 128 lanes x {mhz:.0f} MHz (median under load) / 8 instr per sample"}


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    out, pool, (w, n, K, ms_per_step, clk) = run_ours(a)
    if out is None:
        return
    cores = os.cpu_count() or 1
    samples_per_env_step = None
    if pool is not None:
        steps, wall, busy, samples = time_oracle(pool, cores, a.workload, n, 1000)
        samples_per_env_step = samples / steps
        out["cpu_baseline"] = {"value": steps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{n} envs x 1000 steps of the same workload (f32 oracle, "
                                         f"{cores} spawned processes sharded by env)",
                               "wall_s": wall}
        pool.close()
    if samples_per_env_step is None:
        samples_per_env_step = 1500.0
    out["roofline"] = roofline_alu(samples_per_env_step, n, K, ms_per_step, clk)
    out["roofline"]["samples_per_env_step"] = samples_per_env_step
    print(json.dumps(out))


# ------------------------------------------------------------ reference arm
def run_reference(a):
    """The CPU oracle on this host's cores: each bench step rolls all envs of
    the workload for a bounded number of steps."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import workload

    w = workload(a.workload)
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores)
    per_step = 100  # vectorized steps per bench step (bounded sample)
    for _ in range(a.warmup):
        time_oracle(pool, cores, a.workload, w.n_envs, per_step // 10 or 1)
    tot = 0.0
    steps = 0
    for _ in range(a.steps):
        s, wall, _, _ = time_oracle(pool, cores, a.workload, w.n_envs, per_step)
        tot += wall
        steps += s
    pool.close()
    v = steps / tot
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n_envs": w.n_envs, "rollout_steps_per_bench_step": per_step},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{w.n_envs} envs x {per_step} steps per bench step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
