"""The debug build of the library (SG_DEBUG_BOUNDS: every skip-map load of
the march, every bit-row load of the collision test and every ring entry the
learner samples is checked against its array and would report SG_DEV_BOUNDS
instead of reading outside it).  On tiny and degenerate maps, uneven beams,
every rollout launch, the fused Q rollout and a TD step, the debug build must
give the float32 oracle's results bit for bit with no bounds report.  It runs
in a child process, because the library variant is chosen once per process
(SG_LIB_VARIANT=debug)."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_matches_oracle_without_bounds_reports():
    env = dict(os.environ, SG_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", "import tests.test_debug_bounds as t; t.child()"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "DEBUG_BUILD_OK" in r.stdout


def child():
    import torch

    from oracle import qnet as OQ
    from oracle.sim import OracleSim
    from paper_2305_04180_gb300 import QNet, Replay, Sim, _lib
    from tests._helpers import bits, gpu_state_to_oracle
    from workloads import workload
    from workloads.configs import base_params
    from workloads.maps import empty_map, make_map, random_tiny_map

    L = _lib.load()
    assert L._name.endswith("libsparrowgb_debug.so"), L._name

    def teacher_forced(p, maps, env_map, beams=None, steps=40, seed=0):
        g = Sim(p, maps, env_map, beams)
        o = OracleSim(p, maps, env_map, beams, prec="f32")
        g.reset()
        o.reset()
        rng = np.random.default_rng(seed)
        for t in range(steps):
            a = rng.integers(0, 5, size=g.n).astype(np.uint8)
            f, u = g.get_state()
            o.set_state(*gpu_state_to_oracle(f, u))
            obs, rew, done = g.step(torch.from_numpy(a).cuda())
            oobs, orew, odone, _ = o.step(a)
            assert np.array_equal(done.cpu().numpy(), odone), t
            assert np.array_equal(bits(rew.cpu().numpy()), bits(orew)), t
            assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs)), t
        assert g.status() == 0, "bounds report"
        return g

    dr = {k: v for k, v in workload("dr1024").params.items() if k.endswith(("_lo", "_hi"))}
    p = base_params(n_beams=64, **dr)
    rng = np.random.default_rng(1)
    # tiny, degenerate and mixed maps; beams 2..64; both skip structures
    for sectors in (1, 16):
        q = dict(p, march_sectors=sectors)
        for maps in ([random_tiny_map(7, 20, 20, 0.1)], [np.ones((1, 1), np.uint8)], [empty_map(400)],
                     [random_tiny_map(8, 37, 5, 0.3), random_tiny_map(9, 8, 8, 0.2), make_map(3, 128)]):
            n = 23
            env_map = rng.integers(0, len(maps), n).astype(np.int32)
            beams = rng.choice([2, 3, 16, 32, 33, 64], n).astype(np.int32)
            teacher_forced(q, maps, env_map, beams, steps=30, seed=sectors)
    # every rollout launch of the network-free policy, on the 1,024-env workload's maps
    w = workload("dr1024", n_envs=64)
    maps = w.maps()
    for launch in (dict(kernel="grid"), dict(kernel="queue", warps_per_block=4, order="cost"),
                   dict(kernel="split", warps_per_block=8, warps_per_env=2),
                   dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=64)):
        g = Sim(w.params, maps, w.env_map)
        g.set_launch(**launch)
        g.reset()
        rew = torch.empty((200, g.n), device="cuda")
        g.rollout(200, rew_seq=rew)
        o = OracleSim(w.params, maps, w.env_map, prec="f32")
        o.reset()
        orew = np.stack([o.step(o.random_actions(t))[1] for t in range(200)])
        assert np.array_equal(bits(rew.cpu().numpy()), bits(orew)), launch
        assert g.status() == 0, launch
    # the fused Q rollout into a ring, and a TD step sampling from it
    w = workload("qnet4096", n_envs=200)
    g = Sim(w.params, w.maps(), w.env_map)
    qn = QNet(g.obs_dim, 256, seed=3)
    th = (OQ.flatten(OQ.init_params(5, g.obs_dim)) * 2.0).astype(np.float32)
    qn.set_params(th)
    rp = Replay(16, g.n, g.obs_dim)
    g.reset()
    for rows in (16, 128):
        qn.set_rollout_rows(rows)
        g.rollout(20, policy="eps_q", qnet=qn, eps=torch.from_numpy(w.eps).cuda(), replay=rp)
    loss = torch.zeros(1, device="cuda")
    qn.train_step(rp, 256, lr=1e-4, seed=1, loss=loss)
    torch.cuda.synchronize()
    assert np.isfinite(loss.item())
    assert g.status() == 0
    print("DEBUG_BUILD_OK")
