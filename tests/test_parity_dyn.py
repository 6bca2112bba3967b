"""GPU parity of the moving-obstacle extension against the strict-float32
oracle (through the C ABI): reset, the lane-per-env step, the one-warp-per-env,
work-list and pipelined rollouts and the fused Q-network rollout, all bit-exact in
observations, rewards, done flags, terminal observations and the whole state
including the discs.  The split rollout refuses obstacles.
"""

import numpy as np
import pytest
import torch

from oracle.sim import OracleSim
from tests._helpers import bits, gpu_state_to_oracle, oracle_state_to_gpu
from workloads import workload
from workloads.configs import DR_RANGES, base_params
from workloads.maps import make_map, random_tiny_map

pytestmark = pytest.mark.gpu


def _pair(params, maps, env_map, env_beams=None):
    from paper_2305_04180_gb300 import Sim

    g = Sim(params, maps, env_map, env_beams)
    o = OracleSim(params, maps, env_map, env_beams, prec="f32")
    return g, o


def _w_pair(name="dyn1024", n=None):
    w = workload(name, n_envs=n)
    maps = w.maps()
    return (*_pair(w.params, maps, w.env_map, w.env_beams), w)


def _assert_state_equal(g, o, t):
    f, u, d = g.get_state()
    of, ou, ob, od = o.state()
    gf, gu = oracle_state_to_gpu(of, ou, ob, t)
    assert np.array_equal(bits(f), bits(gf)), np.argwhere(bits(f) != bits(gf))[:5]
    assert np.array_equal(u, gu), np.argwhere(u != gu)[:5]
    assert np.array_equal(bits(d), bits(od)), np.argwhere(bits(d) != bits(od))[:5]


@pytest.mark.parametrize("n", [1024, 37])
def test_reset_bit_exact_with_obstacles(n):
    g, o, _ = _w_pair(n=n)
    obs = g.reset().cpu().numpy()
    oobs = o.reset()
    assert np.array_equal(bits(obs), bits(oobs))
    _assert_state_equal(g, o, 0)


def _teacher_forced(g, o, steps, seed=0):
    n = g.n
    g.reset()
    o.reset()
    term = torch.full((n, g.obs_dim), float("nan"), device="cuda")
    rng = np.random.default_rng(seed)
    n_done = n_col = 0
    for t in range(steps):
        a = rng.integers(0, 5, size=n).astype(np.uint8)
        o.set_state(*gpu_state_to_oracle(*g.get_state()))
        obs, rew, done = g.step(torch.from_numpy(a).cuda(), term_obs=term)
        oobs, orew, odone, oterm = o.step(a)
        d = done.cpu().numpy()
        assert np.array_equal(d, odone), (t, np.argwhere(d != odone)[:5])
        assert np.array_equal(bits(rew.cpu().numpy()), bits(orew)), t
        assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs)), t
        if d.any():
            tg = term.cpu().numpy()[d != 0]
            assert np.array_equal(bits(tg), bits(oterm[d != 0])), t
        _assert_state_equal(g, o, t + 1)
        n_done += int((d != 0).sum())
        n_col += int((d & 1).sum())
    return n_done, n_col


def test_step_teacher_forced_with_obstacles():
    """1024 envs, 4 discs each, every randomisation on: 300 steps
    (307,200 env-steps), each teacher-forced from the GPU's state."""
    g, o, _ = _w_pair()
    n_done, n_col = _teacher_forced(g, o, 300, seed=1)
    assert n_col > 100


def test_step_fast_crowded_obstacles_small_maps():
    """Eight large, fast discs (up to 40 cells per step: mirrored and clamped
    at the walls, stopped at occupied cells), uneven beams, a march step
    below one cell, tiny and mid-sized maps, N not a multiple of a CTA."""
    p = base_params(n_beams=64, march_step=0.37, range_max=60.0, n_dyn=8, dyn_radius=12.0, dyn_speed_lo=50.0,
                    dyn_speed_hi=400.0, dyn_keepout=20.0, **DR_RANGES)
    maps = [make_map(21, 128), random_tiny_map(22, 60, 60, 0.15), make_map(23, 200, 90)]
    n = 45
    rng = np.random.default_rng(4)
    env_map = rng.integers(0, 3, n).astype(np.int32)
    beams = rng.choice([2, 16, 33, 64], n).astype(np.int32)
    g, o = _pair(p, maps, env_map, beams)
    n_done, n_col = _teacher_forced(g, o, 150, seed=5)
    assert n_col > 50


@pytest.mark.parametrize("launch", [dict(kernel="grid", warps_per_block=4),
                                    dict(kernel="queue", warps_per_block=8, order="cost"),
                                    dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"),
                                    dict(kernel="pipe", warps_per_block=16, obs_warps=7, order="map", segment=64)])
def test_rollout_free_running_with_obstacles(launch):
    """400 free-running steps with on-device random actions: every step's
    action, reward, done flags and observation, and the final state, equal
    the oracle's."""
    g, o, _ = _w_pair(n=96)
    g.set_launch(**launch)
    g.reset()
    o.reset()
    K, n = 400, g.n
    obs = g.new_obs()
    obs_seq = torch.empty((K, n, g.obs_dim), dtype=torch.float32, device="cuda")
    act = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    g.rollout(K, obs=obs, obs_seq=obs_seq, act_seq=act, rew_seq=rew, done_seq=done)
    act, rew, done, obs_seq = act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), obs_seq.cpu().numpy()
    n_col = 0
    for k in range(K):
        a = o.random_actions(k)
        assert np.array_equal(act[k], a), k
        oobs, orew, odone, _ = o.step(a)
        assert np.array_equal(done[k], odone), k
        assert np.array_equal(bits(rew[k]), bits(orew)), k
        assert np.array_equal(bits(obs_seq[k]), bits(oobs)), k
        n_col += int((odone & 1).sum())
    assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs))
    _assert_state_equal(g, o, K)
    assert n_col > 20


@pytest.mark.parametrize("rows", [16, 32])
def test_q_rollout_with_obstacles(rows):
    """The fused eps-greedy Q-network rollout (both CTA shapes) with moving
    obstacles: the actions it chose, replayed on the oracle, give the same
    rewards, done flags, observations and final state bit for bit, and the
    transitions in the ring are the oracle's."""
    from paper_2305_04180_gb300 import QNet, Replay

    g, o, w = _w_pair(n=80)
    q = QNet(g.obs_dim, 256, seed=3)
    q.set_rollout_rows(rows)
    eps = torch.linspace(0.0, 0.5, g.n, device="cuda")
    rp = Replay(64, g.n, g.obs_dim)
    obs = g.reset()
    o.reset()
    prev = obs.cpu().numpy().copy()
    K, n = 50, g.n
    act = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    obs_seq = torch.empty((K, n, g.obs_dim), dtype=torch.float32, device="cuda")
    g.rollout(K, policy="eps_q", qnet=q, eps=eps, replay=rp, obs=obs, obs_seq=obs_seq, act_seq=act, rew_seq=rew,
              done_seq=done)
    act, rew, done, obs_seq = act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), obs_seq.cpu().numpy()
    for k in range(K):
        oobs, orew, odone, oterm = o.step(act[k])
        assert np.array_equal(done[k], odone), k
        assert np.array_equal(bits(rew[k]), bits(orew)), k
        assert np.array_equal(bits(obs_seq[k]), bits(oobs)), k
        s, s2, ra, rr, rt = rp.read(k * n, n)
        assert np.array_equal(ra, act[k]) and np.array_equal(bits(rr), bits(orew)), k
        expect_s2 = np.where((odone != 0)[:, None], oterm, oobs)
        assert np.array_equal(bits(s2), bits(expect_s2)), k
        assert np.array_equal(bits(s), bits(prev)), k
        prev = oobs
    _assert_state_equal(g, o, K)


def test_split_rollout_refuses_obstacles():
    from paper_2305_04180_gb300._lib import SgError

    g, _, _ = _w_pair(n=8)
    with pytest.raises(SgError):
        g.set_launch(kernel="split", warps_per_block=8, warps_per_env=2)
    assert g.launch_config()["kernel"] == "grid"


@pytest.mark.parametrize("cfg", [dict(warps_per_block=8, obs_warps=7),
                                 dict(warps_per_block=16, obs_warps=3, order="map", segment=32)])
def test_pipelined_rollout_with_obstacles_and_frequent_episode_ends(cfg):
    """The pipelined rollout's pose warp runs the discs ahead with the pose
    chain and restarts after every episode end inside a chunk: eight fast
    discs on small maps, truncation every 37 steps (scans of the pre-reset
    discs), collisions with discs and walls.  Every step's action, reward,
    done flags and observation and the final state equal the oracle's."""
    p = base_params(n_beams=32, t_max=37, n_dyn=8, dyn_radius=10.0, dyn_speed_lo=40.0, dyn_speed_hi=300.0,
                    dyn_keepout=15.0, **DR_RANGES)
    maps = [make_map(31, 128), random_tiny_map(32, 70, 70, 0.12), make_map(33, 256)]
    n = 48
    env_map = (np.arange(n) % 3).astype(np.int32)
    g, o = _pair(p, maps, env_map)
    g.set_launch(kernel="pipe", **cfg)
    g.reset()
    o.reset()
    K = 300
    obs = g.new_obs()
    obs_seq = torch.empty((K, n, g.obs_dim), dtype=torch.float32, device="cuda")
    act = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    g.rollout(K, obs=obs, obs_seq=obs_seq, act_seq=act, rew_seq=rew, done_seq=done)
    assert g.status() == 0
    act, rew, done, obs_seq = act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), obs_seq.cpu().numpy()
    kinds = np.zeros(3, int)
    for k in range(K):
        a = o.random_actions(k)
        assert np.array_equal(act[k], a), k
        oobs, orew, odone, _ = o.step(a)
        assert np.array_equal(done[k], odone), k
        assert np.array_equal(bits(rew[k]), bits(orew)), k
        assert np.array_equal(bits(obs_seq[k]), bits(oobs)), k
        kinds += [int(((odone & 1) != 0).sum()), int(((odone & 2) != 0).sum()), int((odone == 4).sum())]
    assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs))
    _assert_state_equal(g, o, K)
    assert kinds[0] > 50 and kinds[2] > 50


def test_checkpoint_resume_with_obstacles():
    """The state blob carries the discs: a run resumed from a checkpoint
    continues bit-identically."""
    g, _, _ = _w_pair(n=64)
    g.reset()
    g.rollout(60)
    st = g.get_state()
    assert len(st) == 3 and st[2].shape == (16, 64)
    ra = torch.empty((60, 64), device="cuda")
    rb = torch.empty((60, 64), device="cuda")
    g.rollout(60, rew_seq=ra)
    end_a = g.get_state()
    g.set_state(*st)
    g.rollout(60, rew_seq=rb)
    end_b = g.get_state()
    assert torch.equal(ra, rb)
    for x, y in zip(end_a, end_b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_zero_obstacles_is_the_plain_simulator():
    """n_dyn = 0 with the other obstacle fields set runs the plain kernels:
    the same bits as a configuration without them, and no disc state."""
    w = workload("dr1024", n_envs=64)
    maps = w.maps()
    from paper_2305_04180_gb300 import Sim

    a = Sim(w.params, maps, w.env_map)
    b = Sim(dict(w.params, n_dyn=0, dyn_radius=8.0, dyn_speed_lo=1.0, dyn_speed_hi=2.0, dyn_keepout=5.0), maps,
            w.env_map)
    for s in (a, b):
        s.reset()
    ra = torch.empty((100, 64), device="cuda")
    rb = torch.empty((100, 64), device="cuda")
    a.rollout(100, rew_seq=ra)
    b.rollout(100, rew_seq=rb)
    assert torch.equal(ra, rb)
    assert len(b.get_state()) == 2 and b.info.state_bytes == a.info.state_bytes
