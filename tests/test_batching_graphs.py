"""Uneven batching (per-env maps, beams and dynamics; persistent work-list
kernel), CUDA-graph replay of rollouts and of actor-learner iterations, and
the autotuner.  Launch configuration and graphs must never change results."""

import numpy as np
import pytest
import torch

from oracle.sim import OracleSim
from tests._helpers import bits
from workloads.configs import DR_RANGES, base_params
from workloads.maps import make_map

pytestmark = pytest.mark.gpu


def _uneven(n=96, seed=0):
    rng = np.random.default_rng(seed)
    sides = [128, 256, 366, 512]
    maps = [make_map(300 + m, sides[m % 4]) for m in range(12)]
    env_map = rng.integers(0, 12, n).astype(np.int32)
    beams = rng.choice([16, 32, 64], n).astype(np.int32)
    return base_params(n_beams=64, **DR_RANGES), maps, env_map, beams


def _run(sim, K):
    n = sim.n
    out = dict(obs_seq=torch.empty((K, n, sim.obs_dim), device="cuda"),
               rew=torch.empty((K, n), device="cuda"),
               done=torch.empty((K, n), dtype=torch.uint8, device="cuda"))
    sim.rollout(K, obs_seq=out["obs_seq"], rew_seq=out["rew"], done_seq=out["done"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_uneven_launch_configurations_agree_and_match_oracle():
    from paper_2305_04180_gb300 import Sim

    p, maps, env_map, beams = _uneven()
    K = 50
    results = []
    cfgs = (None, dict(kernel="queue", warps_per_block=8, order="cost"), dict(kernel="grid", warps_per_block=2),
            dict(kernel="queue", warps_per_block=16), dict(kernel="split", warps_per_block=8, warps_per_env=3),
            dict(kernel="split", warps_per_block=8, warps_per_env=8), dict(kernel="split", warps_per_block=4, warps_per_env=5),
            dict(kernel="pipe", warps_per_block=8, obs_warps=3), dict(kernel="pipe", warps_per_block=16, obs_warps=4),
            dict(kernel="pipe", warps_per_block=4, obs_warps=1), dict(kernel="pipe", warps_per_block=12, obs_warps=3, order="map"),
            dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"))
    for cfg in cfgs:
        s = Sim(p, maps, env_map, beams)
        if cfg:
            s.set_launch(**cfg)
            assert s.launch_config()["kernel"] == cfg["kernel"]
        s.reset()
        results.append((_run(s, K), s.get_state()))
    ref, (f0, u0) = results[0]
    for r, (f, u) in results[1:]:
        for k in ref:
            assert np.array_equal(bits(r[k]) if r[k].dtype == np.float32 else r[k],
                                  bits(ref[k]) if ref[k].dtype == np.float32 else ref[k]), k
        assert np.array_equal(bits(f), bits(f0)) and np.array_equal(u, u0)
    # sampled envs replayed on the oracle
    o = OracleSim(p, maps, env_map, beams, prec="f32")
    for i in (0, 5, 17, 42, 95):
        o.reset_env(i, 0)
        for k in range(K):
            obs, rew, done, _ = o.step_one(i, o.random_action(i, k))
            assert done == ref["done"][k, i] and bits(np.float32(rew)) == bits(ref["rew"][k, i])
            assert np.array_equal(bits(obs), bits(ref["obs_seq"][k, i]))


def test_pipelined_pose_chain_with_frequent_episode_ends():
    """Fast robots (dt up to 1 s), a short episode limit and a wide robot
    disc end episodes by collision, arrival and truncation several times per
    32-step chunk: the pipelined kernel's chunked pose chain (motion run ahead,
    steps tested together, restart after each episode end) must give the
    one-step-at-a-time results, and sampled envs must match the oracle."""
    from paper_2305_04180_gb300 import Sim

    rng = np.random.default_rng(7)
    sides = [128, 128, 256, 366]
    maps = [make_map(500 + m, sides[m % 4]) for m in range(8)]
    n = 40
    env_map = rng.integers(0, 8, n).astype(np.int32)
    beams = rng.choice([16, 32, 64], n).astype(np.int32)
    p = base_params(n_beams=64, **dict(DR_RANGES, dt_lo=0.2, dt_hi=1.0, cap_hi=2.0), t_max=9, robot_radius=12.0,
                    goal_radius=90.0)
    K = 100
    results = []
    for cfg in (None, dict(kernel="pipe", warps_per_block=16, obs_warps=7),
                dict(kernel="pipe", warps_per_block=8, obs_warps=3, order="map"),
                dict(kernel="pipe", warps_per_block=2, obs_warps=1)):
        s = Sim(p, maps, env_map, beams)
        if cfg:
            s.set_launch(**cfg)
        s.reset()
        results.append((_run(s, K), s.get_state()))
    ref, (f0, u0) = results[0]
    d = ref["done"]
    assert (d & 1).any() and (d & 2).any() and (d & 4).any()
    per_chunk = np.stack([(d[c:c + 32] != 0).sum(axis=0) for c in range(0, K, 32)])
    assert per_chunk.max() >= 3  # several restarts of the chain inside one chunk
    for r, (f, u) in results[1:]:
        for k in ref:
            assert np.array_equal(bits(r[k]) if r[k].dtype == np.float32 else r[k],
                                  bits(ref[k]) if ref[k].dtype == np.float32 else ref[k]), k
        assert np.array_equal(bits(f), bits(f0)) and np.array_equal(u, u0)
    o = OracleSim(p, maps, env_map, beams, prec="f32")
    for i in (0, 9, 23, 39):
        o.reset_env(i, 0)
        for k in range(K):
            obs, rew, done, _ = o.step_one(i, o.random_action(i, k))
            assert done == d[k, i] and bits(np.float32(rew)) == bits(ref["rew"][k, i]), (i, k)
            assert np.array_equal(bits(obs), bits(ref["obs_seq"][k, i])), (i, k)


@pytest.mark.parametrize("K", [1, 31, 32, 33, 64, 97])
def test_pipelined_rollout_lengths(K):
    """Rollouts of 1 to 4 chunks, full and ragged: the pipelined kernel's
    chunk hand-over (records written / consumed) gives the one-warp-per-env
    results and final state."""
    from paper_2305_04180_gb300 import Sim

    p, maps, env_map, beams = _uneven(50, seed=3)
    out = []
    for cfg in (None, dict(kernel="pipe", warps_per_block=16, obs_warps=7), dict(kernel="pipe", warps_per_block=16,
                                                                                obs_warps=4),
                dict(kernel="pipe", warps_per_block=16, obs_warps=7, order="map"),
                dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=32),
                dict(kernel="pipe", warps_per_block=16, obs_warps=4, segment=64)):
        s = Sim(p, maps, env_map, beams)
        if cfg:
            s.set_launch(**cfg)
        s.reset()
        obs = s.new_obs()
        r = _run_obs(s, K, obs)
        out.append((r, obs.cpu().numpy(), s.get_state()))
    (ref, obs0, (f0, u0)) = out[0]
    for r, ob, (f, u) in out[1:]:
        for k in ref:
            assert np.array_equal(bits(r[k]) if r[k].dtype == np.float32 else r[k],
                                  bits(ref[k]) if ref[k].dtype == np.float32 else ref[k]), k
        assert np.array_equal(bits(ob), bits(obs0))
        assert np.array_equal(bits(f), bits(f0)) and np.array_equal(u, u0)


@pytest.mark.parametrize("n,K,seg,cfg", [(4, 640, 32, dict(warps_per_block=8, obs_warps=7)),
                                         (7, 333, 64, dict(warps_per_block=16, obs_warps=7)),
                                         (50, 500, 96, dict(warps_per_block=12, obs_warps=3, order="map"))])
def test_time_sliced_pipelined_rollout(n, K, seg, cfg):
    """The time-sliced pipelined rollout: with few envs and many segments
    nearly every item waits for the previous segment of its envs on another
    CTA.  Every output and the final state equal the unsliced launch's, no
    wait times out, and the slicing repeats bit for bit."""
    from paper_2305_04180_gb300 import Sim

    p, maps, env_map, beams = _uneven(n, seed=5)
    out = []
    for c in (dict(cfg, kernel="pipe"), dict(cfg, kernel="pipe", segment=seg), dict(cfg, kernel="pipe", segment=seg)):
        s = Sim(p, maps, env_map, beams)
        s.set_launch(**c)
        s.reset()
        obs = s.new_obs()
        r = _run_obs(s, K, obs)
        assert s.status() == 0
        out.append((r, obs.cpu().numpy(), s.get_state()))
    (ref, obs0, (f0, u0)) = out[0]
    for r, ob, (f, u) in out[1:]:
        for k in ref:
            assert np.array_equal(bits(r[k]) if r[k].dtype == np.float32 else r[k],
                                  bits(ref[k]) if ref[k].dtype == np.float32 else ref[k]), k
        assert np.array_equal(bits(ob), bits(obs0))
        assert np.array_equal(bits(f), bits(f0)) and np.array_equal(u, u0)


def test_time_sliced_wait_bound_reports_timeout_and_recovers():
    """Failure detection of the time-sliced rollout's bounded waits: with a
    one-sleep bound, an item that must wait for the previous segment of its
    envs gives up at once.  The launch ends, the status word reads
    SG_DEV_TIMEOUT, and the next launches on the same context (default
    bound) give the unsliced results."""
    from paper_2305_04180_gb300 import Sim

    p, maps, env_map, beams = _uneven(4, seed=6)
    K = 640
    s = Sim(p, maps, env_map, beams)
    s.set_launch(kernel="pipe", warps_per_block=8, obs_warps=7, segment=32, wait_iters=1)
    s.reset()
    rew = torch.empty((K, 4), device="cuda")
    s.rollout(K, rew_seq=rew)
    torch.cuda.synchronize()
    assert s.status() == 2  # SG_DEV_TIMEOUT
    assert s.status() == 0  # reading clears it
    ref = Sim(p, maps, env_map, beams)
    ref.set_launch(kernel="pipe", warps_per_block=8, obs_warps=7)
    ref.reset()
    r0 = _run_obs(ref, K, ref.new_obs())
    s.set_launch(kernel="pipe", warps_per_block=8, obs_warps=7, segment=32)
    s.reset()
    r1 = _run_obs(s, K, s.new_obs())
    assert s.status() == 0
    for k in r0:
        assert np.array_equal(r0[k].view(np.uint8), r1[k].view(np.uint8)), k


def _run_obs(sim, K, obs):
    n = sim.n
    out = dict(obs_seq=torch.empty((K, n, sim.obs_dim), device="cuda"),
               rew=torch.empty((K, n), device="cuda"),
               done=torch.empty((K, n), dtype=torch.uint8, device="cuda"))
    sim.rollout(K, obs=obs, obs_seq=out["obs_seq"], rew_seq=out["rew"], done_seq=out["done"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_graph_replay_equals_direct_calls():
    from paper_2305_04180_gb300 import Sim
    from paper_2305_04180_gb300.graph import Graph

    p, maps, env_map, beams = _uneven(64, seed=1)
    a = Sim(p, maps, env_map, beams)
    b = Sim(p, maps, env_map, beams)
    a.reset()
    b.reset()
    st = torch.cuda.Stream()
    rew_g = torch.empty((4, 16, a.n), device="cuda")
    g = Graph()
    with g.capture(st):
        for c in range(4):
            a.rollout(16, rew_seq=rew_g[c], stream=st)
    assert g.num_nodes() >= 4
    rew_d = torch.empty((4, 16, b.n), device="cuda")
    for rep in range(3):
        g.launch(st)
        st.synchronize()
        for c in range(4):
            b.rollout(16, rew_seq=rew_d[c])
        torch.cuda.synchronize()
        assert torch.equal(rew_g, rew_d), rep
    fa, ua = a.get_state()
    fb, ub = b.get_state()
    assert np.array_equal(bits(fa), bits(fb)) and np.array_equal(ua, ub)
    assert ua[2, 0] == 3 * 64  # 3 replays x 4 rollouts x 16 steps


def _trainer(sim_seed=3, two_streams=True):
    from paper_2305_04180_gb300 import Sim
    from paper_2305_04180_gb300.trainer import ColorTrainer

    p = base_params(**DR_RANGES)
    maps = [make_map(s) for s in range(1, 5)]
    sim = Sim(dict(p, seed=sim_seed), maps, (np.arange(64) % 4).astype(np.int32))
    sim.reset()
    return ColorTrainer(sim, batch=128, slots=32, lr=5e-4, tps=8, learn_start=0, two_streams=two_streams, seed=2)


def test_graph_actor_learner_iteration_sequential_is_deterministic():
    """The captured (sequential) iteration equals the same calls made directly."""
    ta = _trainer()
    tb = _trainer()
    ta.sim.rollout(8, policy="eps_q", qnet=ta.actor, eps=ta.eps, replay=ta.replay)
    tb.sim.rollout(8, policy="eps_q", qnet=tb.actor, eps=tb.eps, replay=tb.replay)
    g = ta.capture_iteration(8, 4, concurrent=False)
    for _ in range(5):
        g.launch(ta.s_actor)
        tb.sim.vem_eps(**tb.vem, out=tb.eps)  # the graph recomputes the VEM noise before its rollout
        tb.sim.rollout(8, policy="eps_q", qnet=tb.actor, eps=tb.eps, replay=tb.replay)
        for _ in range(4):
            tb.learner.train_step(tb.replay, tb.batch, lr=tb.lr, target_every=tb.target_every, seed=tb.seed)
        tb.actor.copy_from(tb.learner)
    torch.cuda.synchronize()
    assert np.array_equal(ta.learner.get_params(), tb.learner.get_params())
    assert np.array_equal(ta.actor.get_params(), tb.learner.get_params())
    assert ta.replay.steps_recorded() == tb.replay.steps_recorded() == 48
    assert ta.learner.optimizer_state()[2] == 20


def test_graph_actor_learner_iteration_concurrent_runs():
    """Concurrent branches: counters advance, upload happens, values stay finite."""
    t = _trainer(sim_seed=4)
    t.sim.rollout(8, policy="eps_q", qnet=t.actor, eps=t.eps, replay=t.replay)
    g = t.capture_iteration(8, 4, concurrent=True)
    for _ in range(6):
        g.launch(t.s_actor)
    torch.cuda.synchronize()
    assert t.replay.steps_recorded() == 8 + 6 * 8
    assert t.learner.optimizer_state()[2] == 24
    th = t.learner.get_params()
    assert np.isfinite(th).all() and np.array_equal(t.actor.get_params(), th)
    assert np.isfinite(t.loss.item())


def test_autotune_applies_a_candidate_and_results_do_not_change(tmp_path):
    from paper_2305_04180_gb300 import Sim
    from paper_2305_04180_gb300.autotune import CANDIDATES, autotune_rollout

    p, maps, env_map, beams = _uneven(80, seed=2)
    a = Sim(p, maps, env_map, beams)
    b = Sim(p, maps, env_map, beams)
    a.reset()
    b.reset()
    cache = str(tmp_path / "tune.json")
    res = autotune_rollout(a, K=8, reps=1, cache_path=cache)
    assert not res["cached"] and len(res["table"]) == len(CANDIDATES)
    assert res["config"] in CANDIDATES
    assert np.array_equal(bits(_run(a, 20)["rew"]), bits(_run(b, 20)["rew"]))
    again = autotune_rollout(a, K=8, reps=1, cache_path=cache)
    assert again["cached"] and again["config"] == res["config"]


def test_checkpoint_resume_is_bit_identical():
    """Train, checkpoint the whole loop (env state, networks, Adam moments,
    ring, counters), continue; a loop with the same configuration that has
    drifted elsewhere, restored from the checkpoint, continues to exactly the
    same parameters and env state."""
    ta = _trainer(sim_seed=6, two_streams=False)
    ta.run(48, rollout_k=8)
    ck = ta.state_dict()
    ta.run(40, rollout_k=8)
    tb = _trainer(sim_seed=6, two_streams=False)
    tb.run(24, rollout_k=8)  # somewhere else; the checkpoint overwrites all of it
    tb.load_state_dict(ck)
    tb.run(40, rollout_k=8)
    assert np.array_equal(ta.learner.get_params(), tb.learner.get_params())
    assert np.array_equal(ta.learner.get_params("target"), tb.learner.get_params("target"))
    fa, ua = ta.sim.get_state()
    fb, ub = tb.sim.get_state()
    assert np.array_equal(bits(fa), bits(fb)) and np.array_equal(ua, ub)
    assert ta.updates == tb.updates and ta.replay.steps_recorded() == tb.replay.steps_recorded()


def test_async_state_upload_matches_synchronous_and_is_stream_ordered():
    """sg_sim_set_state_async restores exactly what sg_sim_set_state does,
    and, queued on a stream behind a rollout, replaces the state only after
    that rollout (the next rollout then repeats the first from the same
    start state, bit for bit)."""
    from paper_2305_04180_gb300 import Sim

    params, maps, env_map, beams = _uneven(n=64, seed=5)
    s = Sim(params, maps, env_map, beams)
    s.reset()
    _run(s, 7)
    f0, u0 = s.get_state()
    blob = s.state_blob(f0, u0)
    ref = _run(s, 20)
    f1, u1 = s.get_state()
    # a synchronous restore and an asynchronous one give the same state
    s.set_state(f0, u0)
    fa, ua = s.get_state()
    _run(s, 5)
    s.set_state_async(blob)
    torch.cuda.synchronize()
    fb, ub = s.get_state()
    assert np.array_equal(bits(fa), bits(fb)) and np.array_equal(ua, ub)
    # on one stream: rollout, upload, rollout (no host synchronisation between)
    st = torch.cuda.Stream()
    n, K = s.n, 20
    bufs = [dict(obs_seq=torch.empty((K, n, s.obs_dim), device="cuda"), rew=torch.empty((K, n), device="cuda"),
                 done=torch.empty((K, n), dtype=torch.uint8, device="cuda")) for _ in range(2)]
    s.set_state_async(blob, st)
    for b in bufs:
        if b is bufs[1]:
            s.set_state_async(blob, st)
        s.rollout(K, obs_seq=b["obs_seq"], rew_seq=b["rew"], done_seq=b["done"], stream=st)
    torch.cuda.synchronize()
    for b in bufs:
        for k in ("obs_seq", "rew", "done"):
            assert np.array_equal(b[k].cpu().numpy(), ref[k]), k
    fc, uc = s.get_state()
    assert np.array_equal(bits(fc), bits(f1)) and np.array_equal(uc, u1)
    from paper_2305_04180_gb300 import _lib

    assert s.L.sg_sim_set_state_async(s.handle, blob.data_ptr(), int(blob.numel()) - 4, None) == _lib.SG_E_INVAL
