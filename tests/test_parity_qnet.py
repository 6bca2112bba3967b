"""GPU parity of the learned part against the float64 oracle (through the C ABI).

* Forward: the tensor-core Q-values against the oracle's bf16 recipe (same
  roundings, float64 sums) and against exact float64; the max relative Q
  error is printed and bounded.
* Fused eps-greedy rollout: exploration decisions and random actions exact;
  greedy actions equal the oracle's argmax wherever its top-2 margin exceeds
  the Q error bound (otherwise either near-tied action is valid); the
  simulator part of every step bit-exact given the chosen actions; replay
  contents exact.
* TD learner: targets, loss and gradient against the oracle's bf16 recipe;
  Adam update against the oracle's Adam on the same gradient; target sync.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from oracle import qnet as OQ
from oracle.sim import OracleSim, lib as olib
from tests._helpers import bits, gpu_state_to_oracle, ring_sample_entries
from workloads import workload

pytestmark = pytest.mark.gpu

Q_REL_TOL = 4e-3  # max |Q_gpu - Q_bf16_recipe| / max|Q| (float32 vs float64 sums, bf16 re-rounding)


def _theta(seed, n_in=37, scale=1.0, arch="dueling"):
    p = OQ.init_params(seed, n_in, arch)
    for k in p:
        p[k] = p[k] * scale
    return OQ.flatten(p).astype(np.float32)


def _qnet(n_in=37, max_batch=256, seed=0, arch="dueling"):
    from paper_2305_04180_gb300 import QNet

    return QNet(n_in, max_batch, seed, arch=arch)


@pytest.mark.parametrize("arch,n_in,count", [("dueling", 37, 77062), ("paper", 32, 41989)])
def test_params_roundtrip_and_count(arch, n_in, count):
    q = _qnet(n_in, arch=arch)
    assert q.n_params == count == OQ.n_params(n_in, arch)
    # the library's own initialisation is finite, non-zero and in the fan-in bounds
    th0 = q.get_params("online")
    assert np.isfinite(th0).all() and np.abs(th0).max() <= 1.0 / np.sqrt(min(n_in, 128)) + 1e-6
    assert np.count_nonzero(th0) > 0.99 * th0.size
    th = _theta(1, n_in, arch=arch)
    q.set_params(th)
    assert np.array_equal(q.get_params("online"), th) and np.array_equal(q.get_params("target"), th)
    th2 = _theta(2, n_in, arch=arch)
    q.set_params(th2, "target")
    assert np.array_equal(q.get_params("online"), th) and np.array_equal(q.get_params("target"), th2)


@pytest.mark.parametrize("n_in,M,arch", [(37, 1, "dueling"), (37, 53, "dueling"), (37, 4096, "dueling"),
                                         (69, 300, "dueling"), (21, 17, "dueling"), (32, 300, "paper"),
                                         (32, 1, "paper"), (37, 77, "paper"), (48, 300, "dueling"),
                                         (64, 129, "dueling"), (65, 257, "dueling")])
def test_forward_against_oracle(n_in, M, arch):
    rng = np.random.default_rng(n_in + M)
    q = _qnet(n_in, arch=arch)
    th = _theta(3, n_in, scale=2.0, arch=arch)
    q.set_params(th)
    obs = rng.uniform(-1, 1, size=(M, n_in)).astype(np.float32)
    got = q.forward(torch.from_numpy(obs).cuda()).cpu().numpy().astype(np.float64)
    p = OQ.unflatten(th.astype(np.float64), n_in, arch)
    ref_bf = OQ.forward(p, obs, bf16=True)
    ref_64 = OQ.forward(p, obs)
    scale = np.abs(ref_64).max()
    err_bf = np.abs(got - ref_bf).max() / scale
    err_64 = np.abs(got - ref_64).max() / scale
    print(f"max relative Q error: vs bf16 recipe {err_bf:.2e}, vs exact float64 {err_64:.2e}")
    assert err_bf <= Q_REL_TOL
    assert err_64 <= 5e-2


@pytest.mark.parametrize("M,stride,n_in", [(65536, 1, 37), (1 << 20, 61, 37), (65536 + 77, 1, 69)])
def test_forward_multi_tile_against_oracle(M, stride, n_in):
    """The batched tcgen05 forward at sizes where every persistent CTA runs
    many 128-row tiles (65,536 rows: about 3 per CTA; 2^20 rows: about 54),
    so that the next tile's layer 1 running beside this tile's layer-2
    epilogue and head, the next tile's input conversion during layer 2, the
    activations kept in tensor memory and the barrier phases across tiles
    are all exercised; at the widest input (69: five 16-column groups of
    layer 1) with a ragged last tile of 77 rows.  Rows are compared element
    by element with the oracle's bf16 recipe: all of them at 65,536, every
    61st at 2^20 (17,190 rows spread over every tile)."""
    rng = np.random.default_rng(M)
    q = _qnet(n_in)
    th = _theta(4, n_in, scale=2.0)
    q.set_params(th)
    obs = rng.uniform(-1, 1, size=(M, n_in)).astype(np.float32)
    got = q.forward(torch.from_numpy(obs).cuda()).cpu().numpy().astype(np.float64)
    rows = np.arange(0, M, stride)
    p = OQ.unflatten(th.astype(np.float64), n_in)
    ref_bf = OQ.forward(p, obs[rows], bf16=True)
    scale = np.abs(ref_bf).max()
    err = np.abs(got[rows] - ref_bf) / scale
    print(f"M={M}: max relative Q error vs bf16 recipe {err.max():.2e} over {rows.size} rows")
    assert np.isfinite(got).all()
    assert err.max() <= Q_REL_TOL
    # a tile's rows do not leak into another's: permuting the batch permutes the output
    perm = rng.permutation(M)
    got_p = q.forward(torch.from_numpy(obs[perm]).cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(got_p, got[perm])


def test_grid_limits_do_not_change_results():
    """sg_qnet_set_grid_limit caps the tcgen05 rollout's and learner's
    grids (so that a concurrent actor and learner keep SMs of their own);
    with caps of 30 rollout CTAs (40 blocks of 128 envs: a time-sliced
    rollout over a resident grid instead of one CTA per block) and 8 learner
    CTAs (16 jobs per CTA) the actions,
    rewards, ring contents, final state, loss and gradient equal the
    uncapped runs bit for bit."""
    from paper_2305_04180_gb300 import Replay, Sim

    w = workload("qnet4096", n_envs=5120)
    maps = w.maps()
    q = _qnet(w.params["n_beams"] + 5, max_batch=4096)
    q.set_params(_theta(22, q.n_in, scale=3.0))
    q.set_rollout_rows(128)
    eps = torch.from_numpy(_eps_spread(5120)).cuda()
    out = []
    for caps in ((0, 0), (30, 8)):
        q.set_grid_limit(rollout=caps[0], learner=caps[1])
        s = Sim(w.params, maps, w.env_map)
        rp = Replay(48, s.n, s.obs_dim)
        s.reset()
        K = 24
        act = torch.empty((K, s.n), dtype=torch.uint8, device="cuda")
        rew = torch.empty((K, s.n), device="cuda")
        s.rollout(K, policy="eps_q", qnet=q, eps=eps, replay=rp, act_seq=act, rew_seq=rew)
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(q.n_params, device="cuda")
        q2 = _qnet(q.n_in, max_batch=4096)
        q2.set_params(q.get_params())
        q2.set_grid_limit(learner=caps[1])
        q2.train_step(rp, 4096, gamma=0.98, lr=0.0, seed=7, loss=loss, grad=grad)
        torch.cuda.synchronize()
        assert s.status() == 0
        out.append((act.cpu().numpy(), rew.cpu().numpy(), rp.read(0, K * s.n), s.get_state(),
                    loss.cpu().numpy(), grad.cpu().numpy()))
    q.set_grid_limit()
    (a0, r0, ring0, st0, l0, g0), (a1, r1, ring1, st1, l1, g1) = out
    assert np.array_equal(a0, a1) and np.array_equal(bits(r0), bits(r1))
    for x, y in zip(ring0, ring1):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    for x, y in zip(st0, st1):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert np.isfinite(l0).all() and np.array_equal(bits(l0), bits(l1))
    assert np.array_equal(bits(g0), bits(g1))
    assert q.L.sg_qnet_set_grid_limit(q.handle, -1, 0) != 0


def _margin_ok(q_ref, act, tol):
    """Greedy action equals the argmax, or the argmax is within tol of it."""
    best = q_ref.max(axis=1)
    chosen = q_ref[np.arange(len(act)), act]
    return best - chosen <= tol


@pytest.mark.parametrize("rows,arch", [(16, "dueling"), (32, "dueling"), (32, "paper"), (128, "dueling"),
                                       (128, "paper")])
def test_fused_rollout_teacher_forced(rows, arch):
    """Step by step (K = 1 rollouts) from the GPU's own state: every decision
    checked, every simulator output bit-exact, the replay ring exact; for
    CTAs of 16 and of 32 envs (mma.sync) and of 128 envs (tcgen05)."""
    from paper_2305_04180_gb300 import Replay, Sim

    w = workload("qnet4096", n_envs=70)
    maps = w.maps()
    g = Sim(w.params, maps, w.env_map)
    o = OracleSim(w.params, maps, w.env_map, prec="f32")
    q = _qnet(g.obs_dim, arch=arch)
    q.set_rollout_rows(rows)
    th = _theta(5, g.obs_dim, scale=3.0, arch=arch)
    q.set_params(th)
    p = OQ.unflatten(th.astype(np.float64), g.obs_dim, arch)
    n = g.n
    rp = Replay(8, n, g.obs_dim)
    eps = torch.from_numpy(w.eps).cuda()
    obs = g.reset()
    o.reset()
    obs_prev = obs.cpu().numpy()
    act = torch.empty((1, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((1, n), dtype=torch.float32, device="cuda")
    done = torch.empty((1, n), dtype=torch.uint8, device="cuda")
    n_greedy = n_explore = 0
    for t in range(40):
        f, u = g.get_state()
        o.set_state(*gpu_state_to_oracle(f, u))
        g.rollout(1, policy="eps_q", qnet=q, eps=eps, replay=rp, obs=obs, act_seq=act, rew_seq=rew, done_seq=done)
        a = act.cpu().numpy()[0]
        # exploration draws and random actions are exact
        explore = o.explore_uniform(t) < w.eps
        rand_a = o.random_actions(t)
        assert np.array_equal(a[explore], rand_a[explore]), t
        # greedy actions: argmax of the oracle's bf16-recipe Q of the previous obs
        qref = OQ.forward(p, obs_prev, bf16=True)
        tol = Q_REL_TOL * np.abs(qref).max()
        ok = _margin_ok(qref, a, 2 * tol)
        assert np.all(ok[~explore]), (t, np.argwhere(~ok & ~explore))
        n_greedy += int((~explore).sum())
        n_explore += int(explore.sum())
        # the simulator part with the chosen actions is bit-exact
        oobs, orew, odone, oterm = o.step(a)
        d = done.cpu().numpy()[0]
        assert np.array_equal(d, odone), t
        assert np.array_equal(bits(rew.cpu().numpy()[0]), bits(orew)), t
        assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs)), t
        # the transition in the ring: slot t mod 8
        s, s2, ra, rr, rt = rp.read((t % 8) * n, n)
        assert np.array_equal(bits(s), bits(obs_prev)), t
        expect_s2 = np.where((odone != 0)[:, None], oterm, oobs)
        assert np.array_equal(bits(s2), bits(expect_s2)), t
        assert np.array_equal(ra, a) and np.array_equal(bits(rr), bits(orew))
        assert np.array_equal(rt, ((odone & 3) != 0).astype(np.uint8))
        obs_prev = oobs
    assert rp.steps_recorded() == 40
    assert n_greedy > 1000 and n_explore > 50


@pytest.mark.parametrize("rows", [0, 128])
def test_fused_rollout_free_running_matches_stepwise(rows):
    """A K-step fused rollout equals K single-step rollouts from the same start
    (the default CTAs, and the tcgen05 kernel's 128-env CTAs over a ragged
    last CTA)."""
    from paper_2305_04180_gb300 import Sim

    w = workload("qnet4096", n_envs=48 if rows == 0 else 300)
    maps = w.maps()
    a = Sim(w.params, maps, w.env_map)
    b = Sim(w.params, maps, w.env_map)
    q = _qnet(a.obs_dim)
    q.set_rollout_rows(rows)
    q.set_params(_theta(6, a.obs_dim, scale=3.0))
    eps = torch.from_numpy(w.eps).cuda()
    a.reset()
    b.reset()
    K = 70
    ra = torch.empty((K, a.n), device="cuda")
    rb = torch.empty((K, b.n), device="cuda")
    aa = torch.empty((K, a.n), dtype=torch.uint8, device="cuda")
    ab = torch.empty((K, b.n), dtype=torch.uint8, device="cuda")
    a.rollout(K, policy="eps_q", qnet=q, eps=eps, rew_seq=ra, act_seq=aa)
    for k in range(K):
        b.rollout(1, policy="eps_q", qnet=q, eps=eps, rew_seq=rb[k:k + 1], act_seq=ab[k:k + 1])
    assert torch.equal(aa, ab) and torch.equal(ra, rb)


def test_time_sliced_tc_rollout_equals_single_steps():
    """More than one wave of 128-env CTAs (20,480 envs): the tcgen05 rollout
    is sliced into segments over a resident grid, and a later segment takes
    its first observation from the replay ring.  A 16-step rollout equals 16
    single-step rollouts (no slicing, every first observation scanned from
    the state): actions, rewards, done flags, ring contents, final state."""
    from paper_2305_04180_gb300 import Replay, Sim

    w = workload("qnet4096", n_envs=20480)
    maps = w.maps()
    q = _qnet(w.params["n_beams"] + 5)
    q.set_params(_theta(21, q.n_in, scale=3.0))
    q.set_rollout_rows(128)
    eps = torch.from_numpy(_eps_spread(20480)).cuda()
    out = []
    for stepwise in (False, True):
        s = Sim(w.params, maps, w.env_map)
        rp = Replay(24, s.n, s.obs_dim)
        s.reset()
        K = 16
        act = torch.empty((K, s.n), dtype=torch.uint8, device="cuda")
        rew = torch.empty((K, s.n), device="cuda")
        done = torch.empty((K, s.n), dtype=torch.uint8, device="cuda")
        if stepwise:
            for k in range(K):
                s.rollout(1, policy="eps_q", qnet=q, eps=eps, replay=rp, act_seq=act[k:k + 1], rew_seq=rew[k:k + 1],
                          done_seq=done[k:k + 1])
        else:
            s.rollout(K, policy="eps_q", qnet=q, eps=eps, replay=rp, act_seq=act, rew_seq=rew, done_seq=done)
        torch.cuda.synchronize()
        assert s.status() == 0
        out.append((act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), rp.read(0, K * s.n), s.get_state()))
    (a0, r0, d0, ring0, st0), (a1, r1, d1, ring1, st1) = out
    assert np.array_equal(a0, a1) and np.array_equal(bits(r0), bits(r1)) and np.array_equal(d0, d1)
    for x, y in zip(ring0, ring1):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    for x, y in zip(st0, st1):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert (d0 != 0).sum() > 100


def _eps_spread(n):
    return np.linspace(0.01, 0.3, n).astype(np.float32)


def test_fused_rollout_tile_heights_agree():
    """CTAs of 16 and of 32 envs compute identical Q-values, so identical
    trajectories (the same MMA order per row)."""
    from paper_2305_04180_gb300 import Sim

    w = workload("qnet4096", n_envs=100)
    maps = w.maps()
    q = _qnet(w.params["n_beams"] + 5)
    q.set_params(_theta(12, q.n_in, scale=3.0))
    eps = torch.from_numpy(w.eps).cuda()
    out = []
    for rows in (16, 32):
        q.set_rollout_rows(rows)
        s = Sim(w.params, maps, w.env_map)
        s.reset()
        act = torch.empty((60, s.n), dtype=torch.uint8, device="cuda")
        rew = torch.empty((60, s.n), device="cuda")
        s.rollout(60, policy="eps_q", qnet=q, eps=eps, act_seq=act, rew_seq=rew)
        out.append((act, rew, s.get_state()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2][1], out[1][2][1])


def test_full_learned_workload_sampled_against_oracle():
    """The 65,536-env learned-loop workload at full size (1,024 maps of sides
    256..1,024, 16..64 beams, every randomisation on) through the fused
    rollout: 32 steps on the GPU with its actions recorded, then sampled envs
    replayed on the oracle with those actions: the exploration decision and
    random action of every step exact, the simulator part (rewards, done
    flags, final state) bit-exact."""
    from paper_2305_04180_gb300 import Sim

    w = workload("full65536")
    maps = w.maps()
    g = Sim(w.params, maps, w.env_map, w.env_beams)
    q = _qnet(g.obs_dim, max_batch=256)
    q.set_params(_theta(12, g.obs_dim, scale=2.0))
    g.reset()
    K = 32
    act = torch.empty((K, g.n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, g.n), device="cuda")
    done = torch.empty((K, g.n), dtype=torch.uint8, device="cuda")
    g.rollout(K, policy="eps_q", qnet=q, eps=torch.from_numpy(w.eps).cuda(), act_seq=act, rew_seq=rew,
              done_seq=done)
    act, rew, done = act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy()
    f, u = g.get_state()
    sample = [0, 1, 1023, 1024, 30000, 65535] + list(range(5, 65536, 6553))
    keep = {int(w.env_map[i]) for i in sample}
    tiny = np.ones((1, 1), np.uint8)
    o = OracleSim(w.params, [maps[m] if m in keep else tiny for m in range(len(maps))], w.env_map, w.env_beams,
                  prec="f32")
    p = OQ.unflatten(_theta(12, g.obs_dim, scale=2.0).astype(np.float64), g.obs_dim)
    n_explore = n_greedy = 0
    for i in sample:
        ob = o.reset_env(i, 0)
        for k in range(K):
            a = int(act[k, i])
            if o.L.orc_explore_uniform(C.byref(o.cfg), i, k) < w.eps[i]:
                assert a == o.random_action(i, k), (i, k)
                n_explore += 1
            else:
                # greedy: the oracle's argmax of its bf16-recipe Q of the
                # observation the step starts from, up to near ties
                qref = OQ.forward(p, np.asarray(ob, np.float32)[None], bf16=True)
                tol = Q_REL_TOL * np.abs(qref).max()
                assert _margin_ok(qref, np.array([a]), 2 * tol)[0], (i, k, qref, a)
                n_greedy += 1
            ob, orew, odone, _ = o.step_one(i, a)
            assert odone == done[k, i] and bits(np.float32(orew)) == bits(rew[k, i]), (i, k)
        assert np.array_equal(bits(o.f[:, i]), bits(f[:, i])), i
        assert np.array_equal(o.u[:, i], u[:2, i]), i
    assert n_explore > 10 and n_greedy > 300


def _fill_replay(n_envs=64, steps=40, seed_theta=7, arch="dueling", max_batch=256):
    from paper_2305_04180_gb300 import Replay, Sim

    w = workload("qnet4096", n_envs=n_envs)
    g = Sim(w.params, w.maps(), w.env_map)
    q = _qnet(g.obs_dim, arch=arch, max_batch=max_batch)
    q.set_params(_theta(seed_theta, g.obs_dim, scale=2.0, arch=arch))
    rp = Replay(32, g.n, g.obs_dim)
    g.reset()
    g.rollout(steps, policy="eps_q", qnet=q, eps=torch.from_numpy(w.eps).cuda(), replay=rp)
    torch.cuda.synchronize()
    return g, q, rp


def _oracle_batch(rp, seed, tstep, batch):
    steps = rp.steps_recorded()
    idx = ring_sample_entries(seed, tstep, batch, steps, rp.slots, rp.n_envs, rp.reserve)
    s, s2, a, r, t = rp.read(0, rp.capacity)
    return idx, dict(s=s[idx].astype(np.float64), a=a[idx].astype(np.int64), r=r[idx].astype(np.float64),
                     s2=s2[idx].astype(np.float64), term=t[idx].astype(np.float64))


@pytest.mark.parametrize("batch,arch", [(256, "dueling"), (100, "dueling"), (256, "paper"), (37, "paper")])
def test_td_loss_and_gradient_against_oracle(batch, arch):
    g, q, rp = _fill_replay(arch=arch)
    th_on = _theta(8, g.obs_dim, scale=2.0, arch=arch)
    th_tg = _theta(9, g.obs_dim, scale=2.0, arch=arch)
    q.set_params(th_on, "online")
    q.set_params(th_tg, "target")
    seed = 1234
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(q.n_params, device="cuda")
    q.train_step(rp, batch, gamma=0.98, lr=0.0, seed=seed, loss=loss, grad=grad)
    _, bt = _oracle_batch(rp, seed, 0, batch)
    pon = OQ.unflatten(th_on.astype(np.float64), g.obs_dim, arch)
    ptg = OQ.unflatten(th_tg.astype(np.float64), g.obs_dim, arch)
    ref_loss, ref_g = OQ.td_loss_grad(pon, ptg, bt, 0.98, bf16=True)
    _, ref_g64 = OQ.td_loss_grad(pon, ptg, bt, 0.98, bf16=False)
    gl = float(loss.item())
    gg = grad.cpu().numpy().astype(np.float64)
    rflat = OQ.flatten(ref_g)
    r64 = OQ.flatten(ref_g64)
    rel_loss = abs(gl - ref_loss) / max(1e-6, abs(ref_loss))
    rel_g = np.linalg.norm(gg - rflat) / np.linalg.norm(rflat)
    rel_g64 = np.linalg.norm(gg - r64) / np.linalg.norm(r64)
    print(f"TD loss rel err {rel_loss:.2e}; grad rel err vs bf16 recipe {rel_g:.2e}, vs float64 {rel_g64:.2e}")
    assert rel_loss <= 1e-2
    assert rel_g <= 3e-2
    assert rel_g64 <= 1e-1
    # every block of the gradient, not just the norm
    for name, sl in _blocks(g.obs_dim, arch):
        nb = np.linalg.norm(rflat[sl])
        if nb > 0:
            assert np.linalg.norm(gg[sl] - rflat[sl]) / nb <= 6e-2, name


# Element-wise bound of the TD gradient against the oracle's bf16 recipe:
# |g - g_ref| <= TD_ATOL * max|g_ref over the parameter block| + TD_RTOL * |g_ref|.
# The two sides round the same quantities to bf16 (weights, activations, the
# backpropagated dZ), but their float32 and float64 sums differ, so a value
# close to a bf16 rounding boundary can land one bf16 step (2^-8 relative)
# apart and carry that into the products it feeds; TD_ATOL bounds such
# contributions relative to the block's scale, TD_RTOL the float32 sums.
TD_RTOL = 1e-2
TD_ATOL = 2e-3


def _td_case(batch, arch, n_envs=64, steps=40):
    g, q, rp = _fill_replay(arch=arch, n_envs=n_envs, steps=steps, max_batch=batch)
    th_on = _theta(8, g.obs_dim, scale=2.0, arch=arch)
    th_tg = _theta(9, g.obs_dim, scale=2.0, arch=arch)
    q.set_params(th_on, "online")
    q.set_params(th_tg, "target")
    return g, q, rp, th_on, th_tg


def _gpu_loss_grad(q, rp, batch, seed):
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(q.n_params, device="cuda")
    q.train_step(rp, batch, gamma=0.98, lr=0.0, seed=seed, loss=loss, grad=grad)
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("batch,arch,n_envs", [(256, "dueling", 64), (4096, "dueling", 256), (256, "paper", 64),
                                               (4096, "paper", 256)])
def test_td_gradient_elementwise_against_oracle(batch, arch, n_envs):
    """Every entry of the TD gradient (77,062 parameters of the dueling
    network, 41,989 of the paper's) against the oracle's bf16 recipe, at the
    learner batches of the 4,096-env workload (256) and of the 65,536-env
    learned loop (4,096)."""
    g, q, rp, th_on, th_tg = _td_case(batch, arch, n_envs=n_envs)
    seed = 77
    gl, gg = _gpu_loss_grad(q, rp, batch, seed)
    _, bt = _oracle_batch(rp, seed, 0, batch)
    pon = OQ.unflatten(th_on.astype(np.float64), g.obs_dim, arch)
    ptg = OQ.unflatten(th_tg.astype(np.float64), g.obs_dim, arch)
    ref_loss, ref_g = OQ.td_loss_grad(pon, ptg, bt, 0.98, bf16=True)
    rflat = OQ.flatten(ref_g)
    assert np.isfinite(gg).all()
    assert abs(gl - ref_loss) <= 1e-4 * max(1e-6, abs(ref_loss)), (gl, ref_loss)
    worst = 0.0
    for name, sl in _blocks(g.obs_dim, arch):
        r = rflat[sl]
        e = np.abs(gg[sl] - r)
        bound = TD_ATOL * np.abs(r).max() + TD_RTOL * np.abs(r)
        ratio = (e / np.maximum(bound, 1e-30)).max()
        worst = max(worst, ratio)
        print(f"batch {batch} {arch} {name}: max |g - g_ref| {e.max():.3e} (block max |g_ref| "
              f"{np.abs(r).max():.3e}), max error / bound {ratio:.3f}")
        assert np.all(e <= bound), (name, int(np.argmax(e / np.maximum(bound, 1e-30))))
    print(f"batch {batch} {arch}: loss {gl:.6f} vs {ref_loss:.6f}; worst error / bound {worst:.3f}")


@pytest.mark.parametrize("n_in", [69, 48])
def test_td_gradient_widest_inputs_at_batch_4096(n_in):
    """The tcgen05 learner at batch 4,096 with inputs of 69 (five 16-column
    groups of layer 1, dW1 of N = 80) and 48 (no zero padding) on a
    synthetic ring: loss and every gradient entry against the oracle's bf16
    recipe at the bound of the other TD parity tests."""
    from paper_2305_04180_gb300 import Replay

    rng = np.random.default_rng(n_in)
    n_envs, slots = 512, 16
    rp = Replay(slots, n_envs, n_in)
    cap = rp.capacity
    s_ = rng.uniform(-1, 1, size=(cap, n_in)).astype(np.float32)
    s2 = rng.uniform(-1, 1, size=(cap, n_in)).astype(np.float32)
    a = rng.integers(0, 5, size=cap).astype(np.uint8)
    r = rng.normal(size=cap).astype(np.float32)
    t = (rng.uniform(size=cap) < 0.05).astype(np.uint8)
    rp.write(0, s_, s2, a, r, t, steps_recorded=slots)
    q = _qnet(n_in, max_batch=4096)
    th_on, th_tg = _theta(10, n_in, scale=2.0), _theta(11, n_in, scale=2.0)
    q.set_params(th_on, "online")
    q.set_params(th_tg, "target")
    batch, seed = 4096, 13
    gl, gg = _gpu_loss_grad(q, rp, batch, seed)
    _, bt = _oracle_batch(rp, seed, 0, batch)
    pon = OQ.unflatten(th_on.astype(np.float64), n_in)
    ptg = OQ.unflatten(th_tg.astype(np.float64), n_in)
    ref_loss, ref_g = OQ.td_loss_grad(pon, ptg, bt, 0.98, bf16=True)
    rflat = OQ.flatten(ref_g)
    assert np.isfinite(gg).all()
    assert abs(gl - ref_loss) <= 1e-4 * max(1e-6, abs(ref_loss)), (gl, ref_loss)
    for name, sl in _blocks(n_in):
        ref = rflat[sl]
        e = np.abs(gg[sl] - ref)
        bound = TD_ATOL * np.abs(ref).max() + TD_RTOL * np.abs(ref)
        assert np.all(e <= bound), (name, int(np.argmax(e / np.maximum(bound, 1e-30))))


def test_td_gradient_finite_differences_at_batch_4096():
    """Central finite differences of the GPU's own loss at batch 4,096 (lr = 0
    evaluations by the learner).  gamma = 0 makes the TD target y = r a
    constant, as the semi-gradient assumes (with gamma > 0 the online
    network's argmax inside the double-DQN target flips under a perturbation
    and the loss is not differentiable there).  Every perturbation moves the
    bf16 weight image exactly: weights go to bf16 values, and the difference
    of the two parameter vectors that were actually used enters the
    directional derivative g . (theta+ - theta-).

    * Head (W3, b3: the loss is smooth in them): 16 single entries, the
      largest gradients of each block, within 1e-2 relative.
    * Hidden layers (W1, b1, W2, b2): the activations are rounded to bf16, so
      the loss is a fine staircase in these parameters; a random direction
      over the whole block, moving every entry by 5% of its size, gives a
      secant that is checked in sign and size (within 35%; the oracle's bf16
      recipe shows up to 15% on such secants)."""
    batch = 4096
    g, q, rp, th_on, th_tg = _td_case(batch, "dueling", n_envs=256)
    seed = 91
    rng = np.random.default_rng(4)

    def loss_grad(th):
        q.set_params(th, "online")
        q.set_params(th_tg, "target")
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(q.n_params, device="cuda")
        q.train_step(rp, batch, gamma=0.0, lr=0.0, seed=seed, loss=loss, grad=grad)
        torch.cuda.synchronize()
        return float(loss.item()), grad.cpu().numpy().astype(np.float64)

    _, gg = loss_grad(th_on)
    blocks = dict(_blocks(g.obs_dim))

    def moved(sl, delta, is_w):
        th = th_on.copy()
        v = (th_on[sl].astype(np.float64) + delta).astype(np.float32)
        th[sl] = OQ.bf16_round(v) if is_w else v
        return th

    worst = {}
    for name in ("W3", "b3"):
        sl = blocks[name]
        for j in np.argsort(np.abs(gg[sl]))[::-1][:8]:
            k = sl.start + int(j)
            # W3: 16 bf16 steps of the weight; b3 (float32 in the image): 5%.
            # The float32 loss itself carries ~1e-7 relative rounding, so the
            # step must move it by far more than that.
            h = 16.0 * 2.0 ** (np.floor(np.log2(abs(float(th_on[k])))) - 7) if name == "W3" \
                else 5e-2 * abs(float(th_on[k])) + 1e-3
            kp = moved(slice(k, k + 1), h, name == "W3")
            km = moved(slice(k, k + 1), -h, name == "W3")
            lp, lm = loss_grad(kp)[0], loss_grad(km)[0]
            an = gg[k] * (float(kp[k]) - float(km[k]))
            rel = abs((lp - lm) - an) / abs(an)
            worst[name] = max(worst.get(name, 0.0), rel)
            assert rel <= 1e-2, (name, k, lp - lm, an)
    for name in ("W1", "b1", "W2", "b2"):
        sl = blocks[name]
        for trial in range(3):
            d = rng.choice([-1.0, 1.0], size=sl.stop - sl.start) * np.abs(th_on[sl]) * 5e-2
            kp = moved(sl, d, name.startswith("W"))
            km = moved(sl, -d, name.startswith("W"))
            lp, lm = loss_grad(kp)[0], loss_grad(km)[0]
            an = float(gg @ (kp.astype(np.float64) - km.astype(np.float64)))
            rel = abs((lp - lm) - an) / abs(an)
            worst[name] = max(worst.get(name, 0.0), rel)
            assert rel <= 0.35, (name, trial, lp - lm, an)
    print("finite differences, worst relative difference per block: "
          + ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))


@pytest.mark.parametrize("batch", [256, 4096])
def test_td_step_with_invalid_action_changes_nothing(batch):
    """A sampled transition whose action is outside the action table (written
    into the ring on purpose) makes the whole step fail: NaN loss and
    gradient, parameters, Adam moments and the step count unchanged (the
    16-sample learner at 256, the tcgen05 learner at 4,096)."""
    g, q, rp, th_on, _ = _td_case(batch, "dueling")
    s, s2, a, r, t = rp.read(0, rp.capacity)
    a = a.copy()
    a[::7] = 9
    rp.write(0, s, s2, a, r, t, rp.steps_recorded())
    m0, v0, st0 = q.optimizer_state()
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(q.n_params, device="cuda")
    q.train_step(rp, batch, gamma=0.98, lr=1e-3, seed=3, loss=loss, grad=grad)
    torch.cuda.synchronize()
    assert np.isnan(loss.item()) and torch.isnan(grad).all()
    assert np.array_equal(q.get_params("online"), th_on)
    m1, v1, st1 = q.optimizer_state()
    assert st1 == st0 and np.array_equal(m1, m0) and np.array_equal(v1, v0)
    # valid actions again: the next step updates
    a[::7] = 0
    rp.write(0, s, s2, a, r, t, rp.steps_recorded())
    q.train_step(rp, batch, gamma=0.98, lr=1e-3, seed=3, loss=loss)
    torch.cuda.synchronize()
    assert np.isfinite(loss.item()) and q.optimizer_state()[2] == st0 + 1


def _blocks(n_in, arch="dueling"):
    o = 0
    out = []
    for name, shp in OQ.param_shapes(n_in, arch):
        k = int(np.prod(shp))
        out.append((name, slice(o, o + k)))
        o += k
    return out


@pytest.mark.parametrize("arch", ["dueling", "paper"])
def test_adam_step_and_target_sync(arch):
    g, q, rp = _fill_replay(arch=arch)
    th = _theta(10, g.obs_dim, scale=1.0, arch=arch)
    q.set_params(th)
    grad = torch.zeros(q.n_params, device="cuda")
    q.train_step(rp, 64, lr=0.0, seed=7, grad=grad)  # gradient at step 0
    g0 = grad.cpu().numpy().astype(np.float64)
    q.train_step(rp, 64, lr=1e-3, target_every=3, seed=7)  # the same batch (step 0), now updating
    th1 = q.get_params("online").astype(np.float64)
    ref, m, v = OQ.adam_step(th.astype(np.float64), g0, np.zeros_like(g0), np.zeros_like(g0), 1, lr=1e-3)
    assert np.max(np.abs(th1 - ref)) <= 2e-6
    mg, vg, steps = q.optimizer_state()
    assert steps == 1
    assert np.allclose(mg, m, rtol=1e-5, atol=1e-12) and np.allclose(vg, v, rtol=1e-4, atol=1e-15)
    # target copy unchanged until the step count reaches 3
    assert np.array_equal(q.get_params("target"), th.astype(np.float32))
    q.train_step(rp, 64, lr=1e-3, target_every=3, seed=7)
    assert np.array_equal(q.get_params("target"), th.astype(np.float32))
    q.train_step(rp, 64, lr=1e-3, target_every=3, seed=7)
    assert np.array_equal(q.get_params("target"), q.get_params("online"))
    # the inference copy follows the master weights: forward equals a fresh net with those weights
    obs = torch.rand((40, g.obs_dim), device="cuda")
    q2 = _qnet(g.obs_dim, arch=arch)
    q2.set_params(q.get_params("online"))
    assert torch.equal(q.forward(obs), q2.forward(obs))
