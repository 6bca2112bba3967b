"""GPU parity of the simulator against the CPU oracle (through the C ABI).

Bar: against the strict-float32 oracle everything is bit-exact (state, obs,
rewards, done flags, term obs, atlas).  Against the float64 oracle pose and
velocity agree within 1e-5 relative and noise-free ranges are equal in
>= 99.99% of beams, otherwise within one march step.
"""

import math

import numpy as np
import pytest
import torch

from oracle.sim import OracleSim, pack_map
from tests._helpers import bits, gpu_state_to_oracle, oracle_state_to_gpu, step_rel_error
from workloads import workload
from workloads.configs import base_params
from workloads.maps import empty_map, make_map, random_tiny_map

pytestmark = pytest.mark.gpu


def _sim(params, maps, env_map, env_beams=None):
    from paper_2305_04180_gb300 import Sim

    return Sim(params, maps, env_map, env_beams)


def _pair(w_or_params, maps=None, env_map=None, env_beams=None):
    if maps is None:
        w = w_or_params
        maps = w.maps()
        params, env_map, env_beams = w.params, w.env_map, w.env_beams
    else:
        params = w_or_params
    g = _sim(params, maps, env_map, env_beams)
    o = OracleSim(params, maps, env_map, env_beams, prec="f32")
    return g, o, maps


def _assert_state_equal(g, o, t):
    f, u = g.get_state()
    of, ou, ob = o.state()
    gf, gu = oracle_state_to_gpu(of, ou, ob, t)
    assert np.array_equal(bits(f), bits(gf)), np.argwhere(bits(f) != bits(gf))[:5]
    assert np.array_equal(u, gu), np.argwhere(u != gu)[:5]


def test_atlas_bit_exact():
    maps = [make_map(1), make_map(2, 128), make_map(3, 200, 77), random_tiny_map(4, 33, 5, 0.5),
            random_tiny_map(5, 1, 1, 1.0), make_map(6, 1024)]
    g = _sim(base_params(), maps, np.arange(6, dtype=np.int32) % 6)
    atlas, offs, rw = g.atlas()
    for m, grid in enumerate(maps):
        h = grid.shape[0]
        ref = pack_map(grid, int(rw[m]))
        got = atlas[offs[m]: offs[m] + h * rw[m]].reshape(h, rw[m])
        assert np.array_equal(got, ref)
        assert rw[m] % 4 == 0  # rows are 16-byte aligned


@pytest.mark.parametrize("name,n", [("plain16", 16), ("dr1024", 1024), ("dr1024", 37)])
def test_reset_bit_exact(name, n):
    g, o, _ = _pair(workload(name, n_envs=n))
    obs = g.reset().cpu().numpy()
    oobs = o.reset()
    assert np.array_equal(bits(obs), bits(oobs))
    _assert_state_equal(g, o, 0)


def _teacher_forced(g, o, steps, seed=0, act_fn=None):
    """Every step both sides start from the same state bits and take the same
    actions; every output must match bit for bit."""
    n = g.n
    obs = g.reset()
    o.reset()
    term = torch.full((n, g.obs_dim), float("nan"), device="cuda")
    rng = np.random.default_rng(seed)
    checked = 0
    for t in range(steps):
        a = rng.integers(0, 5, size=n).astype(np.uint8) if act_fn is None else act_fn(t)
        f, u = g.get_state()
        o.set_state(*gpu_state_to_oracle(f, u))
        at = torch.from_numpy(a).cuda()
        obs, rew, done = g.step(at, term_obs=term)
        oobs, orew, odone, oterm = o.step(a)
        d = done.cpu().numpy()
        assert np.array_equal(d, odone), (t, np.argwhere(d != odone)[:5])
        assert np.array_equal(bits(rew.cpu().numpy()), bits(orew)), t
        assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs)), t
        if d.any():
            tg = term.cpu().numpy()[d != 0]
            assert np.array_equal(bits(tg), bits(oterm[d != 0])), t
        _assert_state_equal(g, o, t + 1)
        checked += n
    return checked


def test_step_teacher_forced_plain16():
    g, o, _ = _pair(workload("plain16"))
    assert _teacher_forced(g, o, 400) == 6400


def test_step_teacher_forced_domain_randomised():
    """1024 envs over 32 maps with every randomisation on (delay, K, cap,
    noise, control interval): 1,000 steps = 1,024,000 env-steps, every one
    teacher-forced from the GPU's state."""
    g, o, _ = _pair(workload("dr1024"))
    assert _teacher_forced(g, o, 1000, seed=1) == 1024000


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"),
                                    dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=512)])
def test_rollout_plain16_million_env_steps(launch):
    """The 16-env workload free-running for 62,500 steps (10^6 env-steps):
    every step's action, reward and done flags and the final state equal the
    oracle's."""
    w = workload("plain16")
    g, o, _ = _pair(w)
    if launch:
        g.set_launch(**launch)
    g.reset()
    o.reset()
    K = 62500
    n = g.n
    act = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    obs = g.new_obs()
    g.rollout(K, obs=obs, act_seq=act, rew_seq=rew, done_seq=done)
    oobs, oact, orew, odone = o.rollout_random(K, 0)
    assert np.array_equal(act.cpu().numpy(), oact)
    assert np.array_equal(done.cpu().numpy(), odone)
    assert np.array_equal(bits(rew.cpu().numpy()), bits(orew))
    assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs))
    _assert_state_equal(g, o, K)
    assert int((odone != 0).sum()) > 1000


def test_step_uneven_beams_and_ragged_batch():
    """Per-env beam counts 2..64 on mixed map sizes, N not a multiple of the
    envs per block."""
    p = base_params(n_beams=64, **{k: v for k, v in workload("dr1024").params.items() if k.endswith(("_lo", "_hi"))})
    maps = [make_map(11, 128), make_map(12, 366), make_map(13, 512), make_map(14, 256, 300)]
    n = 29
    rng = np.random.default_rng(2)
    env_map = rng.integers(0, 4, n).astype(np.int32)
    beams = rng.choice([2, 3, 16, 31, 32, 33, 64], n).astype(np.int32)
    g, o, _ = _pair(p, maps, env_map, beams)
    _teacher_forced(g, o, 150, seed=3)


def test_step_degenerate_cases():
    """N = 1; a map smaller than the start offset (the robot starts outside
    and collides every step); a 1x1 map; a map with no obstacle and no
    border; the out-of-range action index sets the device status bit."""
    p = base_params()
    for maps in ([random_tiny_map(7, 20, 20, 0.1)], [np.ones((1, 1), np.uint8)], [empty_map(400)]):
        g, o, _ = _pair(p, maps, np.zeros(1, np.int32))
        _teacher_forced(g, o, 30, seed=4)
        assert g.status() == 0
    g, o, _ = _pair(p, [make_map(1)], np.zeros(3, np.int32))
    bad = np.array([0, 7, 255], np.uint8)
    _teacher_forced(g, o, 5, act_fn=lambda t: bad)
    assert g.status() == 1
    assert g.status() == 0  # reading clears it


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"),
                                    dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=512)])
def test_rollout_random_free_running_bit_exact(launch):
    """1000 free-running steps with on-device random actions: every step's
    action, reward, done flags and observation, and the final state, equal
    the oracle's (one warp per env, and the pipelined kernel the benchmark
    times)."""
    w = workload("plain16")
    g, o, _ = _pair(w)
    if launch:
        g.set_launch(**launch)
    g.reset()
    o.reset()
    K = 1000
    n = g.n
    obs = g.new_obs()
    obs_seq = torch.empty((K, n, g.obs_dim), dtype=torch.float32, device="cuda")
    act = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    rew = torch.empty((K, n), dtype=torch.float32, device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    g.rollout(K, obs=obs, obs_seq=obs_seq, act_seq=act, rew_seq=rew, done_seq=done)
    act, rew, done, obs_seq = act.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), obs_seq.cpu().numpy()
    ndone = 0
    for k in range(K):
        a = o.random_actions(k)
        assert np.array_equal(act[k], a), k
        oobs, orew, odone, _ = o.step(a)
        assert np.array_equal(done[k], odone), k
        assert np.array_equal(bits(rew[k]), bits(orew)), k
        assert np.array_equal(bits(obs_seq[k]), bits(oobs)), k
        ndone += int((odone != 0).sum())
    assert np.array_equal(bits(obs.cpu().numpy()), bits(oobs))
    _assert_state_equal(g, o, K)
    assert ndone > 100  # episodes did end and reset


def test_rollout_continues_across_calls_and_matches_steps():
    """Two rollouts of K/2 equal one of K; state and RNG counters persist."""
    w = workload("dr1024", n_envs=64)
    maps = w.maps()
    a = _sim(w.params, maps, w.env_map)
    b = _sim(w.params, maps, w.env_map)
    a.reset()
    b.reset()
    ra = torch.empty((100, 64), device="cuda")
    rb = torch.empty((100, 64), device="cuda")
    a.rollout(100, rew_seq=ra)
    b.rollout(50, rew_seq=rb[:50])
    b.rollout(50, rew_seq=rb[50:])
    assert torch.equal(ra, rb)
    fa, ua = a.get_state()
    fb, ub = b.get_state()
    assert np.array_equal(bits(fa), bits(fb)) and np.array_equal(ua, ub)


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"),
                                    dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=512)])
def test_rollout_full_size_sampled_against_oracle(launch):
    """The 1024-env, 32-map domain-randomised workload (one warp per env, and
    the pipelined launch the benchmark times): 300 steps on the GPU, then a
    sample of envs replayed one by one on the oracle from the same start."""
    w = workload("dr1024")
    maps = w.maps()
    g = _sim(w.params, maps, w.env_map)
    if launch:
        g.set_launch(**launch)
    g.reset()
    K = 300
    rew = torch.empty((K, g.n), device="cuda")
    done = torch.empty((K, g.n), dtype=torch.uint8, device="cuda")
    g.rollout(K, rew_seq=rew, done_seq=done)
    rew = rew.cpu().numpy()
    done = done.cpu().numpy()
    f, u = g.get_state()
    o = OracleSim(w.params, maps, w.env_map, prec="f32")
    for i in [0, 1, 31, 32, 500, 777, 1023]:
        o.reset_env(i, 0)
        for k in range(K):
            _, orew, odone, _ = o.step_one(i, o.random_action(i, k))
            assert odone == done[k, i] and bits(np.float32(orew)) == bits(rew[k, i]), (i, k)
        assert np.array_equal(bits(o.f[:, i]), bits(f[:, i]))
        assert np.array_equal(o.u[:, i], u[:2, i])


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map"),
                                    dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map", segment=512)])
def test_uneven_full_size_sampled_against_oracle(launch):
    """The 8,192-env uneven workload at full size (one map per env, sides
    128..1,024, 16/32/64 beams, per-env dynamics): 64 steps on the GPU, then
    sampled envs (every map size and beam count) replayed one by one on the
    oracle, which holds only their maps (1x1 placeholders for the others, so
    env indices and random streams are unchanged)."""
    w = workload("uneven8192")
    maps = w.maps()
    g = _sim(w.params, maps, w.env_map, w.env_beams)
    if launch:
        g.set_launch(**launch)
    g.reset()
    K = w.steps
    rew = torch.empty((K, g.n), device="cuda")
    done = torch.empty((K, g.n), dtype=torch.uint8, device="cuda")
    g.rollout(K, rew_seq=rew, done_seq=done)
    rew = rew.cpu().numpy()
    done = done.cpu().numpy()
    f, u = g.get_state()
    sides = np.array([m.shape[1] for m in maps])
    sample = [0, 1, 8191]
    for side in np.unique(sides):
        for nb in (16, 32, 64):
            cand = np.flatnonzero((sides[w.env_map] == side) & (w.env_beams == nb))
            if cand.size:
                sample.append(int(cand[len(cand) // 2]))
    keep = {int(w.env_map[i]) for i in sample}
    tiny = np.ones((1, 1), np.uint8)
    o = OracleSim(w.params, [maps[m] if m in keep else tiny for m in range(len(maps))], w.env_map, w.env_beams,
                  prec="f32")
    for i in sample:
        o.reset_env(i, 0)
        for k in range(K):
            _, orew, odone, _ = o.step_one(i, o.random_action(i, k))
            assert odone == done[k, i] and bits(np.float32(orew)) == bits(rew[k, i]), (i, k)
        assert np.array_equal(bits(o.f[:, i]), bits(f[:, i])), i
        assert np.array_equal(o.u[:, i], u[:2, i]), i
    assert len(sample) >= 12


def test_against_float64_oracle_tolerances():
    """Teacher forced against the float64 oracle (noise off so that ranges
    are comparable): pose/velocity within 1e-5 relative; ranges equal in
    >= 99.99% of beams and otherwise one march step apart; discrete flags
    equal wherever they are not decided within float rounding."""
    p = dict(workload("dr1024").params, sigma_lo=0.0, sigma_hi=0.0)
    maps = [make_map(s) for s in range(1, 33)]
    env_map = (np.arange(1024) % 32).astype(np.int32)
    g = _sim(p, maps, env_map)
    o = OracleSim(p, maps, env_map, prec="f64")
    g.reset()
    rng = np.random.default_rng(8)
    tot = diff = 0
    for t in range(60):
        f, u = g.get_state()
        of, ou, ob = gpu_state_to_oracle(f, u)
        o.set_state(of.astype(np.float64), ou, ob)
        a = rng.integers(0, 5, size=1024).astype(np.uint8)
        obs, rew, done = g.step(torch.from_numpy(a).cuda())
        oobs, orew, odone, _ = o.step(a)
        d = done.cpu().numpy()
        live = (d == 0) & (odone == 0)
        f2, _ = g.get_state()
        rel = step_rel_error(f[:, live], f2[:, live], o.f[:, live])
        assert rel.max() <= 1e-5
        gr = np.rint(obs.cpu().numpy()[live, :32] * 100.0)
        orr = np.rint(oobs[live, :32] * 100.0)
        dd = np.abs(gr - orr)
        assert dd.max() <= 1.0
        tot += dd.size
        diff += int((dd > 0).sum())
        assert (d != odone).mean() <= 1e-3
    assert diff / tot <= 1e-4, (diff, tot)


@pytest.mark.parametrize("sectors", [4, 16, 32])
def test_sector_skip_planes_are_safe(sectors):
    """Every value of the march's sector skip planes is a safe skip, checked
    by brute force independently of how the library builds them: from points
    spread over a free cell (its corners pulled in by 1e-3 and interior
    points), along directions spread over the sector widened by 5 mrad, the
    march samples 1 .. J-1 cells ahead all fall in free cells of the map.
    Also J is at least the Chebyshev skip of the cell (so the planes never
    slow the march down), and occupied cells hold 0."""
    maps = [random_tiny_map(11, 37, 29, 0.15), make_map(5, 96), random_tiny_map(12, 64, 16, 0.05)]
    g = _sim(dict(base_params(), march_sectors=sectors), maps, np.arange(len(maps), dtype=np.int32))
    planes, offs, S = g.sector_skip()
    assert S == sectors
    clr, coffs = g.clearance()
    frac = np.array([1e-3, 0.27, 0.5, 0.81, 1 - 1e-3])
    qx, qy = (a.ravel() for a in np.meshgrid(frac, frac))
    rng = np.random.default_rng(sectors)
    longer = 0
    for m, grid in enumerate(maps):
        h, w = grid.shape
        cheb = clr[coffs[m]:coffs[m] + w * h].reshape(h, w).astype(np.int64)
        for sct in range(S):
            J = planes[offs[m] + sct * w * h:offs[m] + (sct + 1) * w * h].reshape(h, w).astype(np.int64)
            assert np.all((J == 0) == (grid != 0)), (m, sct)
            assert np.all(J >= cheb), (m, sct)
            longer += int((J > cheb).sum())
            a0 = -np.pi + sct * 2 * np.pi / S - 5e-3
            a1 = -np.pi + (sct + 1) * 2 * np.pi / S + 5e-3
            ang = np.concatenate([[a0, a1], rng.uniform(a0, a1, size=5)])
            # the 150 largest skips of the plane and 250 random cells with J > 1
            ys, xs = np.nonzero(J > 1)
            if ys.size == 0:
                continue
            pick = np.unique(np.concatenate([np.argsort(J[ys, xs])[-150:],
                                             rng.choice(ys.size, size=min(250, ys.size), replace=False)]))
            cy, cx, jj = ys[pick], xs[pick], J[ys[pick], xs[pick]]
            j = np.arange(1, int(jj.max()), dtype=np.float64)
            px = (cx[:, None] + qx[None, :])[:, :, None, None] + j * np.cos(ang)[None, None, :, None]
            py = (cy[:, None] + qy[None, :])[:, :, None, None] + j * np.sin(ang)[None, None, :, None]
            ix, iy = np.floor(px).astype(np.int64), np.floor(py).astype(np.int64)
            live = np.broadcast_to((j[None, :] < jj[:, None])[:, None, None, :], ix.shape)
            inside = (ix >= 0) & (iy >= 0) & (ix < w) & (iy < h)
            assert inside[live].all(), (m, sct)
            free = np.zeros_like(live)
            free[inside] = grid[iy[inside], ix[inside]] == 0
            assert free[live].all(), (m, sct)
    assert longer > 0


def test_march_sectors_leave_results_unchanged():
    """The acceleration structure does not change the step: rollouts with the
    Chebyshev skip map alone and with 4, 16 or 32 sector planes are
    bit-identical (every one is also checked against the oracle elsewhere)."""
    w = workload("dr1024", n_envs=96)
    maps = w.maps()
    out = []
    for sectors in (1, 4, 16, 32):
        g = _sim(dict(w.params, march_sectors=sectors), maps, w.env_map, w.env_beams)
        assert g.info.march_sectors == sectors
        g.reset()
        K = 64
        obs_seq = torch.empty((K, g.n, g.obs_dim), device="cuda")
        rew = torch.empty((K, g.n), device="cuda")
        g.rollout(K, obs_seq=obs_seq, rew_seq=rew)
        out.append((obs_seq.cpu().numpy(), rew.cpu().numpy()))
    for o in out[1:]:
        assert np.array_equal(bits(o[0]), bits(out[0][0])) and np.array_equal(bits(o[1]), bits(out[0][1]))


def test_clearance_matches_chessboard_distance_transform():
    """The march's skip map is the skip value of scipy's chessboard distance
    transform of the free cells (outside of the map counted as occupied,
    capped at 255): 0 on occupied cells, max(1, c - 1) elsewhere."""
    ndimage = pytest.importorskip("scipy.ndimage")
    maps = [make_map(1), make_map(2, 128), make_map(3, 200, 77), random_tiny_map(4, 33, 5, 0.5),
            np.ones((1, 1), np.uint8), empty_map(700), empty_map(9, 600)]
    g = _sim(base_params(), maps, np.arange(len(maps), dtype=np.int32))
    clr, offs = g.clearance()
    for m, grid in enumerate(maps):
        h, w = grid.shape
        pad = np.ones((h + 2, w + 2), np.uint8)
        pad[1:-1, 1:-1] = grid != 0
        ref = ndimage.distance_transform_cdt(pad == 0, metric="chessboard")[1:-1, 1:-1]
        ref = np.minimum(ref, 255).astype(np.int32)
        ref = np.where(ref == 0, 0, np.maximum(1, ref - 1)).astype(np.uint8)
        got = clr[offs[m]: offs[m] + h * w].reshape(h, w)
        assert np.array_equal(got, ref), m


@pytest.mark.parametrize("delta,rmax", [(0.5, 60.0), (1.5, 120.0), (1.0, 250.0)])
def test_step_other_march_steps(delta, rmax):
    """Sample spacing below one cell (clearance skipping on), above one cell
    (skipping off), and a range beyond the clearance cap."""
    p = dict(workload("dr1024").params, march_step=delta, range_max=rmax)
    maps = [make_map(s) for s in range(1, 5)] + [empty_map(600)]
    env_map = (np.arange(40) % 5).astype(np.int32)
    g, o, _ = _pair(p, maps, env_map)
    _teacher_forced(g, o, 60, seed=5)


def test_maximum_map_range_and_beams():
    """The largest map side (16,384 cells), the longest range (4,096 samples
    per beam) and the most beams (64): teacher-forced steps bit-exact against
    the oracle, and a pipelined rollout from the same start equal to it."""
    side = 16384
    grid = empty_map(side)
    rng = np.random.default_rng(8)
    for _ in range(300):
        x0, y0 = rng.integers(0, 4000, 2)
        wx, wy = rng.integers(2, 60, 2)
        grid[y0:y0 + wy, x0:x0 + wx] = 1
    grid[:80, :80] = 0  # a clear start
    p = base_params(n_beams=64, range_max=4096.0, march_step=1.0, **{k: v for k, v in workload("dr1024").params.items()
                                                                       if k.endswith(("_lo", "_hi"))})
    n = 6
    env_map = np.zeros(n, np.int32)
    g, o, _ = _pair(p, [grid], env_map)
    _teacher_forced(g, o, 25, seed=9)
    # the pipelined kernel from a fresh start against the one-warp-per-env kernel
    runs = []
    for launch in (None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, segment=32)):
        s = _sim(p, [grid], env_map)
        if launch:
            s.set_launch(**launch)
        s.reset()
        rew = torch.empty((100, n), device="cuda")
        obs = s.new_obs()
        s.rollout(100, obs=obs, rew_seq=rew)
        torch.cuda.synchronize()
        assert s.status() == 0
        runs.append((rew.cpu().numpy(), obs.cpu().numpy(), s.get_state()))
    (r0, b0, (f0, u0)), (r1, b1, (f1, u1)) = runs
    assert np.array_equal(bits(r0), bits(r1)) and np.array_equal(bits(b0), bits(b1))
    assert np.array_equal(bits(f0), bits(f1)) and np.array_equal(u0, u1)


@pytest.mark.parametrize("launch", [None, dict(kernel="pipe", warps_per_block=8, obs_warps=7, order="map",
                                                segment=32)])
def test_maximum_env_count_sampled_against_oracle(launch):
    """2^24 envs (the largest batch) on the 32-map domain-randomised
    workload: 64 free-running steps (two 32-step segments in the time-sliced
    launch), then envs at both ends and in between replayed one by one on
    the oracle."""
    n = 1 << 24
    w = workload("dr1024", n_envs=n)
    maps = w.maps()
    g = _sim(w.params, maps, w.env_map)
    if launch:
        g.set_launch(**launch)
    g.reset()
    K = 64
    rew = torch.empty((K, n), device="cuda")
    done = torch.empty((K, n), dtype=torch.uint8, device="cuda")
    obs = g.new_obs()
    g.rollout(K, obs=obs, rew_seq=rew, done_seq=done)
    torch.cuda.synchronize()
    assert g.status() == 0
    sample = np.array([0, 1, 31, 4095, 1 << 20, (1 << 23) + 7, n - 33, n - 2, n - 1])
    idx = torch.from_numpy(sample).cuda()
    rew_s = rew[:, idx].cpu().numpy()
    done_s = done[:, idx].cpu().numpy()
    obs_s = obs[idx].cpu().numpy()
    o = OracleSim(w.params, maps, w.env_map, prec="f32")
    for j, i in enumerate(sample):
        o.reset_env(int(i), 0)
        for k in range(K):
            oobs, orew, odone, _ = o.step_one(int(i), o.random_action(int(i), k))
            assert odone == done_s[k, j] and bits(np.float32(orew)) == bits(rew_s[k, j]), (i, k)
        assert np.array_equal(bits(oobs), bits(obs_s[j])), i
