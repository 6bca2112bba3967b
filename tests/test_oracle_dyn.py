"""Pins of the oracle's dynamic obstacles (the extension the paper names as
future work in Sec. 5) against closed forms and invariants that do not come
from the oracle: straight-line motion folded at the walls (a triangle wave),
the stop-and-reverse rule at occupied cells, the centre-distance collision
threshold, the first march sample inside a disc from the ray-circle
intersection, the episode draws' ranges and uniformity, and the order of the
step (obstacles move before the collision test and the scan).  CPU only.
"""

import math

import numpy as np
import pytest

from oracle.sim import OracleSim
from workloads.configs import base_params
from workloads.maps import empty_map, make_map

R_O = 8.0


def _params(n_dyn=1, **kw):
    p = base_params(n_dyn=n_dyn, dyn_radius=R_O, dyn_speed_lo=10.0, dyn_speed_hi=10.0, dyn_keepout=60.0,
                    t_max=10 ** 6)
    p.update(kw)
    return p


def _sim(prec, grid, n_envs=1, **kw):
    return OracleSim(_params(**kw), [grid], np.zeros(n_envs, np.int32), prec=prec)


def _set_obstacle(o, i, k, x, y, vx, vy):
    f, u, b, d = o.state()
    d[4 * k:4 * k + 4, i] = (x, y, vx, vy)
    o.set_state(f, u, b, d)


def _set_pose(o, i, x, y, phi):
    f, u, b, d = o.state()
    f[0, i], f[1, i], f[2, i], f[3, i], f[4, i] = x, y, phi, 0.0, 0.0
    o.set_state(f, u, b, d)


def _fold(s, lo, L):
    """Unfolded travel s from lo folded into [lo, lo + L] (mirror walls):
    position and the sign of the velocity (+1 moving up)."""
    q = math.fmod(s, 2 * L)
    if q < 0:
        q += 2 * L
    return (lo + q, 1.0) if q <= L else (lo + 2 * L - q, -1.0)


@pytest.mark.parametrize("vx,vy", [(37.0, 11.0), (-23.5, 41.25), (5.0, -60.0)])
def test_motion_is_a_triangle_wave_between_the_walls(vx, vy):
    W, H, dt, n = 160, 120, 0.1, 700
    o = _sim("f64", empty_map(W, H))
    o.reset()
    x0, y0 = 50.3, 70.9
    _set_obstacle(o, 0, 0, x0, y0, vx, vy)
    for _ in range(n):
        o.dyn_advance(0, dt)
    x, y, gvx, gvy = o.dyn[:, 0]
    ex, sx = _fold(x0 - R_O + n * dt * vx, R_O, W - 2 * R_O)
    ey, sy = _fold(y0 - R_O + n * dt * vy, R_O, H - 2 * R_O)
    assert abs(x - ex) < 1e-9 and abs(y - ey) < 1e-9
    # the velocity keeps its magnitude and points along the folded motion
    assert gvx == pytest.approx(sx * math.copysign(abs(vx), vx)) and gvy == pytest.approx(sy * math.copysign(abs(vy), vy))


def test_occupied_cell_stops_and_reverses():
    g = empty_map(400)
    g[:, 200:211] = 1  # a wall of columns 200..210
    o = _sim("f64", g)
    o.reset()
    _set_obstacle(o, 0, 0, 150.0, 100.5, 10.0, 0.0)
    xs = []
    for _ in range(14):
        o.dyn_advance(0, 0.5)
        xs.append(float(o.dyn[0, 0]))
    # 5 cells per step: 155 .. 195, then 200.0 would be in column 200: stay
    # at 195 with the velocity reversed, then back 190, 185, ...
    assert xs[:9] == [155.0 + 5 * k for k in range(9)]
    assert xs[9] == 195.0
    assert xs[10:] == [190.0, 185.0, 180.0, 175.0]
    assert o.dyn[1, 0] == 100.5 and o.dyn[2, 0] == -10.0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_obstacles_stay_in_the_box_and_off_occupied_cells(prec):
    g = make_map(7, 366)
    n = 64
    o = OracleSim(_params(n_dyn=6, dyn_speed_lo=5.0, dyn_speed_hi=60.0), [g], np.zeros(n, np.int32), prec=prec)
    o.reset()
    f, _, _, d = o.state()
    free0 = np.array([[g[int(d[4 * k + 1, i]), int(d[4 * k, i])] == 0 for i in range(n)] for k in range(6)])
    for _ in range(300):
        for i in range(n):
            o.dyn_advance(i, 0.2)
        x, y = o.dyn[0::4], o.dyn[1::4]
        assert (x >= R_O).all() and (x <= 366 - R_O).all() and (y >= R_O).all() and (y <= 366 - R_O).all()
        cells = g[np.floor(y).astype(int), np.floor(x).astype(int)]
        # an obstacle that started on a free cell never enters an occupied one
        assert not (cells[free0] != 0).any()


@pytest.mark.parametrize("prec,eps", [("f64", 1e-9), ("f32", 1e-4)])
def test_collision_threshold_is_the_sum_of_radii(prec, eps):
    o = _sim(prec, empty_map(400), n_dyn=2, robot_radius=10.0)
    o.reset()
    rng = np.random.default_rng(3)
    rr = 10.0 + R_O
    for _ in range(200):
        cx, cy = rng.uniform(100, 300, 2)
        a = rng.uniform(-math.pi, math.pi)
        _set_obstacle(o, 0, 0, cx, cy, 0.0, 0.0)
        _set_obstacle(o, 0, 1, 5.0e3, 5.0e3, 0.0, 0.0)  # far away
        for scale, want in ((1 - eps, True), (1 + eps, False)):
            x = cx + rr * scale * math.cos(a)
            y = cy + rr * scale * math.sin(a)
            assert o.dyn_collide(0, x, y) == want


def _first_inside(px, py, ux, uy, cx, cy, r, delta, kmax):
    """First k >= 1 with |p + k delta u - c| <= r, from the ray-circle
    intersection [t1, t2]; None when no sample up to kmax is inside.  Also
    returns how close t1/delta, t2/delta come to an integer (ties)."""
    dx, dy = px - cx, py - cy
    bq = dx * ux + dy * uy
    cq = dx * dx + dy * dy - r * r
    disc = bq * bq - cq
    if disc < 0:
        return None, 1.0
    sq = math.sqrt(disc)
    t1, t2 = -bq - sq, -bq + sq
    k = max(1, math.ceil(t1 / delta))
    tie = min(abs(t1 / delta - round(t1 / delta)), abs(t2 / delta - round(t2 / delta)))
    if k * delta > t2 or k > kmax:
        return None, tie
    return k, tie


@pytest.mark.parametrize("delta", [1.0, 0.37])
def test_lidar_hits_the_first_sample_inside_a_disc(delta):
    rmax = 100.0
    nb = 32
    o = OracleSim(_params(n_dyn=3, march_step=delta, range_max=rmax, n_beams=nb), [empty_map(2000)],
                  np.zeros(1, np.int32), prec="f64")
    kmax = math.floor(rmax / delta)
    fov = o.params["fov"]
    rng = np.random.default_rng(11)
    checked = hits = 0
    for _ in range(300):
        x, y = 1000.0 + rng.uniform(0, 1), 1000.0 + rng.uniform(0, 1)
        phi = rng.uniform(-math.pi, math.pi)
        discs = []
        for _ in range(3):
            # aim at a random beam direction, at a lateral offset up to 1.5 r
            j = rng.integers(nb)
            beta = phi + (j * (fov / (nb - 1)) - fov * 0.5)
            ux, uy = -math.cos(beta), -math.sin(beta)
            t = rng.uniform(-5, rmax + 10)
            b = rng.uniform(-1.5, 1.5) * R_O
            discs.append((x + t * ux - b * uy, y + t * uy + b * ux))
        got, _ = o.lidar_dyn(0, discs, x, y, phi, nb)
        for j in range(nb):
            beta = phi + (j * (fov / (nb - 1)) - fov * 0.5)
            ux, uy = -math.cos(beta), -math.sin(beta)
            best, near_tie = kmax + 1, 1.0
            for cx, cy in discs:
                k, tie = _first_inside(x, y, ux, uy, cx, cy, R_O, delta, kmax)
                near_tie = min(near_tie, tie)
                if k is not None:
                    best = min(best, k)
            if near_tie < 1e-7:
                continue
            checked += 1
            hits += best <= kmax
            assert got[j] == best, (j, got[j], best)
    assert checked > 8000 and hits > 500


def test_no_obstacles_means_no_disc_hits():
    o = OracleSim(_params(n_dyn=0), [empty_map(2000)], np.zeros(1, np.int32), prec="f64")
    h, r = o.lidar_dyn(0, [], 1000.5, 1000.5, 0.3, 32)
    assert (h == math.floor(100.0 / 1.0) + 1).all() and (r == 100.0).all()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_episode_draws(prec):
    g = make_map(5, 366)
    n, nd = 512, 8
    lo, hi, keep = 4.0, 30.0, 60.0
    o = OracleSim(_params(n_dyn=nd, dyn_speed_lo=lo, dyn_speed_hi=hi, dyn_keepout=keep), [g],
                  np.zeros(n, np.int32), prec=prec)
    o.reset()
    d = o.state()[3]
    x, y, vx, vy = d[0::4].ravel(), d[1::4].ravel(), d[2::4].ravel(), d[3::4].ravel()
    assert (x >= R_O).all() and (x <= 366 - R_O).all() and (y >= R_O).all() and (y <= 366 - R_O).all()
    sp = np.hypot(vx, vy)
    tol = 1e-4 if prec == "f32" else 1e-9
    assert (sp >= lo - tol).all() and (sp <= hi + tol).all()
    # headings uniform: the mean unit vector is near zero (4096 draws)
    assert abs(np.mean(vx / sp)) < 0.05 and abs(np.mean(vy / sp)) < 0.05
    # accepted centres: on a free cell and farther than the keep-out from S and G
    S, G = (30.0, 30.0), (336.0, 336.0)
    ok = ((g[np.floor(y).astype(int), np.floor(x).astype(int)] == 0)
          & (np.hypot(x - S[0], y - S[1]) > keep) & (np.hypot(x - G[0], y - G[1]) > keep))
    assert ok.mean() > 0.995
    # the same draws on a second reset; different ones for the next episode
    o2 = OracleSim(o.params, [g], np.zeros(n, np.int32), prec=prec)
    o2.reset()
    assert np.array_equal(o2.dyn, o.dyn)
    o2.reset_env(3, 1)
    assert not np.array_equal(o2.dyn[:, 3], o.dyn[:, 3])


def test_draws_are_uniform_over_the_box_on_an_empty_map():
    W = 400
    n = 2048
    o = OracleSim(_params(n_dyn=2, dyn_keepout=0.0, dyn_speed_lo=1.0, dyn_speed_hi=30.0), [empty_map(W)],
                  np.zeros(n, np.int32), prec="f64")
    o.reset()
    x, y = o.dyn[0::4].ravel(), o.dyn[1::4].ravel()
    vx, vy = o.dyn[2::4].ravel(), o.dyn[3::4].ravel()
    # position, heading and speed are independent draws
    th, sp = np.arctan2(vy, vx), np.hypot(vx, vy)
    for a in (x, y):
        for b in (th, sp):
            assert abs(np.corrcoef(a, b)[0, 1]) < 0.1
    bx = np.minimum(((x - R_O) / (W - 2 * R_O) * 4).astype(int), 3)
    by = np.minimum(((y - R_O) / (W - 2 * R_O) * 4).astype(int), 3)
    cnt = np.bincount(bx * 4 + by, minlength=16)
    e = x.size / 16
    assert ((cnt - e) ** 2 / e).sum() < 40.0  # 15 dof


def _still_sim(prec, nb=3):
    # one action that targets zero velocity: the robot stays put
    return OracleSim(_params(n_dyn=1, n_beams=nb, actions=[(0.0, 0.0)], fov=float(np.float32(1.5 * math.pi))),
                     [empty_map(2000)], np.zeros(1, np.int32), prec=prec)


def test_step_moves_obstacles_before_collision_and_scan():
    o = _still_sim("f64")
    o.reset()
    _set_pose(o, 0, 1000.0, 1000.0, 0.0)  # forward is (-1, 0)
    f, u, b, d = o.state()
    f[5, 0] = 0.1  # dt
    o.set_state(f, u, b, d)
    # disc 30 cells ahead coming closer at 50 cells/s: 5 cells per step
    _set_obstacle(o, 0, 0, 970.0, 1000.0, 50.0, 0.0)
    obs, rew, done, _ = o.step(np.zeros(1, np.uint8))
    assert done[0] == 0
    assert o.dyn[0, 0] == 975.0
    # the centre beam (offset 0) enters the moved disc at 25 - 8 = 17 cells
    assert obs[0, 1] == pytest.approx(17.0 / 100.0)
    # two more steps: 980 (distance 20 > 18), then 985 (15 <= 18): collision
    o.step(np.zeros(1, np.uint8))
    ep = o.u[1, 0]
    _, rew, done, term = o.step(np.zeros(1, np.uint8))
    assert done[0] & 1 and rew[0] == -10.0
    # AutoReset re-drew the obstacles as episode ep + 1 of this env
    ref = _still_sim("f64")
    ref.reset()
    ref.reset_env(0, int(ep) + 1)
    assert np.array_equal(o.dyn, ref.dyn) and o.u[1, 0] == ep + 1


def test_moving_away_does_not_collide():
    o = _still_sim("f64")
    o.reset()
    _set_pose(o, 0, 1000.0, 1000.0, 0.0)
    _set_obstacle(o, 0, 0, 1000.0, 1017.0, 0.0, 50.0)  # 17 < 18 now, moving away
    _, _, done, _ = o.step(np.zeros(1, np.uint8))
    assert done[0] & 1 == 0


def test_without_obstacles_the_step_is_unchanged():
    g = make_map(2, 366)
    n = 32
    a = OracleSim(base_params(), [g], np.zeros(n, np.int32), prec="f32")
    p = base_params(n_dyn=0, dyn_radius=8.0, dyn_speed_lo=1.0, dyn_speed_hi=2.0, dyn_keepout=10.0)
    b = OracleSim(p, [g], np.zeros(n, np.int32), prec="f32")
    oa, ob = a.reset(), b.reset()
    assert np.array_equal(oa, ob)
    rng = np.random.default_rng(0)
    for _ in range(50):
        act = rng.integers(0, 5, n).astype(np.uint8)
        ra, rb = a.step(act), b.step(act)
        for x, y in zip(ra, rb):
            assert np.array_equal(x, y)
