"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one part of the step against a closed form, a library
routine, an independent algorithm or a value printed in the paper, so that a
dropped term, a wrong sign, a swapped axis or an off-by-one in the oracle
fails here.  All CPU-only.
"""

import json
import math
import os

import numpy as np
import pytest

from tests._helpers import step_rel_error
from oracle.sim import OracleSim, lib, pack_map, sincos
from workloads.configs import ACTION_TABLE, base_params
from workloads.maps import empty_map, make_map, random_tiny_map

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _ulp(x):
    return float(np.spacing(np.float32(abs(x))))


# --------------------------------------------------------------- constants
def test_action_table_and_reward_constants_match_paper():
    g = _golden("paper_constants.json")
    t = g["action_table"]
    assert list(ACTION_TABLE) == [tuple(t[k]) for k in (
        "turn_left", "go_straight_turn_left", "go_straight", "go_straight_turn_right", "turn_right")]
    p = base_params()
    sp = g["sim_params"]
    assert p["k_lo"] == sp["K"] and p["dt_lo"] == sp["control_interval_s"]
    assert p["v_nom"] == sp["max_linear_velocity_cm_s"] and p["w_nom"] == sp["max_angular_velocity_rad_s"]
    assert p["near_dist"] == g["reward"]["near_obstacle_cm"]


def test_splitmix64_published_sequence():
    g = _golden("splitmix64.json")
    L = lib("f32")
    got = [format(L.orc_splitmix_at(g["seed"], c), "016x") for c in range(len(g["first_outputs_hex"]))]
    assert got == g["first_outputs_hex"]


def test_rng_nesting_and_independence():
    L = lib("f32")
    # nested counter hash: four levels of "SplitMix64 value at counter"
    s = 123
    h = L.orc_splitmix_at(L.orc_splitmix_at(L.orc_splitmix_at(L.orc_splitmix_at(s, 7), 3), 5), 9)
    assert h == L.orc_rng(s, 7, 3, 5, 9)
    # the top 24 bits are uniform: chi-square over 16 buckets
    vals = np.array([L.orc_rng(1, 2, i, 0, 0) >> 60 for i in range(16000)])
    cnt = np.bincount(vals, minlength=16)
    chi2 = ((cnt - 1000) ** 2 / 1000).sum()
    assert chi2 < 40.0  # 15 dof, p ~ 5e-4


# ------------------------------------------------------ elementary functions
def test_sincos_f32_within_2ulp_of_libm():
    xs = np.linspace(-9.0, 9.0, 40001).astype(np.float32)
    worst = 0.0
    for x in xs[::3]:
        s, c = sincos(float(x), "f32")
        es, ec = math.sin(float(x)), math.cos(float(x))
        assert abs(s - es) <= 1.2e-7 and abs(c - ec) <= 1.2e-7
        for v, e in ((s, es), (c, ec)):
            if abs(e) > 1e-3:
                worst = max(worst, abs(v - e) / _ulp(e))
    assert worst <= 2.0
    # exact special values
    assert sincos(0.0, "f32") == (0.0, 1.0)


def test_atan2_and_log_f32_against_libm():
    L = lib("f32")
    rng = np.random.default_rng(0)
    for _ in range(5000):
        y, x = (rng.normal(size=2) * 10 ** rng.uniform(-3, 3)).astype(np.float32)
        a = L.orc_atan2(float(y), float(x))
        e = math.atan2(float(y), float(x))
        assert abs(a - e) <= 4e-7 and abs(a - e) <= 4 * _ulp(e)
    # quadrant and axis cases
    for y, x, e in ((0.0, 1.0, 0.0), (1.0, 0.0, math.pi / 2), (0.0, -1.0, math.pi), (-1.0, 0.0, -math.pi / 2),
                    (1.0, 1.0, math.pi / 4), (-1.0, -1.0, -3 * math.pi / 4)):
        assert abs(L.orc_atan2(y, x) - e) < 3e-7
    for x in np.concatenate([rng.uniform(1e-7, 1.0, 5000), [2.0 ** -24, 0.5, 1.0]]).astype(np.float32):
        a, e = L.orc_log(float(x)), math.log(float(x))
        assert abs(a - e) <= 1e-6 and (abs(e) < 1e-3 or abs(a - e) <= 3 * _ulp(e))
    assert L.orc_log(1.0) == 0.0


# ----------------------------------------------------------- map packing
def test_pack_map_matches_numpy_packbits():
    for seed, w, h in ((1, 366, 366), (2, 128, 77), (3, 33, 5)):
        g = make_map(seed, w, h) if w > 100 else random_tiny_map(seed, w, h, 0.4)
        rw = ((w + 127) // 128) * 4
        padded = np.zeros((h, rw * 32), np.uint8)
        padded[:, :w] = g != 0
        ref = np.packbits(padded, axis=1, bitorder="little").view("<u4")
        assert np.array_equal(pack_map(g, rw), ref)


# ---------------------------------------------------------- kinematics
def _kin_sim(prec, K, dt, actions, w=2048, delay=0, cap=1.0):
    p = base_params(k_lo=K, k_hi=K, dt_lo=dt, dt_hi=dt, delay_lo=delay, delay_hi=delay,
                    actions=actions, t_max=10 ** 6, cap_lo=cap, cap_hi=cap)
    return OracleSim(p, [empty_map(w)], np.zeros(1, np.int32), prec=prec)


def _place(o, x, y, phi, vl=0.0, va=0.0):
    o.reset()
    f, u, b = o.state()
    f[0, 0], f[1, 0], f[2, 0], f[3, 0], f[4, 0] = x, y, phi, vl, va
    o.set_state(f, u, b)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 2e-4)])
def test_straight_line_closed_form(prec, tol):
    """Eq. 5-6 from rest with target (v, 0): v_n = v (1 - K^n) and the
    displacement is dt v (n - K (1 - K^n) / (1 - K)) along (-cos phi0, -sin phi0)."""
    K, dt, v = 0.6, 0.1, 18.0
    o = _kin_sim(prec, K, dt, [(v, 0.0)])
    x0, y0, phi0 = 1000.5, 1000.25, 0.3
    _place(o, x0, y0, phi0)
    for n in range(1, 201):
        o.step([0])
        f = o.f[:, 0]
        vn = v * (1 - K ** n)
        disp = dt * v * (n - K * (1 - K ** n) / (1 - K))
        assert abs(f[3] - vn) <= tol * max(1, vn)
        assert abs(f[0] - (x0 - disp * math.cos(phi0))) <= tol * max(1.0, disp)
        assert abs(f[1] - (y0 - disp * math.sin(phi0))) <= tol * max(1.0, disp)
        assert f[2] == np.asarray(phi0, o.dtype)  # heading untouched
        assert o.u[1, 0] == 0  # no reset happened


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_pure_rotation_closed_form(prec, tol):
    K, dt, w = 0.6, 0.1, 1.0
    o = _kin_sim(prec, K, dt, [(0.0, w)])
    x0, y0, phi0 = 1000.5, 1000.25, -2.0
    _place(o, x0, y0, phi0)
    for n in range(1, 61):
        o.step([0])
        f = o.f[:, 0]
        ang = phi0 + dt * w * (n - K * (1 - K ** n) / (1 - K))
        wrapped = (ang + math.pi) % (2 * math.pi) - math.pi
        assert abs(f[2] - wrapped) <= tol * 4
        assert f[0] == np.asarray(x0, o.dtype) and f[1] == np.asarray(y0, o.dtype)
        assert abs(f[4] - w * (1 - K ** n)) <= tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 3e-4)])
def test_arc_uses_old_heading(prec, tol):
    """Eq. 6 integrates the new velocity along the *old* heading: with target
    (v, w) from rest, x_n = x0 - sum_k dt v_k cos(phi_{k-1}) where v_k and
    phi_k follow the closed forms of the straight-line and rotation cases."""
    K, dt, v, w = 0.6, 0.1, 18.0, 1.0
    o = _kin_sim(prec, K, dt, [(v, w)])
    x0, y0, phi0 = 1000.5, 1000.25, 0.3
    _place(o, x0, y0, phi0)
    xs, ys = x0, y0
    for n in range(1, 81):
        o.step([0])
        vn = v * (1 - K ** n)
        phi_prev = phi0 + dt * w * ((n - 1) - K * (1 - K ** (n - 1)) / (1 - K))
        xs -= dt * vn * math.cos(phi_prev)
        ys -= dt * vn * math.sin(phi_prev)
        f = o.f[:, 0]
        assert abs(f[0] - xs) <= tol * 10 and abs(f[1] - ys) <= tol * 10


@pytest.mark.parametrize("cap", [0.5, 1.5])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 2e-4)])
def test_velocity_cap_scales_both_targets(prec, tol, cap):
    """Velocity range (Sec. 4.3.2, reading 6): the episode's factor cap scales
    both entries of the action table, so from rest with action (v, w) the
    closed forms of the straight-line and rotation cases hold with cap v and
    cap w: v_n = cap v (1 - K^n), w_n = cap w (1 - K^n), and the heading
    advances by dt cap w (n - K (1 - K^n) / (1 - K)).  A dropped cap, or a cap
    on one of the two targets only, fails one of the three."""
    K, dt, v, w = 0.6, 0.1, 18.0, 1.0
    o = _kin_sim(prec, K, dt, [(v, 0.0), (0.0, w)], cap=cap)
    x0, y0, phi0 = 1000.5, 1000.25, 0.3
    _place(o, x0, y0, phi0)
    assert o.f[7, 0] == np.asarray(cap, o.dtype)  # lo == hi: the draw is cap itself
    for n in range(1, 121):
        o.step([0])
        f = o.f[:, 0]
        vn = cap * v * (1 - K ** n)
        disp = dt * cap * v * (n - K * (1 - K ** n) / (1 - K))
        assert abs(f[3] - vn) <= tol * max(1, vn)
        assert abs(f[0] - (x0 - disp * math.cos(phi0))) <= tol * max(1.0, disp)
        assert abs(f[1] - (y0 - disp * math.sin(phi0))) <= tol * max(1.0, disp)
    o = _kin_sim(prec, K, dt, [(v, 0.0), (0.0, w)], cap=cap)
    phi0 = -2.0
    _place(o, x0, y0, phi0)
    for n in range(1, 41):
        o.step([1])
        f = o.f[:, 0]
        ang = phi0 + dt * cap * w * (n - K * (1 - K ** n) / (1 - K))
        wrapped = (ang + math.pi) % (2 * math.pi) - math.pi
        assert abs(f[2] - wrapped) <= tol * 4
        assert abs(f[4] - cap * w * (1 - K ** n)) <= tol
        assert f[3] == 0.0


def test_inertia_limits():
    # K = 0: the velocity equals the target after one step
    o = _kin_sim("f64", 0.0, 0.1, [(7.0, 0.5)])
    _place(o, 1000.0, 1000.0, 0.0)
    o.step([0])
    assert o.f[3, 0] == 7.0 and o.f[4, 0] == 0.5
    # K = 1: the velocity never changes
    o = _kin_sim("f64", 1.0, 0.1, [(7.0, 0.5)])
    _place(o, 1000.0, 1000.0, 0.0, vl=3.0, va=-0.25)
    for _ in range(5):
        o.step([0])
    assert o.f[3, 0] == 3.0 and o.f[4, 0] == -0.25


@pytest.mark.parametrize("d", [1, 2])
def test_delay_shifts_action_sequence(d):
    """With delay d the executed targets are the inputs shifted by d steps,
    with zero target during the first d steps of the episode."""
    acts = [(18.0, 1.0), (0.36, -1.0), (18.0, 0.0), (0.0, 0.0)]
    seq = np.random.default_rng(d).integers(0, 3, size=40)
    a = _kin_sim("f32", 0.6, 0.1, acts, delay=d)
    b = _kin_sim("f32", 0.6, 0.1, acts, delay=0)
    _place(a, 1000.0, 1000.0, 0.4)
    _place(b, 1000.0, 1000.0, 0.4)
    a.b[2, 0] = d  # the reset drew delay d (lo == hi); b has 0
    shifted = np.concatenate([[3] * d, seq[:-d]])
    for t in range(len(seq)):
        a.step([seq[t]])
        b.step([shifted[t]])
        assert np.array_equal(a.f[:5, 0], b.f[:5, 0])


# ------------------------------------------------------------ LiDAR
def _lidar_sim(prec, grid, fov=0.0, rmax=100.0, delta=1.0, nb=2):
    p = base_params(fov=fov, range_max=rmax, march_step=delta, n_beams=nb)
    return OracleSim(p, [grid], np.zeros(1, np.int32), prec=prec)


def _dir(prec, phi):
    s, c = sincos(phi, prec)
    return -c, -s


@pytest.mark.parametrize("prec,eps", [("f64", 1e-9), ("f32", 2e-4)])
def test_lidar_half_plane_walls(prec, eps):
    """A wall filling every cell with cx >= X0 (and the three rotations): the
    range is in [d, d + delta) for the exact distance d to the wall's face."""
    W = 400
    X0 = 300
    rng = np.random.default_rng(7)
    for orient in range(4):
        g = np.zeros((W, W), np.uint8)
        if orient == 0:
            g[:, X0:] = 1
        elif orient == 1:
            g[:, :W - X0] = 1
        elif orient == 2:
            g[X0:, :] = 1
        else:
            g[:W - X0, :] = 1
        o = _lidar_sim(prec, g)
        for _ in range(200):
            x = rng.uniform(215, 295) if orient in (0, 2) else rng.uniform(105, 185)
            y = rng.uniform(150, 250)
            if orient >= 2:
                x, y = rng.uniform(150, 250), x
            phi = rng.uniform(-math.pi, math.pi)
            hits, ranges = o.lidar(0, x, y, phi)
            x, y, phi = (float(np.asarray(v, o.dtype)) for v in (x, y, phi))
            ux, uy = _dir(prec, phi)
            if orient == 0:
                dist = (X0 - x) / ux if ux > 0 else math.inf
            elif orient == 1:
                dist = (x - (W - X0)) / -ux if ux < 0 else math.inf
            elif orient == 2:
                dist = (X0 - y) / uy if uy > 0 else math.inf
            else:
                dist = (y - (W - X0)) / -uy if uy < 0 else math.inf
            r = float(ranges[0])
            if dist > 100.0 + eps:
                assert r == 100.0
            elif dist < 100.0 - 1.0 - eps:
                assert dist - eps <= r < dist + 1.0 + eps


def _ray_circle(px, py, ux, uy, r):
    """Entry distance and chord of the ray p + t u (|u| = 1, t >= 0) through the
    circle of radius r at the origin, or (inf, 0)."""
    bq = px * ux + py * uy
    cq = px * px + py * py - r * r
    disc = bq * bq - cq
    if disc < 0:
        return math.inf, 0.0
    t0, t1 = -bq - math.sqrt(disc), -bq + math.sqrt(disc)
    if t1 < 0:
        return math.inf, 0.0
    return max(t0, 0.0), t1 - max(t0, 0.0)


@pytest.mark.parametrize("prec,eps", [("f64", 1e-9), ("f32", 1e-4)])
def test_lidar_disc_obstacle(prec, eps):
    """A rasterised disc of radius rc lies between the exact discs of radius
    rc -/+ sqrt(2)/2.  The range is never shorter than the distance to the outer
    circle, and when the ray's chord through the inner circle is at least one
    march step the range is at most one step past the inner circle."""
    W, ox, oy, rc = 400, 200, 200, 20
    cy, cx = np.mgrid[0:W, 0:W]
    g = ((2 * cx + 1 - 2 * ox) ** 2 + (2 * cy + 1 - 2 * oy) ** 2 <= 4 * rc * rc).astype(np.uint8)
    o = _lidar_sim(prec, g)
    rng = np.random.default_rng(3)
    halo = math.sqrt(2.0) / 2 + 1e-6
    inner_hits = 0
    for _ in range(600):
        x, y = rng.uniform(110, 290, size=2)
        if math.hypot(x - ox, y - oy) < rc + 2:
            continue
        phi = rng.uniform(-math.pi, math.pi)
        _, ranges = o.lidar(0, x, y, phi)
        x, y, phi = (float(np.asarray(v, o.dtype)) for v in (x, y, phi))
        ux, uy = _dir(prec, phi)
        r = float(ranges[0])
        t_out, _ = _ray_circle(x - ox, y - oy, ux, uy, rc + halo)
        t_in, chord = _ray_circle(x - ox, y - oy, ux, uy, rc - halo)
        if t_out >= 100.0:
            assert r == 100.0
            continue
        assert r >= t_out - eps
        if chord >= 1.0 + eps and t_in + 1.0 < 100.0:
            assert r <= t_in + 1.0 + eps
            inner_hits += 1
    assert inner_hits > 50


def _dda_first_blocked(grid, x, y, ux, uy, tmax):
    """Amanatides & Woo (1987) voxel traversal: entry distance and chord of
    the first occupied (or outside) cell along the ray."""
    H, W = grid.shape
    ix, iy = math.floor(x), math.floor(y)
    sx = 1 if ux > 0 else -1
    sy = 1 if uy > 0 else -1
    tdx = abs(1.0 / ux) if ux != 0 else math.inf
    tdy = abs(1.0 / uy) if uy != 0 else math.inf
    tx = ((ix + 1 - x) / ux if ux > 0 else (x - ix) / -ux) if ux != 0 else math.inf
    ty = ((iy + 1 - y) / uy if uy > 0 else (y - iy) / -uy) if uy != 0 else math.inf
    t_entry = 0.0
    while t_entry <= tmax + 2:
        t_exit = min(tx, ty)
        if ix < 0 or iy < 0 or ix >= W or iy >= H or grid[iy, ix]:
            return t_entry, t_exit - t_entry
        if tx < ty:
            ix += sx
            tx += tdx
        else:
            iy += sy
            ty += tdy
        t_entry = t_exit
    return math.inf, 0.0


@pytest.mark.parametrize("prec,eps", [("f64", 1e-9), ("f32", 1e-4)])
@pytest.mark.parametrize("side", [8, 16])
def test_lidar_brute_force_tiny_maps(prec, eps, side):
    """Every free cell centre x 64 headings on a random tiny map, against an
    exact voxel traversal: no sample before the first blocked cell can hit,
    and when that cell's chord is at least one march step the hit comes
    within one step of entering it."""
    g = random_tiny_map(side, side, side, 0.25)
    o = _lidar_sim(prec, g, rmax=40.0, delta=1.0)
    n = 0
    for cy in range(side):
        for cx in range(side):
            if g[cy, cx]:
                continue
            x, y = cx + 0.5, cy + 0.5
            for k in range(64):
                phi = -math.pi + k * (2 * math.pi / 64) + 0.013
                hits, ranges = o.lidar(0, x, y, phi)
                ux, uy = _dir(prec, float(np.asarray(phi, o.dtype)))
                de, chord = _dda_first_blocked(g, x, y, ux, uy, 40.0)
                h = int(hits[0])
                assert h <= 40  # every ray leaves a tiny map within range
                assert h * 1.0 >= de - eps
                if chord >= 1.0 + eps:
                    assert h * 1.0 < de + 1.0 + eps
                n += 1
    assert n > 1000


def test_lidar_empty_map_border_distance():
    W = 200
    o = _lidar_sim("f64", empty_map(W), rmax=100.0)
    rng = np.random.default_rng(11)
    for _ in range(300):
        x, y = rng.uniform(1, W - 1, size=2)
        phi = rng.uniform(-math.pi, math.pi)
        _, ranges = o.lidar(0, x, y, phi)
        ux, uy = -math.cos(phi), -math.sin(phi)
        tx = (W - x) / ux if ux > 0 else (x / -ux if ux < 0 else math.inf)
        ty = (W - y) / uy if uy > 0 else (y / -uy if uy < 0 else math.inf)
        d = min(tx, ty)
        r = float(ranges[0])
        if d >= 100.0:
            assert r == 100.0
        else:
            assert d - 1e-9 <= r < d + 1.0 + 1e-9


def test_lidar_first_sample_is_one_step_out():
    """Samples start one march step from the robot: on a fully occupied map
    every beam hits at k = 1 (range = delta); on a huge empty map no beam
    hits (index K + 1, range = range_max)."""
    o = _lidar_sim("f64", np.ones((50, 50), np.uint8), delta=0.5, rmax=20.0, nb=8, fov=4.0)
    hits, ranges = o.lidar(0, 25.3, 24.6, 0.7)
    assert np.all(hits == 1) and np.all(ranges == 0.5)
    o = _lidar_sim("f64", empty_map(600), delta=0.5, rmax=20.0, nb=8, fov=4.0)
    hits, ranges = o.lidar(0, 300.3, 300.6, 0.7)
    assert np.all(hits == 41) and np.all(ranges == 20.0)


def test_beam_fan_layout():
    """270 degree fan, both ends included: beam j points at phi - 135deg +
    j * 270deg / (B - 1).  Checked on a map with a single wall so that beam j's
    range reveals its direction."""
    W = 400
    g = np.zeros((W, W), np.uint8)
    g[:, 300:] = 1
    p = base_params(n_beams=32, range_max=200.0)
    o = OracleSim(p, [g], np.zeros(1, np.int32), prec="f64")
    x, y, phi = 200.0, 200.0, math.pi  # heading (-cos pi, -sin pi) = +x
    _, ranges = o.lidar(0, x, y, phi)
    for j in range(32):
        beta = phi - 0.75 * math.pi + j * 1.5 * math.pi / 31
        ux = -math.cos(beta)
        if ux > 0.6:
            d = 100.0 / ux
            assert d - 1e-9 <= ranges[j] < d + 1.0 + 1e-9
        elif ux < 0:
            assert ranges[j] == 200.0


# ------------------------------------------------------------ collision
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_collision_disc_threshold(prec):
    W = 200
    g = np.zeros((W, W), np.uint8)
    g[100, 120] = 1  # centre (120.5, 100.5)
    o = _lidar_sim(prec, g)
    r = 10.0
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.uniform(-math.pi, math.pi)
        for d, expect in ((r - 1e-3, True), (r + 1e-3, False)):
            x = 120.5 + d * math.cos(a)
            y = 100.5 + d * math.sin(a)
            assert o.collide(0, x, y) == expect
    # leaving the map is a collision; the far interior is not
    assert o.collide(0, -0.01, 50.0) and o.collide(0, 50.0, 200.0)
    assert not o.collide(0, 50.0, 50.0)


# ------------------------------------------------------- reward and obs
def _reward_sim(grid, **kw):
    p = base_params(k_lo=1.0, k_hi=1.0, t_max=10 ** 6, **kw)  # K = 1: the robot stays put
    return OracleSim(p, [grid], np.zeros(1, np.int32), prec="f64")


def test_reward_on_the_start_goal_line():
    """At S heading to G: d1 = D, d2 = 0, alpha = 0, v = 0 and no obstacle
    within 30 cells -> r = 0.3*0 + 0.1*1 + 0.3*0 + 0.3*1 + 0.1*0 = 0.4."""
    W = 366
    o = _reward_sim(empty_map(W))
    D = math.hypot(W - 60, W - 60)
    _place(o, 30.0, 30.0, -0.75 * math.pi)
    obs, rew, done, _ = o.step([2])
    assert done[0] == 0
    assert abs(rew[0] - 0.4) < 1e-12
    B = 32
    assert abs(obs[0, B] - 1.0) < 1e-12 and abs(obs[0, B + 1]) < 1e-12 and abs(obs[0, B + 2]) < 1e-12
    # half way, off the line by delta to the left of the heading
    delta = 12.0
    mx = 30 + (W - 60) / 2 - delta / math.sqrt(2)
    my = 30 + (W - 60) / 2 + delta / math.sqrt(2)
    _place(o, mx, my, -0.75 * math.pi)
    obs, rew, done, _ = o.step([2])
    d1 = math.hypot(W - 30 - mx, W - 30 - my)
    alpha = math.atan2(delta, D / 2)  # goal seen to the right of the heading -> negative
    exp = 0.3 * (1 - d1 / D) + 0.1 * (1 - 2 * delta / D) + 0.3 * (1 - alpha / math.pi)
    assert abs(rew[0] - exp) < 1e-9
    assert abs(obs[0, B + 2] + alpha / math.pi) < 1e-9


@pytest.mark.parametrize("phi,axes", [(math.pi - 1e-12, "x"), (-math.pi / 2, "y"), (0.0, "-x")])
def test_goal_in_robot_frame(phi, axes):
    """Observation goal terms: (forward, left) components of G - P in the
    robot frame (forward = (-cos phi, -sin phi)), divided by D, and
    alpha = atan2(left, forward)."""
    W = 366
    o = _reward_sim(empty_map(W))
    x, y = 150.0, 120.0
    _place(o, x, y, phi)
    obs = o.step([2])[0][0]
    ddx, ddy = W - 30 - x, W - 30 - y
    fwd, left = {"x": (ddx, ddy), "y": (ddy, -ddx), "-x": (-ddx, -ddy)}[axes]
    D = math.hypot(W - 60, W - 60)
    B = 32
    assert abs(obs[B] - fwd / D) < 1e-9 and abs(obs[B + 1] - left / D) < 1e-9
    assert abs(obs[B + 2] - math.atan2(left, fwd) / math.pi) < 1e-9


def test_reward_velocity_and_near_obstacle_terms():
    W = 366
    g = empty_map(W)
    g[200:206, 100:140] = 1  # a bar 25 cells below the robot
    o = _reward_sim(g)
    _place(o, 120.0, 175.0, -0.75 * math.pi, vl=10.0)  # 10 > 0.5 * 18
    obs, rew, done, _ = o.step([2])
    x, y = 120.0 + 0.1 * 10 * math.cos(-0.75 * math.pi) * -1, 175.0 + 0.1 * 10 * math.sin(-0.75 * math.pi) * -1
    # recompute the smooth terms in closed form at the new pose
    D = math.hypot(W - 60, W - 60)
    d1 = math.hypot(W - 30 - x, W - 30 - y)
    d2 = abs((W - 60) * (y - 30) - (W - 60) * (x - 30)) / D
    fwd = (W - 30 - x) * math.cos(math.pi / 4) + (W - 30 - y) * math.sin(math.pi / 4)
    left = -(W - 30 - x) * math.sin(math.pi / 4) + (W - 30 - y) * math.cos(math.pi / 4)
    alpha = math.atan2(left, fwd)
    exp = 0.3 * (1 - d1 / D) + 0.1 * (1 - 2 * d2 / D) + 0.3 * 1 + 0.3 * (1 - abs(alpha) / math.pi) + 0.1 * -1
    assert done[0] == 0
    assert abs(rew[0] - exp) < 1e-9


@pytest.mark.parametrize("cap", [0.5, 1.5])
def test_velocity_observation_terms_use_nominal_maxima(cap):
    """Observation (reading 16): the last two entries are v_l / 18 and
    v_a / 1, the nominal maxima of the simulation-parameter table, not the
    episode's capped maxima; checked at a hand-set velocity with cap != 1
    (K = 1 keeps the velocity through the step)."""
    W = 366
    o = _reward_sim(empty_map(W), cap_lo=cap, cap_hi=cap)
    B = 32
    for vl, va in ((10.0, 0.5), (3.25, -0.75), (0.0, 1.25)):
        _place(o, 150.0, 120.0, 0.7, vl=vl, va=va)
        obs = o.step([2])[0][0]
        assert o.f[7, 0] == cap
        assert abs(obs[B + 3] - vl / 18.0) < 1e-12
        assert abs(obs[B + 4] - va / 1.0) < 1e-12


def test_velocity_reward_threshold_scales_with_cap():
    """r_v = [v_l > v_max / 2] with v_max the episode's capped maximum
    18 cap (reading 15): the reward jumps by the weight 0.3 as v_l crosses
    9 cap, and does not jump at the uncapped threshold 9."""
    W = 366

    def rew(cap, vl):
        o = _reward_sim(empty_map(W), cap_lo=cap, cap_hi=cap)
        _place(o, 150.0, 120.0, 0.7, vl=vl)
        obs, r, done, _ = o.step([2])
        assert done[0] == 0 and obs[0, :32].min() == 1.0  # no obstacle: r_d = 0
        return float(r[0])

    for cap in (0.5, 1.5):
        thr = 9.0 * cap
        jump = rew(cap, thr + 0.01) - rew(cap, thr - 0.01)
        assert abs(jump - 0.3) < 1e-4, (cap, jump)
        flat = rew(cap, 9.0 + 0.01) - rew(cap, 9.0 - 0.01)
        assert abs(flat) < 1e-4, (cap, flat)


def test_near_obstacle_term_uses_noise_free_ranges():
    """r_d = -1 when the nearest noise-free range is below 30 (reading 17):
    with sensor noise sigma = 2 the reward equals the noise-free run's bit for
    bit, while the noisy minimum lands on the other side of 30 in many of the
    same steps (so a reward that read the noisy ranges would differ)."""
    W = 400
    g = np.zeros((W, W), np.uint8)
    g[:, 300:] = 1  # half plane: the nearest beam sees the wall at about 300 - x
    crossed = steps = 0
    for x in np.arange(268.0, 273.0, 0.25):
        a = _reward_sim(g, sigma_lo=0.0, sigma_hi=0.0)
        b = _reward_sim(g, sigma_lo=2.0, sigma_hi=2.0)
        for o in (a, b):
            _place(o, float(x), 200.0, math.pi)  # heading +x, the wall straight ahead
        for _ in range(12):
            oa, ra, da, _ = a.step([2])
            ob, rb, db, _ = b.step([2])
            assert da[0] == 0 and db[0] == 0
            assert ra[0] == rb[0]
            clean, noisy = oa[0, :32].min() * 100.0, ob[0, :32].min() * 100.0
            crossed += (clean < 30.0) != (noisy < 30.0)
            steps += 1
    assert crossed >= steps // 10, (crossed, steps)


def test_terminal_rewards_and_autoreset():
    W = 366
    g = empty_map(W, border=True)
    g[100, 100] = 1
    o = _reward_sim(g)
    # collide: an occupied cell within the robot disc
    _place(o, 100.5, 95.0, 0.0)
    obs, rew, done, term = o.step([2])
    assert rew[0] == -10.0 and done[0] & 1
    # the new episode: ep_id 1, fresh state equal to an explicit reset
    assert o.u[1, 0] == 1 and o.u[0, 0] == 0
    ref = OracleSim(o.params, [g], np.zeros(1, np.int32), prec="f64")
    ref.reset()
    obs_ref = ref.reset_env(0, 1)
    assert np.array_equal(obs[0], obs_ref)
    assert np.array_equal(o.f[:, 0], ref.f[:, 0])
    # arrive: within the goal radius of G = (W - 30, W - 30), collision wins when both
    _place(o, W - 30.0 - 5.0, W - 30.0 + 3.0, 0.0)
    obs, rew, done, term = o.step([2])
    assert rew[0] == 75.0 and done[0] == 2
    assert abs(term[0, 32] * math.hypot(W - 60, W - 60) - (-(5.0 * 1.0 + (-3.0) * 0.0))) < 1e-9


def test_truncation_flag():
    p = base_params(k_lo=1.0, k_hi=1.0, t_max=3)
    o = OracleSim(p, [empty_map(366)], np.zeros(1, np.int32), prec="f64")
    _place(o, 100.0, 100.0, 0.0)
    dones = [int(o.step([2])[2][0]) for _ in range(3)]
    assert dones == [0, 0, 4]


# ------------------------------------------------ noise and diversity
def test_sensor_noise_statistics():
    """Noise is additive N(0, sigma^2) on the reported ranges only."""
    W = 400
    g = np.zeros((W, W), np.uint8)
    g[:, 300:] = 1
    sigma = 2.0
    p = base_params(sigma_lo=sigma, sigma_hi=sigma, k_lo=1.0, k_hi=1.0, t_max=10 ** 7)
    o = OracleSim(p, [g], np.zeros(1, np.int32), prec="f64")
    phi = 2.9
    _place(o, 230.0, 200.0, phi)
    clean = o.lidar(0, 230.0, 200.0, phi)[1]
    diffs = []
    for _ in range(4000):
        obs = o.step([2])[0]
        rng_ = obs[0, :32] * 100.0
        m = (clean > 5) & (clean < 95)
        diffs.append((rng_ - clean)[m])
    d = np.concatenate(diffs)
    n = d.size
    assert n > 20000
    assert abs(d.mean()) < 3 * sigma / math.sqrt(n)
    assert abs(d.var() - sigma ** 2) < 3 * sigma ** 2 * math.sqrt(2.0 / n)
    assert np.array_equal(o.lidar(0, 230.0, 200.0, phi)[1], clean)  # noise never touches the march


def test_domain_randomisation_ranges_and_determinism():
    from workloads.configs import DR_RANGES
    p = base_params(**DR_RANGES)
    o = OracleSim(p, [make_map(1)], np.zeros(64, np.int32), prec="f32")
    o.reset()
    f, u, b = o.state()
    assert np.all((f[5] >= 0.05) & (f[5] <= 0.2))
    assert np.all((f[6] >= 0.6) & (f[6] <= 1.0))
    assert np.all((f[7] >= 0.5) & (f[7] <= 1.5))
    assert np.all((f[8] >= 0.0) & (f[8] <= 2.0))
    assert set(np.unique(b[2])) == {0, 1, 2}
    assert np.all(np.abs(f[0] - 30) <= 5) and np.all(np.abs(f[1] - 30) <= 5)
    assert np.all((f[2] >= -math.pi) & (f[2] <= math.pi))
    # same key, same draw; different episode, different draw
    a1 = o.reset_env(3, 7)
    s1 = o.f[:, 3].copy()
    a2 = o.reset_env(3, 7)
    assert np.array_equal(a1, a2) and np.array_equal(s1, o.f[:, 3])
    o.reset_env(3, 8)
    assert not np.array_equal(s1, o.f[:, 3])


def test_envs_are_independent():
    """A vectorized step equals per-env steps: resets of done envs leave the
    others untouched."""
    from workloads.configs import DR_RANGES
    p = base_params(**DR_RANGES)
    maps = [make_map(1), make_map(2)]
    em = np.array([0, 1, 0, 1], np.int32)
    v = OracleSim(p, maps, em, prec="f32")
    v.reset()
    for t in range(60):
        v.step(v.random_actions(t))
    # rerun envs one by one from scratch and compare the final state
    for i in range(4):
        s = OracleSim(p, maps, em, prec="f32")
        s.reset()
        for t in range(60):
            a = s.random_actions(t)
            keep = s.state()
            s.step(a)
            f, u, b = s.state()
            for j in range(4):
                if j != i:
                    f[:, j], u[:, j], b[:, j] = keep[0][:, j], keep[1][:, j], keep[2][:, j]
            s.set_state(f, u, b)
        assert np.array_equal(s.f[:, i], v.f[:, i])
        assert np.array_equal(s.u[:, i], v.u[:, i])


def test_random_actions_and_vem_fraction():
    p = base_params()
    o = OracleSim(p, [make_map(1)], np.zeros(8, np.int32), prec="f32")
    acts = np.concatenate([o.random_actions(t) for t in range(2000)])
    cnt = np.bincount(acts, minlength=5)
    assert ((cnt - acts.size / 5) ** 2 / (acts.size / 5)).sum() < 20.0  # 4 dof
    eps = np.linspace(0.01, 0.3, 8).astype(np.float32)
    u = np.stack([o.explore_uniform(t) for t in range(4000)])
    frac = (u < eps).mean(axis=0)
    se = np.sqrt(eps * (1 - eps) / 4000)
    assert np.all(np.abs(frac - eps) < 4 * se)


def test_f32_and_f64_oracles_agree_on_a_rollout():
    """The two precisions take the same discrete decisions on a seeded
    domain-randomised workload (teacher forced: both start every step from the
    same float32 state), and pose / velocity agree to 1e-5 relative."""
    from workloads import workload
    w = workload("dr1024", n_envs=32, steps=200)
    a = OracleSim(w.params, w.maps(), w.env_map, prec="f32")
    b = OracleSim(w.params, w.maps(), w.env_map, prec="f64")
    a.reset()
    b.reset()
    for t in range(200):
        b.set_state(a.f.astype(np.float64), a.u, a.b)
        f_old = a.f.copy()
        act = a.random_actions(t)
        _, _, da, _ = a.step(act)
        _, _, db, _ = b.step(act)
        assert np.array_equal(da, db)
        live = da == 0
        rel = step_rel_error(f_old[:, live], a.f[:, live], b.f[:, live])
        assert rel.max() <= 1e-5


def test_f32_and_f64_lidar_agree():
    """Noise-free ranges of the two precisions are equal in >= 99.99% of beams
    and otherwise differ by exactly one march step."""
    maps = [make_map(s) for s in range(1, 5)]
    p = base_params()
    a = OracleSim(p, maps, np.zeros(1, np.int32), prec="f32")
    b = OracleSim(p, maps, np.zeros(1, np.int32), prec="f64")
    rng = np.random.default_rng(9)
    tot = diff = 0
    for _ in range(1500):
        m = int(rng.integers(0, 4))
        x, y = (float(np.float32(v)) for v in rng.uniform(20, 346, size=2))
        phi = float(np.float32(rng.uniform(-math.pi, math.pi)))
        ha, _ = a.lidar(m, x, y, phi)
        hb, _ = b.lidar(m, x, y, phi)
        tot += ha.size
        d = np.abs(ha - hb)
        assert d.max() <= 1
        diff += int((d > 0).sum())
    assert diff / tot <= 1e-3, diff
