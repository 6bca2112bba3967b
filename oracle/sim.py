"""ctypes front end of ``sparrow_oracle.c`` (test infrastructure only).

Builds the C oracle with gcc on first use (``build_oracle``), in two
precisions, and wraps it in :class:`OracleSim`, a slow per-env loop over the
whole step that mirrors the library's public calls (reset / step / rollout).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparrow_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

N_F, N_U, N_B = 9, 2, 3  # float, u32 and u8 state rows per env
F_NAMES = ("x", "y", "phi", "vl", "va", "dt", "K", "cap", "sigma")
U_NAMES = ("ep_step", "ep_id")
B_NAMES = ("q0", "q1", "delay")


def _so_path(prec: str) -> str:
    return os.path.join(_BUILD, f"libsparrow_oracle_{prec}.so")


def build_oracle(force: bool = False) -> None:
    """Compile both precisions of the C oracle with gcc (no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    for prec, flag in (("f32", "-DORC_F32"), ("f64", "-DORC_F64")):
        out = _so_path(prec)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fno-builtin-sincosf", flag, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


class _Config(C.Structure):
    _fields_ = [
        ("n_beams", C.c_int32), ("n_actions", C.c_int32), ("t_max", C.c_int32),
        ("delay_lo", C.c_int32), ("delay_hi", C.c_int32), ("n_dyn", C.c_int32),
        ("fov", C.c_double), ("range_max", C.c_double), ("march_step", C.c_double),
        ("robot_radius", C.c_double), ("goal_radius", C.c_double), ("near_dist", C.c_double),
        ("start_offset", C.c_double), ("start_jitter", C.c_double),
        ("dt_lo", C.c_double), ("dt_hi", C.c_double), ("k_lo", C.c_double), ("k_hi", C.c_double),
        ("cap_lo", C.c_double), ("cap_hi", C.c_double), ("sigma_lo", C.c_double), ("sigma_hi", C.c_double),
        ("v_nom", C.c_double), ("w_nom", C.c_double),
        ("action_v", C.c_double * 8), ("action_w", C.c_double * 8),
        ("seed", C.c_uint64),
        ("dyn_radius", C.c_double), ("dyn_speed_lo", C.c_double), ("dyn_speed_hi", C.c_double),
        ("dyn_keepout", C.c_double),
    ]


class _Maps(C.Structure):
    _fields_ = [("n_maps", C.c_int32), ("pad0", C.c_int32),
                ("w", C.c_void_p), ("h", C.c_void_p), ("off", C.c_void_p), ("grids", C.c_void_p)]


class _Envs(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("pad0", C.c_int32),
                ("env_map", C.c_void_p), ("env_beams", C.c_void_p),
                ("f", C.c_void_p), ("u", C.c_void_p), ("b", C.c_void_p), ("dyn", C.c_void_p)]


def lib(prec: str = "f32"):
    """The loaded oracle library of precision ``prec`` ('f32' or 'f64')."""
    with _LOCK:
        if prec not in _LIBS:
            build_oracle()
            L = C.CDLL(_so_path(prec))
            R = C.c_float if prec == "f32" else C.c_double
            vp = C.c_void_p
            L.orc_rng.restype = C.c_uint64
            L.orc_rng.argtypes = [C.c_uint64] * 5
            L.orc_splitmix_at.restype = C.c_uint64
            L.orc_splitmix_at.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_sincos.argtypes = [R, vp, vp]
            L.orc_atan2.restype = R
            L.orc_atan2.argtypes = [R, R]
            L.orc_log.restype = R
            L.orc_log.argtypes = [R]
            L.orc_pack_map.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp]
            L.orc_lidar.argtypes = [vp, vp, C.c_int32, R, R, R, C.c_int32, vp, vp]
            L.orc_lidar_dyn.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, R, R, R, C.c_int32, vp, vp]
            L.orc_dyn_advance.argtypes = [vp, vp, vp, C.c_int32, R]
            L.orc_dyn_collide.restype = C.c_int32
            L.orc_dyn_collide.argtypes = [vp, vp, C.c_int32, R, R]
            L.orc_collide.restype = C.c_int32
            L.orc_collide.argtypes = [vp, vp, C.c_int32, R, R]
            L.orc_reset_env.argtypes = [vp, vp, vp, C.c_int32, C.c_uint32, vp]
            L.orc_reset.argtypes = [vp, vp, vp, vp]
            L.orc_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_step_one.argtypes = [vp, vp, vp, C.c_int32, C.c_uint8, vp, vp, vp, vp, vp]
            L.orc_random_action.restype = C.c_uint8
            L.orc_random_action.argtypes = [vp, C.c_int32, C.c_uint64]
            L.orc_explore_uniform.restype = R
            L.orc_explore_uniform.argtypes = [vp, C.c_int32, C.c_uint64]
            L.orc_march_samples.restype = C.c_uint64
            L.orc_march_samples.argtypes = []
            L.orc_reset_march_samples.argtypes = []
            L.orc_rollout_random_range.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, vp]
            L.orc_rollout_random.argtypes = [vp, vp, vp, C.c_int32, C.c_uint64, vp, vp, vp, vp, vp, vp]
            _LIBS[prec] = L
        return _LIBS[prec]


def rng_u64(seed, stream, env, a, b) -> int:
    """The counter-based SplitMix64 hash (oracle side)."""
    return int(lib("f32").orc_rng(seed, stream, env, a, b))


def pack_map(grid: np.ndarray, row_words: int | None = None) -> np.ndarray:
    """Bit-packed rows of a uint8 grid, as the oracle defines the layout."""
    g = np.ascontiguousarray(grid, dtype=np.uint8)
    h, w = g.shape
    if row_words is None:
        row_words = ((w + 127) // 128) * 4
    out = np.zeros((h, row_words), dtype=np.uint32)
    lib("f32").orc_pack_map(g.ctypes.data, w, h, row_words, out.ctypes.data)
    return out


def make_config(params: dict) -> _Config:
    c = _Config()
    acts = params["actions"]
    c.n_beams = int(params["n_beams"])
    c.n_actions = len(acts)
    c.t_max = int(params["t_max"])
    c.delay_lo = int(params["delay_lo"])
    c.delay_hi = int(params["delay_hi"])
    for k in ("fov", "range_max", "march_step", "robot_radius", "goal_radius", "near_dist",
              "start_offset", "start_jitter", "dt_lo", "dt_hi", "k_lo", "k_hi", "cap_lo", "cap_hi",
              "sigma_lo", "sigma_hi", "v_nom", "w_nom"):
        setattr(c, k, float(params[k]))
    for i, (v, w) in enumerate(acts):
        c.action_v[i] = float(v)
        c.action_w[i] = float(w)
    c.seed = int(params["seed"]) & 0xFFFFFFFFFFFFFFFF
    # dynamic obstacles (optional; none by default)
    c.n_dyn = int(params.get("n_dyn", 0))
    for k in ("dyn_radius", "dyn_speed_lo", "dyn_speed_hi", "dyn_keepout"):
        setattr(c, k, float(params.get(k, 0.0)))
    return c


class OracleSim:
    """The vectorized environment, one env at a time, on the CPU.

    ``prec`` selects strict float32 ('f32') or float64 ('f64').  State lives
    in three numpy arrays: ``f`` [9, n] reals (x, y, phi, vl, va, dt, K, cap,
    sigma), ``u`` [2, n] uint32 (ep_step, ep_id) and ``b`` [3, n] uint8
    (q0, q1, delay); with dynamic obstacles also ``dyn`` [4 n_dyn, n] reals
    (obstacle o at rows 4o..4o+3: x, y, vx, vy).
    """

    def __init__(self, params: dict, maps, env_map, env_beams=None, prec: str = "f32"):
        self.prec = prec
        self.L = lib(prec)
        self.dtype = np.float32 if prec == "f32" else np.float64
        self.params = dict(params)
        self.cfg = make_config(params)
        self.B = int(params["n_beams"])
        self.obs_dim = self.B + 5
        self.maps = [np.ascontiguousarray(m, dtype=np.uint8) for m in maps]
        self._w = np.array([m.shape[1] for m in self.maps], np.int32)
        self._h = np.array([m.shape[0] for m in self.maps], np.int32)
        sizes = np.array([m.size for m in self.maps], np.int64)
        self._off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self._grids = np.concatenate([m.ravel() for m in self.maps]) if self.maps else np.zeros(1, np.uint8)
        self.cmaps = _Maps(len(self.maps), 0, self._w.ctypes.data, self._h.ctypes.data,
                           self._off.ctypes.data, self._grids.ctypes.data)
        self.env_map = np.ascontiguousarray(env_map, dtype=np.int32)
        self.n = int(self.env_map.size)
        self.env_beams = None if env_beams is None else np.ascontiguousarray(env_beams, dtype=np.int32)
        self.f = np.zeros((N_F, self.n), self.dtype)
        self.u = np.zeros((N_U, self.n), np.uint32)
        self.b = np.zeros((N_B, self.n), np.uint8)
        self.status = np.zeros(1, np.uint32)
        self.n_dyn = int(self.cfg.n_dyn)
        self.dyn = np.zeros((4 * self.n_dyn, self.n), self.dtype)
        self.cenvs = _Envs(self.n, 0, self.env_map.ctypes.data,
                           self.env_beams.ctypes.data if self.env_beams is not None else None,
                           self.f.ctypes.data, self.u.ctypes.data, self.b.ctypes.data,
                           self.dyn.ctypes.data if self.n_dyn else None)

    # -- state ------------------------------------------------------------
    def set_state(self, f, u, b, dyn=None):
        self.f[...] = np.asarray(f, self.dtype)
        self.u[...] = u
        self.b[...] = b
        if self.n_dyn:
            self.dyn[...] = np.asarray(dyn, self.dtype).reshape(self.dyn.shape)

    def state(self):
        """(f, u, b), plus dyn when the envs have dynamic obstacles."""
        base = (self.f.copy(), self.u.copy(), self.b.copy())
        return base + (self.dyn.copy(),) if self.n_dyn else base

    def dyn_advance(self, i: int, dt: float):
        """One motion step of env i's obstacles alone (dt: control interval)."""
        self.L.orc_dyn_advance(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), int(i), dt)

    def dyn_collide(self, i: int, x: float, y: float) -> bool:
        return bool(self.L.orc_dyn_collide(C.byref(self.cfg), C.byref(self.cenvs), int(i), x, y))

    def lidar_dyn(self, map_id: int, discs, x: float, y: float, phi: float, nb: int):
        """Hit indices and noise-free ranges of nb beams with obstacle discs
        (centres [(x, y), ...]) in the way."""
        d = np.ascontiguousarray(np.asarray(discs, self.dtype).reshape(-1))
        hits = np.zeros(nb, np.int32)
        ranges = np.zeros(nb, self.dtype)
        self.L.orc_lidar_dyn(C.byref(self.cfg), C.byref(self.cmaps), int(map_id), d.ctypes.data if d.size else None,
                             d.size // 2, x, y, phi, int(nb), hits.ctypes.data, ranges.ctypes.data)
        return hits, ranges

    # -- calls ------------------------------------------------------------
    def reset(self):
        obs = np.zeros((self.n, self.obs_dim), self.dtype)
        self.L.orc_reset(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), obs.ctypes.data)
        return obs

    def reset_env(self, i: int, ep_id: int):
        obs = np.zeros(self.obs_dim, self.dtype)
        self.L.orc_reset_env(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), int(i),
                             int(ep_id), obs.ctypes.data)
        return obs

    def step(self, actions, obs=None, term_obs=None):
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        assert a.size == self.n
        obs = np.zeros((self.n, self.obs_dim), self.dtype) if obs is None else obs
        term = np.zeros((self.n, self.obs_dim), self.dtype) if term_obs is None else term_obs
        rew = np.zeros(self.n, self.dtype)
        done = np.zeros(self.n, np.uint8)
        self.L.orc_step(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), a.ctypes.data,
                        obs.ctypes.data, rew.ctypes.data, done.ctypes.data, term.ctypes.data,
                        self.status.ctypes.data)
        return obs, rew, done, term

    def step_one(self, i: int, a: int):
        """Step env i alone; returns (obs row, reward, done, term row)."""
        obs = np.zeros(self.obs_dim, self.dtype)
        term = np.zeros(self.obs_dim, self.dtype)
        rew = np.zeros(1, self.dtype)
        done = np.zeros(1, np.uint8)
        self.L.orc_step_one(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), int(i), int(a),
                            obs.ctypes.data, rew.ctypes.data, done.ctypes.data, term.ctypes.data,
                            self.status.ctypes.data)
        return obs, rew[0], int(done[0]), term

    def random_action(self, i: int, t: int) -> int:
        return int(self.L.orc_random_action(C.byref(self.cfg), int(i), int(t)))

    def random_actions(self, t: int) -> np.ndarray:
        return np.array([self.L.orc_random_action(C.byref(self.cfg), i, int(t)) for i in range(self.n)],
                        np.uint8)

    def explore_uniform(self, t: int) -> np.ndarray:
        return np.array([self.L.orc_explore_uniform(C.byref(self.cfg), i, int(t)) for i in range(self.n)],
                        self.dtype)

    def rollout_random(self, K: int, t0: int, obs=None):
        obs = np.zeros((self.n, self.obs_dim), self.dtype) if obs is None else obs
        term = np.zeros((self.n, self.obs_dim), self.dtype)
        act = np.zeros((K, self.n), np.uint8)
        rew = np.zeros((K, self.n), self.dtype)
        done = np.zeros((K, self.n), np.uint8)
        self.L.orc_rollout_random(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), int(K),
                                  int(t0), obs.ctypes.data, term.ctypes.data, act.ctypes.data,
                                  rew.ctypes.data, done.ctypes.data, self.status.ctypes.data)
        return obs, act, rew, done

    def rollout_random_range(self, i0: int, i1: int, K: int, t0: int = 0):
        """Step envs [i0, i1) alone for K random-action steps (timing)."""
        self.L.orc_rollout_random_range(C.byref(self.cfg), C.byref(self.cmaps), C.byref(self.cenvs), int(i0),
                                        int(i1), int(K), int(t0), self.status.ctypes.data)

    # -- single-query helpers for the pins ---------------------------------
    def lidar(self, map_id: int, x: float, y: float, phi: float, nb: int | None = None):
        nb = self.B if nb is None else nb
        hits = np.zeros(nb, np.int32)
        ranges = np.zeros(nb, self.dtype)
        self.L.orc_lidar(C.byref(self.cfg), C.byref(self.cmaps), int(map_id), x, y, phi, int(nb),
                         hits.ctypes.data, ranges.ctypes.data)
        return hits, ranges

    def collide(self, map_id: int, x: float, y: float) -> bool:
        return bool(self.L.orc_collide(C.byref(self.cfg), C.byref(self.cmaps), int(map_id), x, y))


def sincos(a, prec="f32"):
    L = lib(prec)
    R = C.c_float if prec == "f32" else C.c_double
    s, c = R(), R()
    L.orc_sincos(a, C.byref(s), C.byref(c))
    return s.value, c.value
