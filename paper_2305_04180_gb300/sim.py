"""Python front end of the simulator handle (``sg_sim_*`` entry points)."""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check

STATE_F = ("x", "y", "phi", "vl", "va", "dt", "K", "cap", "sigma")
STATE_U = ("ep_step", "ep_id", "t", "fifo")


def make_config(params: dict, n_envs: int) -> _lib.sg_sim_config:
    """Fill an ``sg_sim_config`` from a parameter dict (see workloads)."""
    c = _lib.sg_sim_config()
    acts = params["actions"]
    c.n_envs = int(n_envs)
    c.n_beams = int(params["n_beams"])
    c.n_actions = len(acts)
    c.t_max = int(params["t_max"])
    c.delay_lo = int(params["delay_lo"])
    c.delay_hi = int(params["delay_hi"])
    for k in ("fov", "range_max", "march_step", "robot_radius", "goal_radius", "near_dist", "start_offset",
              "start_jitter", "dt_lo", "dt_hi", "k_lo", "k_hi", "cap_lo", "cap_hi", "sigma_lo", "sigma_hi",
              "v_nom", "w_nom"):
        setattr(c, k, float(params[k]))
    for i, (v, w) in enumerate(acts):
        c.action_v[i] = float(v)
        c.action_w[i] = float(w)
    c.seed = int(params["seed"]) & 0xFFFFFFFFFFFFFFFF
    # dynamic obstacles: optional, none by default
    c.n_dyn = int(params.get("n_dyn", 0))
    for k in ("dyn_radius", "dyn_speed_lo", "dyn_speed_hi", "dyn_keepout"):
        setattr(c, k, float(params.get(k, 0.0)))
    # direction sectors of the march's skip planes (0: chosen by the library)
    c.march_sectors = int(params.get("march_sectors", 0))
    return c


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Sim:
    """N vectorized environments on one GPU (``sg_sim_t``).

    ``maps`` is a list of uint8 numpy grids (rows = y), ``env_map`` the map of
    each env, ``env_beams`` optional per-env beam counts.
    """

    def __init__(self, params: dict, maps, env_map, env_beams=None, device=None):
        self.L = _lib.load()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        env_map = np.ascontiguousarray(env_map, dtype=np.int32)
        self.n = int(env_map.size)
        self.cfg = make_config(params, self.n)
        self.n_dyn = int(self.cfg.n_dyn)
        self.params = dict(params)
        grids = [np.ascontiguousarray(m, dtype=np.uint8) for m in maps]
        ptrs = (C.c_void_p * len(grids))(*[g.ctypes.data for g in grids])
        w = np.array([g.shape[1] for g in grids], np.int32)
        h = np.array([g.shape[0] for g in grids], np.int32)
        eb = None if env_beams is None else np.ascontiguousarray(env_beams, dtype=np.int32)
        self.env_beams = eb
        self.env_map_host = env_map
        self.map_shapes = [tuple(g.shape) for g in grids]
        self.handle = C.c_void_p()
        with torch.cuda.device(dev):
            check(self.L.sg_sim_create(C.byref(self.cfg), len(grids), ptrs, w.ctypes.data, h.ctypes.data,
                                       env_map.ctypes.data, None if eb is None else eb.ctypes.data,
                                       C.byref(self.handle)), "sg_sim_create")
        info = _lib.sg_sim_info()
        check(self.L.sg_sim_info_get(self.handle, C.byref(info)), "sg_sim_info_get")
        self.info = info
        self.obs_dim = int(info.obs_dim)
        self.n_maps = len(grids)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.L.sg_sim_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers --------------------------------------------------------
    def new_obs(self):
        return torch.empty((self.n, self.obs_dim), dtype=torch.float32, device=self.device)

    # -- calls ----------------------------------------------------------
    def reset(self, seed=None, obs=None, stream=None):
        obs = self.new_obs() if obs is None else obs
        seed = int(self.cfg.seed if seed is None else seed) & 0xFFFFFFFFFFFFFFFF
        check(self.L.sg_sim_reset(self.handle, seed, _ptr(obs), _stream(stream)), "sg_sim_reset")
        return obs

    def step(self, actions, obs=None, rew=None, done=None, term_obs=None, stream=None):
        assert actions.dtype == torch.uint8 and actions.is_cuda and actions.numel() == self.n
        obs = self.new_obs() if obs is None else obs
        rew = torch.empty(self.n, dtype=torch.float32, device=self.device) if rew is None else rew
        done = torch.empty(self.n, dtype=torch.uint8, device=self.device) if done is None else done
        check(self.L.sg_sim_step(self.handle, _ptr(actions), _ptr(obs), _ptr(rew), _ptr(done), _ptr(term_obs),
                                 _stream(stream)), "sg_sim_step")
        return obs, rew, done

    def vem_eps(self, e_min=0.01, e_max=0.8, or_start=None, or_final=None, decay_steps=500_000, out=None,
                stream=None):
        """VEM exploration noise per env at the current interacting-step count
        (sg_vem_eps).  OR defaults to the paper's Sparrow schedule scaled to N:
        from N envs down to 3/16 of them (16 -> 3 at N = 16)."""
        out = torch.empty(self.n, dtype=torch.float32, device=self.device) if out is None else out
        or_start = float(self.n if or_start is None else or_start)
        or_final = float(max(2.0, 3.0 * self.n / 16.0) if or_final is None else or_final)
        check(self.L.sg_vem_eps(self.handle, float(e_min), float(e_max), or_start, or_final, float(decay_steps),
                                _ptr(out), _stream(stream)), "sg_vem_eps")
        return out

    def rollout(self, K, policy="random", qnet=None, eps=None, replay=None, obs=None, obs_seq=None, act_seq=None,
                rew_seq=None, done_seq=None, stream=None):
        pol = {"random": _lib.SG_POLICY_RANDOM, "eps_q": _lib.SG_POLICY_EPS_Q}[policy]
        check(self.L.sg_sim_rollout(self.handle, int(K), pol, None if qnet is None else qnet.handle, _ptr(eps),
                                    None if replay is None else replay.handle, _ptr(obs), _ptr(obs_seq),
                                    _ptr(act_seq), _ptr(rew_seq), _ptr(done_seq), _stream(stream)),
              "sg_sim_rollout")
        return obs

    def set_launch(self, kernel="grid", warps_per_block=4, warps_per_env=1, obs_warps=0, blocks_per_sm=0,
                   order="index", segment=0, wait_iters=0):
        """Launch configuration of the network-free rollout (sg_sim_set_launch);
        accepts the keys of ``launch_config()``.  segment: time slicing of the
        pipelined kernel (steps, a multiple of 32; 0 = none); wait_iters: the
        bound of its waits (0 = about a second)."""
        # order 1 is "cost" (longest first) for the work-list kernel and "map"
        # (envs grouped by map) for the pipelined one
        orders = {"queue": ("index", "cost"), "pipe": ("index", "map")}.get(kernel, ("index",))
        if order not in orders:
            raise ValueError(f"order {order!r} is not one of {orders} for kernel {kernel!r}")
        L = _lib.sg_launch(_lib.SG_ROLLOUT_KERNELS[kernel], int(warps_per_block), int(warps_per_env),
                           int(obs_warps), int(blocks_per_sm), orders.index(order), int(segment),
                           int(wait_iters))
        check(self.L.sg_sim_set_launch(self.handle, C.byref(L)), "sg_sim_set_launch")

    def launch_config(self) -> dict:
        L = _lib.sg_launch()
        check(self.L.sg_sim_get_launch(self.handle, C.byref(L)), "sg_sim_get_launch")
        kinds = {v: k for k, v in _lib.SG_ROLLOUT_KERNELS.items()}
        return dict(kernel=kinds[L.kernel], warps_per_block=L.warps_per_block, warps_per_env=L.warps_per_env,
                    obs_warps=L.obs_warps, blocks_per_sm=L.blocks_per_sm,
                    order="index" if L.order == 0 else ("map" if L.kernel == _lib.SG_ROLLOUT_KERNELS["pipe"]
                                                         else "cost"),
                    segment=L.segment, wait_iters=L.wait_iters)

    def get_state(self):
        """(f [9, N] float32, u [4, N] uint32) host copies of the env state,
        plus dyn [4 n_dyn, N] float32 when the envs have dynamic obstacles."""
        nbytes = C.c_size_t(int(self.info.state_bytes))
        buf = np.zeros(int(self.info.state_bytes), np.uint8)
        check(self.L.sg_sim_get_state(self.handle, buf.ctypes.data, C.byref(nbytes)), "sg_sim_get_state")
        f = buf[: 36 * self.n].view(np.float32).reshape(9, self.n).copy()
        u = buf[36 * self.n:52 * self.n].view(np.uint32).reshape(4, self.n).copy()
        if not self.n_dyn:
            return f, u
        d = buf[52 * self.n:].view(np.float32).reshape(4 * self.n_dyn, self.n).copy()
        return f, u, d

    def set_state(self, f, u, dyn=None):
        f = np.ascontiguousarray(f, np.float32).reshape(9, self.n)
        u = np.ascontiguousarray(u, np.uint32).reshape(4, self.n)
        parts = [f.ravel().view(np.uint8), u.ravel().view(np.uint8)]
        if self.n_dyn:
            parts.append(np.ascontiguousarray(dyn, np.float32).reshape(4 * self.n_dyn, self.n).ravel().view(np.uint8))
        buf = np.concatenate(parts)
        check(self.L.sg_sim_set_state(self.handle, buf.ctypes.data, buf.size), "sg_sim_set_state")

    def state_blob(self, f, u, dyn=None, pin=True):
        """The state blob of set_state as a (page-locked) uint8 host tensor,
        for set_state_async."""
        f = np.ascontiguousarray(f, np.float32).reshape(9, self.n)
        u = np.ascontiguousarray(u, np.uint32).reshape(4, self.n)
        parts = [f.ravel().view(np.uint8), u.ravel().view(np.uint8)]
        if self.n_dyn:
            parts.append(np.ascontiguousarray(dyn, np.float32).reshape(4 * self.n_dyn, self.n).ravel().view(np.uint8))
        buf = torch.from_numpy(np.concatenate(parts))
        return buf.pin_memory() if pin else buf

    def set_state_async(self, blob, stream=None):
        """sg_sim_set_state_async: upload a state blob (state_blob) ordered
        on the stream; blob must stay alive until the copy has run."""
        check(self.L.sg_sim_set_state_async(self.handle, C.c_void_p(blob.data_ptr()), int(blob.numel()),
                                            _stream(stream)), "sg_sim_set_state_async")

    def atlas(self):
        words = C.c_size_t(0)
        check(self.L.sg_sim_get_atlas(self.handle, None, C.byref(words), None, None), "sg_sim_get_atlas")
        out = np.zeros(words.value, np.uint32)
        offs = np.zeros(self.n_maps, np.int64)
        rw = np.zeros(self.n_maps, np.int32)
        check(self.L.sg_sim_get_atlas(self.handle, out.ctypes.data, C.byref(words), offs.ctypes.data,
                                      rw.ctypes.data), "sg_sim_get_atlas")
        return out, offs, rw

    def clearance(self):
        """(bytes, per-map offsets) of the march's clearance maps."""
        nbytes = C.c_size_t(0)
        check(self.L.sg_sim_get_clearance(self.handle, None, C.byref(nbytes), None), "sg_sim_get_clearance")
        out = np.zeros(nbytes.value, np.uint8)
        offs = np.zeros(self.n_maps, np.int64)
        check(self.L.sg_sim_get_clearance(self.handle, out.ctypes.data, C.byref(nbytes), offs.ctypes.data),
              "sg_sim_get_clearance")
        return out, offs

    def sector_skip(self):
        """(bytes, per-map offsets, sectors) of the march's sector skip planes
        (empty when the simulator uses the Chebyshev skip map alone)."""
        nbytes = C.c_size_t(0)
        check(self.L.sg_sim_get_sector_skip(self.handle, None, C.byref(nbytes), None), "sg_sim_get_sector_skip")
        out = np.zeros(nbytes.value, np.uint8)
        offs = np.zeros(self.n_maps, np.int64)
        check(self.L.sg_sim_get_sector_skip(self.handle, out.ctypes.data, C.byref(nbytes), offs.ctypes.data),
              "sg_sim_get_sector_skip")
        return out, offs, int(self.info.march_sectors)

    def status(self):
        v = C.c_uint32(0)
        rc = self.L.sg_sim_status(self.handle, C.byref(v))
        if rc not in (_lib.SG_OK, _lib.SG_E_DEVICE):
            check(rc, "sg_sim_status")
        return int(v.value)
