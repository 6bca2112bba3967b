"""Python front end of the learned part (``sg_qnet_*``, ``sg_replay_*``,
``sg_td_train_step``): argument marshalling only."""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class QNet:
    """Q-network on the device (``sg_qnet_t``): arch "dueling" (256-256, value
    and advantage heads) or "paper" (the paper's 256-128 network, plain
    Q-value head)."""

    def __init__(self, n_in: int, max_batch: int = 256, seed: int = 0, arch: str = "dueling"):
        self.L = _lib.load()
        self.n_in = int(n_in)
        self.arch = arch
        self.handle = C.c_void_p()
        check(self.L.sg_qnet_create(self.n_in, _lib.SG_QNET_ARCHS[arch], int(max_batch), int(seed) & (2**64 - 1),
                                    C.byref(self.handle)), "sg_qnet_create")
        n = C.c_int64()
        check(self.L.sg_qnet_num_params(self.handle, C.byref(n)), "sg_qnet_num_params")
        self.n_params = int(n.value)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.L.sg_qnet_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta, which: str = "both"):
        th = np.ascontiguousarray(theta, np.float32)
        assert th.size == self.n_params
        w = {"online": 0, "target": 1, "both": 2}[which]
        check(self.L.sg_qnet_set_params(self.handle, th.ctypes.data, th.size, w), "sg_qnet_set_params")

    def get_params(self, which: str = "online") -> np.ndarray:
        th = np.zeros(self.n_params, np.float32)
        check(self.L.sg_qnet_get_params(self.handle, th.ctypes.data, th.size, {"online": 0, "target": 1}[which]),
              "sg_qnet_get_params")
        return th

    def optimizer_state(self):
        m = np.zeros(self.n_params, np.float32)
        v = np.zeros(self.n_params, np.float32)
        steps = C.c_uint64()
        check(self.L.sg_qnet_get_optimizer(self.handle, m.ctypes.data, v.ctypes.data, self.n_params,
                                           C.byref(steps)), "sg_qnet_get_optimizer")
        return m, v, int(steps.value)

    def set_rollout_rows(self, rows: int):
        """Envs per CTA of the fused rollout (16 or 32 on the mma.sync kernel,
        128 on the tcgen05 kernel, or 0 = automatic)."""
        check(self.L.sg_qnet_set_rollout_rows(self.handle, int(rows)), "sg_qnet_set_rollout_rows")

    def set_grid_limit(self, rollout: int = 0, learner: int = 0):
        """CTA caps of the tcgen05 fused rollout and TD step run with this
        network (0 = every SM): concurrent actor and learner keep SMs of
        their own."""
        check(self.L.sg_qnet_set_grid_limit(self.handle, int(rollout), int(learner)), "sg_qnet_set_grid_limit")

    def copy_from(self, src: "QNet", stream=None):
        """This network's online weights <- src's (model upload), stream-ordered."""
        check(self.L.sg_qnet_copy_params(self.handle, src.handle, _stream(stream)), "sg_qnet_copy_params")

    def set_optimizer_state(self, m, v, steps: int):
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        check(self.L.sg_qnet_set_optimizer(self.handle, m.ctypes.data, v.ctypes.data, self.n_params, int(steps)),
              "sg_qnet_set_optimizer")

    def state_dict(self):
        """Everything needed to resume learning: online and target
        parameters, Adam moments, optimiser step count."""
        m, v, steps = self.optimizer_state()
        return dict(online=self.get_params("online"), target=self.get_params("target"), m=m, v=v, steps=steps)

    def load_state_dict(self, d):
        self.set_params(d["online"], "online")
        self.set_params(d["target"], "target")
        self.set_optimizer_state(d["m"], d["v"], d["steps"])

    def forward(self, obs: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        assert obs.is_cuda and obs.dtype == torch.float32 and obs.shape[1] == self.n_in
        obs = obs.contiguous()
        out = torch.empty((obs.shape[0], 5), dtype=torch.float32, device=obs.device) if out is None else out
        check(self.L.sg_qnet_forward(self.handle, _ptr(obs), int(obs.shape[0]), _ptr(out), _stream(stream)),
              "sg_qnet_forward")
        return out

    def train_step(self, replay, batch: int, gamma: float = 0.98, lr: float = 1e-4, target_every: int = 200,
                   seed: int = 0, loss=None, grad=None, stream=None):
        check(self.L.sg_td_train_step(self.handle, replay.handle, int(batch), float(gamma), float(lr),
                                      int(target_every), int(seed) & (2**64 - 1), _ptr(loss), _ptr(grad),
                                      _stream(stream)), "sg_td_train_step")
        return loss


class Replay:
    """Device replay ring (``sg_replay_t``) of slots_per_env x n_envs entries;
    the learner never samples the ``reserve`` newest slots' successors (see
    sg_replay_create)."""

    def __init__(self, slots_per_env: int, n_envs: int, obs_dim: int, reserve: int = 0):
        self.L = _lib.load()
        self.slots, self.n_envs, self.obs_dim = int(slots_per_env), int(n_envs), int(obs_dim)
        self.reserve = int(reserve)
        self.handle = C.c_void_p()
        check(self.L.sg_replay_create(self.slots, self.n_envs, self.obs_dim, self.reserve, C.byref(self.handle)),
              "sg_replay_create")
        self.capacity = self.slots * self.n_envs

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.L.sg_replay_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def steps_recorded(self) -> int:
        v = C.c_uint64()
        check(self.L.sg_replay_info(self.handle, None, C.byref(v), None, None, None, None, None), "sg_replay_info")
        return int(v.value)

    def write(self, first: int, s, s2, a, r, t, steps_recorded: int):
        """Write entries [first, first+len(a)) and set the recorded-step count."""
        arrs = [np.ascontiguousarray(x, dt) for x, dt in ((s, np.float32), (s2, np.float32), (a, np.uint8),
                                                          (r, np.float32), (t, np.uint8))]
        check(self.L.sg_replay_write(self.handle, int(first), int(arrs[2].size), *[x.ctypes.data for x in arrs],
                                     int(steps_recorded)), "sg_replay_write")

    def state_dict(self):
        return dict(entries=self.read(0, self.capacity), steps=self.steps_recorded())

    def load_state_dict(self, d):
        self.write(0, *d["entries"], steps_recorded=d["steps"])

    def read(self, first: int, count: int):
        """Host copies (s, s2, a, r, term) of entries [first, first+count)."""
        s = np.zeros((count, self.obs_dim), np.float32)
        s2 = np.zeros((count, self.obs_dim), np.float32)
        a = np.zeros(count, np.uint8)
        r = np.zeros(count, np.float32)
        t = np.zeros(count, np.uint8)
        check(self.L.sg_replay_read(self.handle, int(first), int(count), s.ctypes.data, s2.ctypes.data,
                                    a.ctypes.data, r.ctypes.data, t.ctypes.data), "sg_replay_read")
        return s, s2, a, r, t
