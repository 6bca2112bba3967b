"""ctypes binding of ``libsparrowgb.so`` (include/sparrow_gb.h).

Argument marshalling only: every step of the simulator runs in the CUDA
library.  Each C entry point is exposed under its own name; there is no CPU
fallback -- if the library is missing the import of this module fails.
"""

from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SG_OK = 0
SG_E_INVAL = -1
SG_E_ALIGN = -2
SG_E_OOM = -3
SG_E_CUDA = -4
SG_E_DEVICE = -5
SG_E_TIMEOUT = -6
SG_DEV_BAD_ACTION = 0x1
SG_DEV_TIMEOUT = 0x2
SG_DEV_BOUNDS = 0x4
SG_QNET_ARCHS = {"dueling": 0, "paper": 1}
SG_POLICY_RANDOM = 0
SG_POLICY_EPS_Q = 1


class SgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what} failed: {code} ({_strerror(code)}) {_last_cuda()}")


class sg_sim_config(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("n_beams", C.c_int32), ("n_actions", C.c_int32), ("t_max", C.c_int32),
        ("delay_lo", C.c_int32), ("delay_hi", C.c_int32),
        ("fov", C.c_float), ("range_max", C.c_float), ("march_step", C.c_float),
        ("robot_radius", C.c_float), ("goal_radius", C.c_float), ("near_dist", C.c_float),
        ("start_offset", C.c_float), ("start_jitter", C.c_float),
        ("dt_lo", C.c_float), ("dt_hi", C.c_float), ("k_lo", C.c_float), ("k_hi", C.c_float),
        ("cap_lo", C.c_float), ("cap_hi", C.c_float), ("sigma_lo", C.c_float), ("sigma_hi", C.c_float),
        ("v_nom", C.c_float), ("w_nom", C.c_float),
        ("action_v", C.c_float * 8), ("action_w", C.c_float * 8),
        ("seed", C.c_uint64),
        ("n_dyn", C.c_int32), ("dyn_radius", C.c_float), ("dyn_speed_lo", C.c_float),
        ("dyn_speed_hi", C.c_float), ("dyn_keepout", C.c_float),
        ("march_sectors", C.c_int32),
    ]


class sg_launch(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("warps_per_block", C.c_int32), ("warps_per_env", C.c_int32),
                ("obs_warps", C.c_int32), ("blocks_per_sm", C.c_int32), ("order", C.c_int32),
                ("segment", C.c_int32), ("wait_iters", C.c_int32)]


SG_ROLLOUT_KERNELS = {"grid": 0, "queue": 1, "split": 2, "pipe": 3}


class sg_sim_info(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("n_beams", C.c_int32), ("obs_dim", C.c_int32), ("n_maps", C.c_int32),
                ("atlas_words", C.c_int64), ("state_bytes", C.c_int64), ("device", C.c_int32),
                ("march_sectors", C.c_int32)]


_vp = C.c_void_p
_i32 = C.c_int32
# name -> (restype, argtypes); the order follows include/sparrow_gb.h
SIGNATURES = {
    "sg_sim_create": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sg_sim_destroy": (C.c_int, [_vp]),
    "sg_sim_info_get": (C.c_int, [_vp, _vp]),
    "sg_sim_reset": (C.c_int, [_vp, C.c_uint64, _vp, _vp]),
    "sg_sim_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sg_sim_rollout": (C.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sg_sim_set_launch": (C.c_int, [_vp, _vp]),
    "sg_sim_get_launch": (C.c_int, [_vp, _vp]),
    "sg_sim_get_state": (C.c_int, [_vp, _vp, _vp]),
    "sg_sim_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "sg_sim_set_state_async": (C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    "sg_sim_get_atlas": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sg_sim_get_clearance": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sg_sim_get_sector_skip": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sg_sim_status": (C.c_int, [_vp, _vp]),
    "sg_qnet_create": (C.c_int, [_i32, _i32, _i32, C.c_uint64, _vp]),
    "sg_qnet_destroy": (C.c_int, [_vp]),
    "sg_qnet_num_params": (C.c_int, [_vp, _vp]),
    "sg_qnet_set_params": (C.c_int, [_vp, _vp, C.c_int64, _i32]),
    "sg_qnet_get_params": (C.c_int, [_vp, _vp, C.c_int64, _i32]),
    "sg_qnet_get_optimizer": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp]),
    "sg_qnet_set_optimizer": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_uint64]),
    "sg_qnet_set_rollout_rows": (C.c_int, [_vp, _i32]),
    "sg_qnet_set_grid_limit": (C.c_int, [_vp, _i32, _i32]),
    "sg_qnet_copy_params": (C.c_int, [_vp, _vp, _vp]),
    "sg_qnet_forward": (C.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "sg_replay_create": (C.c_int, [_i32, _i32, _i32, _i32, _vp]),
    "sg_replay_destroy": (C.c_int, [_vp]),
    "sg_replay_info": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sg_replay_read": (C.c_int, [_vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp]),
    "sg_replay_write": (C.c_int, [_vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_uint64]),
    "sg_td_train_step": (C.c_int, [_vp, _vp, _i32, C.c_float, C.c_float, _i32, C.c_uint64, _vp, _vp, _vp]),
    "sg_vem_eps": (C.c_int, [_vp, C.c_float, C.c_float, C.c_double, C.c_double, C.c_double, _vp, _vp]),
    "sg_td_grad_noalloc": (C.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _i32, C.c_float, _vp, _vp, _vp]),
    "sg_probe_read": (C.c_int, [_vp, C.c_size_t, _i32, _vp, _i32, _vp]),
    "sg_graph_begin": (C.c_int, [_vp]),
    "sg_graph_end": (C.c_int, [_vp, _vp]),
    "sg_graph_launch": (C.c_int, [_vp, _vp]),
    "sg_graph_num_nodes": (C.c_int, [_vp, _vp]),
    "sg_graph_destroy": (C.c_int, [_vp]),
    "sg_strerror": (C.c_char_p, [C.c_int]),
    "sg_last_cuda_error": (C.c_char_p, []),
}

_LIB = None


def load(build_if_missing: bool = True):
    """Load the library (building it first if it is absent or stale).  The
    environment variable SG_LIB_VARIANT=debug selects the debug build
    (bounds checks that report SG_DEV_BOUNDS, see sg_sim_status) for the
    whole process."""
    global _LIB
    if _LIB is not None:
        return _LIB
    import torch  # noqa: F401  -- loads the CUDA runtime the library links against

    variant = os.environ.get("SG_LIB_VARIANT", "")
    if variant not in _build.VARIANTS:
        raise ImportError(f"SG_LIB_VARIANT={variant!r}: expected one of {sorted(_build.VARIANTS)}")
    path = _build.VARIANTS[variant][0]
    if build_if_missing and not _build.up_to_date(variant):
        _build.build(variant=variant)
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run paper_2305_04180_gb300.build.build()")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _strerror(code):
    try:
        return load(False).sg_strerror(code).decode()
    except Exception:
        return "?"


def _last_cuda():
    try:
        return load(False).sg_last_cuda_error().decode()
    except Exception:
        return ""


def check(code, what):
    if code != SG_OK:
        raise SgError(code, what)
    return code
