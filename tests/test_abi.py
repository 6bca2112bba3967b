"""The C ABI library builds, loads and exports every symbol its header
declares (CPU only: no compute call is made without a GPU)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sparrow_gb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sg_sim_create", "sg_sim_reset", "sg_sim_step", "sg_sim_rollout", "sg_sim_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2305_04180_gb300 import build

    path = build.build()
    lib = C.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2305_04180_gb300 import _lib

    assert set(_lib.SIGNATURES) == set(_declared())


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2305_04180_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "sparrow_oracle" not in src, f


def test_strerror_without_gpu():
    from paper_2305_04180_gb300 import build

    lib = C.CDLL(build.build())
    lib.sg_strerror.restype = C.c_char_p
    assert lib.sg_strerror(0) == b"ok"
    assert lib.sg_strerror(-1) == b"invalid argument"


def test_create_rejects_bad_config_without_touching_the_gpu():
    """Argument validation happens on the host before any CUDA call."""
    from paper_2305_04180_gb300 import _lib
    from paper_2305_04180_gb300.sim import make_config
    from workloads.configs import base_params

    lib = _lib.load()
    cfg = make_config(base_params(), 4)
    cfg.n_beams = 1  # below the minimum of 2
    h = C.c_void_p()
    grid = (C.c_uint8 * 16)()
    ptrs = (C.c_void_p * 1)(C.addressof(grid))
    w = (C.c_int32 * 1)(4)
    em = (C.c_int32 * 4)(0, 0, 0, 0)
    assert lib.sg_sim_create(C.byref(cfg), 1, ptrs, w, w, em, None, C.byref(h)) == _lib.SG_E_INVAL
    cfg = make_config(base_params(), 4)
    em_bad = (C.c_int32 * 4)(0, 0, 0, 3)  # map index out of range
    assert lib.sg_sim_create(C.byref(cfg), 1, ptrs, w, w, em_bad, None, C.byref(h)) == _lib.SG_E_INVAL
    assert lib.sg_sim_step(None, None, None, None, None, None, None) == _lib.SG_E_INVAL


@pytest.mark.parametrize("field,value", [("n_envs", 0), ("n_envs", (1 << 24) + 1), ("n_beams", 65),
                                         ("range_max", 4097.0), ("march_step", 0.0), ("t_max", 0),
                                         ("delay_hi", 3), ("n_dyn", -1)])
def test_create_rejects_each_limit_plus_one(field, value):
    """One past each documented limit is refused on the host (the limits
    themselves: 2^24 envs, 64 beams, 4,096 samples per beam, map sides of
    16,384, are exercised on the GPU)."""
    from paper_2305_04180_gb300 import _lib
    from paper_2305_04180_gb300.sim import make_config
    from workloads.configs import base_params

    lib = _lib.load()
    cfg = make_config(base_params(march_step=1.0), 4)
    setattr(cfg, field, value)
    h = C.c_void_p()
    grid = (C.c_uint8 * 16)()
    ptrs = (C.c_void_p * 1)(C.addressof(grid))
    w = (C.c_int32 * 1)(4)
    em = (C.c_int32 * 4)(0, 0, 0, 0)
    assert lib.sg_sim_create(C.byref(cfg), 1, ptrs, w, w, em, None, C.byref(h)) == _lib.SG_E_INVAL
    assert not h.value


@pytest.mark.parametrize("side", [(16385, 4), (4, 16385), (0, 4)])
def test_create_rejects_map_sides_past_the_limit(side):
    from paper_2305_04180_gb300 import _lib
    from paper_2305_04180_gb300.sim import make_config
    from workloads.configs import base_params

    lib = _lib.load()
    cfg = make_config(base_params(), 1)
    h = C.c_void_p()
    grid = (C.c_uint8 * 16)()
    ptrs = (C.c_void_p * 1)(C.addressof(grid))
    mw = (C.c_int32 * 1)(side[0])
    mh = (C.c_int32 * 1)(side[1])
    em = (C.c_int32 * 1)(0)
    assert lib.sg_sim_create(C.byref(cfg), 1, ptrs, mw, mh, em, None, C.byref(h)) == _lib.SG_E_INVAL
    assert lib.sg_sim_create(C.byref(cfg), 0, ptrs, mw, mh, em, None, C.byref(h)) == _lib.SG_E_INVAL
    assert lib.sg_sim_rollout(None, 0, 0, *([None] * 9)) == _lib.SG_E_INVAL
