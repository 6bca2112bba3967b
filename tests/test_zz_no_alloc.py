"""The allocation-free TD gradient (sg_td_grad_noalloc) against the learner's
regular entry point and against the float64 oracle.

sg_td_grad_noalloc serves callers that cannot allocate device memory (a
fixed memory budget, another framework's allocator, contexts where cudaMalloc
is not allowed): they pass parameters and a batch, and the library keeps its
intermediates in a static device array.  Here its loss and gradient must equal
those of sg_td_train_step (lr = 0) on the same transitions bit for bit (the
same kernels in the same summation order at these batches), on two calls in a
row (the shared scratch is reused); at the widest input (69) they must match the oracle's
bf16 recipe element by element; a batch with an action outside the table
must give NaN; and oversized requests must be refused.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from oracle import qnet as OQ
from tests._helpers import ring_sample_entries
from workloads import workload

pytestmark = pytest.mark.gpu

# element-wise bound against the oracle's bf16 recipe (the learner's TD parity tests use the same)
TD_RTOL = 1e-2
TD_ATOL = 2e-3


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _setup():
    from paper_2305_04180_gb300 import QNet, Replay, Sim

    w = workload("qnet4096", n_envs=64)
    g = Sim(w.params, w.maps(), w.env_map)
    q = QNet(g.obs_dim, 256, seed=11)
    rp = Replay(32, g.n, g.obs_dim)
    g.reset()
    g.rollout(40, policy="eps_q", qnet=q, eps=torch.from_numpy(w.eps).cuda(), replay=rp)
    torch.cuda.synchronize()
    return g, q, rp


def _regular(q, rp, th_on, th_tg, batch, seed):
    """Loss and gradient from sg_td_train_step (lr = 0), and the transitions
    it sampled (the learner's counter-RNG sample rule)."""
    q.set_params(th_on, "online")
    q.set_params(th_tg, "target")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(q.n_params, device="cuda")
    q.train_step(rp, batch, gamma=0.98, lr=0.0, seed=seed, loss=loss, grad=grad)
    torch.cuda.synchronize()
    idx = ring_sample_entries(seed, 0, batch, rp.steps_recorded(), rp.slots, rp.n_envs, rp.reserve)
    s, s2, a, r, t = rp.read(0, rp.capacity)
    return float(loss.item()), grad.cpu().numpy(), (s[idx], a[idx], r[idx], s2[idx], t[idx])


def _noalloc(th_on, th_tg, n_in, batch_arrays, gamma=0.98):
    from paper_2305_04180_gb300 import _lib

    L = _lib.load()
    s, a, r, s2, t = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in batch_arrays)
    pon = torch.from_numpy(np.ascontiguousarray(th_on, np.float32)).cuda()
    ptg = torch.from_numpy(np.ascontiguousarray(th_tg, np.float32)).cuda()
    loss = torch.full((1,), float("nan"), device="cuda")
    grad = torch.full((pon.numel(),), float("nan"), device="cuda")
    rc = L.sg_td_grad_noalloc(_ptr(pon), _ptr(ptg), n_in, _ptr(s), _ptr(a), _ptr(r), _ptr(s2), _ptr(t),
                              s.shape[0], gamma, _ptr(loss), _ptr(grad),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, (rc, L.sg_last_cuda_error())
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy()


def _theta(seed, n_in, scale):
    p = OQ.init_params(seed, n_in)
    return (OQ.flatten(p) * scale).astype(np.float32)


def test_noalloc_matches_regular_entry_point_twice():
    """Two calls in a row, at batches 256 and 100: at batches up to 256 both
    entry points run the same 16-sample kernels in the same summation order,
    so loss and gradient are bit-equal."""
    g, q, rp = _setup()
    n_in = g.obs_dim
    for call, (batch, seed, s_on, s_tg) in enumerate(((256, 5, 21, 22), (100, 9, 23, 24))):
        th_on, th_tg = _theta(s_on, n_in, 2.0), _theta(s_tg, n_in, 2.0)
        loss_ref, grad_ref, arrays = _regular(q, rp, th_on, th_tg, batch, seed)
        loss, grad = _noalloc(th_on, th_tg, n_in, arrays)
        assert np.isfinite(grad).all(), call
        assert np.float32(loss) == np.float32(loss_ref), (call, loss, loss_ref)
        assert np.array_equal(grad.view(np.uint32), grad_ref.view(np.uint32)), call


def test_noalloc_widest_input_against_oracle():
    """n_in = 69 (the widest input, whose weight image sizes the scratch) at
    batch 256, on synthetic transitions: loss and every gradient entry against
    the float64 oracle's bf16 recipe, twice (the scratch keeps the first
    call's contents)."""
    n_in, batch = 69, 256
    rng = np.random.default_rng(69)
    for call in range(2):
        th_on, th_tg = _theta(31 + call, n_in, 2.0), _theta(41 + call, n_in, 2.0)
        s = rng.uniform(-1, 1, size=(batch, n_in)).astype(np.float32)
        s2 = rng.uniform(-1, 1, size=(batch, n_in)).astype(np.float32)
        a = rng.integers(0, 5, size=batch).astype(np.uint8)
        r = rng.normal(size=batch).astype(np.float32)
        t = (rng.uniform(size=batch) < 0.1).astype(np.uint8)
        loss, grad = _noalloc(th_on, th_tg, n_in, (s, a, r, s2, t))
        bt = dict(s=s.astype(np.float64), a=a.astype(np.int64), r=r.astype(np.float64), s2=s2.astype(np.float64),
                  term=t.astype(np.float64))
        pon = OQ.unflatten(th_on.astype(np.float64), n_in)
        ptg = OQ.unflatten(th_tg.astype(np.float64), n_in)
        ref_loss, ref_g = OQ.td_loss_grad(pon, ptg, bt, 0.98, bf16=True)
        rflat = OQ.flatten(ref_g)
        assert abs(loss - ref_loss) <= 1e-2 * abs(ref_loss), (call, loss, ref_loss)
        o = 0
        for name, shp in OQ.param_shapes(n_in):
            k = int(np.prod(shp))
            rb, gb = rflat[o:o + k], grad[o:o + k].astype(np.float64)
            bound = TD_ATOL * np.abs(rb).max() + TD_RTOL * np.abs(rb)
            assert np.all(np.abs(gb - rb) <= bound), (call, name)
            o += k


def test_noalloc_invalid_action_gives_nan():
    """An action index outside the table in the caller's batch: loss and
    gradient are NaN (no partial result), and the next valid call is
    unaffected."""
    n_in, batch = 37, 64
    rng = np.random.default_rng(5)
    th_on, th_tg = _theta(51, n_in, 2.0), _theta(52, n_in, 2.0)
    s = rng.uniform(-1, 1, size=(batch, n_in)).astype(np.float32)
    a = rng.integers(0, 5, size=batch).astype(np.uint8)
    r = rng.normal(size=batch).astype(np.float32)
    t = np.zeros(batch, np.uint8)
    good = _noalloc(th_on, th_tg, n_in, (s, a, r, s, t))
    bad_a = a.copy()
    bad_a[17] = 200
    loss, grad = _noalloc(th_on, th_tg, n_in, (s, bad_a, r, s, t))
    assert np.isnan(loss) and np.isnan(grad).all()
    again = _noalloc(th_on, th_tg, n_in, (s, a, r, s, t))
    assert again[0] == good[0] and np.array_equal(again[1].view(np.uint32), good[1].view(np.uint32))


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2305_04180_gb300 import _lib

    L = _lib.load()
    n_in, batch = 37, 257
    x = torch.zeros((batch, 69), device="cuda")
    b = torch.zeros(batch, dtype=torch.uint8, device="cuda")
    th = torch.zeros(OQ.n_params(69), device="cuda")
    grad = torch.zeros(OQ.n_params(69), device="cuda")
    rc = L.sg_td_grad_noalloc(_ptr(th), _ptr(th), n_in, _ptr(x), _ptr(b), _ptr(x), _ptr(x), _ptr(b), batch, 0.98,
                              None, _ptr(grad), None)
    assert rc == _lib.SG_E_INVAL and b"256" in L.sg_last_cuda_error()
    rc = L.sg_td_grad_noalloc(_ptr(th), _ptr(th), 70, _ptr(x), _ptr(b), _ptr(x), _ptr(x), _ptr(b), 16, 0.98,
                              None, _ptr(grad), None)
    assert rc == _lib.SG_E_INVAL and b"69" in L.sg_last_cuda_error()
