"""The allocation-free TD gradient (sg_td_grad_noalloc) against the learner's
regular entry point.

sg_td_grad_noalloc serves callers that cannot allocate device memory (a
fixed memory budget, another framework's allocator, contexts where cudaMalloc
is not allowed): they pass parameters and a batch, and the library keeps its
intermediates in a static device array.  Here its loss and gradient must equal
those of sg_td_train_step (lr = 0) on the same transitions, on two calls in a
row (the shared scratch is reused), and oversized requests must be refused.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from oracle import qnet as OQ
from tests._helpers import ring_sample_entries
from workloads import workload

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5  # same kernels and summation order: expected equal, tolerance as elsewhere


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
    g, q, rp = _setup()
    n_in = g.obs_dim
    for call, (batch, seed, s_on, s_tg) in enumerate(((256, 5, 21, 22), (100, 9, 23, 24))):
        th_on, th_tg = _theta(s_on, n_in, 2.0), _theta(s_tg, n_in, 2.0)
        loss_ref, grad_ref, arrays = _regular(q, rp, th_on, th_tg, batch, seed)
        loss, grad = _noalloc(th_on, th_tg, n_in, arrays)
        assert np.isfinite(grad).all(), call
        assert abs(loss - loss_ref) <= REL_TOL * max(1e-6, abs(loss_ref)), (call, loss, loss_ref)
        rel = np.linalg.norm(grad - grad_ref) / np.linalg.norm(grad_ref)
        assert rel <= REL_TOL, (call, rel)


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
