"""Shared test plumbing: state conversion between the library blob and the
oracle's arrays, and small input builders.  Holds none of the step's
arithmetic."""

from __future__ import annotations

import numpy as np


def gpu_state_to_oracle(f, u, dyn=None):
    """Library state (f [9,N] f32; u [4,N]: ep_step, ep_id, t, fifo; dyn
    [4 n_dyn, N] with moving obstacles) -> oracle arrays (f [9,N]; u [2,N];
    b [3,N]: q0, q1, delay; dyn passed through)."""
    fifo = u[3].astype(np.uint32)
    b = np.stack([fifo & 0xFF, (fifo >> 8) & 0xFF, (fifo >> 16) & 0xFF]).astype(np.uint8)
    out = (f.copy(), u[:2].copy(), b)
    return out if dyn is None else out + (dyn.copy(),)


def oracle_state_to_gpu(f, u2, b, t):
    fifo = b[0].astype(np.uint32) | (b[1].astype(np.uint32) << 8) | (b[2].astype(np.uint32) << 16)
    t = np.broadcast_to(np.asarray(t, np.uint32), fifo.shape)
    return np.asarray(f, np.float32).copy(), np.stack([u2[0], u2[1], t, fifo]).astype(np.uint32)


def bits(a):
    """Float array as its bit pattern (for bit-exact comparisons that also
    distinguish -0.0 and NaN payloads)."""
    a = np.ascontiguousarray(a, np.float32)
    return a.view(np.uint32)


def ring_sample_entries(seed, tstep, batch, steps, slots, n_envs, reserve=0):
    """Ring entries the learner samples at optimiser step tstep: uniform over
    the min(steps, slots - reserve) most recent slots (counter RNG from the
    oracle), newest slot first."""
    from oracle.sim import lib as olib

    V = min(steps, slots - reserve)
    out = []
    for i in range(batch):
        j = olib("f32").orc_rng(seed, 4, tstep, i, 0) % (V * n_envs)
        slot = (steps - 1 - j // n_envs) % slots
        out.append(slot * n_envs + j % n_envs)
    return np.array(out)
