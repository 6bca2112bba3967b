"""Shared test plumbing: state conversion between the library blob and the
oracle's arrays, small input builders, and the error measure of the float64
tolerance checks.  Holds none of the step's arithmetic."""

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


def step_rel_error(f_old, f_new, f_ref):
    """Relative error of a float32 step's pose and velocity (rows x, y, phi,
    v_l, v_a of the [9, N] state) against the float64 oracle's step from the
    same state f_old.

    Each component is a sum of two terms (Eq. 5: K v + (1 - K) v_hat; Eq. 6:
    x - dt v_l cos(phi), y - dt v_l sin(phi), phi + dt v_a, then the wrap by
    2 pi), and float32 rounds a sum relative to the size of its terms, so the
    error is divided by |term 1| + |term 2| (the terms taken from f_old and
    the float64 result; 2 pi added where the heading wrapped).  Where the two
    terms do not cancel this is |x| within a factor 2; where they do (a
    heading or angular velocity passing through zero) dividing by |x| alone
    would turn one float32 rounding of the terms into an arbitrarily large
    "relative" error.  Returns a [5, N] array."""
    o = np.asarray(f_old, np.float64)
    r = np.asarray(f_ref, np.float64)
    g = np.asarray(f_new, np.float64)
    dt, K = o[5], o[6]
    c, s = np.cos(o[2]), np.sin(o[2])
    wrapped = np.abs(o[2] + dt * r[4] - r[2]) > np.pi
    scale = np.stack([
        np.abs(o[0]) + np.abs(dt * r[3] * c),
        np.abs(o[1]) + np.abs(dt * r[3] * s),
        np.abs(o[2]) + np.abs(dt * r[4]) + np.where(wrapped, 2 * np.pi, 0.0),
        np.abs(K * o[3]) + np.abs(r[3] - K * o[3]),
        np.abs(K * o[4]) + np.abs(r[4] - K * o[4]),
    ])
    err = np.abs(g[:5] - r[:5])
    return np.where(err == 0, 0.0, err / np.maximum(scale, np.finfo(np.float64).tiny))
