"""Actor-learner loop of the paper's ASL framework (Sec. 3.1, Alg. 1-2) over
the library's fused rollout and TD learner.

Host-side orchestration only: every step of the simulation, inference and
learning runs in the CUDA library.  The actor rolls the vectorized envs out
with its own copy of the network (VEM eps-greedy, transitions into the device
ring); the learner samples mini-batches and optimises its network; every
`upload_every` optimisation steps the actor takes the learner's weights
(Alg. 2 step 3, Alg. 1 step 1).

* VEM (Sec. 3.1.1): before every rollout chunk the per-env exploration noise
  is recomputed on the device from the envs' step counter (sg_vem_eps), so the
  exploring interval shrinks with the interacting steps, also inside captured
  graphs.  Default: the paper's Sparrow schedule (E_min 0.01, E_max 0.8, OR
  from N envs to 3N/16 over 500K interacting steps).
* TPS and the time feedback mechanism (Sec. 3.1.2, Eq. 1-4): the number of
  optimisation steps per vectorized step is held at rho = N * TPS / B
  (Eq. 2) by count.  With two streams the actor and the learner run
  concurrently and are coupled by events the way the TFM couples them by
  sleeping: the actor may run at most one rollout chunk ahead of the learner
  (the faster side waits on the slower one's event instead of sleeping for
  xi), and the measured periods V^T (per vectorized step) and B^T (per
  optimisation step) and xi = rho B^T - V^T are reported by tfm_report().
"""

from __future__ import annotations

from collections import deque

import torch

from .graph import Graph
from .qnet import QNet, Replay


class ColorTrainer:
    def __init__(self, sim, *, batch=256, slots=128, gamma=0.98, lr=1e-4, target_every=200, upload_every=50,
                 tps=256, learn_start=30000, eps=None, vem="paper", seed=0, two_streams=False, max_rollout_k=8,
                 arch="dueling"):
        """eps: a fixed per-env noise tensor (no schedule); otherwise vem is
        "paper", a dict of sg_vem_eps arguments, or None (fixed linear
        0.01 .. 0.81 over the envs).  arch: the Q-network ("dueling" or the
        paper's "paper")."""
        self.sim = sim
        n = sim.n
        self.batch, self.gamma, self.lr = batch, gamma, lr
        self.target_every, self.upload_every, self.tps = target_every, upload_every, tps
        self.learn_start, self.seed = learn_start, seed
        self.learner = QNet(sim.obs_dim, batch, seed=seed, arch=arch)
        self.actor = QNet(sim.obs_dim, batch, seed=seed, arch=arch)
        self.actor.copy_from(self.learner)
        # concurrent rollouts of up to max_rollout_k steps must not be sampled
        self.max_rollout_k = max_rollout_k
        self.replay = Replay(slots, n, sim.obs_dim, reserve=max_rollout_k if two_streams else 0)
        if eps is not None or vem is None:
            self.vem = None
            self.eps = eps if eps is not None else torch.linspace(0.01, 0.81, n, device="cuda")
        else:
            self.vem = (dict(e_min=0.01, e_max=0.8, or_start=float(n), or_final=max(2.0, 3.0 * n / 16.0),
                             decay_steps=500_000) if vem == "paper" else dict(vem))
            self.eps = sim.vem_eps(**self.vem)
        # per chunk (the last 4096): k, n_upd, actor start/end, learner start/end events
        self._tfm = deque(maxlen=4096)
        self.updates = 0
        self.transitions = 0
        self._carry = 0.0
        self.two_streams = two_streams
        self.s_actor = torch.cuda.Stream() if two_streams else torch.cuda.current_stream()
        self.s_learner = torch.cuda.Stream() if two_streams else torch.cuda.current_stream()
        self.loss = torch.zeros(1, device="cuda")

    def state_dict(self):
        """Checkpoint of the whole loop: env state, both networks with the
        learner's optimiser, the ring, and the loop counters.  The
        configuration (parameters, maps, seeds) is not part of it: restore
        into a loop built with the same configuration."""
        torch.cuda.synchronize()
        return dict(sim=self.sim.get_state(), learner=self.learner.state_dict(),
                    actor=self.actor.get_params("online"), replay=self.replay.state_dict(),
                    counters=(self.updates, self.transitions, self._carry))

    def load_state_dict(self, d):
        torch.cuda.synchronize()
        self.sim.set_state(*d["sim"])
        self.learner.load_state_dict(d["learner"])
        self.actor.set_params(d["actor"], "online")
        self.replay.load_state_dict(d["replay"])
        self.updates, self.transitions, self._carry = d["counters"]

    def steps_per_vec_step(self):
        """Optimisation steps per vectorized step (Eq. 2): N * TPS / B."""
        return self.sim.n * self.tps / self.batch

    def _actor_chunk(self, k, stream):
        """Alg. 1 steps 2-5 for k vectorized steps: VEM noise, fused policy
        and env steps, transitions into the ring."""
        if self.vem is not None:
            self.sim.vem_eps(**self.vem, out=self.eps, stream=stream)
        self.sim.rollout(k, policy="eps_q", qnet=self.actor, eps=self.eps, replay=self.replay, stream=stream)

    def _learner_steps(self, n_upd, stream):
        """Alg. 2 steps 1-3 n_upd times: sample, DDQN update, model upload every
        upload_every steps (the actor's copy is refreshed on its own stream
        after the learner's step, and the learner waits for the copy)."""
        for _ in range(n_upd):
            self.learner.train_step(self.replay, self.batch, gamma=self.gamma, lr=self.lr,
                                    target_every=self.target_every, seed=self.seed, loss=self.loss, stream=stream)
            self.updates += 1
            if self.updates % self.upload_every == 0:
                up = torch.cuda.Event()
                up.record(stream)
                self.s_actor.wait_event(up)
                self.actor.copy_from(self.learner, stream=self.s_actor)
                back = torch.cuda.Event()
                back.record(self.s_actor)
                stream.wait_event(back)

    def tfm_report(self):
        """Measured periods of the time feedback mechanism over the chunks run
        so far (synchronises): V^T per vectorized step and B^T per optimisation
        step (ms, means over chunks), rho, xi = rho B^T - V^T (> 0: the actor is
        the faster side and waits), the idle time of each stream between its
        chunks, and the achieved TPS = B x B_step / T_step (Eq. 1)."""
        torch.cuda.synchronize()
        v, b, a_idle, l_idle = [], [], [], []
        prev = None
        for k, n_upd, a0, a1, l0, l1 in self._tfm:
            v.append(a0.elapsed_time(a1) / k)
            if n_upd and l0 is not None:
                b.append(l0.elapsed_time(l1) / n_upd)
            if prev is not None:
                a_idle.append(prev[0].elapsed_time(a0))
                if l0 is not None and prev[1] is not None:
                    l_idle.append(prev[1].elapsed_time(l0))
            prev = (a1, l1)
        rho = self.steps_per_vec_step()
        vt = sum(v) / len(v) if v else None
        bt = sum(b) / len(b) if b else None
        t_step = self.transitions
        return dict(rho=rho, v_period_ms=vt, b_period_ms=bt,
                    xi_ms=(rho * bt - vt) if (vt is not None and bt is not None) else None,
                    actor_idle_ms_per_chunk=sum(a_idle) / len(a_idle) if a_idle else 0.0,
                    learner_idle_ms_per_chunk=sum(l_idle) / len(l_idle) if l_idle else 0.0,
                    tps=self.batch * self.updates / t_step if t_step else 0.0, chunks=len(self._tfm))

    def run(self, vec_steps: int, rollout_k: int = 8):
        """Collect vec_steps vectorized steps in chunks of rollout_k, training
        rho = N * TPS / B optimisation steps per vectorized step once
        learn_start transitions are in the ring.  With two streams, chunk c of
        the actor runs while the learner trains on chunk c - 1 and waits for
        the learner to finish chunk c - 2 (at most one chunk of lag)."""
        assert rollout_k <= self.max_rollout_k
        done = 0
        learner_done = []  # learner end events of the last chunks
        while done < vec_steps:
            k = min(rollout_k, vec_steps - done)
            if self.two_streams and len(learner_done) >= 2:
                self.s_actor.wait_event(learner_done[-2])
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(self.s_actor):
                a0.record(self.s_actor)
                self._actor_chunk(k, self.s_actor)
                a1.record(self.s_actor)
            done += k
            self.transitions += k * self.sim.n
            l0 = l1 = None
            n_upd = 0
            if self.transitions >= self.learn_start:
                self.s_learner.wait_event(a1)
                self._carry += k * self.steps_per_vec_step()
                n_upd = int(self._carry)
                self._carry -= n_upd
                l0 = torch.cuda.Event(enable_timing=True)
                l1 = torch.cuda.Event(enable_timing=True)
                l0.record(self.s_learner)
                self._learner_steps(n_upd, self.s_learner)
                l1.record(self.s_learner)
                learner_done = (learner_done + [l1])[-2:]
            self._tfm.append((k, n_upd, a0, a1, l0, l1))
        torch.cuda.synchronize()
        return self

    def capture_iteration(self, rollout_k: int, td_steps: int, concurrent: bool = True, learner_sms: int = 0):
        """One actor-learner iteration as a CUDA graph: the actor's fused
        rollout of rollout_k steps and td_steps learner steps, then the model
        upload.  concurrent=True forks the two as branches of the graph that
        overlap on the GPU (the ring's reserve keeps the learner off the
        slots being written; which completed slots it samples then depends on
        timing); concurrent=False runs the learner after the rollout and is
        deterministic.  learner_sms > 0 (concurrent only): the learner's TD
        steps run on at most that many CTAs and the rollout on the other SMs,
        so the branches overlap instead of taking turns.  Requires
        two_streams=True, rollout_k <= max_rollout_k."""
        assert self.two_streams and rollout_k <= self.max_rollout_k
        g = Graph()
        main = self.s_actor
        torch.cuda.synchronize()
        split = concurrent and learner_sms > 0
        if split:
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            assert 0 < learner_sms < sms
            self.actor.set_grid_limit(rollout=sms - learner_sms)
            self.learner.set_grid_limit(learner=learner_sms)
        try:
            self._capture_body(g, main, rollout_k, td_steps, concurrent)
        finally:
            if split:
                self.actor.set_grid_limit()
                self.learner.set_grid_limit()
        return g

    def _capture_body(self, g, main, rollout_k, td_steps, concurrent):
        with g.capture(main):
            if concurrent:
                fork = torch.cuda.Event()
                fork.record(main)
                self.s_learner.wait_event(fork)
            self._actor_chunk(rollout_k, main)
            if not concurrent:
                after = torch.cuda.Event()
                after.record(main)
                self.s_learner.wait_event(after)
            for _ in range(td_steps):
                self.learner.train_step(self.replay, self.batch, gamma=self.gamma, lr=self.lr,
                                        target_every=self.target_every, seed=self.seed, loss=self.loss,
                                        stream=self.s_learner)
            # the upload at the end of the iteration (every td_steps updates)
            join = torch.cuda.Event()
            join.record(self.s_learner)
            main.wait_event(join)
            self.actor.copy_from(self.learner, stream=main)
