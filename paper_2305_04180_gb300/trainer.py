"""Actor-learner loop of the paper's ASL framework (Sec. 3.1, Alg. 1-2) over
the library's fused rollout and TD learner.

Host-side orchestration only: every step of the simulation, inference and
learning runs in the CUDA library.  The actor rolls the vectorized envs out
with its own copy of the network (VEM eps-greedy, transitions into the device
ring); the learner samples mini-batches and optimises its network; every
`upload_every` optimisation steps the actor takes the learner's weights
(Alg. 2 step 3, Alg. 1 step 1).  The number of optimisation steps per
vectorized step follows Eq. 2: B_step / V_step = N * TPS / B.
"""

from __future__ import annotations

import torch

from .graph import Graph
from .qnet import QNet, Replay


class ColorTrainer:
    def __init__(self, sim, *, batch=256, slots=128, gamma=0.98, lr=1e-4, target_every=200, upload_every=50,
                 tps=256, learn_start=30000, eps=None, seed=0, two_streams=False, max_rollout_k=8):
        self.sim = sim
        n = sim.n
        self.batch, self.gamma, self.lr = batch, gamma, lr
        self.target_every, self.upload_every, self.tps = target_every, upload_every, tps
        self.learn_start, self.seed = learn_start, seed
        self.learner = QNet(sim.obs_dim, batch, seed=seed)
        self.actor = QNet(sim.obs_dim, batch, seed=seed)
        self.actor.copy_from(self.learner)
        # concurrent rollouts of up to max_rollout_k steps must not be sampled
        self.max_rollout_k = max_rollout_k
        self.replay = Replay(slots, n, sim.obs_dim, reserve=max_rollout_k if two_streams else 0)
        self.eps = eps if eps is not None else torch.linspace(0.01, 0.81, n, device="cuda")
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

    def run(self, vec_steps: int, rollout_k: int = 8):
        """Collect vec_steps vectorized steps in chunks of rollout_k, training
        in between once learn_start transitions are in the ring."""
        assert rollout_k <= self.max_rollout_k
        done = 0
        while done < vec_steps:
            k = min(rollout_k, vec_steps - done)
            with torch.cuda.stream(self.s_actor):
                self.sim.rollout(k, policy="eps_q", qnet=self.actor, eps=self.eps, replay=self.replay,
                                 stream=self.s_actor)
                ev = torch.cuda.Event()
                ev.record(self.s_actor)
            done += k
            self.transitions += k * self.sim.n
            if self.transitions < self.learn_start:
                continue
            self.s_learner.wait_event(ev)
            self._carry += k * self.steps_per_vec_step()
            n_upd = int(self._carry)
            self._carry -= n_upd
            for _ in range(n_upd):
                self.learner.train_step(self.replay, self.batch, gamma=self.gamma, lr=self.lr,
                                        target_every=self.target_every, seed=self.seed, loss=self.loss,
                                        stream=self.s_learner)
                self.updates += 1
                if self.updates % self.upload_every == 0:
                    up = torch.cuda.Event()
                    up.record(self.s_learner)
                    self.s_actor.wait_event(up)
                    self.actor.copy_from(self.learner, stream=self.s_actor)
                    back = torch.cuda.Event()
                    back.record(self.s_actor)
                    self.s_learner.wait_event(back)
        torch.cuda.synchronize()
        return self

    def capture_iteration(self, rollout_k: int, td_steps: int, concurrent: bool = True):
        """One actor-learner iteration as a CUDA graph: the actor's fused
        rollout of rollout_k steps and td_steps learner steps, then the model
        upload.  concurrent=True forks the two as branches of the graph that
        overlap on the GPU (the ring's reserve keeps the learner off the
        slots being written; which completed slots it samples then depends on
        timing); concurrent=False runs the learner after the rollout and is
        deterministic.  Requires two_streams=True, rollout_k <= max_rollout_k."""
        assert self.two_streams and rollout_k <= self.max_rollout_k
        g = Graph()
        main = self.s_actor
        torch.cuda.synchronize()
        with g.capture(main):
            if concurrent:
                fork = torch.cuda.Event()
                fork.record(main)
                self.s_learner.wait_event(fork)
            self.sim.rollout(rollout_k, policy="eps_q", qnet=self.actor, eps=self.eps, replay=self.replay,
                             stream=main)
            if not concurrent:
                after = torch.cuda.Event()
                after.record(main)
                self.s_learner.wait_event(after)
            for _ in range(td_steps):
                self.learner.train_step(self.replay, self.batch, gamma=self.gamma, lr=self.lr,
                                        target_every=self.target_every, seed=self.seed, loss=self.loss,
                                        stream=self.s_learner)
            join = torch.cuda.Event()
            join.record(self.s_learner)
            main.wait_event(join)
            self.actor.copy_from(self.learner, stream=main)
        return g
