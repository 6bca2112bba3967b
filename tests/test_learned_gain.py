"""What the trained network gains over the network-free policy.

The ASL loop (fused eps-greedy rollouts into the device ring, double-DQN
learner with Adam, model upload every 50 steps, Eq. 2 schedule) trains on 8
seeded maps with every randomisation of the "Color" setup on; then the greedy
network and the uniformly random policy each run 400 steps of 256 envs on 8
held-out maps from the same seeds.  The trained network must earn clearly more
reward per step and collide far less.
"""

import numpy as np
import pytest
import torch

from workloads.configs import DR_RANGES, base_params
from workloads.maps import make_map

pytestmark = pytest.mark.gpu


def _evaluate(params, maps, n, qnet=None, steps=400, seed=99):
    from paper_2305_04180_gb300 import Sim

    sim = Sim(dict(params, seed=seed), maps, (np.arange(n) % len(maps)).astype(np.int32))
    sim.reset()
    rew = torch.empty((steps, n), device="cuda")
    done = torch.empty((steps, n), dtype=torch.uint8, device="cuda")
    if qnet is None:
        sim.rollout(steps, rew_seq=rew, done_seq=done)
    else:
        sim.rollout(steps, policy="eps_q", qnet=qnet, eps=torch.zeros(n, device="cuda"), rew_seq=rew,
                    done_seq=done)
    torch.cuda.synchronize()
    d = done.cpu().numpy()
    return dict(mean_rew=float(rew.mean().item()), collide=int(((d & 1) != 0).sum()),
                arrive=int(((d & 2) != 0).sum()))


def test_trained_network_beats_network_free_policy():
    from paper_2305_04180_gb300 import Sim
    from paper_2305_04180_gb300.trainer import ColorTrainer

    p = base_params(**DR_RANGES)
    train_maps = [make_map(s) for s in range(1, 9)]
    test_maps = [make_map(s) for s in range(101, 109)]
    n = 256
    sim = Sim(p, train_maps, (np.arange(n) % 8).astype(np.int32))
    sim.reset()
    tr = ColorTrainer(sim, batch=256, slots=64, lr=5e-4, tps=8, learn_start=5000, target_every=200,
                      upload_every=50, seed=1)
    tr.run(1500, rollout_k=8)
    assert tr.updates > 10000
    rnd = _evaluate(p, test_maps, n)
    trained = _evaluate(p, test_maps, n, qnet=tr.learner)
    print(f"held-out maps, 256 envs x 400 steps: random {rnd}, trained {trained}")
    assert trained["mean_rew"] >= rnd["mean_rew"] + 0.2
    assert trained["collide"] <= 0.6 * rnd["collide"]
    assert trained["arrive"] >= rnd["arrive"]
