"""Float64 oracle of the learned part: the Q-networks, double-DQN TD loss with
Huber, its gradient, and Adam.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU legs use it.

Passages followed:
* Sec. 3.1 / Alg. 1-2 (Actor and Learner of ASL): the actor maps the batched
  state to actions with the policy net, the learner samples a mini-batch and
  optimises with the underlying DRL algorithm, DDQN (Sec. 4.1, double
  Q-learning: the online net picks the next action, the target net values it).
* Two networks: "dueling", in -> 256 -> 256 -> (1 + 5) with
  Q = V + A - mean(A) (the dueling architecture cited in Sec. 2); "paper",
  the four fully connected layers [32, 256, 128, 5] of Sec. 4.3.2
  ("Task2Task generalization"), in -> 256 -> 128 -> 5 with Q the outputs.
  Both use ReLU between layers.
* Appendix hyperparameter table, Sparrow column: gamma 0.98, lr 1e-4, Adam,
  batch 256, target update every 200 optimisation steps.
Readings where the paper is silent: Huber loss with delta 1 on the TD error,
mean over the batch; Adam with beta = (0.9, 0.999), eps = 1e-8 (Kingma & Ba);
terminal = collided or arrived (truncation bootstraps); ties in argmax go to
the lowest index.

Parameter layout (flat, float, the order the library's qnet_set/get_params
use): W1 [h1][in], b1 [h1], W2 [h2][h1], b2 [h2], W3 [out][h2], b3 [out];
for "dueling" row 0 of W3 / b3 is the value head, rows 1..5 the advantages.
The architecture of a parameter dict follows from its shapes.
"""

from __future__ import annotations

import numpy as np

HIDDEN = 256
N_ACT = 5
N_OUT = N_ACT + 1
# hidden widths and head outputs of the two networks
ARCHS = {"dueling": (256, 256, N_ACT + 1), "paper": (256, 128, N_ACT)}


def param_shapes(n_in: int = 37, arch: str = "dueling"):
    h1, h2, out = ARCHS[arch]
    return [("W1", (h1, n_in)), ("b1", (h1,)), ("W2", (h2, h1)), ("b2", (h2,)), ("W3", (out, h2)), ("b3", (out,))]


def arch_of(p: dict) -> str:
    return "dueling" if p["W3"].shape[0] == N_ACT + 1 else "paper"


def n_params(n_in: int = 37, arch: str = "dueling") -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(n_in, arch))


def unflatten(theta, n_in: int = 37, arch: str = "dueling") -> dict:
    out, o = {}, 0
    for name, shp in param_shapes(n_in, arch):
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], np.float64).reshape(shp)
        o += k
    assert o == len(theta)
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel()
                           for name, _ in param_shapes(p["W1"].shape[1], arch_of(p))])


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32 -- the rounding a float32 -> bf16 conversion performs."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(a)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out.reshape(a.shape)


def forward(p: dict, s, bf16: bool = False, keep: bool = False):
    """Q-values [B, 5] of states s [B, in].

    bf16=False: exact float64.  bf16=True: the tensor-core recipe -- states,
    weights and hidden activations rounded to bfloat16, products summed and
    biases added in float64 (a stand-in for float32 accumulation).
    """
    s = np.asarray(s, np.float64)
    W1, b1, W2, b2, W3, b3 = (p[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    if bf16:
        r = lambda t: bf16_round(t).astype(np.float64)  # noqa: E731
        s, W1, W2, W3 = r(s), r(W1), r(W2), r(W3)
    z1 = s @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    if bf16:
        h1 = bf16_round(h1).astype(np.float64)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    if bf16:
        h2 = bf16_round(h2).astype(np.float64)
    o = h2 @ W3.T + b3
    if o.shape[1] == N_ACT:
        Q = o  # the paper's network: the outputs are the Q-values
    else:
        V = o[:, :1]
        A = o[:, 1:]
        Q = V + A - A.mean(axis=1, keepdims=True)
    if keep:
        return Q, dict(s=s, z1=z1, h1=h1, z2=z2, h2=h2, o=o)
    return Q


def argmax_lowest(Q) -> np.ndarray:
    """Greedy action: argmax over actions, the lowest index on ties."""
    return np.argmax(np.asarray(Q), axis=1)


def huber(d, delta: float = 1.0):
    d = np.asarray(d, np.float64)
    a = np.abs(d)
    return np.where(a <= delta, 0.5 * d * d, delta * (a - 0.5 * delta))


def td_targets(p_online: dict, p_target: dict, r, s2, term, gamma: float, bf16: bool = False):
    """Double-DQN target y = r + gamma (1 - term) Q_target(s2, argmax_a Q_online(s2, a))."""
    a_star = argmax_lowest(forward(p_online, s2, bf16))
    q_t = forward(p_target, s2, bf16)
    boot = q_t[np.arange(len(a_star)), a_star]
    return np.asarray(r, np.float64) + gamma * (1.0 - np.asarray(term, np.float64)) * boot


def td_loss_grad(p_online: dict, p_target: dict, batch: dict, gamma: float, bf16: bool = False):
    """Mean Huber TD loss over the batch and its gradient w.r.t. the online
    parameters (the target y is held constant).  Returns (loss, grads dict)."""
    s, a, r, s2, term = (batch[k] for k in ("s", "a", "r", "s2", "term"))
    a = np.asarray(a, np.int64)
    B = len(a)
    y = td_targets(p_online, p_target, r, s2, term, gamma, bf16)
    Q, c = forward(p_online, s, bf16, keep=True)
    q_sa = Q[np.arange(B), a]
    d = q_sa - y
    loss = huber(d).mean()
    g = np.clip(d, -1.0, 1.0) / B                  # dL/dq_sa
    dQ = np.zeros_like(Q)
    dQ[np.arange(B), a] = g
    if arch_of(p_online) == "paper":
        do = dQ  # the outputs are the Q-values
    else:
        # Q_k = V + A_k - mean(A):  dV = sum_k dQ_k,  dA_j = dQ_j - mean_k dQ_k
        do = np.concatenate([dQ.sum(axis=1, keepdims=True), dQ - dQ.mean(axis=1, keepdims=True)], axis=1)
    W2 = p_online["W2"]
    W3 = p_online["W3"]
    if bf16:
        W2 = bf16_round(W2).astype(np.float64)
        W3 = bf16_round(W3).astype(np.float64)
    grads = {}
    grads["W3"] = do.T @ c["h2"]
    grads["b3"] = do.sum(axis=0)
    dz2 = (do @ W3) * (c["z2"] > 0)
    grads["W2"] = dz2.T @ c["h1"]
    grads["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (c["z1"] > 0)
    grads["W1"] = dz1.T @ c["s"]
    grads["b1"] = dz1.sum(axis=0)
    return loss, grads


def adam_step(theta, g, m, v, t: int, lr: float = 1e-4, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1.
    Returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int, n_in: int = 37, arch: str = "dueling") -> dict:
    """A seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation (the
    library draws its own; tests set parameters explicitly)."""
    rng = np.random.default_rng(seed)
    p = {}
    shapes = param_shapes(n_in, arch)
    for i, (name, shp) in enumerate(shapes):
        fan_in = shp[1] if len(shp) == 2 else shapes[i - 1][1][1]
        bound = 1.0 / np.sqrt(fan_in)
        p[name] = rng.uniform(-bound, bound, size=shp)
    return p
