"""Pins of the float64 Q-network oracle: central finite differences of the TD
loss, the dueling identity, Huber and double-DQN closed forms on hand
batches, the Adam first step, the bf16 rounding rule, and torch autograd."""

import numpy as np
import pytest

from oracle import qnet as Q


def _batch(rng, B=12, n_in=37):
    return dict(s=rng.normal(size=(B, n_in)), a=rng.integers(0, 5, B), r=rng.normal(size=B),
                s2=rng.normal(size=(B, n_in)), term=(rng.random(B) < 0.3).astype(np.float64))


def test_param_count_and_layout():
    assert Q.n_params(37) == 37 * 256 + 256 + 256 * 256 + 256 + 6 * 256 + 6 == 77062
    p = Q.init_params(0)
    th = Q.flatten(p)
    p2 = Q.unflatten(th)
    assert all(np.array_equal(p[k], p2[k]) for k in p)


def test_dueling_identity():
    """mean_a Q(s, a) equals the value head V(s)."""
    rng = np.random.default_rng(1)
    p = Q.init_params(1)
    s = rng.normal(size=(20, 37))
    q, c = Q.forward(p, s, keep=True)
    assert np.allclose(q.mean(axis=1), c["o"][:, 0], atol=1e-12)
    assert np.allclose(q - q.mean(axis=1, keepdims=True), c["o"][:, 1:] - c["o"][:, 1:].mean(axis=1, keepdims=True))


def test_forward_against_explicit_loops():
    """Tiny network evaluated neuron by neuron."""
    rng = np.random.default_rng(2)
    p = Q.init_params(2, n_in=3)
    s = rng.normal(size=(2, 3))
    q = Q.forward(p, s)
    for b in range(2):
        h1 = [max(0.0, sum(p["W1"][j, i] * s[b, i] for i in range(3)) + p["b1"][j]) for j in range(256)]
        h2 = [max(0.0, sum(p["W2"][j, i] * h1[i] for i in range(256)) + p["b2"][j]) for j in range(256)]
        o = [sum(p["W3"][k, i] * h2[i] for i in range(256)) + p["b3"][k] for k in range(6)]
        mean_a = sum(o[1:]) / 5
        for a in range(5):
            assert abs(q[b, a] - (o[0] + o[1 + a] - mean_a)) < 1e-10


def test_paper_network_count_and_explicit_loops():
    """The [32, 256, 128, 5] network of the Task2Task experiment: parameter
    count by hand, and a tiny instance evaluated neuron by neuron (the
    outputs are the Q-values, no value/advantage split)."""
    assert Q.n_params(32, "paper") == 32 * 256 + 256 + 256 * 128 + 128 + 128 * 5 + 5 == 41989
    p = Q.init_params(7, 32, "paper")
    assert Q.arch_of(p) == "paper" and np.array_equal(Q.flatten(Q.unflatten(Q.flatten(p), 32, "paper")), Q.flatten(p))
    rng = np.random.default_rng(8)
    p = Q.init_params(8, 3, "paper")
    s = rng.normal(size=(2, 3))
    q = Q.forward(p, s)
    assert q.shape == (2, 5)
    for b in range(2):
        h1 = [max(0.0, sum(p["W1"][j, i] * s[b, i] for i in range(3)) + p["b1"][j]) for j in range(256)]
        h2 = [max(0.0, sum(p["W2"][j, i] * h1[i] for i in range(256)) + p["b2"][j]) for j in range(128)]
        for a in range(5):
            o = sum(p["W3"][a, i] * h2[i] for i in range(128)) + p["b3"][a]
            assert abs(q[b, a] - o) < 1e-10


def test_argmax_ties_go_low():
    assert list(Q.argmax_lowest(np.array([[1, 3, 3, 0, 3], [2, 2, 2, 2, 2]]))) == [1, 0]


def test_huber_closed_forms():
    assert Q.huber(0.5) == 0.125 and Q.huber(-0.5) == 0.125
    assert Q.huber(3.0) == 2.5 and Q.huber(-3.0) == 2.5
    assert Q.huber(1.0) == 0.5


def test_double_dqn_target_uses_online_argmax_and_target_value():
    """Hand batch: online net prefers action 2 at s2, target net prefers 0;
    the target takes the target net's value of action 2."""
    p_on = {k: np.zeros(v) for k, v in Q.param_shapes(1)}
    p_tg = {k: np.zeros(v) for k, v in Q.param_shapes(1)}
    # with all weights zero, Q = b3[0] + b3[1:] - mean(b3[1:])
    p_on["b3"] = np.array([0.0, 0.0, 0.0, 5.0, 0.0, 0.0])
    p_tg["b3"] = np.array([1.0, 9.0, 0.0, 2.0, 0.0, 0.0])
    qt = 1.0 + np.array([9.0, 0.0, 2.0, 0.0, 0.0]) - 11.0 / 5
    y = Q.td_targets(p_on, p_tg, r=[0.5, 0.5], s2=np.zeros((2, 1)), term=[0.0, 1.0], gamma=0.98)
    assert np.allclose(y, [0.5 + 0.98 * qt[2], 0.5])


@pytest.mark.parametrize("arch", ["dueling", "paper"])
def test_td_gradient_matches_central_finite_differences(arch):
    rng = np.random.default_rng(3)
    n_in = 6
    p = Q.init_params(3, n_in, arch)
    # larger weights so that the Huber loss sees both branches
    for k in p:
        p[k] = p[k] * 3.0
    pt = Q.init_params(4, n_in, arch)
    batch = _batch(rng, B=10, n_in=n_in)
    batch["r"] = batch["r"] * 3
    loss, g = Q.td_loss_grad(p, pt, batch, 0.98)
    y = Q.td_targets(p, pt, batch["r"], batch["s2"], batch["term"], 0.98)

    def loss_at(theta):
        pp = Q.unflatten(theta, n_in, arch)
        q = Q.forward(pp, batch["s"])
        d = q[np.arange(10), batch["a"]] - y  # target held constant
        return Q.huber(d).mean()

    th = Q.flatten(p)
    gflat = Q.flatten(g)
    h = 1e-6
    idx = rng.choice(th.size, 400, replace=False)
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (loss_at(th + e) - loss_at(th - e)) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])
    assert abs(loss_at(th) - loss) < 1e-12


@pytest.mark.parametrize("arch", ["dueling", "paper"])
def test_td_gradient_matches_torch_autograd(arch):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p = Q.init_params(5, 37, arch)
    pt = Q.init_params(6, 37, arch)
    batch = _batch(rng, B=32)
    loss, g = Q.td_loss_grad(p, pt, batch, 0.98)
    y = torch.tensor(Q.td_targets(p, pt, batch["r"], batch["s2"], batch["term"], 0.98))
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    s = torch.tensor(batch["s"])
    h1 = torch.relu(s @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    o = h2 @ tp["W3"].T + tp["b3"]
    q = o if arch == "paper" else o[:, :1] + o[:, 1:] - o[:, 1:].mean(dim=1, keepdim=True)
    qsa = q[torch.arange(32), torch.tensor(batch["a"])]
    tl = torch.nn.functional.huber_loss(qsa, y, delta=1.0)
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    for k in p:
        assert np.allclose(tp[k].grad.numpy(), g[k], atol=1e-12, rtol=1e-9), k


def test_adam_first_step_closed_form():
    """With m = v = 0 the first bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 0.0, 1e-9])
    th, m, v = Q.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=1e-4)
    assert np.allclose(th, -1e-4 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_rule():
    """float32 -> bfloat16 keeps the top 16 bits, rounding to nearest even;
    checked against torch's conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.normal(size=10000).astype(np.float32) * 10 ** rng.uniform(-5, 5, 10000),
                        np.array([1.0, 1.00390625, 1.01171875, -2.5, 65504.0, 0.0], np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(Q.bf16_round(x).view(np.uint32), ref.view(np.uint32))
    # ties: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> rounds to even (1.0)
    assert Q.bf16_round(np.float32(1.00390625)) == 1.0
