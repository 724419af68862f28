"""Pins of the FP64 learned-beam MLP oracle (no GPU): gradients against
central finite differences, feature layout and a closed-form forward pass,
the first Adam step (lr * sign(g)), and a loss that decreases under training."""
import numpy as np

from oracle import mlp


def tiny_net(seed=0, F=5, E=3, H=(7, 6), n_out=4, n_ant=4):
    g = np.random.default_rng(seed)
    dims = [2 * F + E, *H, n_out]
    W = [g.normal(0, 1 / np.sqrt(dims[i]), (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    b = [g.normal(0, 0.1, dims[i + 1]) for i in range(len(dims) - 1)]
    B = np.stack([g.integers(-3, 4, F), g.normal(0, 2, F), g.normal(0, 2, F)], 1).astype(float)
    return mlp.MLP(B=B, emb=g.normal(0, 0.5, (n_ant, E)), W=W, b=b)


def batch(n=9, seed=1, n_ant=4):
    g = np.random.default_rng(seed)
    return (g.integers(0, n_ant, n), g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi / 2, n),
            g.uniform(100e6, 200e6, n))


def test_gradients_match_central_differences():
    net = tiny_net()
    ant, az, za, nu = batch()
    t = np.random.default_rng(3).normal(size=(9, 4))
    _, g = mlp.loss_and_grads(net, ant, az, za, nu, t)
    h = 1e-6
    for name, p in net.params().items():
        num = np.zeros_like(p)
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = p[i]
            p[i] = old + h
            lp, _ = mlp.loss_and_grads(net, ant, az, za, nu, t)
            p[i] = old - h
            lm, _ = mlp.loss_and_grads(net, ant, az, za, nu, t)
            p[i] = old
            num[i] = (lp - lm) / (2 * h)
        assert np.abs(num - g[name]).max() <= 1e-6 * max(1.0, np.abs(num).max()), name


def test_feature_layout_and_closed_form_forward():
    net = tiny_net()
    F, E = net.B.shape[0], net.emb.shape[1]
    # x = 0 (az = 0, za = 0, nu = nu_mid): sin terms 0, cos terms 1, then the embedding
    f = mlp.features(net, [2], [0.0], [0.0], [net.nu_mid])[0]
    assert np.allclose(f[:F], 0) and np.allclose(f[F:2 * F], 1) and np.allclose(f[2 * F:], net.emb[2])
    # zero hidden weights: h_l = relu(b_l) regardless of input, y = W_out relu(b_L) + b_out
    for w in net.W[:-1]:
        w[:] = 0
    y = mlp.forward(net, *batch())
    want = net.W[-1] @ np.maximum(net.b[-2], 0) + net.b[-1]
    assert np.allclose(y, want[None, :], atol=1e-15)


def test_first_adam_step_is_lr_times_sign():
    net = tiny_net()
    ant, az, za, nu = batch()
    t = np.zeros((9, 4))
    _, g = mlp.loss_and_grads(net, ant, az, za, nu, t)
    before = {k: v.copy() for k, v in net.params().items()}
    mlp.adam_step(net, g, lr=1e-3, eps=1e-300)
    for k, p in net.params().items():
        step = before[k] - p
        nz = g[k] != 0
        assert np.allclose(step[nz], 1e-3 * np.sign(g[k][nz]), rtol=1e-12)


def test_training_decreases_loss():
    net = tiny_net(H=(16, 16))
    g = np.random.default_rng(4)
    ant, az, za, nu = batch(n=256, seed=5)
    t = np.stack([np.cos(za) * np.cos(az), np.sin(az), np.cos(za), 0.1 * (ant == 1)], 1)
    l0, _ = mlp.loss_and_grads(net, ant, az, za, nu, t)
    for _ in range(500):
        _, gr = mlp.loss_and_grads(net, ant, az, za, nu, t)
        mlp.adam_step(net, gr, lr=3e-3)
    l1, _ = mlp.loss_and_grads(net, ant, az, za, nu, t)
    assert l1 < 0.2 * l0
