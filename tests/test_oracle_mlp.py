"""Pins of the warm-start MLP oracle (oracle/mlp.py), CPU only.

Each pin ties the oracle to something other than itself: library routines
(torch's bfloat16 conversion, autograd and Adam in float64), closed forms
(GELU's odd part, the Fourier identity, polygon distances) and central
finite differences."""
import math

import numpy as np
import pytest

from oracle import mlp as M

torch = pytest.importorskip("torch")


def _params(rng, scale=1.0):
    out = []
    for fin, fout in M.LAYERS:
        k = 1.0 / math.sqrt(fin)
        out.append((rng.uniform(-k, k, (fout, fin)) * scale, rng.uniform(-k, k, fout)))
    return out


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 3, 5000), rng.uniform(-1e-3, 1e-3, 500),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -9, 0.0, 65504.0, 3e38]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)
    assert M.bf16(1 + 2 ** -8) == 1.0 and M.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6  # ties to even


def test_gelu_closed_forms_and_derivative():
    z = np.linspace(-6, 6, 241)
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, rtol=0, atol=1e-15)   # z Phi(z) + z Phi(-z) = z
    assert M.gelu(np.array([0.0]))[0] == 0.0 and M.gelu_grad(np.array([0.0]))[0] == 0.5
    h = 1e-5
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-9
    ref = torch.nn.functional.gelu(torch.tensor(z), approximate="none").numpy()
    assert np.max(np.abs(ref - M.gelu(z))) < 1e-15


def test_features_identities():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(-20, 21, 400), rng.uniform(-20, 20, 400)
    d = rng.uniform(0, 20, 400)
    B = rng.normal(0, 1, (M.N_FREQ, 3))
    X = M.features(x, y, d, 0.7, 3.0, B)
    assert X.shape == (400, M.N_IN_PAD)
    s, c = X[:, :M.N_FREQ], X[:, M.N_FREQ:2 * M.N_FREQ]
    assert np.allclose(s * s + c * c, 1.0, atol=1e-14)
    assert np.all(X[:, 2 * M.N_FREQ] == 0.7) and np.all(X[:, 2 * M.N_FREQ + 1] == 0.3)
    assert np.all(X[:, M.N_IN:] == 0.0)
    z = M.compact_inputs(x, y, d)
    assert np.all(np.hypot(z[:, 0], z[:, 1]) < 1.0) and np.all((z[:, 2] >= 0) & (z[:, 2] < 1))


def test_wall_distance_on_a_regular_polygon():
    n, R = 64, 1.0
    th = 2 * np.pi * np.arange(n) / n
    wx, wy = R * np.cos(th), R * np.sin(th)
    # probes on the rays through edge midpoints at radius r: distance r - R cos(pi/n)
    r = np.array([1.5, 3.0, 10.0])
    pm = th[5] + np.pi / n
    px, py = r * np.cos(pm), r * np.sin(pm)
    x = np.concatenate([wx, px])
    y = np.concatenate([wy, py])
    flag = np.concatenate([np.ones(n, np.uint8), np.zeros(3, np.uint8)])
    d = M.wall_distance(x, y, flag)
    assert np.max(np.abs(d[:n])) < 1e-15
    assert np.allclose(d[n:], r - R * np.cos(np.pi / n), rtol=0, atol=1e-13)


def test_output_map_round_trip():
    rng = np.random.default_rng(3)
    o = rng.normal(0, 0.3, (50, 4))
    rho, u, v, p = M.outputs_to_primitive(o, 0.6, -2.0)
    assert np.allclose(M.targets(rho, u, v, p, 0.6, -2.0), o, atol=1e-14)


def _torch_model(params):
    layers = []
    for l, (W, b) in enumerate(params):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.tensor(W))
            lin.bias.copy_(torch.tensor(b))
        layers.append(lin)
        if l < len(params) - 1:
            layers.append(torch.nn.GELU(approximate="none"))
    return torch.nn.Sequential(*layers)


def test_forward_and_gradients_match_torch_autograd():
    rng = np.random.default_rng(4)
    P = _params(rng)
    X = rng.normal(0, 1, (300, M.N_IN_PAD))
    T = rng.normal(0, 0.2, (300, 4))
    loss, grads = M.loss_and_grads(P, X, T)
    net = _torch_model(P)
    o = net(torch.tensor(X[:, :M.N_IN]))
    tl = torch.mean((o - torch.tensor(T)) ** 2)
    tl.backward()
    assert abs(loss - tl.item()) < 1e-14 * max(1.0, loss)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (gW, gb), lin in zip(grads, lins):
        assert np.max(np.abs(gW - lin.weight.grad.numpy())) <= 1e-13 * np.max(np.abs(gW))
        assert np.max(np.abs(gb - lin.bias.grad.numpy())) <= 1e-13 * np.max(np.abs(gb))


def test_gradients_against_central_differences():
    rng = np.random.default_rng(5)
    P = _params(rng)
    X = rng.normal(0, 1, (40, M.N_IN_PAD))
    T = rng.normal(0, 0.2, (40, 4))
    _, grads = M.loss_and_grads(P, X, T)
    h = 1e-6
    for l in (0, 2, 4):
        for (i, j) in ((0, 0), (3, 1), (min(5, P[l][0].shape[0] - 1), 7)):
            Pp = [(W.copy(), b.copy()) for W, b in P]
            Pm = [(W.copy(), b.copy()) for W, b in P]
            Pp[l][0][i, j] += h
            Pm[l][0][i, j] -= h
            fd = (M.loss_and_grads(Pp, X, T)[0] - M.loss_and_grads(Pm, X, T)[0]) / (2 * h)
            assert abs(fd - grads[l][0][i, j]) <= 1e-7 * max(1e-3, abs(fd))


def test_adam_matches_torch():
    rng = np.random.default_rng(6)
    P = _params(rng)
    X = rng.normal(0, 1, (64, M.N_IN_PAD))
    T = rng.normal(0, 0.2, (64, 4))
    net = _torch_model(P)
    opt = torch.optim.Adam(net.parameters(), lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    for _ in range(3):
        _, grads = M.loss_and_grads(P, X, T)
        P = M.adam_step(P, grads, state, 3e-3)
        opt.zero_grad()
        torch.mean((net(torch.tensor(X[:, :M.N_IN])) - torch.tensor(T)) ** 2).backward()
        opt.step()
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (W, b), lin in zip(P, lins):
        assert np.max(np.abs(W - lin.weight.detach().numpy())) < 1e-12
        assert np.max(np.abs(b - lin.bias.detach().numpy())) < 1e-12


def test_first_adam_step_is_lr_times_sign():
    P = [(np.array([[2.0, -3.0]]), np.array([0.5]))]
    g = [(np.array([[0.1, -4.0]]), np.array([1e-3]))]
    Q = M.adam_step(P, g, {}, 0.01)
    assert np.allclose(Q[0][0], [[1.99, -2.99]], atol=1e-9) and np.allclose(Q[0][1], [0.49], atol=1e-6)
