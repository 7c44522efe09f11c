"""Plain NumPy FP64 oracle of the learned warm start (a small MLP).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path never
does.  It shares no code with the CUDA path.

What it computes (the paper's solver is started from the free stream; the
learned start is an extension whose only judge is the solver's residual):

* Wall distance d of a point: distance to the closed wall polygon (wall
  points in caller index order, the polygon also used for Cl and Cd).
* Input map (a reading; the paper has no learned part): the position is
  compactified into the unit disc, zeta = (x - 0.5, y) / (1 + r) with
  r = |(x - 0.5, y)|, and the wall distance into [0, 1), delta = d / (1 + d);
  z = (zeta_x, zeta_y, delta).  Fourier features of z with a fixed matrix
  B in R^{16x3} (entries N(0, 1), seeded): [sin 2 pi B z, cos 2 pi B z], then
  the free stream (M, AoA / 10 deg): 34 inputs, zero-padded to 48.
* Network: 34 -> 128 -> 128 -> 128 -> 128 -> 4, GELU (the erf form,
  z Phi(z)) after each hidden layer, none after the last.
* Outputs o -> primitive state: rho = exp(o_0), u = u_inf + o_1,
  v = v_inf + o_2, p = p_inf exp(o_3) (positive by construction); the
  training target of a sample is (log rho, u - u_inf, v - v_inf,
  log(p / p_inf)), the loss the mean of the squared errors over samples and
  the four outputs.
* Adam (Kingma and Ba, 2015) with bias correction.

Precision: with ``bf16=True`` the functions round to bfloat16 (round to
nearest even) at exactly the places the tensor-core kernels do (inputs,
weights, activations and back-propagated gradients entering a matrix
product), and do everything else in FP64; with ``bf16=False`` they are plain
FP64 (used by the finite-difference pins).
"""
from __future__ import annotations

import math

import numpy as np

N_FREQ = 16
N_IN = 2 * N_FREQ + 2      # 34
N_IN_PAD = 48              # K of the first product (a multiple of 16)
WIDTH = 128
N_OUT = 4
LAYERS = [(N_IN, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, N_OUT)]
GAMMA = 1.4


def bf16(a):
    """Round FP64/FP32 values to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def wall_distance(x, y, flag):
    """Distance of every point to the wall polygon (segments between
    consecutive wall points in index order, closed), by brute force."""
    w = np.flatnonzero(flag == 1)
    ax, ay = x[w], y[w]
    bx, by = np.roll(ax, -1), np.roll(ay, -1)
    d = np.full(x.shape[0], np.inf)
    for s in range(w.shape[0]):
        ex, ey = bx[s] - ax[s], by[s] - ay[s]
        L2 = ex * ex + ey * ey
        t = np.clip(((x - ax[s]) * ex + (y - ay[s]) * ey) / L2, 0.0, 1.0)
        dx, dy = x - (ax[s] + t * ex), y - (ay[s] + t * ey)
        d = np.minimum(d, np.sqrt(dx * dx + dy * dy))
    return d


def compact_inputs(x, y, d):
    """z = (zeta_x, zeta_y, delta) of the input map."""
    X, Y = np.asarray(x, float) - 0.5, np.asarray(y, float)
    r = np.sqrt(X * X + Y * Y)
    return np.stack([X / (1 + r), Y / (1 + r), np.asarray(d, float) / (1 + np.asarray(d, float))], axis=1)


def features(x, y, d, mach, aoa_deg, B, bf16_round=False):
    """[n, 48] network inputs: sin and cos of 2 pi B z, M, AoA/10, zero padding."""
    z = compact_inputs(x, y, d)
    t = 2 * math.pi * (z @ np.asarray(B, float).T)
    n = z.shape[0]
    X = np.zeros((n, N_IN_PAD))
    X[:, :N_FREQ] = np.sin(t)
    X[:, N_FREQ:2 * N_FREQ] = np.cos(t)
    X[:, 2 * N_FREQ] = np.broadcast_to(mach, (n,))
    X[:, 2 * N_FREQ + 1] = np.broadcast_to(np.asarray(aoa_deg, float) / 10.0, (n,))
    return bf16(X) if bf16_round else X


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def forward(params, X, bf16_round=False):
    """params = [(W_l [out, in], b_l [out])]; X [n, 34 or 48].  Returns the
    outputs [n, 4] and the pre-activations / activations for backward."""
    r = bf16 if bf16_round else (lambda a: a)
    A = r(np.asarray(X, float)[:, :N_IN])
    acts, pre = [A], []
    for l, (W, b) in enumerate(params):
        Z = A @ r(np.asarray(W, float)).T + np.asarray(b, float)
        pre.append(Z)
        if l < len(params) - 1:
            A = r(gelu(Z))
            acts.append(A)
    return pre[-1], pre, acts


def targets(rho, u, v, p, mach, aoa_deg):
    """Training targets of samples with free stream (mach, aoa_deg)."""
    a = np.radians(aoa_deg)
    return np.stack([np.log(rho), u - mach * np.cos(a), v - mach * np.sin(a), np.log(p * GAMMA)], axis=1)


def outputs_to_primitive(o, mach, aoa_deg):
    a = np.radians(aoa_deg)
    return (np.exp(o[:, 0]), mach * np.cos(a) + o[:, 1], mach * np.sin(a) + o[:, 2], np.exp(o[:, 3]) / GAMMA)


def loss_and_grads(params, X, T, bf16_round=False):
    """Mean squared error and its gradients [(dW_l, db_l)] by back-propagation."""
    r = bf16 if bf16_round else (lambda a: a)
    o, pre, acts = forward(params, X, bf16_round)
    n = o.shape[0]
    E = o - T
    loss = float(np.mean(E * E))
    G = r(2.0 * E / (n * N_OUT))                 # dL/dZ of the last layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = r(np.asarray(params[l][0], float))
        grads[l] = (G.T @ acts[l], G.sum(axis=0))
        if l > 0:
            G = r((G @ W) * gelu_grad(pre[l - 1]))
    return loss, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (in place on params and state = {"t", "m", "v"})."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (w, g) in enumerate(((W, gW), (b, gb))):
            m = beta1 * state["m"][l][j] + (1 - beta1) * g
            v = beta2 * state["v"][l][j] + (1 - beta2) * g * g
            state["m"][l] = tuple(m if k == j else state["m"][l][k] for k in range(2))
            state["v"][l] = tuple(v if k == j else state["v"][l][k] for k in range(2))
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            new.append(w - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out
