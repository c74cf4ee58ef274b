"""Friction-guess network: plain numpy forward and backward (oracle; test
infrastructure).  Used to check the library's GPU training kernels.

Parameter vector (same layout as the library): W1[H][IN], b1[H], W2[H][H],
b2[H], w3[H], b3, mu[IN], sd[IN], shift, scale; IN = 6, H = 32.
x = (f - mu)/sd, h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3.h2 + b3;
a sample row is [f_0..f_5, z]; loss = mean((y - (z - shift)/scale)^2).
Features of a friction solve (Theta, S, eta_s, psi, a, V0, previous V):
  r = min(Theta/(S a), 700), lc = psi/a - ln(2 V0), xhi = ln(Theta/eta_s),
  xprev = clip(ln V_prev, -700, xhi), ln(eta_s/(S a)) clipped to [-50, 50],
  x_a = clip(r - lc - ln 2, -700, xhi)  (large-argument asymptote of asinh);
the guess is x_a + shift + scale*y.
"""

import numpy as np

IN, H = 6, 32
N_TRAIN = IN * H + H + H * H + H + H + 1
N_PARAM = N_TRAIN + 2 * IN + 2


def unpack(P):
    P = np.asarray(P, np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)),
                        ("b3", (1,)), ("mu", (IN,)), ("sd", (IN,)), ("osc", (2,))):
        size = int(np.prod(shape))
        out[name] = P[o:o + size].reshape(shape)
        o += size
    return out


def forward(P, f):
    p = unpack(P)
    x = (f - p["mu"]) / p["sd"]
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    return h2 @ p["w3"] + p["b3"][0], (x, h1, h2)


def loss_and_grad(P, rows):
    """Mean squared loss and its gradient with respect to the trainable part."""
    p = unpack(P)
    f, z = rows[:, :IN].astype(np.float64), rows[:, IN].astype(np.float64)
    y, (x, h1, h2) = forward(P, f)
    t = (z - p["osc"][0]) / p["osc"][1]
    r = y - t
    n = rows.shape[0]
    loss = np.mean(r * r)
    dy = 2.0 * r / n
    gw3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    da2 = (dy[:, None] * p["w3"][None, :]) * (1.0 - h2 * h2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(0)
    da1 = (da2 @ p["W2"]) * (1.0 - h1 * h1)
    gW1 = da1.T @ x
    gb1 = da1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, gb3])
    return loss, grad


def features(Th, S, eta, psi, a, V0, Vprev):
    lc = psi / a - np.log(2.0 * V0)
    xhi = np.log(Th / eta)
    r = np.minimum(Th / (S * a), 700.0)
    xa = np.clip(r - lc - np.log(2.0), -700.0, xhi)
    xprev = np.clip(np.log(np.maximum(Vprev, 1e-300)), -700.0, xhi)
    le = np.clip(np.log(eta / (S * a)), -50.0, 50.0)
    return np.stack([r, lc, xhi, xprev, le, xa], -1), xa


def guess(P, Th, S, eta, psi, a, V0, Vprev):
    f, xa = features(Th, S, eta, psi, a, V0, Vprev)
    p = unpack(P)
    y, _ = forward(P, f.astype(np.float32).astype(np.float64))
    return np.clip(xa + p["osc"][0] + p["osc"][1] * y, -700.0, np.log(Th / eta))
