"""Friction-guess network: plain numpy forward, backward, training and the
learned Newton start (oracle; test infrastructure).  Used to check the
library's GPU training kernels and its learned start.  The paper has no
learned part; the network proposes the start of the slip-rate Newton solve of
the rate-and-state friction law (Sec. 3) and never changes its answer.

Parameter vector (same layout as the library): W1[H][IN], b1[H], W2[H][H],
b2[H], w3[H], b3, mu[IN], sd[IN], shift, scale; IN = 6, H = 32.
x = (f - mu)/sd, h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3.h2 + b3;
a sample row is [f_0..f_5, z]; loss = mean((y - (z - shift)/scale)^2).
Features of a friction solve (Theta, S, eta_s, psi, a, V0, previous V):
  r = min(Theta/(S a), 700), lc = psi/a - ln(2 V0), xhi = ln(Theta/eta_s),
  xprev = clip(ln V_prev, -700, xhi), ln(eta_s/(S a)) clipped to [-50, 50],
  x_a = clip(r - lc - ln 2, -700, xhi)  (large-argument asymptote of asinh).
Target z = ln V* - x_a with V* the first-pass solution, so the prediction of
ln V* is xhat = x_a + shift + scale*y.
Start of the first-pass Newton at Gauss time point j of a step: the warm
start xprev at j = 0 (or when the previous point was no solve), else
xprev + (xhat_j - xhat_{j-1}): the warm start moved by the change the network
predicts, which is exact where nothing changes.  If Newton from that start
fails, it is rerun from the warm start.
"""

import numpy as np

IN, H = 6, 32
N_TRAIN = IN * H + H + H * H + H + H + 1
N_PARAM = N_TRAIN + 2 * IN + 2
X_FLOOR = -700.0


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


def train(rows, epochs=300, batch=512, lr=3e-3, seed=0):
    """Normalisation from the data (mean, standard deviation of every column),
    Gaussian initialisation scaled by 1/sqrt(fan-in), zero biases, then Adam
    (beta1 0.9, beta2 0.999, eps 1e-8) over mini-batches in row order.
    Returns (P, loss before, loss after)."""
    rows = np.asarray(rows, np.float64)
    rng = np.random.default_rng(seed)
    P = np.zeros(N_PARAM)
    m, s = rows.mean(0), rows.std(0)
    s = np.where(s > 1e-6, s, 1.0)
    P[N_TRAIN:N_TRAIN + IN] = m[:IN]
    P[N_TRAIN + IN:N_TRAIN + 2 * IN] = s[:IN]
    P[N_TRAIN + 2 * IN:] = m[IN], s[IN]
    o = 0
    for fan_in, fan_out in ((IN, H), (H, H), (H, 1)):
        P[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) / np.sqrt(fan_in)
        o += fan_in * fan_out + fan_out
    m1 = np.zeros(N_TRAIN)
    m2 = np.zeros(N_TRAIN)
    loss0 = loss_and_grad(P, rows)[0]
    step = 0
    for _ in range(epochs):
        for r0 in range(0, rows.shape[0], batch):
            _, g = loss_and_grad(P, rows[r0:r0 + batch])
            step += 1
            m1 = 0.9 * m1 + 0.1 * g
            m2 = 0.999 * m2 + 0.001 * g * g
            P[:N_TRAIN] -= lr * (m1 / (1 - 0.9 ** step)) / (np.sqrt(m2 / (1 - 0.999 ** step)) + 1e-8)
    return P, loss0, loss_and_grad(P, rows)[0]


def features(Th, S, eta, psi, a, V0, Vprev):
    lc = psi / a - np.log(2.0 * V0)
    xhi = np.log(Th / eta)
    r = np.minimum(Th / (S * a), 700.0)
    xa = np.clip(r - lc - np.log(2.0), X_FLOOR, xhi)
    xprev = np.clip(np.log(np.maximum(Vprev, 1e-300)), X_FLOOR, xhi)
    le = np.clip(np.log(eta / (S * a)), -50.0, 50.0)
    return np.stack([r, lc, xhi, xprev, le, xa], -1), xa


def predict(P, f):
    """Predicted ln V* = x_a + shift + scale*y (network in FP32 inputs, as the
    library evaluates it)."""
    p = unpack(P)
    y, _ = forward(P, f.astype(np.float32).astype(np.float64))
    return f[..., 5] + p["osc"][0] + p["osc"][1] * y


class LearnedStart:
    """Start guess for the first-pass Newton of the friction solve (the
    `guess` argument of the oracle's rupture step).  With P None it returns
    the plain warm start; with capture=True it records [features, ln V* - x_a]
    rows of the first-pass solves (via `solved`).

    Rule (the learned part is not in the paper): at time point j the network
    is evaluated only at points whose first-pass Newton at point j - 1 needed
    more than one iteration (the state is changing there; where the warm
    start already converges, the network cannot help).  Where it was also
    evaluated at j - 1, the start is the warm start moved by the change of the
    predicted ln V*; everywhere else it is the warm start."""

    def __init__(self, P=None, capture=False):
        self.P = P
        self.capture = capture
        self.rows = []
        self.prev = None
        self.busy = None

    def __call__(self, j, Th, st, psi, V, par):
        S, eta = st["S"], st["eta"]
        solve = (Th > 0) & (S > 0)
        Ths = np.where(solve, Th, 1.0)
        Ss = np.where(solve, S, 1.0)
        f, xa = features(Ths, Ss, eta, psi, par["a"], par["V0"], V)
        self._f, self._xa, self._solve = f, xa, solve
        if self.P is None:
            return V
        if j == 0 or self.prev is None:
            self.prev = np.full(solve.shape, np.nan)
            self.busy = np.zeros(solve.shape, bool)
        ev = solve & self.busy
        xhat = np.where(ev, predict(self.P, f), np.nan)
        xw = f[..., 3]
        use = ev & np.isfinite(self.prev)
        x0 = np.where(use, xw + (xhat - np.where(use, self.prev, 0.0)), xw)
        self.prev = xhat
        return np.where(solve, np.exp(np.clip(x0, X_FLOOR, f[..., 2])), V)

    def solved(self, j, V, iters=None):
        if iters is not None:
            self.busy = self._solve & (np.asarray(iters) > 1)
        if self.capture:
            s = self._solve
            z = np.log(np.maximum(V[s], 1e-300)) - self._xa[s]
            self.rows.append(np.concatenate([self._f[s], z[:, None]], 1))
