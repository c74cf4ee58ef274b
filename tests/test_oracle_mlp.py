"""Pins for the oracle's friction-guess network (forward/backward by hand)."""

import numpy as np

from oracle import mlp


def _params(rng):
    P = rng.standard_normal(mlp.N_PARAM) * 0.3
    p0 = mlp.N_TRAIN
    P[p0:p0 + mlp.IN] = rng.standard_normal(mlp.IN)             # mu
    P[p0 + mlp.IN:p0 + 2 * mlp.IN] = rng.uniform(0.5, 2.0, mlp.IN)  # sd
    P[-2:] = [0.3, 1.7]
    return P


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    P = _params(rng)
    rows = rng.standard_normal((64, mlp.IN + 1))
    loss, g = mlp.loss_and_grad(P, rows)
    assert g.shape == (mlp.N_TRAIN,)
    h = 1e-6
    idx = rng.choice(mlp.N_TRAIN, 60, replace=False)
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.loss_and_grad(Pp, rows)[0] - mlp.loss_and_grad(Pm, rows)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_asymptotic_base_guess_solves_the_large_argument_limit():
    # for c V >> 1 and eta V << Theta: Theta = S a ln(2 c V) exactly gives x_a
    a, V0, psi = 0.01, 1e-6, 0.6
    S, eta, x_true = 40e6, 1e-3, np.log(0.3)
    lc = psi / a - np.log(2 * V0)
    Th = S * a * (np.log(2.0) + lc + x_true)
    _, xa = mlp.features(np.array([Th]), np.array([S]), np.array([eta]), np.array([psi]), a, V0, np.array([1e-12]))
    assert abs(xa[0] - x_true) < 1e-9
