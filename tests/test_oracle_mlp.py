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


def _fault_run(guess, steps=20):
    from oracle import rupture as ru
    from oracle.ader import Oracle
    from synthetic.workloads import fault_box, random_dofs, rs_fault_params
    m, (rho, lam, mu) = fault_box(nx=4, ny=2, nz=4, dz=1e3)
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, rho, lam, mu, 3, cfl=0.5, max_clusters=1)
    par = rs_fault_params(o.f_xyz, o.f_n, seed=1, patch_radius=2e3)
    o.set_fault({k: par[..., i] for i, k in enumerate(ru.PARAMS)})
    o.Q = random_dofs((m.nt, o.B, 9), 4, N=3) * 1e3
    o.fault_guess = guess
    for _ in range(steps):
        o.step_gts()
    return o


def test_learned_start_keeps_the_solution_and_saves_iterations():
    """Train on the first-pass solves of one run, rerun with the learned start:
    the same solution to the Newton tolerance, fewer iterations per solve."""
    cap = mlp.LearnedStart(capture=True)
    plain = _fault_run(cap)
    rows = np.concatenate(cap.rows)
    assert rows.shape[0] > 1000 and np.all(np.isfinite(rows))
    P, l0, l1 = mlp.train(rows, epochs=150)
    assert l1 < 0.1 * l0
    learned = _fault_run(mlp.LearnedStart(P))
    assert learned.newton_solves == plain.newton_solves
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(learned.Q, plain.Q) <= 1e-10
    assert rel(learned.fault["V"], plain.fault["V"]) <= 1e-10
    assert rel(learned.fault["slip"], plain.fault["slip"]) <= 1e-10
    ip, il = plain.newton_iters / plain.newton_solves, learned.newton_iters / learned.newton_solves
    assert il < 0.95 * ip, (ip, il)
