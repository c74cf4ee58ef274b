"""Dynamic-rupture fault solve (oracle; test infrastructure).

Fault conditions, Sec. 3 Eq. (bc-dynrup): |tau| <= tau_S, tau_S V_i = tau_i |V|,
tau_S = S f(|V|, psi), dpsi/dt = g(|V|, psi), with n pointing from the minus
to the plus side, s = n.sigma.n, tau = (I - n n) sigma n, V = (I - n n)(v+ - v-).

Readings (the paper names the law - fast-velocity-weakening rate and state -
but prints neither f nor g):
  * strength S = max(0, -(sigma_n0 + sigma_n^b)): compression is negative in
    the tension-positive convention of Eq. (elasticity-pde);
  * f(V, psi) = a asinh( V/(2 V0) exp(psi/a) )  (regularised rate and state);
  * g(V, psi) = -(V/L)(psi - psi_ss(V)),  psi_ss = a ln( (2V0/V) sinh(f_ss/a) ),
    f_ss = f_w + (f_LV - f_w)/(1 + (V/V_w)^8)^(1/8),  f_LV = f0 - (b-a) ln(V/V0);
  * Godunov states: the normal part is the welded P middle state (the same
    alpha_1 as Eq. boundary-state); the locked shear traction is
    theta = eta_s [(u+ - u-) + tau+/Z_s+ + tau-/Z_s-], eta_s = Z_s- Z_s+/(Z_s- + Z_s+);
    the fault traction is tau0 + theta - eta_s V with V parallel to tau0 + theta
    (Sec. 3, second condition), so |V| solves
        Theta - eta_s |V| = S f(|V|, psi),  Theta = |tau0 + theta|;
    side states: u_b = u- + (tau - tau-)/Z_s-,  u_c = u+ - (tau - tau+)/Z_s+;
  * time: N+1 Gauss-Legendre points per step; between points psi relaxes
    exactly for frozen V; two passes of [psi update, Newton on |V|], the first
    with the previous slip rate, the second with the mid-point of the previous
    and the first pass's slip rate (a Newton start guess never enters the
    state update, so the answer does not depend on it); Newton is safeguarded by the bracket
    [0, Theta/eta_s] in x = ln V, tolerance |dx| <= tol;
  * the fault sits at the equispaced face nodes of the minus element's face;
    the flux there is interpolated (Lagrange on those nodes) and integrated
    against the basis; minus = the lower user tet index of the pair.

Linear slip weakening (Sec. 5, the Scenario-A fault; law of Andrews 1976),
the same Eq. (bc-dynrup) with the state psi = slip path length:
  * f(psi) = mu_s - (mu_s - mu_d) min(psi / D_c, 1),  dpsi/dt = |V|;
  * strength tau_S = C + f(psi) S (cohesion C >= 0, S as above);
  * |V| = max(0, Theta - tau_S) / eta_s: the locked traction if it is below the
    strength, else the strength with the slip rate that the Godunov states
    give (Theta - eta_s |V| = tau_S);
  * time: the same points and two passes as above, the state advancing exactly
    for a frozen slip rate, psi + |V| h.
"""

import numpy as np
from numpy.polynomial.legendre import leggauss

# parameter slots per fault node (rate and state; linear slip weakening uses
# the first four for its own parameters, slots 4..6 unused)
PARAMS = ("a", "b", "L", "f0", "V0", "fw", "Vw", "sn0", "t0x", "t0y", "t0z", "psi", "V")
LSW_PARAMS = ("mu_s", "mu_d", "Dc", "C", "u4", "u5", "u6", "sn0", "t0x", "t0y", "t0z", "psi", "V")
NPAR = len(PARAMS)


def f_ss(V, p):
    fLV = p["f0"] - (p["b"] - p["a"]) * np.log(V / p["V0"])
    return p["fw"] + (fLV - p["fw"]) / (1.0 + (V / p["Vw"]) ** 8) ** 0.125


def log_sinh(x):
    """log(sinh x) for x > 0 without overflow."""
    return x + np.log1p(-np.exp(-2.0 * x)) - np.log(2.0)


def psi_ss(V, p):
    a = p["a"]
    return a * (np.log(2.0 * p["V0"] / V) + log_sinh(f_ss(V, p) / a))


def friction(V, psi, p):
    a = p["a"]
    return a * np.arcsinh(V / (2.0 * p["V0"]) * np.exp(psi / a))


def psi_relax(psi, V, h, p):
    """Exact solution of dpsi/dt = -(V/L)(psi - psi_ss(V)) over h for frozen V
    (V is floored at 1e-300: for V -> 0 the state does not change)."""
    V = np.maximum(V, 1e-300)
    ss = psi_ss(V, p)
    return ss + (psi - ss) * np.exp(-V * h / p["L"])


X_FLOOR = -700.0  # ln of the smallest slip rate represented (e^-700 ~ 1e-304 m/s)


def newton_slip_rate(Theta, S, eta, psi, p, V_start, tol=1e-10, max_iter=100):
    """Solve Theta - eta V - S a asinh(c V) = 0, c = exp(psi/a)/(2 V0), for V >= 0
    (element-wise) by Newton on x = ln V.  In x the function is decreasing and
    concave, so from the right of the root Newton decreases monotonically and
    from the left one step lands on the right; every iterate is clamped to
    [X_FLOOR, ln(Theta/eta)], where g changes sign.  Converged when
    |dx| <= tol (a relative change of V below tol).  Theta = 0 gives V = 0,
    S = 0 gives V = Theta/eta.  Returns (V, iterations, converged)."""
    a = p["a"]
    lc = psi / a - np.log(2.0 * p["V0"])  # ln c
    pos = Theta > 0
    Th = np.where(pos, Theta, 1.0)
    lo = np.full(Theta.shape, X_FLOOR)
    hi = np.log(Th / eta)
    x = np.clip(np.log(np.maximum(V_start, 1e-300)), lo, hi)
    it = np.zeros(Theta.shape, np.int64)
    done = ~pos | (S == 0)
    for _ in range(max_iter):
        if np.all(done):
            break
        V = np.exp(x)
        cv = np.exp(lc + x)
        g = Th - eta * V - S * a * np.arcsinh(cv)
        dg = -eta * V - S * a * cv / np.sqrt(1.0 + cv * cv)
        xn = np.clip(x - g / dg, lo, hi)
        step = np.abs(xn - x)
        it = np.where(done, it, it + 1)
        x = np.where(done, x, xn)
        done |= step <= tol
    V = np.where(pos, np.where(S == 0, Th / eta, np.exp(x)), 0.0)
    return V, it, done


def bisect_slip_rate(Theta, S, eta, psi, p, n=200):
    """Brute-force bisection of the same equation (for pins)."""
    a = p["a"]
    c = np.exp(psi / a) / (2.0 * p["V0"])
    lo = np.zeros_like(Theta)
    hi = Theta / eta
    for _ in range(n):
        m = 0.5 * (lo + hi)
        g = Theta - eta * m - S * a * np.arcsinh(c * m)
        lo = np.where(g > 0, m, lo)
        hi = np.where(g > 0, hi, m)
    return 0.5 * (lo + hi)


def fault_states(n, qm, qp, matm, matp, tau0, sn0):
    """Locked quantities at fault points: returns dict with welded normal
    state (sn_b, vn_b), shear tractions/velocities of both sides, theta,
    eta_s and the strength-free pieces.  All vectors are global 3-vectors."""
    rhom, lamm, mum = matm
    rhop, lamp, mup = matp
    Zpm, Zpp = np.sqrt(rhom * (lamm + 2 * mum)), np.sqrt(rhop * (lamp + 2 * mup))
    Zsm, Zsp = np.sqrt(rhom * mum), np.sqrt(rhop * mup)

    def traction(q):
        s = q[..., :6]
        sx = np.stack([s[..., 0], s[..., 3], s[..., 5]], -1)
        sy = np.stack([s[..., 3], s[..., 1], s[..., 4]], -1)
        sz = np.stack([s[..., 5], s[..., 4], s[..., 2]], -1)
        return sx * n[..., 0:1] + sy * n[..., 1:2] + sz * n[..., 2:3]

    Tm, Tp = traction(qm), traction(qp)
    vm, vp = qm[..., 6:9], qp[..., 6:9]
    snm = np.sum(Tm * n, -1)
    snp = np.sum(Tp * n, -1)
    vnm = np.sum(vm * n, -1)
    vnp = np.sum(vp * n, -1)
    taum = Tm - snm[..., None] * n
    taup = Tp - snp[..., None] * n
    um = vm - vnm[..., None] * n
    up = vp - vnp[..., None] * n
    a1 = Zpm * Zpp / (Zpm + Zpp) * ((snm - snp) / Zpp + vnm - vnp)
    sn_b = snm - a1
    vn_b = vnm - a1 / Zpm
    eta = Zsm * Zsp / (Zsm + Zsp)
    theta = eta[..., None] * ((up - um) + taup / Zsp[..., None] + taum / Zsm[..., None])
    t0s = tau0 - np.sum(tau0 * n, -1)[..., None] * n
    Thv = t0s + theta
    return dict(sn_b=sn_b, vn_b=vn_b, taum=taum, taup=taup, um=um, up=up, eta=eta, theta=theta,
                Thv=Thv, t0s=t0s, Zsm=Zsm, Zsp=Zsp, S=np.maximum(0.0, -(sn0 + sn_b)))


def middle_traction_velocity(st, Vmag, n):
    """Given |V|: perturbation traction and velocities of both sides (Sec. 3 reading)."""
    Th = np.linalg.norm(st["Thv"], axis=-1)
    d = np.where(Th[..., None] > 0, st["Thv"] / np.where(Th > 0, Th, 1.0)[..., None], 0.0)
    tau_tot = (Th - st["eta"] * Vmag)[..., None] * d
    tau_p = tau_tot - st["t0s"]
    ub = st["um"] + (tau_p - st["taum"]) / st["Zsm"][..., None]
    uc = st["up"] - (tau_p - st["taup"]) / st["Zsp"][..., None]
    t_b = st["sn_b"][..., None] * n + tau_p
    vb = st["vn_b"][..., None] * n + ub
    vc = st["vn_b"][..., None] * n + uc
    return t_b, vb, vc, Vmag[..., None] * d, tau_tot


def ahat_apply(n, t, v, rho, lam, mu):
    """n.(A,B,C) q for a state with traction t = sigma n and velocity v
    (only those enter): stress rows -lam (n.v) delta_ij - mu (n_j v_i + n_i v_j),
    velocity rows -t/rho (Eq. elasticity-pde)."""
    nv = np.sum(n * v, -1)
    out = np.empty(t.shape[:-1] + (9,))
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))
    for c, (i, j) in enumerate(pairs):
        out[..., c] = -(mu * (n[..., j] * v[..., i] + n[..., i] * v[..., j]))
        if i == j:
            out[..., c] -= lam * nv
    out[..., 6:9] = -t / rho[..., None]
    return out


def lsw_friction(psi, p):
    """Linear slip weakening: mu_s at psi = 0, mu_d from psi = D_c on."""
    return p["mu_s"] - (p["mu_s"] - p["mu_d"]) * np.minimum(psi / p["Dc"], 1.0)


def lsw_slip_rate(Theta, S, eta, psi, p):
    """|V| = max(0, Theta - tau_S) / eta_s with tau_S = C + f(psi) S."""
    return np.maximum(0.0, Theta - (p["C"] + lsw_friction(psi, p) * S)) / eta


def time_points(N, dt):
    x, w = leggauss(N + 1)
    return 0.5 * dt * (x + 1.0), 0.5 * dt * w


def solve_step(n, qm_t, qp_t, matm, matp, par, dt, N, guess=None, tol=1e-10, max_iter=100, law="rs"):
    """One step at all fault points.
    qm_t, qp_t: (N+1, npts, 9) states of both sides at the Gauss time points.
    par: dict of per-point parameter arrays (PARAMS, or LSW_PARAMS for
    law = "lsw"), psi and V are the state at the step start.  Returns
    (G_minus, G_plus, new psi, new |V|, slip increment (npts,3), iteration
    counts (N+1, 2, npts; zero for the closed-form law), final traction)."""
    if law not in ("rs", "lsw"):
        raise ValueError("law: 'rs' or 'lsw'")
    tj, wj = time_points(N, dt)
    psi = par["psi"].copy()
    V = par["V"].copy()
    tau0 = np.stack([par["t0x"], par["t0y"], par["t0z"]], -1)
    npts = psi.shape[0]
    Gm = np.zeros((npts, 9))
    Gp = np.zeros((npts, 9))
    slip = np.zeros((npts, 3))
    iters = np.zeros((N + 1, 2, npts), np.int64)
    tprev = 0.0
    tau_tot = np.zeros((npts, 3))
    for j in range(N + 1):
        st = fault_states(n, qm_t[j], qp_t[j], matm, matp, tau0, par["sn0"])
        Th = np.linalg.norm(st["Thv"], axis=-1)
        h = tj[j] - tprev
        Vold = V
        if law == "lsw":
            # pass 0 advances the state with the previous slip rate, pass 1
            # with the mid-point of the previous and pass-0 rates
            Vcur = V
            for ps in range(2):
                Vmid = Vold if ps == 0 else 0.5 * (Vold + Vcur)
                psi_new = psi + Vmid * h
                Vcur = lsw_slip_rate(Th, st["S"], st["eta"], psi_new, par)
            psi, V = psi_new, Vcur
            t_b, vb, vc, Vvec, tau_tot = middle_traction_velocity(st, V, n)
            Gm += wj[j] * ahat_apply(n, t_b, vb, *matm)
            Gp += wj[j] * (-ahat_apply(n, t_b, vc, *matp))
            slip += wj[j] * Vvec
            tprev = tj[j]
            continue
        # the start guess only seeds Newton; the state update of the first
        # pass uses the previous slip rate, the second the mid-point
        Vcur = V if guess is None else guess(j, Th, st, psi, V, par)
        psi_new = psi
        for ps in range(2):
            Vmid = Vold if ps == 0 else 0.5 * (Vold + Vcur)
            psi_new = psi_relax(psi, Vmid, h, par)
            Vcur, it, ok = newton_slip_rate(Th, st["S"], st["eta"], psi_new, par, Vcur, tol, max_iter)
            if ps == 0 and guess is not None and not np.all(ok):
                # fallback: rerun the failed points from the warm start
                Vw, itw, okw = newton_slip_rate(Th, st["S"], st["eta"], psi_new, par, V, tol, max_iter)
                bad = ~ok
                Vcur = np.where(bad, Vw, Vcur)
                it = np.where(bad, it + itw, it)
                ok = np.where(bad, okw, ok)
            if not np.all(ok):
                raise RuntimeError("friction Newton did not converge")
            if ps == 0 and hasattr(guess, "solved"):
                guess.solved(j, Vcur, it)
            iters[j, ps] = it
        psi, V = psi_new, Vcur
        t_b, vb, vc, Vvec, tau_tot = middle_traction_velocity(st, V, n)
        Gm += wj[j] * ahat_apply(n, t_b, vb, *matm)
        Gp += wj[j] * (-ahat_apply(n, t_b, vc, *matp))
        slip += wj[j] * Vvec
        tprev = tj[j]
    psi = psi + V * (dt - tprev) if law == "lsw" else psi_relax(psi, V, dt - tprev, par)
    return Gm, Gp, psi, V, slip, iters, tau_tot
