"""ADER-DG solver, FP64, numpy (oracle; test infrastructure).

Per element over a step [t0, t0 + dt] (Sec. 4.1):
  predictor  D^0 = Q,  D^{k+1} = -sum_e K_e^T D^k A*_e^T  (k < N)
             (discrete Cauchy-Kovalewski in strong form: the L2 projection of
             -sum_e A*_e dq/dxi_e; K_e[k,l] = int dphi_k/dxi_e phi_l);
  time integral  I = sum_k (tb^{k+1} - ta^{k+1})/(k+1)! D^k   (Eq. taylor);
  corrector  Q += sum_e K_e I A*_e^T
                  - 1/|J| sum_faces int_face phi (T A^- w^b(I^-, I^+)) dS
             (time-integrated Eq. semi-discrete-form; the face integral is
             a Gauss rule on the physical face: the neighbour's polynomial is
             evaluated at the same physical points through its own inverse map).
Gravitational faces (Sec. 4.3) carry eta at the face quadrature points; per
step the (eta, H) ODE is solved with physics.gravity_ode_taylor and the flux
uses int w1^b = -rho g H, int w7^b = eta^{n+1} - eta^n, w4^b = w6^b = 0.
Local time stepping (Sec. 4.4): see `advance_macro`.

Dofs layout in this module: Q[e, l, p] (element, basis, quantity).
"""

from math import factorial

import numpy as np

from . import basis as ob
from . import physics as ph
from .geometry import Geometry, cfl_dt, clusters
from .quadrature import tet_rule, tri_rule


class Oracle:
    def __init__(self, xyz, tets, face_tag, face_partner, rho, lam, mu, N, cfl=0.5,
                 g=9.81, max_clusters=1, dt=None):
        self.geo = geo = Geometry(xyz, tets, face_tag, face_partner)
        self.N = N
        self.B = ob.n_basis(N)
        E = geo.E
        self.E = E
        self.rho = np.asarray(rho, np.float64)
        self.lam = np.asarray(lam, np.float64)
        self.mu = np.asarray(mu, np.float64)
        self.g = float(g)
        self.Kxi = ob.stiffness(N)
        self.star = ph.star_matrices(geo.Jinv, self.rho, self.lam, self.mu)
        self.Zp, self.Zs = ph.impedances(self.rho, self.lam, self.mu)
        chi, w = tri_rule(2 * N)
        self.chi, self.fw, self.nq = chi, w, w.size
        self.phi_face = np.stack([ob.eval_basis(N, ob.face_to_ref(f, chi)) for f in range(4)])
        self.R = ph.frame(geo.normal)  # (E,4,3,3)
        # neighbour basis values at this face's quadrature points
        self.phi_nbr = np.zeros((E, 4, self.nq, self.B))
        self.face_x = np.zeros((E, 4, self.nq, 3))
        for f in range(4):
            xr = ob.face_to_ref(f, chi)  # (nq,3)
            x = geo.x0[:, None, :] + np.einsum("eda,qa->eqd", geo.J, xr)
            self.face_x[:, f] = x
            nb = geo.nbr[:, f]
            has = nb >= 0
            if np.any(has):
                xs = x[has] + geo.shift[has, f][:, None, :]
                xin = np.einsum("ead,eqd->eqa", geo.Jinv[nb[has]], xs - geo.x0[nb[has]][:, None, :])
                self.phi_nbr[has, f] = ob.eval_basis(N, xin.reshape(-1, 3)).reshape(-1, self.nq, self.B)
        self.eta = np.zeros((E, 4, self.nq))  # nodal eta on gravitational faces
        self.dt_e = cfl_dt(geo, self.rho, self.lam, self.mu, N, cfl)
        self.cluster, self.dtmin = clusters(geo, self.dt_e, max_clusters)
        if dt is not None:
            self.dtmin = float(dt)
        self.Q = np.zeros((E, self.B, 9))
        self.t = 0.0
        self.fault_guess = None
        self._setup_faults()

    # ---------------- dynamic rupture (oracle.rupture) -----------------
    def _setup_faults(self):
        """Fault faces: one per tet pair, minus = lower tet index, n = its outward
        normal; listed cluster-major, then by minus tet, then by face (the
        library's order).  The fault sits at the minus face's equispaced nodes."""
        geo, N = self.geo, self.N
        ff = [(int(e), int(f)) for e, f in np.argwhere(geo.face_tag == 5) if geo.nbr[e, f] > e]
        ff.sort(key=lambda ef: (self.cluster[ef[0]], ef[0], ef[1]))
        self.nff = len(ff)
        if not ff:
            return
        for e, f in ff:
            if self.cluster[e] != self.cluster[geo.nbr[e, f]]:
                raise ValueError("fault sides must share a cluster")
        self.fm = np.array(ff)
        self.fp = np.array([(geo.nbr[e, f], geo.nbr_face[e, f]) for e, f in ff])
        nodes = np.array([[i1 / N, i2 / N] for i2 in range(N + 1) for i1 in range(N + 1 - i2)])
        self.f_nodes = nodes
        Bf = nodes.shape[0]
        em, fm = self.fm[:, 0], self.fm[:, 1]
        ep = self.fp[:, 0]
        self.f_n = geo.normal[em, fm]                                   # (nff,3)
        self.f_xyz = np.stack([geo.to_phys(np.full(Bf, e), ob.face_to_ref(f, nodes)) for e, f in ff])
        self.f_phim = np.stack([ob.eval_basis(N, ob.face_to_ref(f, nodes)) for e, f in ff])
        self.f_phip = np.stack([ob.eval_basis(N, geo.to_ref(np.full(Bf, e2), x))
                                for e2, x in zip(ep, self.f_xyz)])
        # lift: int_face phi_k (sum_n ell_n G_n) dS by the face Gauss rule
        mono = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
        V = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in nodes])
        Vq = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in self.chi])
        self.f_ell = Vq @ np.linalg.inv(V)                              # (nq, Bf)
        xq = np.stack([geo.to_phys(np.full(self.nq, e), ob.face_to_ref(f, self.chi)) for e, f in ff])
        self.f_phiq_m = np.stack([self.phi_face[f] for e, f in ff])     # (nff,nq,B)
        self.f_phiq_p = np.stack([ob.eval_basis(N, geo.to_ref(np.full(self.nq, e2), x)) for e2, x in zip(ep, xq)])
        self.f_area = geo.area[em, fm]
        self.fault = None  # set by set_fault

    def set_fault(self, par, law="rs"):
        """par: dict of (nff, Bf) arrays named as rupture.PARAMS, or rupture.LSW_PARAMS
        for law = "lsw" (linear slip weakening); psi, V: initial state."""
        self.fault = {k: np.array(v, dtype=np.float64) for k, v in par.items()}
        self.fault_law = law
        self.fault["slip"] = np.zeros(self.fault["psi"].shape + (3,))
        self.fault["traction"] = np.zeros(self.fault["psi"].shape + (3,))
        self.newton_solves = 0
        self.newton_iters = 0

    def fault_update(self, sel, D, dt, guess=None):
        """Friction solve over [t0, t0+dt] on fault faces sel (indices into the
        fault list) from the Taylor expansions D (full element arrays) of both
        sides; returns {element: dQ increment}."""
        from . import rupture as ru
        N, Bf = self.N, self.f_nodes.shape[0]
        if self.fault is None:
            raise RuntimeError("fault parameters not set")
        em, ep = self.fm[sel, 0], self.fp[sel, 0]
        tj, _ = ru.time_points(N, dt)
        qm_t = np.zeros((N + 1, sel.size, Bf, 9))
        qp_t = np.zeros((N + 1, sel.size, Bf, 9))
        for j, t in enumerate(tj):
            for k, Dk in enumerate(D):
                c = t ** k / factorial(k)
                qm_t[j] += c * np.einsum("xnl,xlp->xnp", self.f_phim[sel], Dk[em])
                qp_t[j] += c * np.einsum("xnl,xlp->xnp", self.f_phip[sel], Dk[ep])
        flat = lambda a: a.reshape(a.shape[0] * a.shape[1], *a.shape[2:])
        nrm = np.repeat(self.f_n[sel], Bf, axis=0)
        matm = tuple(np.repeat(a[em], Bf) for a in (self.rho, self.lam, self.mu))
        matp = tuple(np.repeat(a[ep], Bf) for a in (self.rho, self.lam, self.mu))
        par = {k: flat(v[sel]) for k, v in self.fault.items() if k not in ("slip", "traction")}
        Gm, Gp, psi, V, dslip, iters, tau = ru.solve_step(
            nrm, qm_t.reshape(N + 1, -1, 9), qp_t.reshape(N + 1, -1, 9), matm, matp, par, dt, N, guess=guess,
            law=self.fault_law)
        self.newton_solves += int(np.sum(iters > 0))
        self.newton_iters += int(iters.sum())
        shp = (sel.size, Bf)
        self.fault["psi"][sel] = psi.reshape(shp)
        self.fault["V"][sel] = V.reshape(shp)
        self.fault["slip"][sel] += dslip.reshape(shp + (3,))
        self.fault["traction"][sel] = tau.reshape(shp + (3,))
        Gm = Gm.reshape(shp + (9,))
        Gp = Gp.reshape(shp + (9,))
        out = {}
        for i, fi in enumerate(sel):
            for (e, phiq, G) in ((em[i], self.f_phiq_m[fi], Gm[i]), (ep[i], self.f_phiq_p[fi], Gp[i])):
                scale = 2.0 * self.f_area[fi] / self.geo.detJ[e]
                Gq = self.f_ell @ G                                       # (nq, 9)
                d = -scale * np.einsum("q,qk,qp->kp", self.fw, phiq, Gq)
                out[int(e)] = out.get(int(e), 0.0) + d
        return out

    # ---------------- predictor -----------------
    def derivatives(self, Q, idx):
        D = [Q]
        KT = self.Kxi.transpose(0, 2, 1)[:, None]           # (3,1,B,B): K_e^T
        sT = self.star[idx].transpose(1, 0, 3, 2)           # (3,x,9,9): A*_e^T
        for _ in range(self.N):
            D.append(-np.sum(np.matmul(np.matmul(KT, D[-1][None]), sT), axis=0))
        return D

    @staticmethod
    def integrate(D, ta, tb):
        """int_{ta}^{tb} of the Taylor expansion (times relative to its centre)."""
        ta = np.asarray(ta, np.float64)
        tb = np.asarray(tb, np.float64)
        out = np.zeros_like(D[0])
        for k, Dk in enumerate(D):
            c = (tb ** (k + 1) - ta ** (k + 1)) / factorial(k + 1)
            out += (c[..., None, None] if np.ndim(c) else c) * Dk
        return out

    # ---------------- corrector -----------------
    def volume(self, I, idx):
        sT = self.star[idx].transpose(1, 0, 3, 2)
        return np.sum(np.matmul(np.matmul(self.Kxi[:, None], I[None]), sT), axis=0)

    def _nbr_state(self, idx, f, Inb):
        return np.einsum("xql,xlp->xqp", self.phi_nbr[idx, f], Inb)

    def face_update(self, idx, I, nbr_integral, D=None, dt=None, eta_new=None):
        """-1/|J| sum_f int phi (T A^- w^b) for elements idx with own
        time integral I.  nbr_integral(f, nb_idx) returns the neighbours'
        integrals over the same interval.  D/dt are needed on gravitational
        faces; the new eta is written to eta_new[(e, f)]."""
        geo = self.geo
        dQ = np.zeros_like(I)
        for f in range(4):
            tag = geo.face_tag[idx, f]
            qm = np.einsum("ql,xlp->xqp", self.phi_face[f], I)
            R = self.R[idx, f][:, None, :, :]
            wm = ph.rotate_in(qm, R)
            wb = np.zeros_like(wm)
            Zpm, Zsm = self.Zp[idx][:, None], self.Zs[idx][:, None]
            inter = (tag == 0) | (tag == 4)
            if np.any(inter):
                s = np.nonzero(inter)[0]
                nb = geo.nbr[idx[s], f]
                qp = self._nbr_state(idx[s], f, nbr_integral(f, idx[s], nb))
                wp = ph.rotate_in(qp, R[s])
                wb[s] = ph.middle_state(wm[s], wp, Zpm[s], self.Zp[nb][:, None], Zsm[s],
                                        self.Zs[nb][:, None])
            for bt in (1, 3, 6):
                s = np.nonzero(tag == bt)[0]
                if s.size:
                    wp = ph.ghost(wm[s], bt)
                    wb[s] = ph.middle_state(wm[s], wp, Zpm[s], Zpm[s], Zsm[s], Zsm[s])
            s = np.nonzero(tag == 2)[0]
            if s.size:
                wb[s] = self._gravity_state(idx[s], f, wm[s], R[s], D, s, dt, eta_new)
            fl = ph.flux_rotated(wb, self.rho[idx][:, None], self.lam[idx][:, None],
                                 self.mu[idx][:, None])
            F = ph.rotate_out(fl, R)
            scale = 2.0 * geo.area[idx, f] / geo.detJ[idx]
            dQ -= scale[:, None, None] * np.einsum("q,qk,xqp->xkp", self.fw, self.phi_face[f], F, optimize=True)
        return dQ

    def _gravity_state(self, e, f, wm_int, R, D, s, dt, eta_new):
        """Time-integrated middle state on gravitational faces (Sec. 4.3)."""
        rho, Z = self.rho[e], self.Zp[e]
        kappa = rho * self.g / Z
        # Taylor coefficients of f = v_n^- + p^-/Z = w7 - w1/Z at the face points
        fc = []
        for m, Dm in enumerate(D):
            qm = np.einsum("ql,xlp->xqp", self.phi_face[f], Dm[s])
            wmm = ph.rotate_in(qm, R)
            fc.append((wmm[..., 6] - wmm[..., 0] / Z[:, None]) / factorial(m))
        fc = np.stack(fc, axis=-1)  # (ns, nq, N+1)
        eta0 = self.eta[e, f]
        eta1, H = ph.gravity_ode_taylor(eta0, fc, kappa[:, None], dt)
        wb = wm_int.copy()
        wb[..., 0] = -rho[:, None] * self.g * H
        wb[..., 6] = eta1 - eta0
        wb[..., 3] = 0.0
        wb[..., 5] = 0.0
        Zs = self.Zs[e][:, None]
        sol = Zs > 0
        for (ts, tv) in ((3, 7), (5, 8)):
            wb[..., tv] = np.where(sol, wm_int[..., tv] - wm_int[..., ts] / np.where(sol, Zs, 1.0),
                                   wm_int[..., tv])
        eta_new.append((e, f, eta1))
        return wb

    # ---------------- time stepping -----------------
    def step_gts(self, dt=None):
        """One global time step (every element with the same dt)."""
        dt = self.dtmin if dt is None else dt
        idx = np.arange(self.E)
        D = self.derivatives(self.Q, idx)
        I = self.integrate(D, 0.0, dt)
        eta_new = []
        dQ = self.volume(I, idx) + self.face_update(
            idx, I, lambda f, s, nb: I[nb], D=D, dt=dt, eta_new=eta_new)
        if self.nff:
            for e, d in self.fault_update(np.arange(self.nff), D, dt, self.fault_guess).items():
                dQ[e] += d
        self.Q = self.Q + dQ
        for e, f, v in eta_new:
            self.eta[e, f] = v
        self.t += dt

    def advance_macro(self, scale=1.0):
        """One macro step of rate-2 LTS (Sec. 4.4), reading:
        ticks s = 0 .. 2^cmax - 1 of length dtmin; at tick s every cluster c
        with s % 2^c == 0 runs its predictor (derivatives kept, own integral,
        buffer reset when s % 2^(c+1) == 0, own integral added to the buffer);
        then every cluster with (s+1) % 2^c == 0 runs its corrector over
        [t_end - 2^c dtmin, t_end], taking from a same-cluster neighbour its
        integral, from a coarser neighbour the integral of its Taylor
        expansion over the sub-interval, from a finer neighbour its buffer.
        `scale` < 1 shortens every cluster step uniformly."""
        c = self.cluster
        cmax = int(c.max())
        dtm = self.dtmin * scale
        E = self.E
        if not hasattr(self, "_D") or self._D is None:
            self._D = [np.zeros_like(self.Q) for _ in range(self.N + 1)]
            self._t0 = np.zeros(E)
            self._Iown = np.zeros_like(self.Q)
            self._buf = np.zeros_like(self.Q)
        for s in range(1 << cmax):
            tick_t = s * dtm
            for cl in range(cmax + 1):
                if s % (1 << cl):
                    continue
                idx = np.nonzero(c == cl)[0]
                if idx.size == 0:
                    continue
                D = self.derivatives(self.Q[idx], idx)
                for k in range(self.N + 1):
                    self._D[k][idx] = D[k]
                self._t0[idx] = tick_t
                Iown = self.integrate(D, 0.0, (1 << cl) * dtm)
                self._Iown[idx] = Iown
                if s % (1 << (cl + 1)) == 0:
                    self._buf[idx] = 0.0
                self._buf[idx] += Iown
            t_end = (s + 1) * dtm
            for cl in range(cmax + 1):
                if (s + 1) % (1 << cl):
                    continue
                idx = np.nonzero(c == cl)[0]
                if idx.size == 0:
                    continue
                t_start = t_end - (1 << cl) * dtm

                def nbr_int(f, sidx, nb, cl=cl, t_start=t_start):
                    out = np.empty((nb.size, self.B, 9))
                    cn = c[nb]
                    same = cn == cl
                    out[same] = self._Iown[nb[same]]
                    fine = cn < cl
                    out[fine] = self._buf[nb[fine]]
                    coarse = np.nonzero(cn > cl)[0]
                    if coarse.size:
                        nbc = nb[coarse]
                        Dn = [Dk[nbc] for Dk in self._D]
                        ta = t_start - self._t0[nbc]
                        tb = ta + (1 << cl) * dtm
                        out[coarse] = self.integrate(Dn, ta, tb)
                    return out

                Dloc = [Dk[idx] for Dk in self._D]
                eta_new = []
                dQ = self.volume(self._Iown[idx], idx) + self.face_update(
                    idx, self._Iown[idx], nbr_int, D=Dloc, dt=(1 << cl) * dtm, eta_new=eta_new)
                if self.nff:
                    sel = np.nonzero(c[self.fm[:, 0]] == cl)[0]
                    if sel.size:
                        pos = {int(e): i for i, e in enumerate(idx)}
                        for e, d in self.fault_update(sel, self._D, (1 << cl) * dtm, self.fault_guess).items():
                            dQ[pos[e]] += d
                self.Q[idx] += dQ
                for e, f, v in eta_new:
                    self.eta[e, f] = v
        self.t += (1 << cmax) * dtm

    # ---------------- input / output helpers -----------------
    def project(self, fn, degree=None):
        """L2 projection of a physical field fn(x (...,3)) -> (...,9)."""
        pts, w = tet_rule(2 * self.N + 4 if degree is None else degree)
        phi = ob.eval_basis(self.N, pts)
        x = self.geo.x0[:, None, :] + np.einsum("eda,qa->eqd", self.geo.J, pts)
        vals = fn(x)
        return np.einsum("q,ql,eqp->elp", w, phi, vals)

    def l2_error(self, fn, Q=None, degree=None):
        Q = self.Q if Q is None else Q
        pts, w = tet_rule(2 * self.N + 4 if degree is None else degree)
        phi = ob.eval_basis(self.N, pts)
        x = self.geo.x0[:, None, :] + np.einsum("eda,qa->eqd", self.geo.J, pts)
        err = np.einsum("ql,elp->eqp", phi, Q) - fn(x)
        return np.sqrt(np.einsum("e,q,eqp->p", self.geo.detJ, w, err ** 2))

    def evaluate(self, e, x, Q=None):
        """q at physical points x (n,3) inside elements e (n,)."""
        Q = self.Q if Q is None else Q
        xi = self.geo.to_ref(e, x)
        phi = np.stack([ob.eval_basis(self.N, xi[i:i + 1])[0] for i in range(len(e))])
        return np.einsum("nl,nlp->np", phi, Q[e])

    def energy(self, Q=None):
        """Mechanical energy sum_K int (1/2 rho |v|^2 + 1/2 s:C^-1:s) plus the
        gravitational surface energy sum int 1/2 rho g eta^2 dS."""
        Q = self.Q if Q is None else Q
        rho, lam, mu = self.rho, self.lam, self.mu
        # orthonormal basis: int_K f g = |J| sum_l F_l G_l
        kin = 0.5 * rho * np.einsum("elp,elp->e", Q[..., 6:], Q[..., 6:])
        tr = Q[..., 0] + Q[..., 1] + Q[..., 2]
        sq = (np.einsum("elp,elp->e", Q[..., :3], Q[..., :3])
              + 2 * np.einsum("elp,elp->e", Q[..., 3:6], Q[..., 3:6]))
        trtr = np.einsum("el,el->e", tr, tr)
        solid = mu > 0
        ms = np.where(solid, mu, 1.0)
        pot_s = 0.5 * (sq / (2 * ms) - lam / (2 * ms * (3 * lam + 2 * ms)) * trtr)
        pot_f = 0.5 * trtr / (9.0 * lam)
        pot = np.where(solid, pot_s, pot_f)
        E = np.sum(self.geo.detJ * (kin + pot))
        gf = np.argwhere(self.geo.face_tag == 2)
        for e, f in gf:
            E += 0.5 * rho[e] * self.g * 2 * self.geo.area[e, f] * np.sum(self.fw * self.eta[e, f] ** 2)
        return E
