"""The pins catch plausible mistakes: each case plants one mistake in an
oracle module (a source replacement, executed in a child process on the CPU;
nothing on disk changes) and runs the pins that cover that part of the
oracle, which must then fail.  The unmutated pins pass in the rest of the
suite."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (id, oracle file, original text, planted text, pin tests (file, -k expression))
CASES = [
    ("absorbing-transparent", "physics.py",
     "if tag == 3:      # absorbing: q+ = 0\n        wp[...] = 0.0",
     "if tag == 3:      # absorbing: q+ = 0\n        wp[...] = wm",
     ("test_oracle_physics.py", "absorbing")),
    ("rigid-mirrors-traction", "physics.py",
     "elif tag == 6:    # rigid wall, free slip\n        wp[..., [6, 3, 5]] *= -1.0",
     "elif tag == 6:    # rigid wall, free slip\n        wp[..., [0, 3, 5]] *= -1.0",
     ("test_oracle_physics.py", "wall_middle")),
    ("free-surface-keeps-shear", "physics.py",
     "elif tag == 1:    # free surface: traction mirrored\n        wp[..., [0, 3, 5]] *= -1.0",
     "elif tag == 1:    # free surface: traction mirrored\n        wp[..., [0]] *= -1.0",
     ("test_oracle_physics.py", "wall_middle")),
    ("lts-coarse-subinterval-from-start", "ader.py",
     "ta = t_start - self._t0[nbc]", "ta = 0.0 * self._t0[nbc]",
     ("test_oracle_scheme.py", "conserves")),
    ("lts-fine-neighbour-last-integral", "ader.py",
     "out[fine] = self._buf[nb[fine]]", "out[fine] = self._Iown[nb[fine]]",
     ("test_oracle_scheme.py", "conserves")),
    ("lts-buffer-never-reset", "ader.py",
     "self._buf[idx] = 0.0", "self._buf[idx] = self._buf[idx]",
     ("test_oracle_scheme.py", "conserves")),
    ("fault-plus-side-scaled-by-minus-volume", "ader.py",
     "scale = 2.0 * self.f_area[fi] / self.geo.detJ[e]", "scale = 2.0 * self.f_area[fi] / self.geo.detJ[em[i]]",
     ("test_oracle_rupture_lsw.py", "locked_fault_in")),
    ("fault-taylor-factor", "ader.py",
     "c = t ** k / factorial(k)\n", "c = t ** k / factorial(k + 1)\n",
     ("test_oracle_rupture_lsw.py", "locked_fault_in")),
    ("fault-lts-step-length", "ader.py",
     "for e, d in self.fault_update(sel, self._D, (1 << cl) * dtm, self.fault_guess).items():",
     "for e, d in self.fault_update(sel, self._D, dtm, self.fault_guess).items():",
     ("test_oracle_rupture_lsw.py", "locked_fault_in")),
    ("energy-poisson-term", "ader.py",
     "pot_s = 0.5 * (sq / (2 * ms) - lam / (2 * ms * (3 * lam + 2 * ms)) * trtr)",
     "pot_s = 0.5 * (sq / (2 * ms) - lam / (ms * (3 * lam + 2 * ms)) * trtr)",
     ("test_oracle_scheme.py", "energy_is")),
    ("energy-surface-term", "ader.py",
     "E += 0.5 * rho[e] * self.g * 2 * self.geo.area[e, f]", "E += 0.5 * rho[e] * self.g * self.geo.area[e, f]",
     ("test_oracle_scheme.py", "energy_is")),
    ("projection-transposed-map", "ader.py",
     'x = self.geo.x0[:, None, :] + np.einsum("eda,qa->eqd", self.geo.J, pts)\n        vals',
     'x = self.geo.x0[:, None, :] + np.einsum("ead,qa->eqd", self.geo.J, pts)\n        vals',
     ("test_oracle_scheme.py", "polynomial")),
    ("cfl-length-halved", "geometry.py",
     "self.h = 6.0 * self.volume / self.area.sum(axis=1)", "self.h = 3.0 * self.volume / self.area.sum(axis=1)",
     ("test_oracle_geometry.py", "")),
    ("clusters-ignore-faults", "geometry.py",
     "lim = np.where(tag == 5, cn, cn + 1)", "lim = cn + 1",
     ("test_oracle_geometry.py", "clusters")),
    ("clusters-round-up", "geometry.py",
     "c = np.floor(np.log2(dt / dtmin) + 1e-12).astype(np.int64)",
     "c = np.ceil(np.log2(dt / dtmin) - 1e-12).astype(np.int64)",
     ("test_oracle_geometry.py", "clusters")),
    ("periodic-shift-sign", "geometry.py",
     "self.shift[e, f] = self.face_centroid[p // 4, p % 4] - self.face_centroid[e, f]",
     "self.shift[e, f] = self.face_centroid[e, f] - self.face_centroid[p // 4, p % 4]",
     ("test_oracle_geometry.py", "neighbours")),
    ("inverse-map-transposed", "geometry.py",
     'np.einsum("...ad,...d->...a", self.Jinv[e], x - self.x0[e])',
     'np.einsum("...da,...d->...a", self.Jinv[e], x - self.x0[e])',
     ("test_oracle_scheme.py", "polynomial")),
    ("rs-no-tail", "rupture.py",
     'psi = psi + V * (dt - tprev) if law == "lsw" else psi_relax(psi, V, dt - tprev, par)',
     'psi = psi + V * (dt - tprev) if law == "lsw" else psi',
     ("test_oracle_rupture.py", "constant_load")),
    ("rs-interval-from-step-start", "rupture.py",
     "        h = tj[j] - tprev\n", "        h = tj[j]\n",
     ("test_oracle_rupture.py", "constant_load")),
    ("basis-jacobi-parameter", "basis.py",
     "f2, f2y, f2t = _G(j, 2 * i + 1, eta, t)", "f2, f2y, f2t = _G(j, 2 * i, eta, t)",
     ("test_oracle_basis.py", "orthonormal")),
    ("basis-gradient-sign", "basis.py",
     "grad[:, l, 1] = -f1s * f2 * f3 + f1 * f2y * f3", "grad[:, l, 1] = f1s * f2 * f3 + f1 * f2y * f3",
     ("test_oracle_basis.py", "gradient")),
    ("stiffness-transposed", "basis.py",
     'return np.einsum("q,qke,ql->ekl", w, g, v)', 'return np.einsum("q,qke,ql->elk", w, g, v)',
     ("test_oracle_basis.py", "stiffness")),
    ("face-vertex-list", "basis.py",
     "FACE_VERTS = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))",
     "FACE_VERTS = ((1, 2, 3), (0, 2, 3), (0, 1, 2), (0, 1, 3))",
     ("test_oracle_basis.py", "face_maps")),
    ("tet-rule-collapse-weight", "quadrature.py",
     "wt = wu * wv * ws * (1 - v) * (1 - s) ** 2", "wt = wu * wv * ws * (1 - v) * (1 - s)",
     ("test_oracle_basis.py", "quadrature")),
    ("tet-rule-too-few-points", "quadrature.py",
     "n = max(1, int(np.ceil((degree + 3) / 2.0)))", "n = max(1, int(np.ceil((degree + 1) / 2.0)))",
     ("test_oracle_basis.py", "quadrature")),
    ("jacobian-normal-stress-mu", "physics.py",
     "M[..., S[(d, d)], 6 + d] -= 2 * mu", "M[..., S[(d, d)], 6 + d] -= mu",
     ("test_oracle_physics.py", "eigenvalues")),
    ("middle-state-impedance", "physics.py",
     "a1 = Zpm * Zpp / (Zpm + Zpp) * ((wm[..., 0:1] - wp[..., 0:1]) / Zpp",
     "a1 = Zpm * Zpp / (Zpm + Zpp) * ((wm[..., 0:1] - wp[..., 0:1]) / Zpm",
     ("test_oracle_physics.py", "both_sides")),
    ("middle-state-shear-impedance", "physics.py",
     "a = Zsm * Zsp / (Zsm + Zsp) * ((wm[..., ts:ts + 1] - wp[..., ts:ts + 1]) / Zsp",
     "a = Zsm * Zsp / (Zsm + Zsp) * ((wm[..., ts:ts + 1] - wp[..., ts:ts + 1]) / Zsm",
     ("test_oracle_physics.py", "both_sides")),
    ("gravity-ode-H-series", "physics.py",
     "H = H + term * dt / (m + 2)", "H = H + term * dt / (m + 1)",
     ("test_oracle_physics.py", "gravity_ode")),
    ("friction-2V0", "rupture.py",
     'return a * np.arcsinh(V / (2.0 * p["V0"]) * np.exp(psi / a))',
     'return a * np.arcsinh(V / p["V0"] * np.exp(psi / a))',
     ("test_oracle_rupture.py", "steady_state")),
    ("locked-traction-impedances-swapped", "rupture.py",
     "theta = eta[..., None] * ((up - um) + taup / Zsp[..., None] + taum / Zsm[..., None])",
     "theta = eta[..., None] * ((up - um) + taup / Zsm[..., None] + taum / Zsp[..., None])",
     ("test_oracle_rupture.py", "locked_fault_is")),
    ("side-velocity-sign", "rupture.py",
     'ub = st["um"] + (tau_p - st["taum"]) / st["Zsm"][..., None]',
     'ub = st["um"] - (tau_p - st["taum"]) / st["Zsm"][..., None]',
     ("test_oracle_rupture.py", "locked_fault_is or slipping")),
    ("gauss-time-weights", "rupture.py",
     "return 0.5 * dt * (x + 1.0), 0.5 * dt * w", "return 0.5 * dt * (x + 1.0), dt * w",
     ("test_oracle_rupture_lsw.py", "locked_fault_in")),
    ("mlp-tanh-derivative", "mlp.py",
     "da2 = (dy[:, None] * p[\"w3\"][None, :]) * (1.0 - h2 * h2)",
     "da2 = (dy[:, None] * p[\"w3\"][None, :]) * (1.0 - h2)",
     ("test_oracle_mlp.py", "gradient")),
    ('predictor-sign', 'ader.py',
     'D.append(-np.sum(np.matmul(np.matmul(KT, D[-1][None]), sT), axis=0))',
     'D.append(np.sum(np.matmul(np.matmul(KT, D[-1][None]), sT), axis=0))',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('time-integral-factorial', 'ader.py',
     'c = (tb ** (k + 1) - ta ** (k + 1)) / factorial(k + 1)',
     'c = (tb ** (k + 1) - ta ** (k + 1)) / factorial(k)',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('volume-operator-transposed', 'ader.py',
     'return np.sum(np.matmul(np.matmul(self.Kxi[:, None], I[None]), sT), axis=0)',
     'return np.sum(np.matmul(np.matmul(self.Kxi.transpose(0, 2, 1)[:, None], I[None]), sT), axis=0)',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('face-scale-factor-2', 'ader.py',
     'scale = 2.0 * geo.area[idx, f] / geo.detJ[idx]',
     'scale = geo.area[idx, f] / geo.detJ[idx]',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('periodic-neighbour-shift-sign', 'ader.py',
     'xs = x[has] + geo.shift[has, f][:, None, :]',
     'xs = x[has] - geo.shift[has, f][:, None, :]',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('gravity-eta-increment', 'ader.py',
     'wb[..., 6] = eta1 - eta0',
     'wb[..., 6] = eta1',
     ('test_oracle_scheme.py', 'surface_gravity_wave_dispersion')),
    ('gravity-kappa', 'ader.py',
     'kappa = rho * self.g / Z',
     'kappa = rho * self.g * Z',
     ('test_oracle_scheme.py', 'surface_gravity_wave_dispersion')),
    ('gravity-forcing-sign', 'ader.py',
     'fc.append((wmm[..., 6] - wmm[..., 0] / Z[:, None]) / factorial(m))',
     'fc.append((wmm[..., 6] + wmm[..., 0] / Z[:, None]) / factorial(m))',
     ('test_oracle_scheme.py', 'surface_gravity_wave_dispersion')),
    ('rotation-transposed', 'physics.py',
     'Sr = np.einsum("...ji,...jk,...kl->...il", R, S, R, optimize=True)',
     'Sr = np.einsum("...ij,...jk,...lk->...il", R, S, R, optimize=True)',
     ('test_oracle_physics.py', 'rotation')),
    ('flux-wrong-direction', 'physics.py',
     'A = jacobians(rho, lam, mu)[..., 0, :, :]',
     'A = jacobians(rho, lam, mu)[..., 1, :, :]',
     ('test_oracle_scheme.py', 'convergence_order')),
    ('gravity-ghost-pressure-sign', 'physics.py',
     'wp[..., 0] = -(2.0 * rho * g * eta - pm)',
     'wp[..., 0] = (2.0 * rho * g * eta - pm)',
     ('test_oracle_physics.py', 'gravity_ghost')),
    ('strength-sign', 'rupture.py',
     'S=np.maximum(0.0, -(sn0 + sn_b)))',
     'S=np.maximum(0.0, -(sn0 - sn_b)))',
     ('test_oracle_rupture_lsw.py', 'normal_stress')),
    ('lsw-min-max', 'rupture.py',
     'np.minimum(psi / p["Dc"], 1.0)',
     'np.maximum(psi / p["Dc"], 1.0)',
     ('test_oracle_rupture_lsw.py', 'coefficient')),
    ('state-relaxation-sign', 'rupture.py',
     'return ss + (psi - ss) * np.exp(-V * h / p["L"])',
     'return ss + (psi - ss) * np.exp(V * h / p["L"])',
     ('test_oracle_rupture.py', 'relaxation')),
    ('basis-norm', 'basis.py',
     'return 1.0 / np.sqrt(np.einsum("q,ql,ql->l", w, v, v))',
     'return 1.0 / np.einsum("q,ql,ql->l", w, v, v)',
     ('test_oracle_basis.py', 'orthonormal')),
    ('tri-rule-weight', 'quadrature.py',
     'wt = wu * wv * (1 - v)\n',
     'wt = wu * wv\n',
     ('test_oracle_basis.py', '')),
    ('inverse-map-transposed-matrix', 'geometry.py',
     'self.Jinv = np.linalg.inv(self.J)',
     'self.Jinv = np.linalg.inv(self.J).transpose(0, 2, 1)',
     ('test_oracle_scheme.py', 'polynomial')),
    ('normal-orientation', 'geometry.py',
     'sgn = np.sign(np.einsum("ij,ij->i", n, a - opp))',
     'sgn = np.ones(n.shape[0])',
     ('test_oracle_geometry.py', '')),
    ('fluid-tangential-velocity-sign', 'physics.py',
     'wv_fluid = np.where(Zsm > 0, wm[..., tv:tv + 1] - wm[..., ts:ts + 1]',
     'wv_fluid = np.where(Zsm > 0, wm[..., tv:tv + 1] + wm[..., ts:ts + 1]',
     ('test_oracle_physics.py', 'both_sides or acoustic_rule')),
    ('impedance-as-speed', 'physics.py',
     'return np.sqrt(rho * (lam + 2 * mu)), np.sqrt(rho * mu)',
     'return np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)',
     ('test_oracle_physics.py', '')),
    ('fault-traction-eta-sign', 'rupture.py',
     'tau_tot = (Th - st["eta"] * Vmag)[..., None] * d',
     'tau_tot = (Th + st["eta"] * Vmag)[..., None] * d',
     ('test_oracle_rupture.py', '')),
    ('fault-flux-velocity-rows', 'rupture.py',
     'out[..., 6:9] = -t / rho[..., None]',
     'out[..., 6:9] = t / rho[..., None]',
     ('test_oracle_rupture.py', '')),
    ('fault-plus-flux-sign', 'rupture.py',
     'Gp += wj[j] * (-ahat_apply(n, t_b, vc, *matp))\n            slip += wj[j] * Vvec\n            tprev = tj[j]\n            continue',
     'Gp += wj[j] * ahat_apply(n, t_b, vc, *matp)\n            slip += wj[j] * Vvec\n            tprev = tj[j]\n            continue',
     ('test_oracle_rupture_lsw.py', 'locked_fault_in')),
    ('lsw-state-uses-current-rate', 'rupture.py',
     'psi_new = psi + Vmid * h',
     'psi_new = psi + Vcur * h',
     ('test_oracle_rupture_lsw.py', '')),
    ('lts-buffer-assigned', 'ader.py',
     'self._buf[idx] += Iown',
     'self._buf[idx] = Iown',
     ('test_oracle_scheme.py', 'conserves')),
    ('subinterval-integral-of-difference', 'ader.py',
     'c = (tb ** (k + 1) - ta ** (k + 1)) / factorial(k + 1)',
     'c = (tb - ta) ** (k + 1) / factorial(k + 1)',
     ('test_oracle_scheme.py', 'conserves')),
    ('lts-predictor-start-time', 'ader.py',
     'self._t0[idx] = tick_t',
     'self._t0[idx] = 0.0',
     ('test_oracle_scheme.py', 'conserves')),
    ('lts-buffer-reset-every-step', 'ader.py',
     'if s % (1 << (cl + 1)) == 0:',
     'if s % (1 << cl) == 0:',
     ('test_oracle_scheme.py', 'conserves')),
    ('macro-scale-ignored', 'ader.py',
     'dtm = self.dtmin * scale',
     'dtm = self.dtmin',
     ('test_oracle_scheme.py', 'gravity_wave_with_lts')),
    ('neighbour-basis-through-own-map', 'ader.py',
     'xin = np.einsum("ead,eqd->eqa", geo.Jinv[nb[has]], xs - geo.x0[nb[has]][:, None, :])',
     'xin = np.einsum("ead,eqd->eqa", geo.Jinv[has], xs - geo.x0[has][:, None, :])',
     ('test_oracle_scheme.py', 'convergence_order')),
]

_CHILD = """
import importlib, sys, traceback
try:
    sys.path.insert(0, {root!r})
    mod = importlib.import_module("oracle." + {stem!r})
    path = {path!r}
    src = open(path).read()
    if src.count({old!r}) != 1:
        raise RuntimeError("the original text is not unique in " + path)
    exec(compile(src.replace({old!r}, {new!r}), path, "exec"), mod.__dict__)
except Exception:
    traceback.print_exc()
    sys.exit(3)  # the mistake could not be planted: distinct from a failing pin
import pytest
args = ["-q", "-x", "-p", "no:cacheprovider", {test!r}]
if {sel!r}:
    args += ["-k", {sel!r}]
sys.exit(pytest.main(args))
"""


def _run(case):
    name, fname, old, new, (tfile, sel) = case
    path = os.path.join(ROOT, "oracle", fname)
    code = _CHILD.format(root=ROOT, stem=fname[:-3], path=path, old=old, new=new,
                         test=os.path.join(ROOT, "tests", tfile), sel=sel)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900,
                          env=env)


@pytest.fixture(scope="module")
def results():
    """All children at once (independent processes, single-threaded BLAS)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip((c[0] for c in CASES), ex.map(_run, CASES)))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pins(case, results):
    name = case[0]
    r = results[name]
    # pytest exit code 1: tests ran and some failed (not 2/4/5: interrupted, usage error, nothing collected;
    # 3: the mistake could not be planted)
    assert r.returncode == 1, f"{name}: pins did not fail (exit {r.returncode})\n{r.stdout[-2000:]}{r.stderr[-2000:]}"
