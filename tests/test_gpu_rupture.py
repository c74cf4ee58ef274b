"""GPU parity of dynamic rupture (Sec. 3, Eq. bc-dynrup) and of the learned
Newton start, against the FP64 oracle."""

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import rupture as ru
from synthetic.workloads import fault_box, lsw_fault_params, random_dofs, rs_fault_params
from tests._cases import make_pair, rel_l2, to_gpu_layout, to_oracle_layout

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _fault_pair(N=3, ocean_layers=0, max_clusters=1, precision=0, law="rs", **kw):
    m, mat = fault_box(nx=4, ny=2, nz=4, dz=1e3, ocean_layers=ocean_layers, **kw)
    o, s = make_pair(m, mat, N, precision=precision, cfl=0.5, max_clusters=max_clusters)
    nff = int(s.info.n_fault_faces)
    assert nff == o.nff > 0
    from paper_2107_06640_gb300 import _lib
    mf, pf, xyz, nrm = _lib.adg_fault_faces(s.ctx, nff, s.Bf)
    assert np.array_equal(mf, o.fm[:, 0] * 4 + o.fm[:, 1])
    assert np.array_equal(pf, o.fp[:, 0] * 4 + o.fp[:, 1])
    assert np.allclose(xyz, o.f_xyz, rtol=0, atol=1e-9) and np.allclose(nrm, o.f_n, atol=1e-14)
    if law == "lsw":
        par = lsw_fault_params(xyz, nrm, seed=1, patch_radius=2e3)
        _lib.adg_set_friction_law(s.ctx, _lib.ADG_FRICTION_LSW)
        names = ru.LSW_PARAMS
    else:
        par = rs_fault_params(xyz, nrm, seed=1, patch_radius=2e3)
        names = ru.PARAMS
    _lib.adg_set_fault(s.ctx, par[:, None, :, :])
    o.set_fault({k: par[..., i] for i, k in enumerate(names)}, law=law)
    return m, o, s, nff


def _read_fault(s, nff):
    from paper_2107_06640_gb300 import _lib
    st = np.empty((nff, 1, s.Bf, 8))
    return _lib.adg_read_fault(s.ctx, st)[:, 0]


def _compare(o, s, nff, tol=FP64_TOL):
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= tol
    st = _read_fault(s, nff)
    assert rel_l2(st[..., 0], o.fault["V"]) <= tol
    assert rel_l2(st[..., 1], o.fault["psi"]) <= tol
    assert rel_l2(st[..., 2:5], o.fault["slip"]) <= tol
    assert rel_l2(st[..., 5:8], o.fault["traction"]) <= tol
    return st


def test_rupture_parity_fp64():
    m, o, s, nff = _fault_pair()
    Q0 = random_dofs((m.nt, s.B, 9), 4, N=3) * 1e3
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(5):
        o.step_gts()
    s.advance(5)
    st = _compare(o, s, nff)
    assert st[..., 0].max() > 0.1          # the nucleation patch ruptured
    from paper_2107_06640_gb300 import _lib
    solves, iters = _lib.adg_fault_stats(s.ctx)
    assert solves > 0 and iters >= solves


def test_rupture_under_ocean_with_lts_fp64():
    m, o, s, nff = _fault_pair(N=2, ocean_layers=1, max_clusters=3)
    for _ in range(2):
        o.advance_macro()
    s.advance(2)
    _compare(o, s, nff)


def test_slip_weakening_parity_fp64():
    """Linear slip weakening (closed-form slip rate): dofs, slip rate, slip
    path, slip and traction against the oracle after 5 steps; the nucleation
    patch ruptures and no Newton solve runs."""
    m, o, s, nff = _fault_pair(law="lsw")
    Q0 = random_dofs((m.nt, s.B, 9), 4, N=3) * 1e3
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(5):
        o.step_gts()
    s.advance(5)
    st = _compare(o, s, nff)
    assert st[..., 0].max() > 0.1 and st[..., 1].max() > 0
    assert np.all(st[..., 0] >= 0) and np.all(st[..., 1] >= 0)
    from paper_2107_06640_gb300 import _lib
    solves, iters = _lib.adg_fault_stats(s.ctx)
    assert solves == 0 and iters == 0


def test_slip_weakening_under_ocean_with_lts_fp64():
    m, o, s, nff = _fault_pair(N=2, ocean_layers=1, max_clusters=3, law="lsw")
    for _ in range(2):
        o.advance_macro()
    s.advance(2)
    _compare(o, s, nff)


def test_rupture_degree4_on_the_tensor_cores_under_ocean():
    """Degree 4 in the 3xTF32 form, the megathrust's configuration: elements
    with a fault or gravitational face take the FP32 CUDA-core kernels, the
    others both tensor-core kernels; the friction solve stays FP64 on FP32
    traces.  Against the FP64 oracle after 4 steps: dofs within 2e-5 as the
    other 3xTF32 steps; the fault state within 1e-3, because a relative error
    d in the traction moves ln V by about d Th / (a S) (Th / (a S) ~ 50 here)."""
    from paper_2107_06640_gb300 import _lib
    m, o, s, nff = _fault_pair(N=4, ocean_layers=1, precision=2)
    assert 0 < int(s.info.tensor_core_updates_per_macro) < m.nt
    Q0 = random_dofs((m.nt, s.B, 9), 4, N=4) * 1e3
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    for _ in range(4):
        o.step_gts()
    s.advance(4)
    assert rel_l2(to_oracle_layout(s.get_dofs()), o.Q) <= 2e-5, rel_l2(to_oracle_layout(s.get_dofs()), o.Q)
    st = _read_fault(s, nff)
    errs = [rel_l2(st[..., 0], o.fault["V"]), rel_l2(st[..., 1], o.fault["psi"]),
            rel_l2(st[..., 2:5], o.fault["slip"]), rel_l2(st[..., 5:8], o.fault["traction"])]
    assert max(errs) <= 1e-3, errs
    assert st[..., 0].max() > 0.1          # the nucleation patch ruptured
    _, launches = _lib.adg_profile(s.ctx, 1)
    assert launches[0] >= 2 and launches[1] >= 2   # tensor-core and CUDA-core launches in both phases


def test_friction_law_switch_needs_new_parameters():
    from paper_2107_06640_gb300 import AdgError, _lib
    m, o, s, nff = _fault_pair(law="lsw")
    _lib.adg_set_friction_law(s.ctx, _lib.ADG_FRICTION_RS)
    with pytest.raises(AdgError):
        s.advance(1)  # parameters cleared by the switch
    with pytest.raises(AdgError):
        _lib.adg_set_friction_law(s.ctx, 7)


def test_mlp_gradient_matches_oracle():
    from paper_2107_06640_gb300 import _lib
    rng = np.random.default_rng(3)
    P = rng.standard_normal(omlp.N_PARAM).astype(np.float32) * 0.3
    P[omlp.N_TRAIN + omlp.IN:omlp.N_TRAIN + 2 * omlp.IN] = rng.uniform(0.5, 2.0, omlp.IN)
    P[-2:] = [0.2, 1.5]
    rows = rng.standard_normal((3000, omlp.IN + 1)).astype(np.float32)
    g, loss = _lib.adg_mlp_gradient(P, rows)
    lo, go = omlp.loss_and_grad(P.astype(np.float64), rows.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_learned_newton_start_same_solution_fewer_iterations():
    """Capture friction solves from one run, train the network on the GPU,
    rerun from the same start with the learned guess: same answer to the
    solver tolerance, fewer Newton iterations."""
    from paper_2107_06640_gb300 import _lib
    m, o, s, nff = _fault_pair()
    Q0 = random_dofs((m.nt, s.B, 9), 4, N=3) * 1e3
    s.set_dofs(to_gpu_layout(Q0))
    start = s.save_state()
    steps = 20
    _lib.adg_fault_stats(s.ctx, reset=True)
    _lib.adg_rupture_capture(s.ctx, 1 << 20)
    s.advance(steps)
    n = _lib.adg_rupture_capture(s.ctx, 0)
    plain_solves, plain_iters = _lib.adg_fault_stats(s.ctx, reset=True)
    plain_Q, plain_fault = s.get_dofs(), _read_fault(s, nff)
    loss = _lib.adg_mlp_train(s.ctx, epochs=300, batch=512, lr=3e-3, seed=0)
    assert n > 1000 and loss[1] < 0.5 * loss[0]
    _lib.adg_mlp_params(s.ctx, enable=1)
    s.load_state(start)
    s.advance(steps)
    mlp_solves, mlp_iters = _lib.adg_fault_stats(s.ctx, reset=True)
    print(f"Newton iterations per solve: plain {plain_iters / plain_solves:.3f} ({plain_solves} solves), "
          f"learned start {mlp_iters / mlp_solves:.3f} ({mlp_solves} solves); {n} training solves; "
          f"loss {loss[0]:.3e} -> {loss[1]:.3e}")
    assert abs(mlp_solves - plain_solves) <= 1e-3 * plain_solves
    assert rel_l2(s.get_dofs(), plain_Q) <= FP64_TOL
    assert rel_l2(_read_fault(s, nff)[..., 0], plain_fault[..., 0]) <= FP64_TOL
    assert mlp_iters / mlp_solves < plain_iters / plain_solves
