"""The launch-shape autotuner (adg_autotune): it picks each kernel kind's
shape from its candidates by timing them on the context's own clusters,
leaves the solution where it was, and the steps after it give bit-identical
results to untuned steps (a launch shape changes how the work is cut, not the
arithmetic of any element)."""

import numpy as np
import pytest

import synthetic as syn
from synthetic.workloads import random_dofs
from tests._cases import small_coupled, to_gpu_layout

pytestmark = pytest.mark.gpu

CANDIDATES = [(64, 128, 256), (64, 128, 256), (1, 2, 4), (1, 2, 4)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _pair(m, mat, **kw):
    from paper_2107_06640_gb300 import Solver
    rho, lam, mu = mat
    mk = lambda: Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=5, cfl=0.5, precision=2, **kw)
    return mk(), mk()


def _fault_context(N=5):
    """A fault box under an ocean (its fault elements take the CUDA-core
    kernels, the rest the tensor-core ones) with rate-and-state parameters."""
    from paper_2107_06640_gb300 import Solver, _lib
    from synthetic.workloads import fault_box, rs_fault_params
    m, (rho, lam, mu) = fault_box(nx=4, ny=2, nz=4, dz=1e3, ocean_layers=1)
    mk = lambda: Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N, cfl=0.5, precision=2)
    out = []
    for _ in range(2):
        s = mk()
        nff = int(s.info.n_fault_faces)
        _, _, xyz, nrm = _lib.adg_fault_faces(s.ctx, nff, s.Bf)
        _lib.adg_set_fault(s.ctx, rs_fault_params(xyz, nrm, seed=1, patch_radius=2e3)[:, None])
        out.append(s)
    return m, out[0], out[1]


@pytest.mark.parametrize("case", ["gts", "lts", "fault"])
def test_autotune_keeps_the_solution_and_the_arithmetic(case):
    from paper_2107_06640_gb300 import _lib
    if case == "lts":
        m, mat = syn.workloads.coupled_box(nxy=4, n_water=2, n_crust=2, L=8e3, depth=4e3, water=1e3, grading=4.0)
        tuned, plain = _pair(m, mat, max_clusters=4)
        assert tuned.info.n_clusters >= 2
    elif case == "fault":
        m, tuned, plain = _fault_context()
    else:
        m, mat = small_coupled()
        tuned, plain = _pair(m, mat)
    Q0 = to_gpu_layout(random_dofs((m.nt, tuned.B, 9), 31, N=5))
    for s in (tuned, plain):
        s.set_dofs(Q0)
        s.advance(1)
    before, t_before = tuned.get_dofs(), tuned.time
    choice, ms = _lib.adg_autotune(tuned.ctx, reps=1, force=True)
    # the tensor-core kinds run in every context (sea-surface elements and
    # elements at LTS cluster borders too); the CUDA-core kinds only in the
    # fault box (its fault elements): each kind that runs is tuned over its
    # three candidates, the others keep 0
    for k in range(4):
        if k < 2 and case != "fault":
            assert choice[k] == 0 and np.all(ms[k] == -1.0), (k, choice, ms)
            continue
        assert choice[k] in CANDIDATES[k], (k, choice)
        assert np.all(ms[k] > 0), (k, ms)
        assert ms[k][CANDIDATES[k].index(choice[k])] == ms[k].min()
    assert np.array_equal(tuned.get_dofs(), before) and tuned.time == t_before
    tuned.advance(2)
    plain.advance(2)
    assert np.array_equal(tuned.get_dofs(), plain.get_dofs())
    # a second context of the same kind takes the cached choice without timing
    if case == "fault":
        again = _fault_context()[1]
    else:
        again = _pair(m, mat, **({"max_clusters": 4} if case == "lts" else {}))[0]
    c2, ms2 = _lib.adg_autotune(again.ctx, reps=1)
    assert np.array_equal(c2, choice) and np.all(ms2 == -1.0)


def test_autotune_needs_an_initialised_context_at_a_macro_boundary():
    from paper_2107_06640_gb300 import _lib
    m, mat = syn.workloads.coupled_box(nxy=4, n_water=2, n_crust=2, L=8e3, depth=4e3, water=1e3, grading=4.0)
    s = _pair(m, mat, max_clusters=4)[0]
    _lib.adg_step_tick(s.ctx)
    with pytest.raises(_lib.AdgError) as ei:
        _lib.adg_autotune(s.ctx, reps=1)
    assert ei.value.code == -3
