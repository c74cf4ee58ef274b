"""The acoustic ocean (adg_set_acoustic_ocean): the fluid as the elastic
system with mu = 0 and stress -p I (Sec. 4.1), kept isotropic by the library
and, with the tensor-core kernels, its plain elements on the 4-quantity (p, v)
local kernel.  Parity against the 9-quantity FP64 oracle on data whose fluid
stress is isotropic (the acoustic subspace is invariant under the scheme,
pinned on the oracle by test_fluid_stress_stays_isotropic)."""

import numpy as np
import pytest

import synthetic as syn
from synthetic.workloads import random_dofs
from tests._cases import (eta_poly, make_pair, node_chi, oracle_eta_at_nodes, rel_l2, small_coupled,
                          to_gpu_layout, to_oracle_layout)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_06640_gb300 import build
    build.build()


def _isotropic(Q, fluid):
    """Q in the oracle layout [nt][B][9]: fluid stress replaced by its mean."""
    Q = Q.copy()
    m = Q[fluid, :, 0:3].mean(axis=2)
    Q[fluid, :, 0] = Q[fluid, :, 1] = Q[fluid, :, 2] = m
    Q[fluid, :, 3:6] = 0.0
    return Q


def _acoustic_pair(m, mat, N, precision, **kw):
    o, s = make_pair(m, mat, N, precision=precision, cfl=0.5, acoustic_ocean=True, **kw)
    return o, s


def _run(m, mat, N, precision, steps=3, seed=41, macro=False, **kw):
    o, s = _acoustic_pair(m, mat, N, precision, **kw)
    fluid = mat[2] == 0.0
    Q0 = _isotropic(random_dofs((m.nt, s.B, 9), seed, N=N) * 1e-3, fluid)
    o.Q = Q0.copy()
    s.set_dofs(to_gpu_layout(Q0))
    ef, nxyz = s.gravity_faces()
    s.set_eta(eta_poly(nxyz[..., 0], nxyz[..., 1])[:, None, :])
    for e, f in np.argwhere(m.face_tag == syn.TAG_GRAVITY):
        o.eta[e, f] = eta_poly(o.face_x[e, f, :, 0], o.face_x[e, f, :, 1])
    for _ in range(steps):
        o.advance_macro() if macro else o.step_gts()
    s.advance(steps)
    eq = rel_l2(to_oracle_layout(s.get_dofs()), o.Q)
    ee = rel_l2(s.read_ssh()[:, 0, :], oracle_eta_at_nodes(o, ef, node_chi(N), N))
    return o, s, eq, ee


@pytest.mark.parametrize("N", [5, 4])
def test_acoustic_local_kernel_matches_the_oracle_3xtf32(N):
    """Ocean (two water layers) over crust, gravitational top, absorbing
    sides: the second water layer's 54 elements take the 4-quantity kernel
    (two tiles of 32, the second ragged), the crust the elastic one, the
    sea-surface layer the elastic one with its gravitational-face path;
    three steps."""
    from paper_2107_06640_gb300 import _lib
    m, mat = small_coupled()
    o, s, eq, ee = _run(m, mat, N, 2)
    assert eq <= 2e-5 and ee <= 1e-6, (eq, ee)
    _, launches = _lib.adg_profile(s.ctx, 1)
    assert launches[0] == 3  # local phase: elastic, acoustic and gravitational-face tensor-core launches
    assert int(s.info.tensor_core_updates_per_macro) == m.nt
    fluid_plain = int(np.sum((mat[2] == 0) & ~np.any(m.face_tag == syn.TAG_GRAVITY, axis=1)))
    assert int(s.info.acoustic_updates_per_macro) == fluid_plain


@pytest.mark.parametrize("N", [5, 4])
def test_acoustic_ocean_under_lts_3xtf32(N):
    m, mat = syn.workloads.coupled_box(nxy=4, n_water=3, n_crust=2, L=8e3, depth=4e3, water=1.5e3, grading=4.0)
    o, s, eq, ee = _run(m, mat, N, 2, steps=1, macro=True, max_clusters=4)
    assert s.info.n_clusters >= 2
    assert eq <= 2e-5 and ee <= 1e-6, (eq, ee)


def test_acoustic_ocean_fp64_projection_path():
    """FP64 (CUDA-core kernels): the projection at upload and the 9-quantity
    kernels on isotropic fluid data equal the oracle to 1e-10."""
    m, mat = small_coupled()
    o, s, eq, ee = _run(m, mat, 3, 0)
    assert eq <= 1e-10 and ee <= 1e-10, (eq, ee)


def test_upload_keeps_only_the_isotropic_fluid_stress():
    from paper_2107_06640_gb300 import Solver
    m, mat = small_coupled()
    rho, lam, mu = mat
    s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=3, cfl=0.5, precision=0, acoustic_ocean=True)
    Q = to_gpu_layout(random_dofs((m.nt, s.B, 9), 42, N=3))
    s.set_dofs(Q)
    got = to_oracle_layout(s.get_dofs())
    want = _isotropic(to_oracle_layout(Q), mu == 0.0)
    assert np.array_equal(got[mu > 0], want[mu > 0])
    assert np.allclose(got, want, rtol=0, atol=1e-15 * np.abs(want).max())


@pytest.mark.parametrize("N", [5, 4])
def test_acoustic_kernel_equals_the_nine_quantity_kernel(N):
    """On isotropic fluid data the 4-quantity local kernel gives the
    9-quantity tensor-core result to FP32 rounding."""
    from paper_2107_06640_gb300 import Solver
    m, mat = small_coupled()
    rho, lam, mu = mat
    B = (N + 1) * (N + 2) * (N + 3) // 6
    Q0 = to_gpu_layout(_isotropic(random_dofs((m.nt, B, 9), 43, N=N), mu == 0.0))
    out = []
    for ac in (False, True):
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N, cfl=0.5, precision=2, acoustic_ocean=ac)
        s.set_dofs(Q0)
        s.advance(3)
        out.append(s.get_dofs())
    assert rel_l2(out[1], out[0]) <= 5e-6, rel_l2(out[1], out[0])
