"""The oracle against values the paper prints (fixtures in tests/golden/,
each with its citation): the wave speeds of the Scenario-A materials as
eigenvalues of the oracle's Jacobians (Sec. 4.4: the largest is the P-wave
speed), and the degrees of freedom per element of the order-6 meshes."""

import os

import numpy as np
import pytest

from oracle import basis as ob
from oracle import physics as ph

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = float(v)
    return out


def _speeds(rho, lam, mu, n):
    """Absolute eigenvalues of the Jacobian in direction n, n_x A + n_y B + n_z C."""
    A = ph.jacobians(rho, lam, mu)
    An = np.einsum("d,dij->ij", n, A)
    return np.sort(np.abs(np.linalg.eigvals(An).real))


@pytest.mark.parametrize("n", [(1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.48, -0.6, 0.64)])
def test_scenario_a_speeds_are_the_jacobian_eigenvalues(n):
    g = _load("scenario_a_materials.txt")
    n = np.asarray(n) / np.linalg.norm(n)
    ev = _speeds(g["solid_rho"], g["solid_lambda"], g["solid_mu"], n)
    # +-c_p, +-c_s twice (two polarisations), and three zero speeds
    assert ev[7:] == pytest.approx([g["solid_cp"]] * 2, rel=1e-13)
    assert ev[3:7] == pytest.approx([g["solid_cs"]] * 4, rel=1e-13)
    assert np.max(ev[:3]) < 1e-6
    # impedances of the same material
    Zp, Zs = ph.impedances(g["solid_rho"], g["solid_lambda"], g["solid_mu"])
    assert Zp == pytest.approx(g["solid_rho"] * g["solid_cp"], rel=1e-13)
    assert Zs == pytest.approx(g["solid_rho"] * g["solid_cs"], rel=1e-13)


def test_ocean_speed_is_the_acoustic_eigenvalue():
    g = _load("scenario_a_materials.txt")
    ev = _speeds(g["ocean_rho"], g["ocean_K"], 0.0, np.array([0.0, 0.6, 0.8]))
    # +-c and seven zero speeds (mu = 0: no shear waves); the zero eigenvalue is
    # defective (a Jordan block), so it is computed only to about sqrt(eps)
    assert ev[7:] == pytest.approx([g["ocean_cp"]] * 2, rel=1e-14)
    assert np.max(ev[:7]) < 1e-7 * g["ocean_cp"]


def test_order_six_meshes_have_nine_times_56_dofs_per_element():
    g = _load("mesh_dofs.txt")
    N = int(g["order"]) - 1
    per = 9 * ob.n_basis(N)
    assert per == 504
    assert per * g["mesh_L_elements"] == pytest.approx(g["mesh_L_dofs"], rel=0.01)
    assert per * g["mesh_M_elements"] == pytest.approx(g["mesh_M_dofs"], rel=0.05)
