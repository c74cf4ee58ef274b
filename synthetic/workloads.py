"""Synthetic workloads shaped like the paper's scenarios (inputs only).

  * periodic unit cube, homogeneous elastic (rho=1, lambda=2, mu=1), P plane
    wave along x (amplitude 1e-3) - the small convergence case;
  * coupled ocean-crust box 100 x 100 x 40 km: a 2 km water layer (4 layers
    of 0.5 km) over elastic crust (35 layers), gravitational free surface on
    top, absorbing elsewhere, Gaussian seafloor velocity pulse (v_z, sigma
    5 km horizontally, 1 km vertically, 1 m/s); `scale` shrinks the hex
    counts for small test versions;
  * the same box with the sea floor warped by +-500 m sin bathymetry and a
    geometric grading of the element size (rate-2 LTS clusters);
  * ensemble of seafloor-uplift scenarios (sum of 8 Gaussian bumps).
Materials of the paper's Scenario A (crust 3775 kg/m^3, 7639.9/4229.4 m/s) are
available as CRUST_A.
"""

import numpy as np

from .materials import CRUST, OCEAN
from .mesh import (TAG_ABSORB, TAG_GRAVITY, TAG_PERIODIC, TAG_RIGID, graded_axis, kuhn_box,
                   unit_cube_periodic)

CRUST_A = (3775.0, 3775.0 * (7639.9 ** 2 - 2 * 4229.4 ** 2), 3775.0 * 4229.4 ** 2)
R_P = np.array([-2.0, -1, -1, 0, 0, 0, 1, 0, 0])  # right-going P eigenvector for rho=1, lam=2, mu=1


def plane_wave_field(t, amp=1e-3):
    """q = amp r sin(2 pi x - 4 pi t) (c_p = 2): closed-form physical field."""
    return lambda x: amp * R_P * np.sin(2 * np.pi * x[..., 0:1] - 4 * np.pi * t)


def plane_wave_case(n=8):
    m = unit_cube_periodic(n)
    nt = m.nt
    return m, (np.ones(nt), np.full(nt, 2.0), np.ones(nt))


def coupled_box(nxy=80, n_water=4, n_crust=35, L=100e3, depth=40e3, water=2e3, bathy=None,
                grading=1.0, rigid_bottom=False):
    """Ocean over crust.  bathy(x, y) -> seafloor z (default flat at -water)."""
    xs = np.linspace(0.0, L, nxy + 1)
    if grading != 1.0:
        half = nxy // 2
        left = graded_axis(0.0, L / 2, half, 1.0 / grading)
        right = graded_axis(L / 2, L, nxy - half, grading)
        xs = np.concatenate([left, right[1:]])
    ys = xs.copy()
    zs = np.concatenate([np.linspace(-depth, -water, n_crust + 1), np.linspace(-water, 0.0, n_water + 1)[1:]])
    warp = None
    if bathy is not None:
        zf = zs[n_crust]

        def warp(xyz, ijk):
            k = ijk[:, 2]
            sf = bathy(xyz[:, 0], xyz[:, 1])
            z = xyz[:, 2].copy()
            lo = k <= n_crust
            # crust nodes: stretch [-depth, zf] -> [-depth, sf]; water: [zf, 0] -> [sf, 0]
            z[lo] = -depth + (z[lo] + depth) * (sf[lo] + depth) / (zf + depth)
            hi = ~lo
            z[hi] = sf[hi] + (z[hi] - zf) * (0.0 - sf[hi]) / (0.0 - zf)
            xyz[:, 2] = z
            return xyz

    tags = {"x-": TAG_ABSORB, "x+": TAG_ABSORB, "y-": TAG_ABSORB, "y+": TAG_ABSORB,
            "z-": TAG_RIGID if rigid_bottom else TAG_ABSORB, "z+": TAG_GRAVITY}
    m = kuhn_box(xs, ys, zs, tags=tags, warp=warp)
    # water: the top n_water layers of hexes
    wet = m.hex_index[:, 2] >= n_crust
    rho = np.where(wet, OCEAN[0], CRUST[0])
    lam = np.where(wet, OCEAN[1], CRUST[1])
    mu = np.where(wet, OCEAN[2], CRUST[2])
    m.extra["seafloor"] = -water
    return m, (rho, lam, mu)


def seafloor_pulse(x0, y0, z0, sigma_h=5e3, sigma_v=1e3, amp=1.0):
    """v_z Gaussian pulse centred on the sea floor (physical field)."""
    def fn(x):
        out = np.zeros(x.shape[:-1] + (9,))
        r2 = ((x[..., 0] - x0) ** 2 + (x[..., 1] - y0) ** 2) / sigma_h ** 2 + (x[..., 2] - z0) ** 2 / sigma_v ** 2
        out[..., 8] = amp * np.exp(-0.5 * r2)
        return out
    return fn


def uplift_scenarios(S, L=100e3, seed=0):
    """S seeded sea-surface uplift fields eta0(x, y): sum of 8 Gaussian bumps,
    amplitude U[0.1, 2] m, width U[3, 10] km, centres uniform in the box."""
    out = []
    for s in range(S):
        rng = np.random.default_rng(seed + s)
        a = rng.uniform(0.1, 2.0, 8)
        w = rng.uniform(3e3, 10e3, 8)
        c = rng.uniform(0.1 * L, 0.9 * L, (8, 2))

        def eta0(x, y, a=a, w=w, c=c):
            r = np.zeros_like(x)
            for b in range(8):
                r += a[b] * np.exp(-((x - c[b, 0]) ** 2 + (y - c[b, 1]) ** 2) / (2 * w[b] ** 2))
            return r
        out.append(eta0)
    return out


def random_dofs(shape, seed, decay=0.5, N=None):
    """Seeded random modal coefficients (any basis layout); optional decay by
    basis index keeps higher modes smaller."""
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal(shape)
    if N is not None and decay:
        B = shape[-1]
        Q *= (1.0 + np.arange(B)) ** (-decay)
    return Q
