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


def fault_box(nx=8, ny=4, nz=4, dz=1e3, dip_deg=15.0, width=None, ocean_layers=0, water=2e3,
              material=CRUST):
    """Megathrust-style box: a Kuhn grid whose hexes are stretched so that the
    index diagonal plane i - k = 0 dips `dip_deg` (dx = dz / tan(dip)); its
    faces between j in [0, width] become a planar fault (tag 5).  Optionally
    `ocean_layers` of water (OCEAN material, gravitational top) sit on top of
    the crust layers.  Sides absorbing."""
    dx = dz / np.tan(np.radians(dip_deg))
    xs = np.arange(nx + 1) * dx
    ys = np.arange(ny + 1) * dx
    if ocean_layers:
        zs = np.concatenate([np.linspace(-water - nz * dz, -water, nz + 1),
                             np.linspace(-water, 0.0, ocean_layers + 1)[1:]])
    else:
        zs = np.linspace(-nz * dz, 0.0, nz + 1)
    width = ny if width is None else width
    tags = {"x-": TAG_ABSORB, "x+": TAG_ABSORB, "y-": TAG_ABSORB, "y+": TAG_ABSORB, "z-": TAG_ABSORB,
            "z+": TAG_GRAVITY if ocean_layers else TAG_ABSORB}
    m = kuhn_box(xs, ys, zs, tags=tags, fault=dict(c=0, jrange=(0, width), krange=(0, nz)))
    wet = m.hex_index[:, 2] >= nz
    rho = np.where(wet, OCEAN[0], material[0])
    lam = np.where(wet, OCEAN[1], material[1])
    mu = np.where(wet, OCEAN[2], material[2])
    return m, (rho, lam, mu)


def rs_fault_params(node_xyz, normal, seed=0, patch_center=None, patch_radius=3e3, sn0=-40e6,
                    tau_ratio=0.55, patch_ratio=0.85, noise=0.05, psi0=0.6, V_init=1e-12):
    """Per-node rate-and-state parameters [nff, Bf, 13] (a, b, L, f0, V0, f_w,
    V_w, sigma_n0, tau0_xyz, psi_init, V_init): a, b, L, f0, V0 uniform with
    seeded +-noise relative perturbations; f_w = 0.1, V_w = 0.1 m/s; uniform
    normal stress sn0 (compression negative); shear prestress along the
    up-dip direction with |tau0| = tau_ratio |sn0|, raised to patch_ratio |sn0|
    inside a circular nucleation patch (overstress)."""
    rng = np.random.default_rng(seed)
    nff, Bf, _ = node_xyz.shape
    base = dict(a=0.01, b=0.014, L=0.2, f0=0.6, V0=1e-6)
    out = np.zeros((nff, Bf, 13))
    for k, (name, v) in enumerate(base.items()):
        out[..., k] = v * (1.0 + noise * rng.uniform(-1.0, 1.0, (nff, Bf)))
    out[..., 5] = 0.1
    out[..., 6] = 0.1
    out[..., 7] = sn0
    up = np.array([0.0, 0.0, 1.0])
    d = up[None, :] - np.sum(normal * up, 1, keepdims=True) * normal
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-30)
    if patch_center is None:
        patch_center = node_xyz.reshape(-1, 3).mean(0)
    r = np.linalg.norm(node_xyz - np.asarray(patch_center)[None, None, :], axis=2)
    mag = np.where(r < patch_radius, patch_ratio, tau_ratio) * abs(sn0)
    out[..., 8:11] = mag[..., None] * d[:, None, :]
    out[..., 11] = psi0
    out[..., 12] = V_init
    return out


def lsw_fault_params(node_xyz, normal, seed=0, patch_center=None, patch_radius=3e3, sn0=-40e6, mu_s=0.6,
                     mu_d=0.4, Dc=0.5, tau_ratio=0.48, patch_ratio=0.62, noise=0.05, C_top=2e6, taper=2e3):
    """Per-node linear slip-weakening parameters [nff, Bf, 13] (mu_s, mu_d,
    D_c, cohesion C, three unused, sigma_n0, tau0_xyz, psi_init = 0,
    V_init = 0): mu_s, mu_d, D_c with seeded +-noise relative perturbations
    (mu_d kept <= mu_s); uniform normal stress sn0 (compression negative);
    shear prestress along the up-dip direction with |tau0| = tau_ratio |sn0|,
    between the dynamic and static strengths, raised to patch_ratio |sn0|
    (above the static strength) in a circular nucleation patch; cohesion
    rising linearly from 0 at depth `taper` below the fault's top edge to C_top
    there, so the fault is stronger toward the seafloor (Sec. 5, Scenario A)."""
    rng = np.random.default_rng(seed)
    nff, Bf, _ = node_xyz.shape
    out = np.zeros((nff, Bf, 13))
    for k, v in enumerate((mu_s, mu_d, Dc)):
        out[..., k] = v * (1.0 + noise * rng.uniform(-1.0, 1.0, (nff, Bf)))
    out[..., 1] = np.minimum(out[..., 1], out[..., 0])
    z = node_xyz[..., 2]
    out[..., 3] = C_top * np.clip(1.0 - (z.max() - z) / taper, 0.0, 1.0)
    out[..., 7] = sn0
    up = np.array([0.0, 0.0, 1.0])
    d = up[None, :] - np.sum(normal * up, 1, keepdims=True) * normal
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-30)
    if patch_center is None:
        patch_center = node_xyz.reshape(-1, 3).mean(0)
    r = np.linalg.norm(node_xyz - np.asarray(patch_center)[None, None, :], axis=2)
    mag = np.where(r < patch_radius, patch_ratio, tau_ratio) * abs(sn0)
    out[..., 8:11] = mag[..., None] * d[:, None, :]
    return out


def random_dofs(shape, seed, decay=0.5, N=None):
    """Seeded standard-normal modal coefficients.  With N given, the axis of
    length B_N = (N+1)(N+2)(N+3)/6 is the basis axis (either dofs layout,
    [..., B, 9] or [..., 9, B]; the last such axis if several match) and mode l
    is scaled by (1 + l)^-decay, so that higher modes are smaller."""
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal(shape)
    if N is not None and decay:
        B = (N + 1) * (N + 2) * (N + 3) // 6
        axes = [i for i, n in enumerate(shape) if n == B]
        if not axes:
            raise ValueError(f"random_dofs: no axis of length B = {B} in {shape}")
        w = (1.0 + np.arange(B)) ** (-decay)
        Q *= w.reshape([-1 if i == axes[-1] else 1 for i in range(len(shape))])
    return Q
