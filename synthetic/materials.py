"""Per-element material parameters (rho, lambda, mu) for the synthetic workloads.

Values are physical constants of the scenarios, not method arithmetic:
  * ELASTIC_UNIT: rho=1, lambda=2, mu=1 (plane-wave convergence case);
  * OCEAN: water, rho=1000 kg/m^3, c=1500 m/s, mu=0 (acoustic);
  * CRUST: rho=2700 kg/m^3, vp=6000 m/s, vs=3464 m/s (elastic).
"""

import numpy as np

ELASTIC_UNIT = (1.0, 2.0, 1.0)
OCEAN = (1000.0, 1000.0 * 1500.0 ** 2, 0.0)
_vs = 3464.0
_vp = 6000.0
CRUST = (2700.0, 2700.0 * (_vp ** 2 - 2 * _vs ** 2), 2700.0 * _vs ** 2)


def elastic_uniform(nt, rho_lam_mu=ELASTIC_UNIT):
    r, l, m = rho_lam_mu
    return (np.full(nt, r), np.full(nt, l), np.full(nt, m))


def ocean_crust(mesh, seafloor_z, water=OCEAN, solid=CRUST):
    """Water above `seafloor_z(x, y)` (decided on the element centroid), crust below."""
    c = mesh.centroids()
    wet = c[:, 2] > seafloor_z(c[:, 0], c[:, 1])
    rho = np.where(wet, water[0], solid[0])
    lam = np.where(wet, water[1], solid[1])
    mu = np.where(wet, water[2], solid[2])
    return rho, lam, mu
