"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only builds *inputs*: tetrahedral meshes (vertex coordinates,
connectivity, boundary tags, periodic partners), per-element material
parameters, seeded random numbers and point-wise physical fields given in
closed form.  It contains none of the ADER-DG method's arithmetic (no basis,
no quadrature, no projection, no flux), so the oracle and the CUDA path can
both consume it without sharing any part of the method.
"""

from .mesh import (  # noqa: F401
    TAG_INTERIOR, TAG_FREE, TAG_GRAVITY, TAG_ABSORB, TAG_PERIODIC, TAG_FAULT,
    TAG_RIGID, Mesh, kuhn_box, graded_axis, unit_cube_periodic,
)
from .materials import (  # noqa: F401
    elastic_uniform, ocean_crust, ELASTIC_UNIT, OCEAN, CRUST,
)
