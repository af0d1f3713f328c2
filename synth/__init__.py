"""Seeded synthetic atmospheres shared by the CPU oracle and the CUDA path.

This package only draws random fields and lays out the model parameters of each
workload (opacity/source-function stratification, sparsity, line parameters,
quadrature directions).  It holds none of the formal-solution arithmetic: no
line-profile evaluation, no ray traversal, no mipmapping.  Both the oracle and
the CUDA path start from the float32 arrays returned here.
"""

from . import atom, mlp  # noqa: F401
from .atmospheres import (  # noqa: F401
    SEED_BASE,
    lognormal_field,
    smooth_uniform_field,
    directions,
    dense_exponential,
    sparse_line_atmosphere,
    gaussian_field,
    random_medium,
    dynamic_line_atmosphere,
    batch_specs,
    rc_directions,
)
from .atmospheres3 import directions3, sparse_line_atmosphere3, random_medium3  # noqa: F401
