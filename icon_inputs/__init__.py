"""Seeded, synthetic inputs shared by the FP64 oracle and the CUDA dycore.

This package holds only input generation: the icosahedral RnBm grid (raw
connectivity and coordinates, as an ICON grid file would provide them), the
stretched vertical grid, a Gaussian mountain with its terrain-following
half-level heights, and analytic initial states.  It contains none of the
dynamical core's discretisation: no operator weights, no metric factors, no
reference state.  Both the oracle (``oracle/``) and the GPU library take their
inputs from here and derive everything else on their own.
"""
from .grid import make_grid, Grid  # noqa: F401
from .vertical import make_vct  # noqa: F401
from .state import (jw_type_state, gaussian_perturbation_centre,  # noqa: F401
                    sample_perturbation_centre, CONSTANTS)
from .perturb import perturb_state  # noqa: F401
from .terrain import mountain_height, terrain_following_z  # noqa: F401
