"""FP64 CPU oracle for the ICON-type nonhydrostatic dynamical core.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (``paper_2608_21150_gb300``); both take their inputs from
``icon_inputs`` and derive every coefficient on their own.

The paper (Sec. 4.1) states the structure of one step -- dynamical substeps
made of a predictor and a corrector, each starting with the advective
tendencies, then the horizontal momentum update (pressure gradient and
advection), divergence damping in the corrector only, a vertically implicit
solve for w and the thermodynamic state, and one diffusion call per step
(Smagorinsky plus fourth-order background) -- but no formula of the
discretisation.  Every formula here is therefore a reading of an ICON-type
scheme on the triangular C-grid; the module docstrings name each one.

Everything is plain numpy in float64, vectorised over the horizontal index
only where that does not reorder the arithmetic of one point.  No ICON code
or data exist to compare against, so agreement with ICON itself cannot be
checked; every function of the oracle is pinned by invariants, closed forms
and convergence (tests/).
"""
from .params import DycoreParams  # noqa: F401
from .geometry import Geometry  # noqa: F401
from .vertical import VerticalGrid  # noqa: F401
from .dycore import Dycore  # noqa: F401
