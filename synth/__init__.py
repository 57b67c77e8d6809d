"""Seeded synthetic inputs for the map-making solver.

This package only *synthesises* data: scan geometry (pixel index and
polarisation angle per sample), stationary-interval boundaries, noise
parameters, a random sky, and the timestream d = A z + n of the data model
(Section 3, Eqs. 1-2).  It contains none of the solver's arithmetic (no
pointing operators, no noise filters, no FFT convolution, no PCG).  Both the
CPU oracle and the GPU library consume what it produces; neither imports the
other.  ``boresight`` produces compressed pointing (nodes and detector
offsets, with the signal at the scan's true positions) and ``extended`` the
extra columns' indices and signals (offsets, chopper bins, half-wave plate).
"""

from .flat import Problem, make_config, make_flat_problem, config_spec  # noqa: F401
from .allsky import make_allsky_problem  # noqa: F401
