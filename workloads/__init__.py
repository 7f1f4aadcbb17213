"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only *describes* problems: voxel material IDs, per-axis cell
sizes, material constants, boundary choices and current-source waveforms.
It performs none of the solver's arithmetic (no field update, no
coefficient averaging, no time-step rule), so the oracle and the CUDA path
both consume it without sharing any of the method.
"""
from .package import (  # noqa: F401
    Material, Source, Problem,
    COPPER, DIELECTRIC, SILICON, UNDERFILL,
    BC_PEC, BC_PMC, BC_CPML,
    tiny_package, layered_package, full_package, uniform_box, crop, paper_setup_package,
)
from .waveforms import (  # noqa: F401
    GaussianDerivative, PRBSBurst, Sampled, Jitter, Ricker, Sine, GaussianPulseTrain, Scaled,
)
