"""B300-native transient EM-thermal-mechanical package solver.

The compute path is libcosim.so (hand-written CUDA for sm_103a behind the C
ABI in include/cosim.h); ``cosim`` is its Python binding.
"""
from .cosim import (  # noqa: F401
    Context, CosimError, load,
    cosim_create, cosim_set_sources, cosim_em_steps, cosim_joule_accumulate, cosim_thermal_steps,
    cosim_stress_solve, cosim_stress_apply, cosim_read_fields, cosim_write_fields, cosim_query,
    cosim_last_error, cosim_destroy,
)
from . import cosim as capi  # noqa: F401
