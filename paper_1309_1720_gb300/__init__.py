"""GB300-native FP64 stepper for 2-D cardiac reaction-diffusion models.

Implements the fused explicit time step of Marcotte & Grigoriev,
"Implementation of PDE models of cardiac dynamics on GPUs using OpenCL"
(diffusion stencil with no-flux or periodic ghost points, FitzHugh-Nagumo and
Bueno-Orovio-Cherry-Fenton local terms, explicit Euler / Heun / RK4 and the
Rush-Larsen / implicit-Euler gate integrators) as
hand-written CUDA kernels for sm_103a behind a C ABI
(include/cardiac_gb300.h).  This package is the Python binding.
"""
from .api import (  # noqa: F401
    ABI_VERSION, BOCF, CLAMP, DIFFUSION, EULER, FHN, HEUN, IMPLICIT_EULER, KARMA, MIRROR, PERIODIC, RK4,
    RUSH_LARSEN, STENCIL5, STENCIL9, FLAG_ALLOW_UNSTABLE, FLAG_PER_STAGE_LAUNCH, FLAG_NEIGHBOR_SYNC,
    FLAG_TANH_AS_HK, FLAG_TEST_STUCK_BARRIER,
    Checkpoints, DEV_NONFINITE, DEV_TIMEOUT, Linearization, Plan, Problem, default_params, n_fields, n_params,
)
from ._lib import CGError  # noqa: F401
