"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds workload parameters and seeded random draws only; it contains
none of the method's arithmetic (no cosmology, no mesh or lensing operations),
so that the oracle and the CUDA path stay independent while still being driven
by identical inputs.
"""
from .configs import WORKLOADS, workload, cosmology_params  # noqa: F401
from .noise import white_noise, serving_arrivals  # noqa: F401
