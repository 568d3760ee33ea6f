"""Seeded synthetic grid instances for contingency-constrained DC OPF.

This package only draws data: topologies, device parameters, load profiles
and outage lists.  It contains none of the message-passing arithmetic, so both
the FP64 oracle and the CUDA path can be fed from it without sharing any of
the method's code.
"""
from .cases import CONFIGS, make_case, case_dims, scale_case  # noqa: F401
