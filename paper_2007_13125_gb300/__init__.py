"""GB300-native parallel-in-time BDF-k / CQ-BDF-k solver (waveform relaxation with
kappa-circulant diagonalisation, Wu & Zhou, arXiv 2007.13125).

The compute path is the C-ABI library ``lib/libpint.so`` (hand-written sm_103a CUDA);
``pint`` is its thin ctypes binding. Nothing here falls back to a CPU implementation:
if the library is missing, every call raises.
"""
from . import pint  # noqa: F401
from .pint import (PintError, Plan, Server, lib, PINT_FP64, PINT_MIXED, PINT_FP32,  # noqa: F401
                   PINT_EIG_TRUNC_DFT, PINT_EIG_CLOSED_FORM)
