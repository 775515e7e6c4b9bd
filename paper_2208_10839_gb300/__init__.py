"""eRTIS in-air imaging sonar energyscape chain on one GB300 (sm_103a).

Matched filter -> delay-and-sum beamforming -> envelope/low-pass/subsample,
as hand-written CUDA kernels behind a C ABI (include/rtis.h, librtis.so).
This package is the thin Python binding of that ABI.
"""
from . import _native  # noqa: F401
from ._native import RtisError, lib  # noqa: F401
from .calibrate import Calibrator  # noqa: F401
from .plan import Batch, FdGemm, Plan, energyscape, pdm_demodulate, process_batch  # noqa: F401

__all__ = ["Plan", "Batch", "Calibrator", "FdGemm", "energyscape", "pdm_demodulate", "process_batch", "RtisError",
           "lib"]
