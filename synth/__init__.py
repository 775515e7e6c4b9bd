"""Seeded synthetic inputs for the eRTIS energyscape chain.

This package only *makes inputs*: microphone geometries, steering-direction
sets, the emitted chirp, and int16 recordings of point-reflector scenes.  It
holds none of the processing arithmetic (matched filter, beamforming,
envelope); both the CUDA library's tests/benchmarks and the FP64 oracle
consume what it produces.
"""
from .scene import *  # noqa: F401,F403
from .pdm import *  # noqa: F401,F403
