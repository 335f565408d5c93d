"""Seeded synthetic event generator shared by the CUDA path, the oracle and the benchmark.

This package simulates a barrel tracking detector (helical charged tracks in a
uniform solenoid field crossing thin cylindrical layers, multiple scattering,
Gaussian hit smearing, uniform noise hits, layer misalignment) and builds
three-hit seeds with a geometric circle estimate.  It contains no step of the
Kalman-filter method itself: no covariance transport, no Jacobian, no gain, no
chi2, no candidate ranking and no duplicate removal.
"""
from .events import (  # noqa: F401
    CONFIGS,
    Batch,
    Detector,
    detector_for,
    make_batch,
    simulate_event,
)
