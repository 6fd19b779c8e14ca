"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module draws random numbers and states workload parameters; it holds none
of the wavefront-sensor arithmetic.  Every random number the simulation needs
(phase-screen spectral noise, subharmonic noise, wind directions, learned-model
initialisation draws, training-sample Fried parameters) is drawn here from
NumPy's PCG64 generator and handed to both implementations as an input, so the
two sides never need a common random generator.

The paper uses proprietary calibration data and no public dataset (Sect. 8;
"Code and Data Availability"), so every workload here is synthetic and shaped
like the systems of Sect. 6, Tab. 2.
"""
from .workloads import (  # noqa: F401
    Layer, Source, Pupil, PwfsGeom, ShGeom, Sensor, Workload, WORKLOADS,
    workload, ARCSEC,
)
from .noise import (  # noqa: F401
    screen_noise, subharmonic_noise, uniform_draws, normal_draws,
)
