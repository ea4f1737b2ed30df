"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws phantoms (speed-of-sound maps and initial-pressure maps),
sensor positions and measurement noise.  It holds none of the method's
arithmetic: no wave propagation, no interpolation, no gradient.  Every random
number the method consumes is drawn here and handed to both implementations
as an input.

The paper's phantoms and breast data are not available, so the workloads are
stand-ins that follow the value ranges of Sec. 4: speed of sound of soft tissue
(inclusions 1400-1650 m/s in a 1500 m/s background, cf. the 1430/1580 m/s
phantom of Sec. 4.1.1), additive Gaussian noise whose standard deviation is 1 %
of each data set's peak-to-peak value (Sec. 4.1.1), and point sensors.
"""
from .phantoms import (ellipse_phantom, blob_p0, vessel_p0, circle_sensors,
                       add_noise, noise_weights, workload, Workload, rng_for,
                       add_noise_torch, warmstart_sample, square_sensors, simple_phantom_c,
                       simple_phantom_p0, SIMPLE_L, SIMPLE_MARGIN, SIMPLE_TARGET)

__all__ = ["ellipse_phantom", "blob_p0", "vessel_p0", "circle_sensors",
           "add_noise", "noise_weights", "workload", "Workload", "rng_for",
           "add_noise_torch", "warmstart_sample", "square_sensors", "simple_phantom_c",
           "simple_phantom_p0", "SIMPLE_L", "SIMPLE_MARGIN", "SIMPLE_TARGET"]
