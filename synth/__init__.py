"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module draws random numbers and random matrices only.  It contains none
of the smoothing method's arithmetic (no staples, no exponentials, no Z(3)
projection, no centrifuge): both sides of every parity check receive the same
inputs from here and compute everything else on their own.

Random streams come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated in counter mode:
value i of stream `seed` is the mix of ``seed + (i + 1) * 0x9E3779B97F4A7C15``.
"""

from .rng import splitmix64, uniform01, gaussian
from .fields import (
    lattice_volume,
    iid_labels,
    haar_su3,
    haar_field,
    random_gauge,
    serving_jobs,
)

__all__ = [
    "splitmix64",
    "uniform01",
    "gaussian",
    "lattice_volume",
    "iid_labels",
    "haar_su3",
    "haar_field",
    "random_gauge",
    "serving_jobs",
]
