"""Cooled hot-start labels built by the oracle, cached on disk.

TEST INFRASTRUCTURE ONLY (the tests, the smoke check and the CPU-baseline and
reference legs of the benchmark).  The synthetic stand-in for a gauge-fixed
ensemble member: every link an independent Haar SU(3) matrix (synth), then
n_cool sweeps of the oracle's annealed MaxReTr cooling (Sec. III: alpha = 1,
plaquette staples, three passes over the SU(2) subgroups), then each link's
Z(3) label (Sec. I, Eq. centre_element).  Labels are cached as .npy files
keyed by the extents, the seed and the number of cooling sweeps, so a
32^3 x 64 input (a few minutes of oracle cooling) is built once per machine.
"""

import os

import numpy as np

from . import oracle as _O

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def cooled_labels(dims, seed, n_cool=20, cache=True):
    """int8 [4][V] labels of the cooled hot start of `dims` from `seed`."""
    import synth
    dims = tuple(int(d) for d in dims)
    path = os.path.join(_CACHE, "cooled_%s_seed%d_cool%d.npy" % ("x".join(map(str, dims)), seed, n_cool))
    if cache and os.path.exists(path):
        lab = np.load(path)
        if lab.shape == (4, int(np.prod(dims))) and lab.dtype == np.int8:
            return lab
    U = synth.haar_field(dims, seed)
    U = _O.cool(dims, U, n_cool)
    lab = _O.labels(dims, U)
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + ".%d.tmp.npy" % os.getpid()
        np.save(tmp, lab)
        os.replace(tmp, path)
    return lab
