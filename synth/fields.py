"""Seeded lattice inputs: label fields, Haar SU(3) links, gauge transforms, job mixes.

Layouts (shared convention of the whole project):
  * lattice extents ``dims = (Lx, Ly, Lz, Lt)``; site index is lexicographic
    with x fastest: s = x + Lx*(y + Ly*(z + Lz*t)).
  * labels: int8 array [4][V] (direction mu major), values in {-1, 0, +1}.
  * links: complex128 array [4][V][3][3] (row-major 3x3), which is the same
    bytes as float64 [4][V][3][3][2].
"""

import numpy as np

from .rng import uniform01, gaussian


def lattice_volume(dims):
    v = 1
    for L in dims:
        v *= int(L)
    return v


def iid_labels(dims, seed, p0=0.7, p_plus=0.15):
    """Independent Z(3) labels: P(0)=p0, P(+1)=p_plus, P(-1)=1-p0-p_plus.

    The 4^4 pure-vortex workload draws n iid with P(0)=0.7, P(+-1)=0.15.
    """
    V = lattice_volume(dims)
    u = uniform01(seed, np.arange(4 * V, dtype=np.uint64))
    lab = np.full(4 * V, -1, dtype=np.int8)
    lab[u < p0 + p_plus] = 1
    lab[u < p0] = 0
    return lab.reshape(4, V)


def haar_su3(n, seed, offset=0):
    """n Haar-distributed SU(3) matrices, complex128 [n][3][3].

    Random-matrix recipe (Mezzadri, Notices AMS 54, 2007): QR of a complex
    Ginibre matrix with the phases of diag(R) moved into Q gives Haar U(3);
    dividing by the principal cube root of the determinant lands in SU(3).
    Matrix m consumes Gaussian stream values offset + 18m ... offset + 18m + 17.
    """
    g = gaussian(seed, 18 * n, offset=offset).reshape(n, 3, 3, 2)
    z = (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    q = q / np.exp(1j * np.angle(det) / 3.0)[:, None, None]
    return np.ascontiguousarray(q)


def haar_field(dims, seed, chunk=1 << 18, workers=None):
    """A hot-start gauge field: every link an independent Haar SU(3) matrix.
    Chunks of the counter-mode stream are drawn on a thread pool (numpy's
    batched QR releases the interpreter lock); the result does not depend on
    the chunking or the number of threads."""
    import concurrent.futures as cf
    import os
    V = lattice_volume(dims)
    n = 4 * V
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def fill(a):
        b = min(n, a + chunk)
        out[a:b] = haar_su3(b - a, seed, offset=18 * a)

    starts = range(0, n, chunk)
    if len(starts) == 1:
        fill(0)
    else:
        with cf.ThreadPoolExecutor(max_workers=workers or min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    return out.reshape(4, V, 3, 3)


def random_gauge(dims, seed):
    """A random gauge transformation G(x): one Haar SU(3) matrix per site."""
    V = lattice_volume(dims)
    return haar_su3(V, seed).reshape(V, 3, 3)


_SERVE_SHAPES = ((8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (24, 24, 24, 48))


def serving_jobs(n_jobs=64, seed=99, rate_hz=1.0, first_job_seed=100,
                 shapes=_SERVE_SHAPES, rho_range=(0.04, 0.1),
                 sweep_range=(50, 300)):
    """A Poisson-arrival job mix for the serving workload.

    Returns a list of dicts with keys: arrival_s, dims, seed, rho, n_sweeps.
    Inter-arrival gaps are exponential with the given rate; shape, rho and
    sweep count are uniform over the stated sets and ranges.
    """
    k = np.arange(n_jobs, dtype=np.uint64) * np.uint64(4)
    gap = -np.log(1.0 - uniform01(seed, k)) / rate_hz
    shp = np.minimum((uniform01(seed, k + np.uint64(1)) * len(shapes)).astype(int),
                     len(shapes) - 1)
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * uniform01(seed, k + np.uint64(2))
    ns = sweep_range[0] + np.minimum(
        (uniform01(seed, k + np.uint64(3)) * (sweep_range[1] - sweep_range[0] + 1)).astype(int),
        sweep_range[1] - sweep_range[0])
    t = np.cumsum(gap)
    jobs = []
    for i in range(n_jobs):
        jobs.append(dict(arrival_s=float(t[i]), dims=tuple(shapes[shp[i]]),
                         seed=first_job_seed + i, rho=float(rho[i]),
                         n_sweeps=int(ns[i])))
    return jobs
