"""Shared helpers of the GPU tests: seeded inputs and the two pipelines."""

import functools

import numpy as np

import oracle as O
import synth


@functools.lru_cache(maxsize=None)
def cooled_labels(dims, seed, n_cool=20):
    """The cooled hot-start workload input: Haar SU(3) links from `seed`,
    n_cool sweeps of oracle MaxReTr cooling, each link projected to Z(3)
    (built by the oracle, cached on disk)."""
    return O.cooled_labels(dims, seed, n_cool)


def oracle_pipeline(dims, labels, omega, cseed, n_sweeps, rho, eps, vp=True,
                    schedule=O.ANNEALED):
    U0 = O.centrifuge(dims, labels, omega, cseed) if omega is not None else O.links_from_labels(dims, labels)
    U, rej = O.smooth(dims, U0, labels, n_sweeps, rho, eps=eps, vp=vp, schedule=schedule)
    return U, rej


def gpu_pipeline(vs, ctx, dims, labels, omega, cseed, n_sweeps, rho, eps, vp=True,
                 precision=None, storage=None, reunit_every=10, kind=None):
    precision = vs.VS_FP64 if precision is None else precision
    storage = vs.VS_LINK18 if storage is None else storage
    kind = vs.VS_ANNEALED if kind is None else kind
    f = vs.vs_field_create(ctx, dims, precision, storage)
    try:
        vs.vs_load_field(f, labels=labels)
        if omega is not None:
            vs.vs_centrifuge(f, omega, cseed)
        stats = vs.vs_smooth(f, n_sweeps, rho, eps, vortex_preserve=vp, stats=True,
                             reunit_every=reunit_every, kind=kind)
        assert vs.vs_field_count_nonfinite(f) == 0
        U = vs.vs_read_field(f)
        cur = vs.vs_current_labels(f)
        S = vs.vs_action(f)
        chk = vs.vs_vortex_check(f)
    finally:
        vs.vs_field_destroy(f)
    return dict(U=U, stats=stats, labels=cur, action=S, check=chk)


def max_abs(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())
