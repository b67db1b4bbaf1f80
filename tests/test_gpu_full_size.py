"""Parity at the benchmark's full size (32^3 x 64), in the configuration bench.py
times (FP32 18-real and 12-real, over-improved, VP on, class launches of 524,288
threads), and at the largest lattice of the scaling sweep (48^3 x 96, 3.06 GB of
FP32 links, 2,654,208 threads per launch): the oracle recomputes sampled link
updates one by one.

After a few GPU sweeps from the cooled hot start, the field is read back; one
colour class is updated by the kernel (vs_subsweep); for a random sample of
the class's links the oracle computes exp(rho Q) U from the field read before
the launch (its own staple sum, generator and exponential) and the
vortex-preservation decision.  Links outside the class must be untouched.
"""

import numpy as np
import pytest

import oracle as O
from tests import lattice_np as L

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")

@pytest.mark.parametrize("DIMS,storage,tol,n_sample", [((32, 32, 32, 64), "link18", 2e-6, 3000),
                                                      ((32, 32, 32, 64), "link12", 3e-6, 3000),
                                                      ((48, 48, 48, 96), "link18", 2e-6, 1500)])
def test_sampled_class_update_at_full_size(DIMS, storage, tol, n_sample):
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, st)
    vs.vs_load_cooled(f, 3, 20)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_smooth(f, 3, 0.06, -0.25, vortex_preserve=True)
    lab = vs.vs_read_labels(f)
    U = vs.vs_read_field(f)                       # FP32 links, exactly as stored
    mu, col, rho = 1, 2, 0.06
    vs.vs_subsweep(f, mu, col, rho, -0.25, 1.0, True)
    U1 = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)

    V = int(np.prod(DIMS))
    changed = np.any(U1 != U, axis=(2, 3))
    assert not changed[[m for m in range(4) if m != mu]].any()
    c0, c1 = O.overimproved_coeffs(-0.25)
    rng = np.random.default_rng(11)
    sample = rng.choice(V, n_sample, replace=False)
    n_class = n_rej = 0
    for s in sample:
        x = np.unravel_index(s, DIMS[::-1])[::-1]
        if O.colour(DIMS, mu, x) != col:
            assert not changed[mu, s]
            continue
        n_class += 1
        S = O.staple_sum(DIMS, U, mu, x, c0, c1)
        Q = O.stout_generator(S @ L.dag(U[mu, s]))
        cand = O.expm(rho * Q) @ U[mu, s]
        accept = O.label_matrix(cand) == lab[mu, s]
        arg = np.angle(np.trace(cand))
        margin = min(abs(arg - np.pi / 3), abs(arg + np.pi / 3), np.pi - abs(arg))
        if margin < 1e-5:
            continue                               # within FP32 noise of a sector edge
        if accept:
            assert np.abs(U1[mu, s] - cand).max() < tol
        else:
            n_rej += 1
            assert np.array_equal(U1[mu, s], U[mu, s])
    assert n_class > n_sample // 6


def _margin(M):
    arg = np.angle(np.trace(M))
    return min(abs(arg - np.pi / 3), abs(arg + np.pi / 3), np.pi - abs(arg))


@pytest.mark.parametrize("projection,tol", [("maxretr", 1e-6), ("ucp", 3e-6)])
def test_sampled_aus_first_class_at_full_size(projection, tol):
    """One AUS sweep (alpha = 0.02, eps = -0.25, VP on; MaxReTr with 3 hits or
    unit circle projection, Sec. II.C) at 32^3 x 64 in FP32 18-real, as the
    benchmark times it.  The sweep's first class launch (mu = 0, colour 0)
    updates its links from the field read before the sweep and no later launch
    of the sweep touches them, so the oracle recomputes a sample of them one by
    one: the blocked matrix (1 - alpha) U + alpha/6 Sigma, its projection back
    to SU(3), and the vortex-preservation decision."""
    DIMS = (32, 32, 32, 64)
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_cooled(f, 3, 20)
    vs.vs_centrifuge(f, 0.02, 1234)
    lab = vs.vs_read_labels(f)
    U = vs.vs_read_field(f)
    alpha, eps = 0.02, -0.25
    if projection == "maxretr":
        vs.vs_smooth_aus(f, 1, alpha, eps, n_hits=3, reunit_every=0, vortex_preserve=True)
    else:
        vs.vs_smooth_ape(f, 1, alpha, eps, reunit_every=0, vortex_preserve=True)
    U1 = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)

    V = int(np.prod(DIMS))
    mu = 0
    c0, c1 = O.overimproved_coeffs(eps)
    rng = np.random.default_rng(12)
    n_class = n_rej = 0
    for s in rng.choice(V, 3000, replace=False):
        x = np.unravel_index(s, DIMS[::-1])[::-1]
        if O.colour(DIMS, mu, x) != 0:
            continue
        n_class += 1
        S = O.staple_sum(DIMS, U, mu, x, c0, c1)
        Vb = (1.0 - alpha) * U[mu, s] + (alpha / 6.0) * S
        if projection == "maxretr":
            cand = O.maxretr(U[mu, s], Vb, 3)
        else:
            cand = O.ucp(Vb)
            if cand is None:
                cand = U[mu, s]
        if _margin(cand) < 1e-5:
            continue                               # within FP32 noise of a sector edge
        if O.label_matrix(cand) == lab[mu, s]:
            assert np.abs(U1[mu, s] - cand).max() < tol
        else:
            n_rej += 1
            assert np.array_equal(U1[mu, s], U[mu, s])
    assert n_class > 500


def test_sampled_ape_simultaneous_at_full_size():
    """One sweep of APE smearing with unit circle projection (simultaneous:
    every link from the previous field; alpha = 0.5, eps = -0.25, VP off) at
    32^3 x 64 in FP32 18-real, as the benchmark times it: the oracle recomputes
    a sample of links in all four directions from the field read before the
    sweep.  1.5e-5, the per-sweep FP32 bound of the projection at this weight."""
    DIMS = (32, 32, 32, 64)
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, DIMS, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_cooled(f, 3, 20)
    vs.vs_centrifuge(f, 0.02, 1234)
    U = vs.vs_read_field(f)
    alpha, eps = 0.5, -0.25
    vs.vs_smooth_ape(f, 1, alpha, eps, schedule=vs.VS_SIMULTANEOUS, reunit_every=0,
                     vortex_preserve=False)
    U1 = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)

    V = int(np.prod(DIMS))
    c0, c1 = O.overimproved_coeffs(eps)
    rng = np.random.default_rng(13)
    for s in rng.choice(V, 1500, replace=False):
        x = np.unravel_index(s, DIMS[::-1])[::-1]
        for mu in range(4):
            S = O.staple_sum(DIMS, U, mu, x, c0, c1)
            cand = O.ucp((1.0 - alpha) * U[mu, s] + (alpha / 6.0) * S)
            if cand is None:
                cand = U[mu, s]
            assert np.abs(U1[mu, s] - cand).max() < 1.5e-5
