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

import functools

import numpy as np
import pytest

import oracle as O
from tests import lattice_np as L
from tests.gpu_common import cooled_labels

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
            continue                               # within the FP32 error band of a sector edge
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


# Every link at full size: the field is an 8^4 field repeated periodically over
# 32^3 x 64.  The colour classes c_mu(x) repeat with period 4 in every direction
# and the schedules treat all sites alike, so the exact result is the oracle's
# 8^4 result repeated; the kernels see 32^3 x 64 with the benchmark's launch
# shapes and distinct coordinates everywhere, and a neighbour index that went
# wrong anywhere would break the repetition.
TILE = (8, 8, 8, 8)
FULL = (32, 32, 32, 64)
REPS = tuple(F // T for F, T in zip(FULL, TILE))


def _tile(a):
    inner = a.shape[2:]
    t = a.reshape((4,) + TILE[::-1] + inner)
    return np.tile(t, (1,) + REPS[::-1] + (1,) * len(inner)).reshape((4, -1) + inner)


def _first_tile_if_periodic(a):
    """Checks bit for bit that a full-size array repeats the 8^4 pattern and
    returns the first copy, as (4, 4096, ...)."""
    inner = a.shape[2:]
    shp = (4,)
    for R, T in zip(REPS[::-1], TILE[::-1]):
        shp += (R, T)
    b = a.reshape(shp + inner)
    first = b[:, :1, :, :1, :, :1, :, :1]
    for mu in range(4):
        assert (b[mu] == first[mu]).all(), "direction %d breaks the period" % mu
    return first.reshape((4, -1) + inner)


@functools.lru_cache(maxsize=None)
def _tile_start():
    """Cooled 8^4 labels, centrifuged, then 12 oracle sweeps of annealed
    over-improved VP smoothing: the sweeps where rejections set in (337 of
    16,384 candidates rejected in the next sweep)."""
    lab = cooled_labels(TILE, 2)
    U = O.centrifuge(TILE, lab, 0.02, 1234)
    U, _ = O.smooth(TILE, U, lab, 12, 0.06, eps=-0.25, vp=True)
    return lab, U


def _split_links(Ug, Uo, U0, edge):
    """Links decided differently (accepted on one side, rejected on the
    other): the accepted candidate must lie within `edge` rad of a sector edge."""
    d = np.abs(Ug - Uo).max(axis=(2, 3))
    split = d > 1e-4
    for mu, s in zip(*np.nonzero(split)):
        acc = Ug[mu, s] if np.abs(Ug[mu, s] - U0[mu, s]).max() > 1e-5 else Uo[mu, s]
        assert _margin(acc) < edge, (mu, s, _margin(acc))
    return d, split


PATHS = [
    # name, precision, storage, tolerance
    ("stout", vs.VS_FP32, vs.VS_LINK18, 1e-6),
    ("stout", vs.VS_FP32, vs.VS_LINK12, 1e-6),
    ("stout", vs.VS_FP64, vs.VS_LINK18, 1e-12),
    ("stout_simultaneous", vs.VS_FP32, vs.VS_LINK18, 1e-6),
    ("aus_maxretr", vs.VS_FP32, vs.VS_LINK18, 1e-6),
    ("aus_ucp", vs.VS_FP32, vs.VS_LINK18, 3e-6),
    ("ape_simultaneous", vs.VS_FP32, vs.VS_LINK18, 1.5e-5),
    ("flow_rk3", vs.VS_FP32, vs.VS_LINK18, 2e-6),
]


@pytest.mark.parametrize("path,prec,storage,tol", PATHS,
                         ids=["%s-%s-%s" % (p[0], "fp32" if p[1] == vs.VS_FP32 else "fp64",
                                             "18" if p[2] == vs.VS_LINK18 else "12") for p in PATHS])
def test_every_link_of_a_periodic_field_at_full_size(path, prec, storage, tol):
    """One sweep (RK3: one step) of each path on the periodic 32^3 x 64 field,
    from the same starting field on both sides: the GPU result repeats bit for
    bit and its first copy matches the oracle's 8^4 sweep link by link, with
    the same VP decisions except candidates at a sector edge (FP32)."""
    lab, U0 = _tile_start()
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, FULL, prec, storage)
    vs.vs_load_field(f, links=_tile(U0))
    assert np.array_equal(_first_tile_if_periodic(vs.vs_read_labels(f)), lab)
    eps, rho, alpha = -0.25, 0.06, 0.02
    n_undec = None                        # undecidable links the GPU counted (VP paths)
    if path == "stout":
        st = vs.vs_smooth(f, 1, rho, eps, vortex_preserve=True, reunit_every=0, stats=True)
        Uo, rej = O.smooth(TILE, U0, lab, 1, rho, eps=eps, vp=True)
        n_undec = st[0]["n_undecidable"]
    elif path == "stout_simultaneous":
        st = vs.vs_smooth(f, 1, rho, eps, vortex_preserve=True, reunit_every=0, kind=vs.VS_SIMULTANEOUS,
                          stats=True)
        Uo, rej = O.smooth(TILE, U0, lab, 1, rho, eps=eps, vp=True, schedule=O.SIMULTANEOUS)
        n_undec = st[0]["n_undecidable"]
    elif path == "aus_maxretr":
        st = vs.vs_smooth_aus(f, 1, alpha, eps, n_hits=3, reunit_every=0, vortex_preserve=True, stats=True)
        Uo, rej = O.aus(TILE, U0, lab, 1, alpha, eps=eps, n_hits=3, vp=True)
        n_undec = st[0]["n_undecidable"]
    elif path == "aus_ucp":
        st = vs.vs_smooth_ape(f, 1, alpha, eps, reunit_every=0, vortex_preserve=True, stats=True)
        Uo, rej = O.ape_ucp(TILE, U0, lab, 1, alpha, eps=eps, vp=True)
        n_undec = st[0]["n_undecidable"]
    elif path == "ape_simultaneous":
        vs.vs_smooth_ape(f, 1, 0.5, eps, schedule=vs.VS_SIMULTANEOUS, reunit_every=0,
                         vortex_preserve=False)
        Uo, rej = O.ape_ucp(TILE, U0, None, 1, 0.5, eps=eps, schedule="simultaneous", vp=False)
    else:
        vs.vs_flow_rk3(f, 1, 0.02, 1.0, reunit_every=0)
        Uo, rej = O.flow_rk3(TILE, U0, 1, 0.02, eps=1.0), None
    assert vs.vs_field_count_nonfinite(f) == 0
    Ug = _first_tile_if_periodic(vs.vs_read_field(f))
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)

    d, split = _split_links(Ug, Uo, U0, 1e-5 if prec == vs.VS_FP32 else 1e-10)
    if prec == vs.VS_FP64 or n_undec is None:
        assert int(split.sum()) == 0
    else:
        # decisions equal the oracle's except for links counted undecidable
        # (each of the 512 copies of the 8^4 tile counts its own)
        assert int(split.sum()) * int(np.prod(REPS)) <= n_undec
    assert float(d[~split].max()) < tol
    if rej is not None and path != "ape_simultaneous":
        assert int(rej.sum()) > 0                  # the sweep exercises rejections
