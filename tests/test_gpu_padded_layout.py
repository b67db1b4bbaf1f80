"""Lattices whose x-rows are padded in the device layout (Lx/4 = 5 or 6 sites
per x mod 4 group, stored in 8 positions): every kernel family against the
FP64 oracle, through the C ABI.  The layout is internal, so every result must
be what the oracle computes on the lexicographic field; unused positions are
never read into a result."""

import numpy as np
import pytest

import oracle as O
import synth
from tests.gpu_common import gpu_pipeline, max_abs, oracle_pipeline

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")

PADDED = [(20, 8, 4, 8), (24, 4, 8, 4)]


@pytest.fixture(scope="module")
def ctx():
    c = vs.vs_create(0)
    yield c
    vs.vs_destroy(c)


def test_plane_stride_includes_the_padding(ctx):
    for dims in PADDED:
        f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
        d = vs.vs_field_describe(f)
        vs.vs_field_destroy(f)
        assert d["n_sites"] == int(np.prod(dims))
        assert d["plane_stride"] == 32 * dims[1] * dims[2] * dims[3]


@pytest.mark.parametrize("dims", PADDED)
@pytest.mark.parametrize("eps", [-0.25, 1.0])
def test_fp64_smoothing_with_vp_matches_oracle(ctx, dims, eps):
    lab = synth.iid_labels(dims, 3)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, 4, 0.3, eps)
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, 4, 0.3, eps)
    assert max_abs(r["U"], Uo) < 1e-11
    assert [s["n_reject"] for s in r["stats"]] == list(rej)
    assert rej.sum() > 0 and r["check"]["n_label_diff"] == 0
    assert abs(r["action"] - O.action(dims, Uo)) < 1e-12


@pytest.mark.parametrize("dims", PADDED)
@pytest.mark.parametrize("storage", ["link18", "link12"])
@pytest.mark.parametrize("eps", [-0.25, 1.0])
def test_fp32_sweeps_on_a_general_field(ctx, dims, storage, eps):
    """A cooled Haar field (every matrix entry matters), VP off, annealed:
    each FP32 sweep from the oracle's FP64 field within 1e-6."""
    U = O.cool(dims, synth.haar_field(dims, 17), 3)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst = 0.0
    for _ in range(3):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth(f, 1, 0.06, eps, vortex_preserve=False, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U, _ = O.smooth(dims, U, None, 1, 0.06, eps=eps, vp=False)
        worst = max(worst, max_abs(Ug, U))
    assert vs.vs_field_count_nonfinite(f) == 0
    vs.vs_field_destroy(f)
    assert worst < 1e-6


@pytest.mark.parametrize("dims", PADDED)
def test_simultaneous_observables_and_vortex_check(ctx, dims):
    U = O.cool(dims, synth.haar_field(dims, 19), 2)
    Uo, _ = O.smooth(dims, U, None, 2, 0.08, eps=-0.25, schedule=O.SIMULTANEOUS, vp=False)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    lab = vs.vs_read_labels(f)
    vs.vs_smooth(f, 2, 0.08, -0.25, vortex_preserve=False, kind=vs.VS_SIMULTANEOUS)
    Ug = vs.vs_read_field(f)
    r = vs.vs_observables(f, per_site=True)
    chk = vs.vs_vortex_check(f)
    cur = vs.vs_current_labels(f)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, Uo) < 1e-11
    SR, Q, SRs, qs = O.observables(dims, Uo, per_site=True)
    S, Ss = O.action(dims, Uo, per_site=True)
    assert np.abs(r["S"] - Ss).max() < 1e-12 and np.abs(r["S_R"] - SRs).max() < 1e-12
    assert np.abs(r["q"] - qs).max() < 1e-12
    want = O.vortex_check(dims, Uo, lab, near_tol=1e-5)
    assert chk["n_label_diff"] == want["n_label_diff"] > 0
    assert chk["n_charge_diff"] == want["n_charge_diff"]
    assert abs(chk["min_margin"] - want["min_margin"]) < 1e-12
    assert np.array_equal(cur, O.labels(dims, Uo))


@pytest.mark.parametrize("dims", PADDED)
@pytest.mark.parametrize("method", ["stout", "aus", "ucp"])
def test_random_gauge_smoothers(ctx, dims, method):
    lab = synth.iid_labels(dims, 5)
    G = synth.random_gauge(dims, 47)
    U0 = O.gauge_transform(dims, O.centrifuge(dims, lab, 0.02, 1234), G)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_gauge_transform(f, G)
    if method == "stout":
        st = vs.vs_smooth(f, 3, 0.3, -0.25, vortex_preserve=True, stats=True)
        Uo, rej = O.smooth(dims, U0, lab, 3, 0.3, eps=-0.25, vp=True, gauge=G)
    elif method == "aus":
        st = vs.vs_smooth_aus(f, 3, 0.7, -0.25, vortex_preserve=True, stats=True)
        Uo, rej = O.aus(dims, U0, lab, 3, 0.7, eps=-0.25, vp=True, gauge=G)
    else:
        st = vs.vs_smooth_ape(f, 3, 0.7, -0.25, vortex_preserve=True, stats=True)
        Uo, rej = O.ape_ucp(dims, U0, lab, 3, 0.7, eps=-0.25, vp=True, gauge=G)
    Ug = vs.vs_read_field(f)
    chk = vs.vs_vortex_check(f)
    d = vs.vs_field_describe(f)
    noalloc = vs.vs_vortex_check_noalloc(d["links"], d["labels"], dims, vs.VS_FP64, vs.VS_LINK18,
                                         d["stream"], gauge=d["gauge"])
    vs.vs_field_destroy(f)
    assert [s["n_reject"] for s in st] == list(rej)
    assert max_abs(Ug, Uo) < 1e-10
    assert chk["n_label_diff"] == 0 and noalloc == chk


@pytest.mark.parametrize("dims", PADDED)
def test_runge_kutta_flow_and_checkpoint(ctx, dims):
    U = O.cool(dims, synth.haar_field(dims, 23), 2)
    Uo = O.flow_rk3(dims, U, 2, 0.02, eps=-0.25)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    vs.vs_flow_rk3(f, 2, 0.02, -0.25, reunit_every=0)
    Ug = vs.vs_read_field(f)
    links, labels, n = vs.vs_field_checkpoint(f)
    g = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_field_restore(g, links, labels, n)
    assert np.array_equal(vs.vs_read_field(g), Ug)
    assert np.array_equal(vs.vs_read_labels(g), vs.vs_read_labels(f))
    vs.vs_field_destroy(g)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, Uo) < 1e-11


def test_served_job_on_a_padded_lattice_equals_the_direct_run(ctx):
    dims = (20, 8, 4, 8)
    lab = synth.iid_labels(dims, 9)
    V = int(np.prod(dims))
    out = np.empty((4, V, 3, 3), dtype=np.complex128)
    sctx = vs.vs_create(0)
    j = vs.make_job(dims, 0.06, 25, labels=lab, omega=0.02, centrifuge_seed=1234, links_out=out)
    r = vs.vs_poll(sctx, vs.vs_submit(sctx, j), -1)
    vs.vs_destroy(sctx)
    assert r["status"] == vs.VS_OK
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_smooth(f, 25, 0.06, -0.25, reunit_every=10)
    U = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert np.array_equal(U, out)


class _DeviceArray:
    """A raw device buffer of the library, seen by torch through the CUDA
    array interface (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (n,), "typestr": typestr,
                                         "version": 3}


@pytest.mark.parametrize("dims", [(8, 4, 4, 8)] + PADDED)
@pytest.mark.parametrize("mode", ["fp32_18", "fp32_12", "fp64_18"])
def test_device_links_follow_the_documented_blocked_layout(ctx, dims, mode):
    """vs_field_desc documents the device layout for callers that read the
    links in place: direction mu at element mu NC P, blocks of 16 plane
    positions, each vector chunk of a block contiguous.  Every stored real of
    every link sits where that description puts it."""
    torch = pytest.importorskip("torch")
    precision = vs.VS_FP64 if mode == "fp64_18" else vs.VS_FP32
    storage = vs.VS_LINK12 if mode == "fp32_12" else vs.VS_LINK18
    U = synth.haar_field(dims, 31)
    f = vs.vs_field_create(ctx, dims, precision, storage)
    try:
        vs.vs_load_field(f, links=U)
        Ur = vs.vs_read_field(f)
        vs.vs_synchronize(f)
        d = vs.vs_field_describe(f)
        P, NC = d["plane_stride"], d["n_components"]
        assert P % 256 == 0
        typestr = "<f8" if precision == vs.VS_FP64 else "<f4"
        raw = torch.as_tensor(_DeviceArray(d["links"], 4 * NC * P, typestr), device="cuda").cpu().numpy()
    finally:
        vs.vs_field_destroy(f)
    V = int(np.prod(dims))
    Ur = Ur.reshape(4, V, 3, 3)
    Lx, Ly, Lz, Lt = dims
    for s in range(V):
        x = (s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz))
        i = vs.vs_layout_index(dims, x)
        b, k = divmod(i, 16)
        for mu in range(4):
            base = mu * NC * P + b * 16 * NC
            ent = Ur[mu, s].reshape(9)
            n_ent = 6 if NC == 12 else 9
            for e in range(n_ent):
                if precision == vs.VS_FP64:
                    off = base + 32 * e + 2 * k
                elif e < 8:
                    off = base + 64 * (e // 2) + 4 * k + 2 * (e % 2)
                else:
                    off = base + 256 + 2 * k
                assert raw[off] == ent[e].real and raw[off + 1] == ent[e].imag, (mu, x, e)
