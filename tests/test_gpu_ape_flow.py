"""GPU parity of the smoothers the paper compares with the annealed stout path:
APE / AUS with unit circle projection (Sec. II.C, Sec. VII.A) and the Wilson
flow integrated by third-order Runge-Kutta (Sec. V.B), through the C ABI,
against the FP64 oracle.  The oracle projects with an eigendecomposition of
V^dag V and the kernels with the scaled Newton polar iteration: two algorithms
for the same function."""

import numpy as np
import pytest

import oracle as O
import synth
from tests.gpu_common import cooled_labels, max_abs

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")


@pytest.fixture(scope="module")
def ctx():
    c = vs.vs_create(0)
    yield c
    vs.vs_destroy(c)


def _field(ctx, dims, lab, precision=None, storage=None, gauge=None, omega=0.02):
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64 if precision is None else precision,
                           vs.VS_LINK18 if storage is None else storage)
    vs.vs_load_field(f, labels=lab)
    if omega is not None:
        vs.vs_centrifuge(f, omega, 1234)
    if gauge is not None:
        vs.vs_gauge_transform(f, gauge)
    return f


@pytest.mark.parametrize("case", ["aus_vp", "aus_random_gauge", "ape_random_gauge"])
def test_ucp_smoothing_fp64_matches_oracle(ctx, case):
    """AUS+UCP as in the paper's Fig. (centrifuge w = 0.02, eps = -0.25,
    alpha = 0.02, vortex preservation, 10 sweeps) and, on the centrifuged field
    after a random gauge transformation, AUS+UCP and APE smearing with UCP at
    alpha = 0.7 / 0.5 (3 sweeps); FP64 against the oracle, reject counts equal."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    U0 = O.centrifuge(dims, lab, 0.02, 1234)
    G = None
    if case == "aus_vp":
        alpha, vp, n, sched = 0.02, True, 10, "annealed"
    else:
        G = synth.random_gauge(dims, 45)
        U0 = O.gauge_transform(dims, U0, G)
        alpha, vp, n = (0.7, False, 3) if case == "aus_random_gauge" else (0.5, False, 3)
        sched = "annealed" if case == "aus_random_gauge" else "simultaneous"
    Uo, rej = O.ape_ucp(dims, U0, lab, n, alpha, eps=-0.25, schedule=sched, vp=vp, gauge=G)
    f = _field(ctx, dims, lab, gauge=G)
    assert max_abs(vs.vs_read_field(f), U0) < 1e-14
    st = vs.vs_smooth_ape(f, n, alpha, -0.25, vortex_preserve=vp, stats=True,
                          schedule=vs.VS_ANNEALED if sched == "annealed" else vs.VS_SIMULTANEOUS)
    Ug = vs.vs_read_field(f)
    chk = vs.vs_vortex_check(f)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, Uo) < 1e-11
    assert [s["n_reject"] for s in st] == list(rej)
    assert all(s["n_singular"] == 0 for s in st)
    if vp:
        assert chk["n_label_diff"] == 0 and chk["n_charge_diff"] == 0


@pytest.mark.parametrize("storage,dims", [("link18", (8, 8, 8, 8)), ("link12", (8, 8, 8, 8)),
                                          ("link18", (4, 4, 12, 20))])
def test_ucp_fp32_each_sweep_within_rounding(ctx, storage, dims):
    """FP32 AUS+UCP from the oracle's FP64 state, one sweep at a time (also on
    a lattice whose class launches end in a partial block)."""
    lab = cooled_labels(dims, 2)
    G = synth.random_gauge(dims, 46)
    U = O.gauge_transform(dims, O.centrifuge(dims, lab, 0.02, 1234), G)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst = 0.0
    for _ in range(10):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth_ape(f, 1, 0.3, -0.25, vortex_preserve=False, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U, _ = O.ape_ucp(dims, U, None, 1, 0.3, eps=-0.25, vp=False)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    assert worst < 3e-6


def test_ape_simultaneous_fp32_each_sweep_within_rounding(ctx):
    """FP32 APE smearing with UCP (simultaneous: every link from the previous
    field, through the alternate buffer) on a randomly gauged field, one sweep
    at a time from the oracle's FP64 state, at the benchmark's alpha = 0.5.
    The FP32 projection (Newton polar iteration stopped at a squared step of
    1e-13, adjugate inverse, cube root of the determinant) leaves a few 1e-6
    per sweep at this blocking weight: measured 7.6e-6, and 7.4e-6 with plain
    loads and a field copy per sweep; 1.5e-5."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    U = O.gauge_transform(dims, O.centrifuge(dims, lab, 0.02, 1234), synth.random_gauge(dims, 47))
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    worst = 0.0
    for _ in range(5):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth_ape(f, 1, 0.5, -0.25, vortex_preserve=False, reunit_every=0, schedule=vs.VS_SIMULTANEOUS)
        Ug = vs.vs_read_field(f)
        U, _ = O.ape_ucp(dims, U, None, 1, 0.5, eps=-0.25, schedule="simultaneous", vp=False)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    assert worst < 1.5e-5


def test_ucp_keeps_a_vortex_field_on_centre_elements(ctx):
    """A Z(3) field in a random gauge: every projected link is G(x) z G^dag(x+mu)
    with z in Z(3) (Sec. II.C); at small alpha z is the original element, so the
    gauge-reversed vortex check sees no label change."""
    dims = (8, 8, 8, 8)
    lab = synth.iid_labels(dims, 47)
    G = synth.random_gauge(dims, 48)
    f = _field(ctx, dims, lab, gauge=G, omega=None)
    vs.vs_smooth_ape(f, 2, 0.02, -0.25, vortex_preserve=False)
    U = vs.vs_read_field(f)
    chk = vs.vs_vortex_check(f)
    vs.vs_field_destroy(f)
    back = O.gauge_transform(dims, U, G.conj().transpose(0, 2, 1))
    diag = back[..., [0, 1, 2], [0, 1, 2]]
    assert np.abs(back - diag[..., :, None] * np.eye(3)).max() < 1e-12
    assert np.abs(diag - diag[..., :1]).max() < 1e-12
    assert chk["n_label_diff"] == 0


@pytest.mark.parametrize("eps", [1.0, -0.25])
def test_flow_rk3_fp64_matches_oracle(ctx, eps):
    """Wilson flow (eps = 1) and over-improved flow (eps = -0.25) by RK3, three
    steps of 0.02 from a lightly cooled Haar field and from the centrifuged
    vortex field; FP64 against the oracle."""
    dims = (8, 8, 8, 8)
    U1 = O.cool(dims, synth.haar_field(dims, 49), 2)
    lab = cooled_labels(dims, 2)
    U2 = O.centrifuge(dims, lab, 0.02, 1234)
    for U in (U1, U2):
        f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
        vs.vs_load_field(f, links=U)
        st = vs.vs_flow_rk3(f, 3, 0.02, eps, stats=True)
        Ug = vs.vs_read_field(f)
        vs.vs_field_destroy(f)
        assert max_abs(Ug, O.flow_rk3(dims, U, 3, 0.02, eps=eps)) < 1e-12
        assert len(st) == 3


@pytest.mark.parametrize("eps", [-0.25, 1.0])
@pytest.mark.parametrize("storage", ["link18", "link12"])
def test_flow_rk3_fp32_each_step_within_rounding(ctx, storage, eps):
    """FP32 Runge-Kutta steps (the over-improved and the Wilson flow, whose
    staples take different link streams) from the oracle's FP64 field, one
    step at a time; also a lattice whose launches end in a partial block."""
    for dims in [(8, 8, 8, 8), (4, 4, 12, 20)]:
        _flow_fp32_steps(ctx, dims, storage, eps)


def _flow_fp32_steps(ctx, dims, storage, eps):
    U = O.cool(dims, synth.haar_field(dims, 50), 2)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst = 0.0
    for _ in range(5):
        vs.vs_load_field(f, links=U)
        vs.vs_flow_rk3(f, 1, 0.05, eps, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U = O.flow_rk3(dims, U, 1, 0.05, eps=eps)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    assert worst < 2e-6


@pytest.mark.parametrize("n_steps", [2, 3])
def test_flow_rk3_reunitarises_the_live_field(ctx, n_steps):
    """The stages alternate between the field and a scratch buffer (6 stages
    end in the field, 9 in the scratch buffer); re-unitarisation after the last
    step must act on the buffer that holds the current links.  Input links
    carry 1e-3 of non-unitary noise, which the flow keeps and only the
    re-unitarisation removes."""
    dims = (8, 4, 4, 8)
    U = O.cool(dims, synth.haar_field(dims, 53), 2)
    rng = np.random.default_rng(54)
    U = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    devs = []
    for every in (0, n_steps):
        vs.vs_load_field(f, links=U)
        vs.vs_flow_rk3(f, n_steps, 0.02, -0.25, reunit_every=every)
        Ug = vs.vs_read_field(f)
        devs.append(np.abs(np.einsum("...ij,...kj->...ik", Ug, Ug.conj()) - np.eye(3)).max())
    vs.vs_field_destroy(f)
    assert devs[0] > 1e-4 and devs[1] < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_rk3_leaves_a_vortex_field_unchanged(ctx, precision):
    """Q = 0 exactly on a centre-vortex field (Sec. V.B): bitwise unchanged."""
    dims = (8, 8, 8, 8)
    lab = synth.iid_labels(dims, 51)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64 if precision == "fp64" else vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    U0 = vs.vs_read_field(f)
    vs.vs_flow_rk3(f, 4, 0.05, -0.25)
    U1 = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert np.array_equal(U0, U1)


def test_ape_and_flow_reject_bad_arguments(ctx):
    dims = (4, 4, 4, 4)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=synth.iid_labels(dims, 52))
    for call in (lambda: vs.vs_smooth_ape(f, 1, 1.5), lambda: vs.vs_smooth_ape(f, 1, 0.1, schedule=7),
                 lambda: vs.vs_flow_rk3(f, 1, -0.1), lambda: vs.vs_flow_rk3(f, -1, 0.1)):
        with pytest.raises(vs.VSError) as ei:
            call()
        assert ei.value.status == vs.VS_EINVAL
    vs.vs_field_destroy(f)
