"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated per test): FP64 GPU vs oracle 1e-11 on links and 1e-11
relative on the action (different exponential algorithm and summation order:
rounding differences of ~1e-16 per operation, amplified by the flow, whose
perturbations grow ~1.5x per sweep on these fields, so FP64 runs are compared
over at most 25 sweeps); FP32 GPU within 1e-6 of FP64 on every single sweep;
Z(3) labels, centre charges and the per-sweep vortex-preservation reject
counts bit-exact (FP64); in FP32 the vortex-preservation decisions equal the
FP64 oracle's except for links the kernels count as undecidable (a candidate
whose trace lies within 2e-6, in trace units, of a sector edge: the FP32
error band of the trace).
"""

import numpy as np
import pytest

import oracle as O
import synth
from tests import lattice_np as L
from tests.gpu_common import cooled_labels, gpu_pipeline, max_abs, oracle_pipeline

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")


@pytest.fixture(scope="module")
def ctx():
    c = vs.vs_create(0)
    yield c
    vs.vs_destroy(c)


# --------------------------------------------------------------------------
# Building blocks
# --------------------------------------------------------------------------

def _herm(rng, n, scale):
    A = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    H = 0.5 * (A + L.dag(A))
    H -= np.trace(H, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    return H * (scale / np.linalg.norm(H, axis=(1, 2)))[:, None, None]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 2e-7)])
def test_exponential_matches_taylor_and_eigendecomposition(ctx, prec, tol):
    rng = np.random.default_rng(5)
    Hs = np.concatenate([_herm(rng, 200, s) for s in (1e-7, 1e-3, 0.05, 0.3, 0.9, 1.5, 3.0)])
    # degenerate and near-degenerate spectra
    for gap in (0.0, 1e-7, 1e-3):
        W = synth.haar_su3(1, 9)[0]
        Hs = np.concatenate([Hs, (W @ np.diag([0.2, 0.2 + gap, -0.4 - gap]) @ L.dag(W))[None]])
    X = 1j * Hs
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    E = vs.vs_debug_expm(ctx, X, p)
    Eeig = L.expm_eigh(X)
    Etay = np.stack([O.expm(x) for x in X])
    scale = np.maximum(1.0, np.linalg.norm(Hs, axis=(1, 2)))
    assert (np.abs(E - Etay).max(axis=(1, 2)) / scale).max() < tol * 4
    assert (np.abs(E - Eeig).max(axis=(1, 2)) / scale).max() < tol * 4
    assert np.array_equal(vs.vs_debug_expm(ctx, np.zeros((1, 3, 3)), p)[0], np.eye(3))


@pytest.mark.parametrize("prec,storage,tol", [("fp64", "link18", 1e-14), ("fp32", "link18", 1e-6),
                                               ("fp32", "link12", 1e-6)])
def test_reunitarise_matches_oracle(ctx, prec, storage, tol):
    """Re-unitarisation of a Haar field with 1e-3 non-unitary noise on every
    entry, against the oracle's Gram-Schmidt; the FP32 result is unitary to
    the rounding of its stored rows.  12-real storage keeps rows 0-1 only, so
    its input row 2 is replaced on load, as the oracle ignores it."""
    dims = (4, 8, 12, 16)
    U = synth.haar_field(dims, 80)
    rng = np.random.default_rng(81)
    U = U + 1e-3 * (rng.normal(size=U.shape) + 1j * rng.normal(size=U.shape))
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64 if prec == "fp64" else vs.VS_FP32,
                           vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12)
    vs.vs_load_field(f, links=U)
    vs.vs_reunitarise(f)
    Ug = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, O.reunit(U)) < tol
    dev = np.abs(np.einsum("...ij,...kj->...ik", Ug, Ug.conj()) - np.eye(3)).max()
    assert dev < (1e-14 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_load_and_centrifuge_match_oracle(ctx, prec):
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    for dims, seed in [((4, 4, 4, 4), 1), ((8, 4, 12, 8), 2)]:
        lab = synth.iid_labels(dims, seed)
        f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18)
        vs.vs_load_field(f, labels=lab)
        assert np.array_equal(vs.vs_read_labels(f), lab)
        Z = vs.vs_read_field(f)
        assert max_abs(Z, O.links_from_labels(dims, lab)) < (1e-15 if prec == "fp64" else 1e-7)
        vs.vs_centrifuge(f, 0.02, 1234)
        U = vs.vs_read_field(f)
        Uo = O.centrifuge(dims, lab, 0.02, 1234)
        assert max_abs(U, Uo) < (1e-14 if prec == "fp64" else 1e-7)
        assert np.array_equal(vs.vs_current_labels(f), lab)
        assert vs.vs_vortex_check(f)["n_label_diff"] == 0
        vs.vs_field_destroy(f)


def test_load_rejects_host_labels_outside_z3(ctx):
    """Host labels are checked before any copy: a value outside {-1, 0, 1}
    anywhere (first or last entry) is VS_EINVAL, naming its position."""
    dims = (4, 4, 4, 8)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    for pos, val in [(0, 2), (-1, -2)]:
        lab = synth.iid_labels(dims, 7).copy()
        lab.reshape(-1)[pos] = val
        with pytest.raises(vs.VSError) as ei:
            vs.vs_load_field(f, labels=lab)
        assert ei.value.status == vs.VS_EINVAL and "outside" in str(ei.value)
    vs.vs_load_field(f, labels=synth.iid_labels(dims, 7))
    vs.vs_field_destroy(f)


@pytest.mark.parametrize("prec,storage", [("fp32", "link18"), ("fp32", "link12"), ("fp64", "link18")])
def test_checkpoint_restore_resumes_bit_for_bit(ctx, prec, storage):
    """N + M sweeps equal N sweeps, checkpoint, restore into another field,
    M sweeps: bit for bit, across a re-unitarisation (every 4 sweeps, N = 3,
    M = 6), with VP against the original reference labels (restored as given,
    not recomputed from the links)."""
    dims = (4, 8, 4, 8)
    lab = cooled_labels(dims, 2)
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12

    def fresh():
        f = vs.vs_field_create(ctx, dims, p, st)
        vs.vs_load_field(f, labels=lab)
        vs.vs_centrifuge(f, 0.02, 1234)
        return f

    a = fresh()
    ra = vs.vs_smooth(a, 9, 0.06, -0.25, reunit_every=4, stats=True)
    Ua = vs.vs_read_field(a)
    vs.vs_field_destroy(a)
    b = fresh()
    rb = vs.vs_smooth(b, 3, 0.06, -0.25, reunit_every=4, stats=True)
    links, labels, n = vs.vs_field_checkpoint(b)
    vs.vs_field_destroy(b)
    assert n == 3 and np.array_equal(labels, lab)
    c = vs.vs_field_create(ctx, dims, p, st)
    vs.vs_field_restore(c, links, labels, n)
    rc = vs.vs_smooth(c, 6, 0.06, -0.25, reunit_every=4, stats=True)
    Uc = vs.vs_read_field(c)
    assert np.array_equal(vs.vs_read_labels(c), lab)
    vs.vs_field_destroy(c)
    assert np.array_equal(Ua, Uc)
    assert [s["n_reject"] for s in ra] == [s["n_reject"] for s in rb + rc]


@pytest.mark.parametrize("prec,storage", [("fp32", "link18"), ("fp32", "link12"), ("fp64", "link18")])
def test_nonfinite_links_are_counted(ctx, prec, storage):
    """The NaN/Inf guard counts exactly the links that carry a non-finite
    entry (in a row that the storage keeps), and none on a smoothed field."""
    dims = (4, 4, 4, 8)
    U = O.cool(dims, synth.haar_field(dims, 5), 1)
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12)
    vs.vs_load_field(f, links=U)
    vs.vs_smooth(f, 2, 0.06, -0.25, vortex_preserve=False)
    assert vs.vs_field_count_nonfinite(f) == 0
    bad = U.copy()
    bad[0, 3, 0, 1] = np.nan
    bad[2, 17, 1, 2] = np.inf
    bad[3, 40, 0, 0] = complex(0.0, -np.inf)
    vs.vs_load_field(f, links=bad)
    assert vs.vs_field_count_nonfinite(f) == 3
    vs.vs_field_destroy(f)


def test_checkpoint_and_centrifuge_refuse_gauge_transformed_fields(ctx):
    """A field in a random gauge keeps G on the device: a checkpoint would
    lose it (EUNSUPPORTED), and the centrifuge, which builds links from the
    labels in the original gauge, would leave links and G inconsistent
    (EINVAL).  A second transform is refused too; a reload drops G."""
    dims = (4, 4, 4, 4)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    lab = synth.iid_labels(dims, 3)
    vs.vs_load_field(f, labels=lab)
    vs.vs_gauge_transform(f, synth.random_gauge(dims, 4))
    with pytest.raises(vs.VSError) as ei:
        vs.vs_field_checkpoint(f)
    assert ei.value.status == vs.VS_EUNSUPPORTED
    for call in (lambda: vs.vs_centrifuge(f, 0.02, 1), lambda: vs.vs_gauge_transform(f, synth.random_gauge(dims, 5))):
        with pytest.raises(vs.VSError) as ei:
            call()
        assert ei.value.status == vs.VS_EINVAL
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1)
    assert vs.vs_vortex_check(f)["n_label_diff"] == 0
    vs.vs_field_destroy(f)


def test_load_links_and_labels_from_fp64_input(ctx):
    dims = (4, 8, 4, 4)
    U = synth.haar_field(dims, 3)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    assert np.array_equal(vs.vs_read_field(f), U)
    assert np.array_equal(vs.vs_read_labels(f), O.labels(dims, U))
    vs.vs_field_destroy(f)


@pytest.mark.parametrize("storage", ["link18", "link12"])
def test_fp32_action_within_rounding(ctx, storage):
    """FP32 action (plaquette products and traces in FP32, the sum over
    plaquettes in FP64) of a Haar field and of a centrifuged vortex field,
    against the oracle's FP64 action of the same links: within 1e-6 absolute
    (a few FP32 roundings per plaquette, ~1e-7 each)."""
    dims = (8, 4, 4, 8)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    for U in (synth.haar_field(dims, 4), O.centrifuge(dims, synth.iid_labels(dims, 6), 0.02, 1234)):
        f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
        vs.vs_load_field(f, links=U)
        S = vs.vs_action(f)
        vs.vs_field_destroy(f)
        assert abs(S - O.action(dims, U)) < 1e-6


def test_action_and_vortex_check_match_oracle(ctx):
    dims = (8, 4, 4, 8)
    U = synth.haar_field(dims, 4)
    lab = synth.iid_labels(dims, 5)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    assert abs(vs.vs_action(f) - O.action(dims, U)) < 1e-13
    vs.vs_field_destroy(f)
    # vortex check: reference labels from a pure Z(3) field, then compare with
    # the labels of a different Z(3) field loaded over it -> counts from the oracle
    Z = O.links_from_labels(dims, lab)
    lab2 = lab.copy()
    lab2[1, ::7] = ((lab2[1, ::7] + 2) % 3) - 1
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    chk = vs.vs_vortex_check(f)
    assert chk["n_label_diff"] == 0 and chk["n_charge_diff"] == 0
    assert abs(vs.vs_action(f) - O.action(dims, Z)) < 1e-13
    vs.vs_field_destroy(f)
    ref = O.vortex_check(dims, O.links_from_labels(dims, lab2), lab)
    assert ref["n_label_diff"] == np.count_nonzero(lab2 != lab)
    assert ref["n_charge_diff"] > 0


# --------------------------------------------------------------------------
# Smoothing parity
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("eps", [1.0, -0.25])
def test_pure_z3_field_is_unchanged(ctx, prec, eps):
    # Sec. II.A: Q = 0 on a vortex field; the kernels return it bit for bit.
    dims = (8, 8, 4, 4)
    lab = synth.iid_labels(dims, 1)
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    r = gpu_pipeline(vs, ctx, dims, lab, None, 0, 3, 0.1, eps, precision=p, reunit_every=0)
    f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    Z = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert np.array_equal(r["U"], Z)
    assert all(s["n_reject"] == 0 for s in r["stats"])


def test_workload_4x4_pure_vortex_fp64(ctx):
    """4^4 pure Z(3) field, P(0)=0.7, seed 1; centrifuge w=0.02 (seed 1234);
    10 standard stout sweeps rho=0.1 with vortex preservation; FP64."""
    dims = (4, 4, 4, 4)
    lab = synth.iid_labels(dims, 1)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, 10, 0.1, 1.0)
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, 10, 0.1, 1.0)
    assert max_abs(r["U"], Uo) < 1e-11
    assert [s["n_reject"] for s in r["stats"]] == list(rej)
    assert np.array_equal(r["labels"], O.labels(dims, Uo))
    assert abs(r["action"] - O.action(dims, Uo)) < 1e-12 * O.action(dims, Uo)
    assert r["check"]["n_label_diff"] == 0 and r["check"]["n_charge_diff"] == 0


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 8, 12, 16)])
def test_overimproved_vp_fp64_on_cooled_input(ctx, dims):
    lab = cooled_labels(dims, 2)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, 20, 0.06, -0.25)
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, 20, 0.06, -0.25)
    assert max_abs(r["U"], Uo) < 1e-11
    assert [s["n_reject"] for s in r["stats"]] == list(rej)
    assert abs(r["action"] / O.action(dims, Uo) - 1) < 1e-11


def test_large_steps_exercise_rejections_fp64(ctx):
    dims = (8, 4, 8, 4)
    lab = synth.iid_labels(dims, 13)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, 6, 0.3, -0.25)
    assert rej.sum() > 0
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, 6, 0.3, -0.25)
    assert [s["n_reject"] for s in r["stats"]] == list(rej)
    # rounding-level differences (the two exponentials differ in the last bits)
    # grow by the Lipschitz factor of the update, ~(1 + rho |dQ/dU|) per sweep:
    # at rho = 0.3 that is a few per sweep, so allow 1e-11 after 6 sweeps.
    assert max_abs(r["U"], Uo) < 1e-11


@pytest.mark.parametrize("kind", ["annealed", "simultaneous"])
@pytest.mark.parametrize("eps", [1.0, -0.25])
def test_full_su3_field_parity(ctx, kind, eps):
    """A general (non-diagonal) SU(3) field exercises every entry of the staple
    products: a cooled Haar field, VP off."""
    dims = (4, 8, 4, 8)
    U = O.cool(dims, synth.haar_field(dims, 17), 3)
    sched = O.ANNEALED if kind == "annealed" else O.SIMULTANEOUS
    Uo, _ = O.smooth(dims, U, None, 3, 0.08, eps=eps, schedule=sched, vp=False)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    vs.vs_smooth(f, 3, 0.08, eps, vortex_preserve=False,
                 kind=vs.VS_ANNEALED if kind == "annealed" else vs.VS_SIMULTANEOUS)
    Ug = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, Uo) < 1e-11


@pytest.mark.parametrize("eps,rho", [(-0.25, 0.35), (1.0, 0.75)])
@pytest.mark.parametrize("n_sweeps", [3, 4])
def test_simultaneous_vp_with_rejections_fp64(ctx, eps, rho, n_sweeps):
    """Simultaneous stout smearing (every link from the previous field; the
    field and a scratch buffer alternate as source and destination) with
    vortex preservation at steps large enough to reject (the largest the
    exponential's range check admits for each eps): a rejected link must
    carry its old value into the destination buffer.  Even and odd sweep
    counts end in either buffer."""
    dims = (8, 4, 8, 4)
    lab = synth.iid_labels(dims, 13)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, n_sweeps, rho, eps, schedule=O.SIMULTANEOUS)
    assert rej.sum() > 0
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, n_sweeps, rho, eps, kind=vs.VS_SIMULTANEOUS)
    assert [s["n_reject"] for s in r["stats"]] == list(rej)
    assert max_abs(r["U"], Uo) < 1e-11
    assert r["check"]["n_label_diff"] == 0


@pytest.mark.parametrize("eps,rho", [(-0.25, 0.35), (1.0, 0.75)])
def test_fp32_simultaneous_vp_each_sweep(ctx, eps, rho):
    """FP32 simultaneous stout sweeps with vortex preservation (the link-ring
    kernels on every link of a direction, writing into the alternate buffer;
    rejected links carry their old value), each from the oracle's FP64 field,
    through the sweeps where rejections set in: within 1e-6, with the same
    decisions except links the GPU counted as undecidable."""
    dims = (8, 4, 8, 4)
    lab = synth.iid_labels(dims, 13)
    U = O.centrifuge(dims, lab, 0.02, 1234)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    worst, ties, n_rej, n_undec = 0.0, 0, 0, 0
    for sweep in range(4):
        vs.vs_load_field(f, links=U)
        st = vs.vs_smooth(f, 1, rho, eps, vortex_preserve=True, reunit_every=0, kind=vs.VS_SIMULTANEOUS,
                          stats=True)[0]
        Ug = vs.vs_read_field(f)
        U, rej, cmargin, _ = O.smooth(dims, U, lab, 1, rho, eps=eps, vp=True, schedule=O.SIMULTANEOUS,
                                      diagnostics=True)
        n_rej += int(rej.sum())
        n_undec += st["n_undecidable"]
        d = np.abs(Ug - U).max(axis=(2, 3))
        split = d > 1e-4
        ties += int(split.sum())
        # decisions differ only where the GPU counted an undecidable link
        assert int(split.sum()) <= st["n_undecidable"], (sweep, cmargin[split], st)
        if st["n_undecidable"] == 0:
            assert st["n_reject"] == int(rej[0])
        worst = max(worst, float(d[~split].max()))
    vs.vs_field_destroy(f)
    print("simultaneous eps=%g: worst %.3g, undecidable %d, split %d" % (eps, worst, n_undec, ties))
    assert n_rej > 100
    assert worst < 1e-6


@pytest.mark.parametrize("storage", ["link18", "link12"])
def test_fp32_vp_candidates_near_an_edge_are_redecided_in_fp64(ctx, storage):
    """Sec. VI test in FP32 with vortex preservation: a candidate whose FP32
    trace lies within the FP32 band of a sector edge is decided again in FP64
    from the same stored links (vs_anneal.fp64_redecide).  Along the 200-sweep
    trajectory, each sweep from the oracle's FP64 field: with the FP64 pass the
    decisions equal the oracle's except for candidates within the band of the
    FP32 link storage (n_undecidable), every re-decided candidate is counted,
    and fewer candidates stay undecidable than with FP32 decisions alone."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    tot = {True: dict(split=0, undec=0, redec=0), False: dict(split=0, undec=0, redec=0)}
    U = O.centrifuge(dims, lab, 0.02, 1234)
    for sweep in range(200):
        Unext, rej, cmargin, _ = O.smooth(dims, U, lab, 1, 0.06, eps=-0.25, vp=True, diagnostics=True)
        for redecide in (True, False):
            vs.vs_load_field(f, links=U)
            s1 = vs.vs_smooth(f, 1, 0.06, -0.25, vortex_preserve=True, reunit_every=0, stats=True,
                              fp64_redecide=redecide)[0]
            Ug = vs.vs_read_field(f)
            split = np.abs(Ug - Unext).max(axis=(2, 3)) > 1e-4
            assert int(split.sum()) <= s1["n_undecidable"], (redecide, sweep, cmargin[split], s1)
            t = tot[redecide]
            t["split"] += int(split.sum())
            t["undec"] += s1["n_undecidable"]
            t["redec"] += s1["n_fp64_redecided"]
            if s1["n_undecidable"] == 0:
                assert s1["n_reject"] == int(rej[0]) and s1["n_label_diff"] == int(rej[0])
        U = Unext
    vs.vs_field_destroy(f)
    print("%s: with FP64 re-decision %s, FP32 alone %s" % (storage, tot[True], tot[False]))
    assert tot[False]["redec"] == 0
    assert tot[False]["undec"] > 0 and tot[True]["redec"] > 0
    assert tot[True]["undec"] <= tot[False]["undec"]
    assert tot[True]["split"] <= tot[False]["split"]


@pytest.mark.parametrize("storage,vp", [("link18", True), ("link12", True), ("link18", False)])
def test_fp32_each_sweep_within_fp32_rounding_of_fp64(ctx, storage, vp):
    """FP32 accuracy along the whole 200-sweep FP64 trajectory.  The annealed
    flow on these fields amplifies any difference, however small, by ~1.5x per
    sweep (two FP64 runs a 1e-10 perturbation apart separate to O(1) within ~60
    sweeps), so FP32 and FP64 runs cannot be compared link by link after many
    free-running sweeps.  What FP32 mode must get right is every step: here
    each sweep starts both sides from the oracle's FP64 field, and the FP32
    result must agree to 1e-6 (a few FP32 roundings), with the same VP
    decisions except for links the GPU counted as undecidable, and the per-sweep
    smallest candidate margin within 2e-6 rad of the oracle's."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    U = O.centrifuge(dims, lab, 0.02, 1234)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst, worst_margin = 0.0, 0.0
    ties = n_undec = n_rej = 0
    for sweep in range(200):
        vs.vs_load_field(f, links=U)
        if vp:
            assert np.array_equal(vs.vs_read_labels(f), lab)
        s1 = vs.vs_smooth(f, 1, 0.06, -0.25, vortex_preserve=vp, reunit_every=0, stats=True)[0]
        Ug = vs.vs_read_field(f)
        U, rej, cmargin, rejected = O.smooth(dims, U, lab, 1, 0.06, eps=-0.25, vp=vp,
                                             diagnostics=True)
        d = np.abs(Ug - U).max(axis=(2, 3))
        split = d > 1e-4                     # decided differently
        ties += int(split.sum())
        n_undec += s1["n_undecidable"]
        n_rej += int(rej[0])
        # FP32 decisions equal the FP64 oracle's except for links the GPU
        # counted as undecidable (trace within the FP32 error band of an edge)
        assert int(split.sum()) <= s1["n_undecidable"], (sweep, cmargin[split], s1)
        if s1["n_undecidable"] == 0:
            assert s1["n_reject"] == int(rej[0])
            if vp:
                assert s1["n_label_diff"] == int(rej[0])
        worst_margin = max(worst_margin, abs(s1["min_margin"] - float(np.nanmin(cmargin))))
        worst = max(worst, float(d[~split].max()))
    vs.vs_field_destroy(f)
    print("%s vp=%d: worst one-sweep link error %.3g, min-margin error %.3g, rejections %d, "
          "undecidable %d, split decisions %d" % (storage, vp, worst, worst_margin, n_rej, n_undec, ties))
    assert worst < 1e-6
    assert worst_margin < 2e-6
    if not vp:
        assert ties == 0


@pytest.mark.parametrize("eps", [-0.25, 1.0])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 4, 12, 20)])
@pytest.mark.parametrize("storage", ["link18", "link12"])
def test_fp32_class_kernel_general_su3_ragged(ctx, dims, storage, eps):
    """The FP32 class kernels (over-improved: the benchmark's path; eps = 1:
    plaquette staples) on a general SU(3) field, so that every entry of the
    two-row chains and rebuilt rows matters, at
    lattices whose class launches end in a partial block: 4^4 (64 threads of a
    128-thread block, and +-2 shifts land on the same site) and 4x4x12x20
    (960 threads, 7.5 blocks).  Each sweep starts both sides from the oracle's
    FP64 field; FP32 within 1e-6."""
    U = O.cool(dims, synth.haar_field(dims, 31), 2)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst = 0.0
    for sweep in range(3):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth(f, 1, 0.06, eps, vortex_preserve=False, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U, _ = O.smooth(dims, U, None, 1, 0.06, eps=eps, vp=False)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    assert worst < 1e-6


def test_zero_sweeps_and_bad_extents(ctx):
    """n_sweeps = 0 leaves the field bit for bit; extents that are not positive
    multiples of 4 (the annealing schedule's requirement) or a lattice above
    2^30 sites are rejected with VS_EINVAL before any allocation."""
    dims = (4, 8, 4, 4)
    U = O.cool(dims, synth.haar_field(dims, 32), 1)
    for prec in (vs.VS_FP64, vs.VS_FP32):
        f = vs.vs_field_create(ctx, dims, prec, vs.VS_LINK18)
        vs.vs_load_field(f, links=U)
        U0 = vs.vs_read_field(f)
        assert vs.vs_smooth(f, 0, 0.06, -0.25, stats=True) == []
        vs.vs_smooth_aus(f, 0, 0.02, -0.25)
        vs.vs_flow_rk3(f, 0, 0.02)
        assert np.array_equal(vs.vs_read_field(f), U0)
        vs.vs_field_destroy(f)
    for bad in [(0, 4, 4, 4), (6, 4, 4, 4), (4, 4, 4, -4), (4, 4, 2, 4), (2048, 2048, 2048, 4)]:
        with pytest.raises(vs.VSError) as ei:
            vs.vs_field_create(ctx, bad, vs.VS_FP32, vs.VS_LINK18)
        assert ei.value.status == vs.VS_EINVAL


def test_calls_on_a_field_never_loaded_are_refused(ctx):
    """A created field holds uninitialised device memory until a load: every
    call that reads the links or the labels refuses it with VS_EINVAL rather
    than returning garbage, and the field still works after a load."""
    dims = (4, 4, 4, 8)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    calls = [lambda: vs.vs_read_field(f), lambda: vs.vs_read_labels(f), lambda: vs.vs_current_labels(f),
             lambda: vs.vs_reunitarise(f), lambda: vs.vs_subsweep(f, 0, 0, 0.05, -0.25),
             lambda: vs.vs_action(f), lambda: vs.vs_observables(f), lambda: vs.vs_vortex_check(f),
             lambda: vs.vs_field_count_nonfinite(f), lambda: vs.vs_centrifuge(f, 0.02, 1),
             lambda: vs.vs_smooth(f, 1, 0.05, -0.25), lambda: vs.vs_smooth_aus(f, 1, 0.02),
             lambda: vs.vs_smooth_ape(f, 1, 0.02), lambda: vs.vs_flow_rk3(f, 1, 0.02),
             lambda: vs.vs_field_checkpoint(f)]
    for call in calls:
        with pytest.raises(vs.VSError) as ei:
            call()
        assert ei.value.status == vs.VS_EINVAL
    lab = synth.iid_labels(dims, 3)
    vs.vs_load_field(f, labels=lab)
    assert np.array_equal(vs.vs_read_labels(f), lab)
    assert vs.vs_vortex_check(f)["n_label_diff"] == 0
    vs.vs_field_destroy(f)


def test_binding_checks_cuda_buffers(ctx):
    """CUDA tensors handed to the binding are checked for element type, size
    and device before the library sees the pointer; a correct one round-trips."""
    torch = pytest.importorskip("torch")
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_field(f, labels=synth.iid_labels(dims, 5))
    assert vs.vs_field_describe(f)["device"] == 0
    with pytest.raises(TypeError):
        vs.vs_read_field(f, torch.empty((4, V, 3, 3), dtype=torch.complex64, device="cuda:0"))
    with pytest.raises(ValueError):
        vs.vs_read_labels(f, torch.empty((4, V - 1), dtype=torch.int8, device="cuda:0"))
    with pytest.raises(ValueError):
        vs.vs_load_field(f, links=torch.empty((4, V, 3, 3), dtype=torch.complex128, device="cuda:0")[:, :, :2])
    out = torch.empty((4, V, 3, 3), dtype=torch.complex128, device="cuda:0")
    vs.vs_read_field(f, out)
    vs.vs_synchronize(f)
    assert np.array_equal(out.cpu().numpy(), vs.vs_read_field(f))
    vs.vs_field_destroy(f)


def test_device_buffers_round_trip(ctx):
    """The device side of the ABI (where = VS_DEVICE, torch CUDA tensors):
    labels loaded from the device, a checkpoint written to device buffers
    and restored from them resumes bit for bit, and a gauge field given on
    the device acts as the same field given on the host."""
    torch = pytest.importorskip("torch")
    dims = (4, 8, 4, 8)
    V = int(np.prod(dims))
    lab = synth.iid_labels(dims, 9)
    lab_d = torch.from_numpy(lab).to("cuda:0")
    G = synth.random_gauge(dims, 11)
    G_d = torch.from_numpy(G).to("cuda:0")
    torch.cuda.synchronize()                      # the library's streams do not wait for torch's
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab_d)
    assert np.array_equal(vs.vs_read_labels(f), lab)
    vs.vs_centrifuge(f, 0.02, 7)
    vs.vs_smooth(f, 3, 0.06, -0.25, reunit_every=2)
    L = torch.empty((4, V, 3, 3), dtype=torch.complex128, device="cuda:0")
    N = torch.empty((4, V), dtype=torch.int8, device="cuda:0")
    _, _, n = vs.vs_field_checkpoint(f, L, N)
    vs.vs_synchronize(f)
    assert n == 3
    assert np.array_equal(L.cpu().numpy(), vs.vs_read_field(f))
    assert np.array_equal(N.cpu().numpy(), lab)
    g = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_field_restore(g, L, N, n)
    vs.vs_smooth(f, 3, 0.06, -0.25, reunit_every=2)
    vs.vs_smooth(g, 3, 0.06, -0.25, reunit_every=2)
    assert np.array_equal(vs.vs_read_field(f), vs.vs_read_field(g))
    vs.vs_field_destroy(g)
    vs.vs_field_destroy(f)
    a = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    b = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    for h, gauge in ((a, G_d), (b, G)):
        vs.vs_load_field(h, labels=lab)
        vs.vs_gauge_transform(h, gauge)
    assert np.array_equal(vs.vs_read_field(a), vs.vs_read_field(b))
    vs.vs_field_destroy(a)
    vs.vs_field_destroy(b)


def test_fp32_vp_200_free_running_sweeps_keep_vortex_structure(ctx):
    """200 free-running FP32 sweeps with VP: every label and centre charge
    equals the original (and the FP64 oracle's), and the mean action, a
    lattice average, agrees with the oracle's to 1e-3 relative although the
    individual links have decorrelated (see the test above)."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    Uo, rej = oracle_pipeline(dims, lab, 0.02, 1234, 200, 0.06, -0.25)
    r = gpu_pipeline(vs, ctx, dims, lab, 0.02, 1234, 200, 0.06, -0.25, precision=vs.VS_FP32)
    assert np.array_equal(r["labels"], lab)
    assert np.array_equal(O.labels(dims, Uo), lab)
    assert r["check"]["n_label_diff"] == 0 and r["check"]["n_charge_diff"] == 0
    So = O.action(dims, Uo)
    print("action fp32 %.9f oracle %.9f rel %.2e" % (r["action"], So, r["action"] / So - 1))
    assert abs(r["action"] / So - 1) < 1e-3


def test_subsweep_matches_single_link_oracle(ctx):
    """One colour class on a full SU(3) field: every updated link equals the
    oracle's exp(rho Q) U from the field before the launch; others untouched."""
    dims = (8, 4, 4, 8)
    U = O.cool(dims, synth.haar_field(dims, 23), 2)
    c0, c1 = O.overimproved_coeffs(-0.25)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    mu, col = 2, 3
    vs.vs_subsweep(f, mu, col, 0.07, -0.25, 1.0, False)
    Ug = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    V = int(np.prod(dims))
    n_upd = 0
    for s in range(V):
        x = np.unravel_index(s, dims[::-1])[::-1]
        for m in range(4):
            if m == mu and O.colour(dims, mu, x) == col:
                S = O.staple_sum(dims, U, mu, x, c0, c1)
                Q = O.stout_generator(S @ L.dag(U[mu, s]))
                ref = O.expm(0.07 * Q) @ U[mu, s]
                assert np.abs(Ug[mu, s] - ref).max() < 1e-13
                n_upd += 1
            else:
                assert np.array_equal(Ug[m, s], U[m, s])
    assert n_upd == V // 4


# --------------------------------------------------------------------------
# Annealed U-link smearing with MaxReTr (Sec. III): the CP / VP / AS recipes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("recipe", ["VP", "CP", "AS"])
def test_aus_maxretr_fp64_matches_oracle(ctx, recipe):
    """AUS with MaxReTr, over-improved eps = -0.25, FP64 against the oracle,
    per-sweep reject counts identical:
      VP / CP: centrifuge (w = 0.02), alpha = 0.02, with / without vortex
               preservation, 10 sweeps (in the original gauge);
      AS:      random gauge, alpha = 0.7, no preservation, 3 sweeps (large steps
               on the rough vortex field amplify rounding quickly).
    On an exactly Z(3) field in its own gauge, MaxReTr candidates can land
    exactly on a sector edge, where the decision is a rounding tie; the AS
    recipe runs in a random gauge, as in the paper, which has no exact ties."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    if recipe == "AS":
        G = synth.random_gauge(dims, 43)
        U0 = O.gauge_transform(dims, O.links_from_labels(dims, lab), G)
        alpha, vp, n = 0.7, False, 3
    else:
        G = None
        U0 = O.centrifuge(dims, lab, 0.02, 1234)
        alpha, vp, n = 0.02, recipe == "VP", 10
    Uo, rej = O.aus(dims, U0, lab, n, alpha, eps=-0.25, vp=vp, gauge=G)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    if recipe == "AS":
        vs.vs_gauge_transform(f, G)
    else:
        vs.vs_centrifuge(f, 0.02, 1234)
    assert max_abs(vs.vs_read_field(f), U0) < 1e-14
    st = vs.vs_smooth_aus(f, n, alpha, -0.25, vortex_preserve=vp, stats=True)
    Ug = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    # alpha = 0.7 on the rough field divides by small k = sqrt(det T) in many
    # subgroup steps, which magnifies rounding differences (observed 1.4e-9
    # after 3 sweeps); alpha = 0.02 stays at the 1e-11 FP64 level
    assert max_abs(Ug, Uo) < (1e-8 if recipe == "AS" else 1e-11)
    assert [s["n_reject"] for s in st] == list(rej)


def test_aus_cooling_equals_hot_start_generator_step(ctx):
    """alpha = 1, eps = 1 is cooling: one AUS sweep on a Haar field equals the
    oracle's cooling sweep (the recipe of the cooled inputs)."""
    dims = (4, 8, 4, 8)
    U = synth.haar_field(dims, 31)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, links=U)
    vs.vs_smooth_aus(f, 2, 1.0, 1.0, vortex_preserve=False)
    Ug = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert max_abs(Ug, O.cool(dims, U, 2)) < 1e-12


@pytest.mark.parametrize("eps,storage,dims", [(-0.25, "link18", (8, 8, 8, 8)), (1.0, "link18", (8, 8, 8, 8)),
                                              (-0.25, "link12", (8, 8, 8, 8)), (-0.25, "link18", (4, 4, 12, 20))])
def test_aus_fp32_each_sweep_within_rounding(ctx, eps, storage, dims):
    """FP32 AUS + MaxReTr with VP on a centrifuged vortex field, one sweep at a
    time from the oracle's FP64 field (18- and 12-real storage; 4x4x12x20 ends
    every class launch in a partial block).  1e-6; 2e-6 for 12-real storage,
    which rebuilds row 2 of every link it reads and of the result (measured
    1.04e-6, the same with plain loads as with the link ring)."""
    lab = cooled_labels(dims, 2)
    U = O.centrifuge(dims, lab, 0.02, 1234)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12)
    worst = 0.0
    for sweep in range(30):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth_aus(f, 1, 0.02, eps, vortex_preserve=True, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U, _ = O.aus(dims, U, lab, 1, 0.02, eps=eps, vp=True)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    assert worst < (1e-6 if storage == "link18" else 2e-6)


@pytest.mark.parametrize("storage", ["link18", "link12"])
def test_fp32_cooling_general_su3_ragged(ctx, storage):
    """FP32 cooling (AUS with alpha = 1, plaquette staples, 3 MaxReTr hits: the
    input generator) from a Haar field, one sweep at a time from the oracle's
    field, on a lattice whose class launches end in a partial block.  On a hot
    field each link takes nine SU(2) rotations normalised by k = |(a, b)|,
    which is small where the random staples nearly cancel (Sec. III.A: near
    the singular subgroup rounding noise decides the rotation), so one FP32
    sweep is 50-120x the unit roundoff away from FP64 (measured 2.4e-6 with
    18-real links and 7.0e-6 with 12-real links, whose row 2 is rebuilt on
    every load; 2.8e-6 and 3.5e-6 with five-operation rebuilds): 1e-5."""
    dims = (4, 4, 12, 20)
    U = synth.haar_field(dims, 33)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    worst = 0.0
    for sweep in range(3):
        vs.vs_load_field(f, links=U)
        vs.vs_smooth_aus(f, 1, 1.0, 1.0, vortex_preserve=False, reunit_every=0)
        Ug = vs.vs_read_field(f)
        U = O.cool(dims, U, 1)
        worst = max(worst, max_abs(Ug, U))
    vs.vs_field_destroy(f)
    print("%s: worst one-sweep cooling error %.3g" % (storage, worst))
    assert worst < 1e-5


# --------------------------------------------------------------------------
# Random gauge (Sec. V.D) with the gauge-reversed vortex-preservation test
# --------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["stout", "aus"])
def test_random_gauge_smoothing_matches_oracle(ctx, method):
    """The VP recipe of the paper: centrifuge, random gauge transformation,
    annealed smoothing with the vortex-preservation test applied to
    G^dag(x) U' G(x+mu); FP64 against the oracle, identical reject counts,
    and zero gauge-reversed label differences."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    G = synth.random_gauge(dims, 41)
    U0 = O.gauge_transform(dims, O.centrifuge(dims, lab, 0.02, 1234), G)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_gauge_transform(f, G)
    assert max_abs(vs.vs_read_field(f), U0) < 1e-14
    if method == "stout":
        Uo, rej = O.smooth(dims, U0, lab, 6, 0.3, eps=-0.25, vp=True, gauge=G)
        st = vs.vs_smooth(f, 6, 0.3, -0.25, vortex_preserve=True, stats=True)
    else:
        Uo, rej = O.aus(dims, U0, lab, 10, 0.02, eps=-0.25, vp=True, gauge=G)
        st = vs.vs_smooth_aus(f, 10, 0.02, -0.25, vortex_preserve=True, stats=True)
    Ug = vs.vs_read_field(f)
    chk = vs.vs_vortex_check(f)
    vs.vs_field_destroy(f)
    assert [s["n_reject"] for s in st] == list(rej)
    assert max_abs(Ug, Uo) < 1e-10
    assert chk["n_label_diff"] == 0 and chk["n_charge_diff"] == 0
    ref = O.vortex_check(dims, Uo, lab, gauge=G)
    assert ref["n_label_diff"] == 0
    if method == "stout":
        assert rej.sum() > 0


# --------------------------------------------------------------------------
# Smoothness observables (Sec. V)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_observables_match_oracle(ctx, prec, tol):
    """Clover F, S_R(x), q(x) and S(x) per site against the oracle, on a
    smoothed centrifuged field and on the uniform two-plane flux field whose
    q(x) is known in closed form."""
    from tests.test_oracle_pins import _uniform_flux_field
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    dims = (8, 8, 4, 8)
    lab = synth.iid_labels(dims, 21)
    U = O.smooth(dims, O.centrifuge(dims, lab, 0.02, 1234), lab, 5, 0.06, eps=-0.25)[0]
    Uf, (p1, p2) = _uniform_flux_field(dims, [(0, 1, 1), (2, 3, 1)])
    for links in (U, Uf):
        f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18)
        vs.vs_load_field(f, links=links)
        r = vs.vs_observables(f, per_site=True)
        vs.vs_field_destroy(f)
        SR, Q, SRs, qs = O.observables(dims, links, per_site=True)
        S, Ss = O.action(dims, links, per_site=True)
        assert np.abs(r["S_R"] - SRs).max() < tol
        assert np.abs(r["q"] - qs).max() < tol
        assert np.abs(r["S"] - Ss).max() < tol
        assert abs(r["mean_SR"] - SR) < tol and abs(r["mean_S"] - S) < tol
        assert abs(r["Q"] - Q) < tol * int(np.prod(dims))
    assert abs(r["q"][0] - np.sin(p1) * np.sin(p2) / (2 * np.pi ** 2)) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_density_correlations_match_oracle(ctx, prec, tol):
    """C^S_XY and C^q_XY (Sec. VII, Eq. correlation_s) between the vortex-only
    field X (after the centrifuge) and the field Y after smoothing with and
    without vortex preservation, as the paper's recipe comparison does:
    vs_correlation of the library's densities (host and device input) against
    the oracle's correlation of the oracle's densities."""
    torch = pytest.importorskip("torch")
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    U0 = O.centrifuge(dims, lab, 0.02, 1234)
    fields = {"X": U0,
              "VP": O.smooth(dims, U0, lab, 10, 0.06, eps=-0.25, vp=True)[0],
              "noVP": O.smooth(dims, U0, lab, 10, 0.3, eps=-0.25, vp=False)[0]}
    dens_o, dens_g = {}, {}
    f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18)
    for k, U in fields.items():
        vs.vs_load_field(f, links=U)
        r = vs.vs_observables(f, per_site=True)
        dens_g[k] = (r["S"], r["q"])
        _, _, _, qo = O.observables(dims, U, per_site=True)
        dens_o[k] = (O.action(dims, U, per_site=True)[1], qo)
    for a, b in (("X", "VP"), ("X", "noVP"), ("VP", "noVP")):
        for d in (0, 1):
            want = O.correlation(dens_o[a][d], dens_o[b][d])
            got = vs.vs_correlation(f, dens_g[a][d], dens_g[b][d])
            dev = vs.vs_correlation(f, torch.from_numpy(dens_g[a][d]).cuda(),
                                    torch.from_numpy(dens_g[b][d]).cuda())
            assert got == dev
            assert abs(got - want) < tol, (a, b, d, got, want)
    # C(a, a) = 1 and C(a, -a) = -1 through the library as well
    S = dens_g["VP"][0]
    assert abs(vs.vs_correlation(f, S, S) - 1) < 1e-14
    assert abs(vs.vs_correlation(f, S, -S) + 1) < 1e-14
    with pytest.raises(vs.VSError):
        vs.vs_correlation(f, np.zeros_like(S), S)
    vs.vs_field_destroy(f)


def _links_at_trace_angles(thetas, dims):
    """Links 2 exp(i theta) diag(1, 0, 0): the trace sits at angle theta."""
    V = int(np.prod(dims))
    th = np.resize(np.asarray(thetas, dtype=np.float64), 4 * V)
    M = np.zeros((4 * V, 3, 3), dtype=np.complex128)
    M[:, 0, 0] = 2.0 * np.exp(1j * th)
    return M.reshape(4, V, 3, 3)


@pytest.mark.parametrize("prec,tol,planted", [("fp64", 1e-12, (1e-7, 5e-6, 2e-5, 1e-3)),
                                               ("fp32", 1e-6, (3e-6, 6e-6, 3e-5, 1e-3))])
def test_vortex_check_margins_match_oracle(ctx, prec, tol, planted):
    """vs_vortex_check's smallest margin and near-edge count (links within
    1e-5 rad of a sector edge) against the oracle's: on a smoothed vortex
    field, and on a field whose traces sit at planted distances from every
    edge (FP32: distances clear of the FP32 rounding of the stored links)."""
    p = vs.VS_FP64 if prec == "fp64" else vs.VS_FP32
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    U = O.smooth(dims, O.centrifuge(dims, lab, 0.02, 1234), lab, 15, 0.06, eps=-0.25, vp=True)[0]
    thetas = [e + sg * d for e in (np.pi / 3, -np.pi / 3, np.pi) for d in planted for sg in (1, -1)]
    Up = _links_at_trace_angles(thetas + [0.1, 2.2, -2.0], dims)
    f = vs.vs_field_create(ctx, dims, p, vs.VS_LINK18)
    for links in (U, Up):
        vs.vs_load_field(f, links=links)
        labg = vs.vs_read_labels(f)
        got = vs.vs_vortex_check(f)
        want = O.vortex_check(dims, links, labg, near_tol=1e-5)
        assert got["n_label_diff"] == want["n_label_diff"] == 0
        assert got["n_near_boundary"] == want["n_near_boundary"]
        assert abs(got["min_margin"] - want["min_margin"]) < tol
    vs.vs_field_destroy(f)
    assert want["n_near_boundary"] > 0


@pytest.mark.parametrize("vp", [True, False])
def test_per_sweep_label_diffs_and_margins_fp64(ctx, vp):
    """The per-sweep diagnostics of vs_smooth (Sec. VI; the n_diff counts of the
    paper's tables): FP64 sweeps against the oracle run one sweep at a time,
    the candidates' label differences from the reference (with VP: the
    rejections; without: the label differences after the sweep) exactly, and
    the smallest candidate margin to 1e-12."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    U = O.centrifuge(dims, lab, 0.02, 1234)
    rho = 0.06 if vp else 0.3
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    st = vs.vs_smooth(f, 8, rho, -0.25, vortex_preserve=vp, stats=True)
    vs.vs_field_destroy(f)
    n_diff_seen = 0
    for k in range(8):
        U, rej, cm, rejected = O.smooth(dims, U, lab, 1, rho, eps=-0.25, vp=vp, diagnostics=True)
        if vp:
            want_diff = int(rej[0])
        else:
            want_diff = int(np.count_nonzero(O.labels(dims, U) != lab))
        assert st[k]["n_label_diff"] == want_diff, (k, st[k], want_diff)
        assert st[k]["n_reject"] == (int(rej[0]) if vp else 0)
        assert st[k]["n_undecidable"] == 0
        # free-running FP64 trajectories drift apart by ~1e-12 over 8 sweeps at rho = 0.3
        assert abs(st[k]["min_margin"] - float(np.nanmin(cm))) < 1e-10
        n_diff_seen += want_diff
    assert n_diff_seen > 0


@pytest.mark.parametrize("method", ["aus", "ucp"])
@pytest.mark.parametrize("vp", [True, False])
def test_aus_and_ucp_per_sweep_label_diffs_fp64(ctx, method, vp):
    """The per-sweep diagnostics of vs_smooth_aus / vs_smooth_ape in the
    paper's AS setting (alpha = 0.7, a random gauge, Sec. V.D and Table
    t:recipes), FP64 against the oracle one sweep at a time: the candidates'
    label differences (in the original gauge, Sec. VI) equal the oracle's
    rejections with vortex preservation, and without it the label differences
    after the sweep; no candidate lies within the FP64 band of an edge."""
    dims = (8, 8, 8, 8)
    lab = cooled_labels(dims, 2)
    G = synth.random_gauge(dims, 43)
    U = O.gauge_transform(dims, O.centrifuge(dims, lab, 0.02, 1234), G)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_gauge_transform(f, G)
    if method == "aus":
        st = vs.vs_smooth_aus(f, 3, 0.7, -0.25, vortex_preserve=vp, stats=True)
    else:
        st = vs.vs_smooth_ape(f, 3, 0.7, -0.25, vortex_preserve=vp, stats=True)
    vs.vs_field_destroy(f)
    seen = 0
    for k in range(3):
        if method == "aus":
            U, rej = O.aus(dims, U, lab, 1, 0.7, eps=-0.25, vp=vp, gauge=G)
        else:
            U, rej = O.ape_ucp(dims, U, lab, 1, 0.7, eps=-0.25, vp=vp, gauge=G)
        want = int(rej[0]) if vp else O.vortex_check(dims, U, lab, gauge=G)["n_label_diff"]
        assert st[k]["n_label_diff"] == want, (k, st[k], want)
        assert st[k]["n_reject"] == (int(rej[0]) if vp else 0)
        assert st[k]["n_undecidable"] == 0 and 0 < st[k]["min_margin"] < np.pi / 3 + 1e-12
        seen += want
    assert seen > 0


@pytest.mark.parametrize("kind,storage", [("annealed", "link18"), ("simultaneous", "link18"),
                                          ("annealed", "link12")])
def test_fp64_redecision_in_a_random_gauge_keeps_every_label(ctx, kind, storage):
    """The FP64 re-decision reads the field's gauge transformation G for the
    gauge-reversed test (Sec. V.D, Sec. VI) and, in the simultaneous schedule,
    writes the alternate buffer: 60 free-running FP32 sweeps with vortex
    preservation re-decide candidates, and every gauge-reversed label and
    centre charge is the original one afterwards."""
    dims = (16, 16, 16, 32)
    lab = cooled_labels(dims, 2)
    G = synth.random_gauge(dims, 43)
    st = vs.VS_LINK18 if storage == "link18" else vs.VS_LINK12
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, st)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_gauge_transform(f, G)
    k = vs.VS_ANNEALED if kind == "annealed" else vs.VS_SIMULTANEOUS
    stats = vs.vs_smooth(f, 60, 0.06, -0.25, kind=k, vortex_preserve=True, stats=True, fp64_redecide=True)
    chk = vs.vs_vortex_check(f)
    vs.vs_field_destroy(f)
    n_redec = sum(s["n_fp64_redecided"] for s in stats)
    print("%s %s: %d re-decided, %d undecidable, %d rejected" % (
        kind, storage, n_redec, sum(s["n_undecidable"] for s in stats), sum(s["n_reject"] for s in stats)))
    assert n_redec > 0
    assert chk["n_label_diff"] == 0 and chk["n_charge_diff"] == 0
