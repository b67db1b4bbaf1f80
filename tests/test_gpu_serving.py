"""Serving layer: continuous batching of smoothing jobs (vs_submit / vs_poll).

A job's result must not depend on what else runs: the same job alone and in a
mix gives bit-identical links.  Admission respects the HBM budget and the slot
count; cancellation, timeouts and allocation failures are reported through
status codes without disturbing other jobs (failures are injected on the host).
"""

import ctypes
import time

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")


def _job(dims, rho, n, seed, **kw):
    V = int(np.prod(dims))
    out = np.empty((4, V, 3, 3), dtype=np.complex128)
    j = vs.make_job(dims, rho, n, seed=seed, n_cool=5, links_out=out, **kw)
    return j, out


def test_job_alone_and_in_mix_are_bit_identical():
    dims = (8, 8, 8, 8)
    ctx = vs.vs_create(0, max_slots=1)
    j, alone = _job(dims, 0.07, 40, seed=100)
    r_alone = vs.vs_poll(ctx, vs.vs_submit(ctx, j), -1)
    vs.vs_destroy(ctx)
    assert r_alone["status"] == vs.VS_OK

    ctx = vs.vs_create(0, max_slots=6)
    others = []
    for k, shp in enumerate([(12, 12, 12, 24), (8, 8, 8, 8), (16, 16, 16, 32), (8, 8, 8, 16)]):
        jo, oo = _job(shp, 0.05 + 0.01 * k, 30 + 10 * k, seed=200 + k)
        others.append((vs.vs_submit(ctx, jo), jo, oo))
    j2, mixed = _job(dims, 0.07, 40, seed=100)
    t = vs.vs_submit(ctx, j2)
    r_mix = vs.vs_poll(ctx, t, -1)
    res = [vs.vs_poll(ctx, tt, -1) for tt, _, _ in others]
    st = vs.vs_serve_stats_get(ctx)
    vs.vs_destroy(ctx)
    assert r_mix["status"] == vs.VS_OK and all(r["status"] == vs.VS_OK for r in res)
    assert np.array_equal(alone, mixed)
    assert r_alone["action"] == r_mix["action"]
    assert r_alone["n_reject"] == r_mix["n_reject"]
    assert st["completed"] == 5


def test_served_job_equals_direct_field_pipeline():
    dims = (8, 8, 4, 8)
    lab = synth.iid_labels(dims, 7)
    ctx = vs.vs_create(0)
    V = int(np.prod(dims))
    out = np.empty((4, V, 3, 3), dtype=np.complex128)
    j = vs.make_job(dims, 0.06, 25, labels=lab, omega=0.02, centrifuge_seed=1234,
                    links_out=out, precision=vs.VS_FP64)
    r = vs.vs_poll(ctx, vs.vs_submit(ctx, j), -1)
    assert r["status"] == vs.VS_OK
    f = vs.vs_field_create(ctx, dims, vs.VS_FP64, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    vs.vs_smooth(f, 25, 0.06, -0.25, reunit_every=10)
    U = vs.vs_read_field(f)
    S = vs.vs_action(f)
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)
    assert np.array_equal(U, out)
    assert S == r["action"]
    # and the served FP64 result agrees with the oracle
    Uo, rej = O.smooth(dims, O.centrifuge(dims, lab, 0.02, 1234), lab, 25, 0.06, eps=-0.25)
    assert np.abs(out - Uo).max() < 1e-11
    assert r["n_reject"] == int(rej.sum())


def test_admission_respects_budget_and_slots():
    dims = (12, 12, 12, 24)
    # a job's device footprint: links and two label planes over the layout's
    # plane stride, the partials, and the host-label staging
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    P = vs.vs_field_describe(f)["plane_stride"]
    vs.vs_field_destroy(f)
    vs.vs_destroy(ctx)
    one = 4 * 18 * 4 * P + 8 * P + 1216 * 8 + 4096 + 4 * 41472
    budget = int(2.5 * one)
    ctx = vs.vs_create(0, hbm_budget_bytes=budget, max_slots=8)
    ts = []
    for k in range(6):
        j = vs.make_job(dims, 0.05, 40, seed=300 + k, n_cool=2)
        ts.append((vs.vs_submit(ctx, j), j))
    res = [vs.vs_poll(ctx, t, -1) for t, _ in ts]
    st = vs.vs_serve_stats_get(ctx)
    vs.vs_destroy(ctx)
    assert all(r["status"] == vs.VS_OK for r in res)
    assert st["peak_bytes_in_use"] <= budget
    assert st["peak_bytes_in_use"] >= 2 * one          # two jobs did share the device
    # later jobs waited for memory to free up
    admits = sorted(r["t_admit_ms"] - r["t_submit_ms"] for r in res)
    assert admits[-1] > admits[0]


def test_job_larger_than_budget_fails_cleanly():
    ctx = vs.vs_create(0, hbm_budget_bytes=1 << 20)
    j = vs.make_job((16, 16, 16, 32), 0.05, 10, seed=1, n_cool=0)
    r = vs.vs_poll(ctx, vs.vs_submit(ctx, j), 10000)
    vs.vs_destroy(ctx)
    assert r["status"] == vs.VS_ENOMEM


def test_cancel_and_poll_timeouts():
    ctx = vs.vs_create(0, max_slots=1)
    long_job = vs.make_job((16, 16, 16, 32), 0.05, 3000, seed=5, n_cool=0)
    short = vs.make_job((8, 8, 8, 8), 0.05, 10, seed=6, n_cool=0)
    t1 = vs.vs_submit(ctx, long_job)
    t2 = vs.vs_submit(ctx, short)
    assert vs.vs_poll(ctx, t2, 0) is None                # EAGAIN: waiting behind t1
    assert vs.vs_poll(ctx, t2, 50) is None               # ETIMEDOUT
    vs.vs_cancel(ctx, t1)
    r1 = vs.vs_poll(ctx, t1, 60000)
    r2 = vs.vs_poll(ctx, t2, 60000)
    with pytest.raises(vs.VSError) as ei:
        vs.vs_poll(ctx, t1, 0)                           # retired ticket
    assert ei.value.status == vs.VS_ENOTFOUND
    st = vs.vs_serve_stats_get(ctx)
    vs.vs_destroy(ctx)
    assert r1["status"] == vs.VS_ECANCELED
    assert r2["status"] == vs.VS_OK
    assert st["cancelled"] == 1 and st["completed"] == 1


def test_queue_cap_gives_ebusy():
    ctx = vs.vs_create(0, max_slots=1, max_queue=2)
    j = vs.make_job((16, 16, 16, 32), 0.05, 2000, seed=5, n_cool=0)
    ts = [vs.vs_submit(ctx, j)]
    time.sleep(0.2)                                      # first job admitted
    ts += [vs.vs_submit(ctx, j), vs.vs_submit(ctx, j)]
    with pytest.raises(vs.VSError) as ei:
        vs.vs_submit(ctx, j)
    assert ei.value.status == vs.VS_EBUSY
    for t in ts:
        vs.vs_cancel(ctx, t)
    vs.vs_destroy(ctx)


def test_submit_rejects_bad_jobs():
    """vs_submit refuses a malformed job before queueing it: extents that are
    not positive multiples of 4, more than 2^30 sites, a negative count, a
    centrifuge angle at or above 1/4, a non-finite step, a label outside
    {-1, 0, 1} (EINVAL); FP64 with 12-real storage (EUNSUPPORTED).  Nothing
    reaches the queue."""
    ctx = vs.vs_create(0)
    dims = (4, 4, 4, 4)
    bad_labels = np.zeros((4, 256), dtype=np.int8)
    bad_labels[2, 17] = 2
    cases = [(vs.make_job((6, 4, 4, 4), 0.05, 1), vs.VS_EINVAL),
             (vs.make_job((2048, 2048, 2048, 4), 0.05, 1), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, -1), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, 1, n_cool=-2), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, 1, omega=0.25), vs.VS_EINVAL),
             (vs.make_job(dims, float("nan"), 1), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, 1, u0=0.0), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, 1, labels=bad_labels), vs.VS_EINVAL),
             (vs.make_job(dims, 0.05, 1, precision=vs.VS_FP64, storage=vs.VS_LINK12), vs.VS_EUNSUPPORTED)]
    for job, status in cases:
        with pytest.raises(vs.VSError) as ei:
            vs.vs_submit(ctx, job)
        assert ei.value.status == status
    assert vs.vs_serve_stats_get(ctx)["submitted"] == 0
    vs.vs_destroy(ctx)


def test_allocation_failure_is_reported_and_isolated():
    """Host-side fault injection: the allocator hook refuses every allocation
    after the first N; the job that hits it reports VS_ENOMEM, memory it did
    get is returned, and jobs after it still run."""
    import torch
    real = vs.TorchAllocator(0)
    state = {"left": 2, "live": 0}

    @vs._ALLOC_FN
    def alloc(n, user):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        state["live"] += 1
        return real._alloc(n, user)

    @vs._FREE_FN
    def free(p, user):
        state["live"] -= 1
        real._free(p, user)

    class Hook:
        alloc_fn = alloc
        free_fn = free

    ctx = vs.vs_create(0, allocator=Hook(), max_slots=1)
    j = vs.make_job((8, 8, 8, 8), 0.05, 10, seed=9, n_cool=0)
    r = vs.vs_poll(ctx, vs.vs_submit(ctx, j), 30000)
    assert r["status"] == vs.VS_ENOMEM
    assert state["live"] == 0                            # nothing leaked
    state["left"] = 1000
    r2 = vs.vs_poll(ctx, vs.vs_submit(ctx, j), 30000)
    vs.vs_destroy(ctx)
    assert r2["status"] == vs.VS_OK
    assert state["live"] == 0
    torch.cuda.synchronize()


def test_chunk_graphs_are_reused_per_shape():
    """Jobs of one shape, one after another (one slot), with different labels,
    step sizes and sweep counts: the first instantiates its chunk graph, the
    next ones take it from the shape's pool and update it with their own
    field and parameters; every result equals the direct field pipeline bit
    for bit (FP32 18-real, two chunks and a partial one each)."""
    dims = (8, 8, 8, 16)
    ctx = vs.vs_create(0, max_slots=1)
    V = int(np.prod(dims))
    specs = [(0.06, 25, 31), (0.08, 23, 32), (0.05, 27, 33)]
    outs, tickets = [], []
    for rho, n, seed in specs:
        lab = synth.iid_labels(dims, seed)
        out = np.empty((4, V, 3, 3), dtype=np.complex128)
        j = vs.make_job(dims, rho, n, labels=lab, omega=0.02, centrifuge_seed=1234, links_out=out)
        tickets.append((vs.vs_submit(ctx, j), j, lab))
        outs.append(out)
    res = [vs.vs_poll(ctx, t, -1) for t, _, _ in tickets]
    st = vs.vs_serve_stats_get(ctx)
    for (rho, n, seed), (t, j, lab), out, r in zip(specs, tickets, outs, res):
        assert r["status"] == vs.VS_OK
        f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
        vs.vs_load_field(f, labels=lab)
        vs.vs_centrifuge(f, 0.02, 1234)
        vs.vs_smooth(f, n, rho, -0.25, reunit_every=10)
        U = vs.vs_read_field(f)
        vs.vs_field_destroy(f)
        assert np.array_equal(U, out), (rho, n, seed)
    vs.vs_destroy(ctx)
    assert st["graphs_instantiated"] == 1 and st["graphs_reused"] == 2, st


def test_served_job_with_fp64_redecision_equals_direct_pipeline():
    """A served FP32 job with the FP64 re-decision (vs_job.fp64_redecide: its
    chunk graphs hold the re-decision launches and are pooled apart from the
    FP32-decision graphs) gives the links of the same pipeline on a field,
    alone and in a mix with FP32-decision jobs of the same shape."""
    from tests.gpu_common import cooled_labels
    dims = (16, 16, 16, 32)
    lab = cooled_labels(dims, 2)
    V = int(np.prod(dims))
    ctx = vs.vs_create(0)
    f = vs.vs_field_create(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
    vs.vs_load_field(f, labels=lab)
    vs.vs_centrifuge(f, 0.02, 1234)
    st = vs.vs_smooth(f, 60, 0.06, -0.25, reunit_every=10, stats=True, fp64_redecide=True)
    U = vs.vs_read_field(f)
    vs.vs_field_destroy(f)
    assert sum(s["n_fp64_redecided"] for s in st) > 0
    outs = []
    for mix in (False, True):
        jobs = []
        if mix:
            for k in range(2):
                o = np.empty((4, V, 3, 3), dtype=np.complex128)
                jobs.append((vs.make_job(dims, 0.05, 40, labels=lab, omega=0.02, centrifuge_seed=1234,
                                         links_out=o), o))
        out = np.empty((4, V, 3, 3), dtype=np.complex128)
        j = vs.make_job(dims, 0.06, 60, labels=lab, omega=0.02, centrifuge_seed=1234, links_out=out,
                        fp64_redecide=True)
        tickets = [vs.vs_submit(ctx, jj) for jj, _ in jobs] + [vs.vs_submit(ctx, j)]
        res = [vs.vs_poll(ctx, t, -1) for t in tickets]
        assert all(r["status"] == vs.VS_OK for r in res)
        outs.append(out)
    vs.vs_destroy(ctx)
    assert np.array_equal(outs[0], U) and np.array_equal(outs[1], U)
