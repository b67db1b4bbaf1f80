"""vs_vortex_check_noalloc: the vortex check for callers that cannot allocate.

Through the C ABI, its reports must equal those of vs_vortex_check (integer
counts exactly, the minimum margin exactly: same kernels, same inputs) on two
calls in a row, so that the shared scratch array carries nothing over from one
call to the next.  Kept in its own file so pytest collects it last.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

vs = pytest.importorskip("paper_2203_09764_gb300.vs")


def _smoothed_field(ctx, dims, precision, storage, gauge=False):
    f = vs.vs_field_create(ctx, dims, precision, storage)
    vs.vs_load_cooled(f, 7, 3)
    vs.vs_centrifuge(f, 0.02, 1234)
    if gauge:
        import synth
        vs.vs_gauge_transform(f, synth.random_gauge(dims, 41))
    # without vortex preservation and with large steps some labels move, so
    # the counts under test are not all zero
    vs.vs_smooth(f, 3, 0.3, -0.25, vortex_preserve=False)
    vs.vs_synchronize(f)
    return f


@pytest.mark.parametrize("precision,storage,dims,gauge", [
    (vs.VS_FP32, vs.VS_LINK18, (16, 16, 16, 32), False),
    (vs.VS_FP64, vs.VS_LINK18, (8, 8, 8, 16), False),
    (vs.VS_FP32, vs.VS_LINK12, (8, 8, 12, 16), False),
    (vs.VS_FP32, vs.VS_LINK18, (8, 8, 8, 16), True),
    (vs.VS_FP64, vs.VS_LINK18, (8, 8, 8, 8), True),
    (vs.VS_FP32, vs.VS_LINK18, (32, 32, 32, 64), False),   # exactly VS_NOALLOC_MAX_LINKS links
])
def test_noalloc_matches_field_check_on_two_calls(precision, storage, dims, gauge):
    """Equal reports on two calls in a row; in a random gauge (Sec. V.D) the
    check reads the field's G, as vs_vortex_check does; and at the largest
    lattice the fixed scratch admits."""
    ctx = vs.vs_create(0)
    try:
        f = _smoothed_field(ctx, dims, precision, storage, gauge)
        ref = vs.vs_vortex_check(f)
        assert ref["n_label_diff"] > 0 and ref["n_charge_diff"] > 0
        d = vs.vs_field_describe(f)
        assert (d["gauge"] is not None) == gauge
        if 4 * int(np.prod(dims)) == vs.VS_NOALLOC_MAX_LINKS:
            assert d["n_sites"] * 4 == vs.VS_NOALLOC_MAX_LINKS
        got = [vs.vs_vortex_check_noalloc(d["links"], d["labels"], dims, precision, storage,
                                          d["stream"], gauge=d["gauge"]) for _ in range(2)]
        if gauge:
            # without G the labels of the gauge-rotated links are tested: a different report
            plain = vs.vs_vortex_check_noalloc(d["links"], d["labels"], dims, precision, storage, d["stream"])
            assert plain["n_label_diff"] != ref["n_label_diff"]
        vs.vs_field_destroy(f)
    finally:
        vs.vs_destroy(ctx)
    for g in got:
        assert g["n_links"] == ref["n_links"]
        assert g["n_label_diff"] == ref["n_label_diff"]
        assert g["n_charge_diff"] == ref["n_charge_diff"]
        assert g["n_near_boundary"] == ref["n_near_boundary"]
        assert g["min_margin"] == ref["min_margin"]


def test_noalloc_rejects_lattices_beyond_its_scratch():
    dims = (32, 32, 32, 128)          # 4 V = 2^24 links > VS_NOALLOC_MAX_LINKS
    with pytest.raises(vs.VSError) as ei:
        vs.vs_vortex_check_noalloc(1, 1, dims, vs.VS_FP32, vs.VS_LINK18)
    assert ei.value.status == vs.VS_EINVAL
    assert "scratch" in str(ei.value)
    assert 4 * 32 * 32 * 32 * 64 <= vs.VS_NOALLOC_MAX_LINKS


_FIRST_CALL_IN_CAPTURE = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2203_09764_gb300 import vs
dims = (8, 8, 8, 8)
V = 8 ** 4
torch.manual_seed(0)
links = torch.randn(4 * 18 * V, device="cuda:0", dtype=torch.float32)   # any values: labels follow
labels = torch.zeros(4 * V, device="cuda:0", dtype=torch.int8)
work = torch.cuda.Stream()
args = (links.data_ptr(), labels.data_ptr(), dims, vs.VS_FP32, vs.VS_LINK18, work)
x = torch.zeros(1024, device="cuda:0")
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    x.add_(1.0)
    first = vs.vs_vortex_check_noalloc(*args)     # the first call on this device, mid-capture
    x.mul_(3.0)
g.replay()
torch.cuda.synchronize()
second = vs.vs_vortex_check_noalloc(*args)
assert first == second, (first, second)
assert first["n_label_diff"] > 0
assert float(x[0]) == 3.0
print("first call in capture ok", first["n_label_diff"])
"""


def test_noalloc_first_call_during_a_capture_in_a_fresh_process():
    """In a process where no vs_create ran, the first call on the device (which
    does the once-per-device set-up) is made while another stream of the
    thread captures a graph in the global mode: it succeeds, leaves the
    capture valid, and a later call reports the same."""
    pytest.importorskip("torch")
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_IN_CAPTURE, root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "first call in capture ok" in r.stdout


def test_noalloc_while_another_stream_captures_a_graph():
    """The use the call exists for: a graph is being captured on another
    stream of this thread (torch's default global capture mode, which forbids
    allocation), and the check runs on the field's own stream in the middle
    of it.  The report equals vs_vortex_check's and the captured graph still
    replays correctly."""
    torch = pytest.importorskip("torch")
    dims = (8, 8, 8, 16)
    ctx = vs.vs_create(0)
    try:
        f = _smoothed_field(ctx, dims, vs.VS_FP32, vs.VS_LINK18)
        ref = vs.vs_vortex_check(f)
        d = vs.vs_field_describe(f)
        args = (d["links"], d["labels"], dims, vs.VS_FP32, vs.VS_LINK18, d["stream"])
        vs.vs_vortex_check_noalloc(*args)            # first call on this device: before any capture
        x = torch.zeros(4096, device="cuda:0")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            got = vs.vs_vortex_check_noalloc(*args)
            x.mul_(3.0)
        g.replay()
        torch.cuda.synchronize()
        vs.vs_field_destroy(f)
    finally:
        vs.vs_destroy(ctx)
    assert got == ref
    assert float(x[0]) == 3.0 and float(x[-1]) == 3.0
