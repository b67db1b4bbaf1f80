"""Host-only checks of the C ABI: the library builds, loads and exports every
function include/vs.h declares; pure host helpers behave.  No GPU needed."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libvs():
    from paper_2203_09764_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared_functions():
    with open(os.path.join(ROOT, "include", "vs.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(vs_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_function_is_exported(libvs):
    names = _declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(libvs, n)]
    assert not missing, missing


def test_binding_names_match_the_abi(libvs):
    from paper_2203_09764_gb300 import vs
    for n in _declared_functions():
        assert hasattr(vs, n), n


def test_layout_index_groups_x_by_residue(libvs):
    from paper_2203_09764_gb300 import vs
    dims = (8, 4, 4, 8)
    seen = set()
    for t in range(8):
        for z in range(4):
            for y in range(4):
                for x in range(8):
                    i = vs.vs_layout_index(dims, (x, y, z, t))
                    row = y + 4 * (z + 4 * t)
                    assert i == row * 8 + (x % 4) * 2 + x // 4
                    seen.add(i)
    assert seen == set(range(8 * 4 * 4 * 8))


@pytest.mark.parametrize("Lx,Qp", [(20, 8), (24, 8), (28, 8), (12, 3), (16, 4), (48, 12)])
def test_layout_index_pads_short_groups_to_a_line(libvs, Lx, Qp):
    """Rows whose x mod 4 groups hold 5, 6 or 7 sites get 8 positions per
    group (a float4 plane's 128-byte line), the others none; positions stay
    distinct and inside the plane."""
    from paper_2203_09764_gb300 import vs
    dims = (Lx, 4, 4, 4)
    seen = set()
    for t in range(4):
        for z in range(4):
            for y in range(4):
                row = y + 4 * (z + 4 * t)
                for x in range(Lx):
                    i = vs.vs_layout_index(dims, (x, y, z, t))
                    assert i == row * 4 * Qp + (x % 4) * Qp + x // 4
                    seen.add(i)
    assert len(seen) == Lx * 64 and max(seen) < 4 * Qp * 64


def test_version_and_error_string(libvs):
    from paper_2203_09764_gb300 import vs
    assert "sm_103a" in vs.vs_version()
    assert isinstance(vs.vs_last_error(), str)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2203_09764_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    txt = f.read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "vs_oracle" not in txt, fn


def test_binding_checks_buffers_before_the_call(libvs):
    """The binding checks what the C side cannot see in a plain pointer: the
    element type, contiguity and byte size of every buffer (host arrays here;
    CUDA tensors also get a device check), so a wrong buffer raises in Python
    instead of reaching a kernel."""
    import numpy as np
    import torch
    from paper_2203_09764_gb300 import vs
    V = 16
    ok = [(np.zeros((4, V, 3, 3), np.complex128), "c", 36 * V),
          (np.zeros((4, V, 3, 3, 2), np.float64), "c", 36 * V),
          (torch.zeros((4, V, 3, 3), dtype=torch.complex128), "c", 36 * V),
          (np.zeros((4, V), np.int8), "i8", 4 * V),
          (torch.zeros((4, V), dtype=torch.int8), "i8", 4 * V)]
    for a, kind, n in ok:
        p, where = vs._buf(None, a, kind, n, "buffer")
        assert where == vs.VS_HOST and p.value
    bad = [(np.zeros((4, V, 3, 3), np.complex64), "c", 36 * V, TypeError),
           (torch.zeros((4, V, 3, 3), dtype=torch.complex64), "c", 36 * V, TypeError),
           (np.zeros((4, V, 3, 3), np.float64), "c", 36 * V, ValueError),        # real, half the bytes
           (np.zeros((4, V - 1, 3, 3), np.complex128), "c", 36 * V, ValueError),
           (np.zeros((4, 2 * V, 3, 3), np.complex128)[:, ::2], "c", 36 * V, ValueError),
           (np.zeros((4, V), np.int16), "i8", 4 * V, TypeError),
           (np.zeros((4, V + 1), np.int8), "i8", 4 * V, ValueError),
           ([0] * (4 * V), "i8", 4 * V, TypeError)]
    for a, kind, n, err in bad:
        with pytest.raises(err):
            vs._buf(None, a, kind, n, "buffer")
    # host link input: complex128 and float64 pairs pass unchanged, others convert
    a = np.zeros((4, V, 3, 3, 2))
    assert vs._host_links(a) is a
    assert vs._host_links(np.zeros((4, V, 3, 3), np.complex64)).dtype == np.complex128


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No fallback: with no libvs.so where the binding looks, importing it
    raises ImportError naming the missing library, and the product package
    never imports the oracle."""
    import subprocess
    import sys
    env = dict(os.environ, VS_BUILD_DIR=str(tmp_path / "empty"))
    r = subprocess.run([sys.executable, "-c", "import paper_2203_09764_gb300.vs"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libvs.so is not built" in r.stderr
    r = subprocess.run([sys.executable, "-c",
                        "import sys, paper_2203_09764_gb300.vs; "
                        "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))"],
                       cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "[]"


def test_oracle_and_product_share_no_code():
    """The oracle and the GPU path are independent: no include or import
    crosses between oracle/ and the product (csrc, include/, the binding),
    and the shared seeded input generators (synth/) import neither."""
    import glob
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    imp = re.compile(r"^\s*(?:from|import)\s+([A-Za-z_][\w.]*)", re.M)

    def text(p):
        with open(p) as f:
            return f.read()

    product_c = glob.glob(os.path.join(ROOT, "paper_2203_09764_gb300", "csrc", "*"))
    product_c += glob.glob(os.path.join(ROOT, "include", "*.h"))
    for p in product_c:
        for h in inc.findall(text(p)):
            assert "oracle" not in h, (p, h)
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        for h in inc.findall(text(p)):
            assert not any(k in h for k in ("vs.h", "csrc", "paper_2203", ".cuh", "vs_")), (p, h)
    for p in glob.glob(os.path.join(ROOT, "paper_2203_09764_gb300", "*.py")):
        for m in imp.findall(text(p)):
            assert not (m == "oracle" or m.startswith("oracle.")), (p, m)
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for m in imp.findall(text(p)):
            assert not m.startswith("paper_2203_09764_gb300"), (p, m)
    for p in glob.glob(os.path.join(ROOT, "synth", "*.py")):
        for m in imp.findall(text(p)):
            assert not (m.startswith("oracle") or m.startswith("paper_2203_09764_gb300")), (p, m)
    assert product_c and glob.glob(os.path.join(ROOT, "oracle", "*.c"))


STRUCTS = ["vs_options", "vs_anneal", "vs_sweep_stats", "vs_vortex_report", "vs_observables_out",
           "vs_field_desc", "vs_job", "vs_result", "vs_serve_stats"]


def test_binding_structs_match_the_header(libvs, tmp_path):
    """Every public struct of include/vs.h and its ctypes mirror in the binding
    agree on size, field names, order and offsets (compiled with the host C
    compiler against the header itself)."""
    import shutil
    import subprocess
    from paper_2203_09764_gb300 import vs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vs.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(vs, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, value = line.split()
            got[(name, field)] = int(value)
    for name in STRUCTS:
        cls = getattr(vs, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
