"""ctypes wrapper of the C oracle (vs_oracle.c), plus build helper.

TEST INFRASTRUCTURE ONLY.  All arrays follow the layouts stated in
``vs_oracle.c``: links complex128 [4][V][3][3], labels int8 [4][V].
"""

import ctypes
import os
import subprocess

import numpy as np

__all__ = [
    "build_oracle", "lib", "max_threads", "use_library", "compile_variant", "source",
    "label_matrix", "labels", "links_from_labels", "splitmix64", "centrifuge_pair",
    "centrifuge", "overimproved_coeffs", "staple_sum", "expm", "stout_generator",
    "colour", "smooth", "action", "centre_charges", "vortex_check", "correlation", "gauge_transform",
    "cool", "aus", "maxretr", "observables", "reunit", "ucp", "ape_ucp", "flow_rk3", "ANNEALED", "SIMULTANEOUS",
]

ANNEALED = 0
SIMULTANEOUS = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vs_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build_oracle(force=False):
    """Compile vs_oracle.c with gcc (IEEE arithmetic, no FMA contraction)."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fcx-limited-range", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


def _bind(path):
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(build_oracle())
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of
    vs_oracle.c (the mutation tests load deliberately broken copies)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _bind(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_variant(src_text, out_path):
    """Compile a modified oracle source (same flags as the real build)."""
    src = out_path[:-3] + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-fcx-limited-range", "-o", out_path, src, "-lm"])
    return out_path


def source():
    with open(_SRC) as f:
        return f.read()


def _declare(L):
    P = ctypes.c_void_p
    u64, dbl = ctypes.c_uint64, ctypes.c_double
    sig = {
        "or_label_matrix": (ctypes.c_int, [P]),
        "or_labels": (ctypes.c_int, [P, P, P, P]),
        "or_links_from_labels": (ctypes.c_int, [P, P, P]),
        "or_splitmix64": (u64, [u64, u64]),
        "or_centrifuge_pair": (ctypes.c_int, [u64, ctypes.c_long, ctypes.c_int, ctypes.c_long]),
        "or_centrifuge": (ctypes.c_int, [P, P, dbl, u64, P, P]),
        "or_overimproved_coeffs": (None, [dbl, dbl, P, P]),
        "or_staple_sum": (ctypes.c_int, [P, P, ctypes.c_int, P, dbl, dbl, P]),
        "or_expm": (ctypes.c_int, [P, P]),
        "or_stout_generator": (ctypes.c_int, [P, P]),
        "or_colour": (ctypes.c_int, [P, ctypes.c_int, P]),
        "or_smooth": (ctypes.c_int, [P, P, P, ctypes.c_int, P, dbl, dbl,
                                     ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P]),
        "or_action": (ctypes.c_int, [P, P, P, P]),
        "or_centre_charges": (ctypes.c_int, [P, P, P]),
        "or_vortex_check": (ctypes.c_int, [P, P, P, P, P, P, P, dbl, P]),
        "or_correlation": (ctypes.c_int, [ctypes.c_long, P, P, P]),
        "or_gauge_transform": (ctypes.c_int, [P, P, P]),
        "or_cool": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "or_aus": (ctypes.c_int, [P, P, P, ctypes.c_int, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                  P, ctypes.c_int, P]),
        "or_maxretr": (ctypes.c_int, [P, P, ctypes.c_int, P]),
        "or_observables": (ctypes.c_int, [P, P, P, P, P, P]),
        "or_ucp": (ctypes.c_int, [P, P]),
        "or_reunit": (ctypes.c_int, [ctypes.c_long, P, P]),
        "or_ape_ucp": (ctypes.c_int, [P, P, P, ctypes.c_int, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                      P, ctypes.c_int, P]),
        "or_flow_rk3": (ctypes.c_int, [P, P, ctypes.c_int, dbl, dbl, dbl, ctypes.c_int]),
        "or_max_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def max_threads():
    return int(lib().or_max_threads())


def _c128(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def label_matrix(M):
    M = _c128(M, (3, 3))
    return int(lib().or_label_matrix(_p(M)))


def labels(dims, links, with_margin=False):
    d = _dims(dims)
    U = _c128(links)
    V = U.size // 36
    lab = np.empty(4 * V, dtype=np.int8)
    mar = np.empty(4 * V, dtype=np.float64) if with_margin else None
    _check(lib().or_labels(_p(d), _p(U), _p(lab), _p(mar) if with_margin else None), "labels")
    lab = lab.reshape(4, V)
    return (lab, mar.reshape(4, V)) if with_margin else lab


def links_from_labels(dims, lab):
    d = _dims(dims)
    lab = np.ascontiguousarray(lab, dtype=np.int8)
    V = lab.size // 4
    U = np.empty((4, V, 3, 3), dtype=np.complex128)
    _check(lib().or_links_from_labels(_p(d), _p(lab), _p(U)), "links_from_labels")
    return U


def splitmix64(seed, i):
    return int(lib().or_splitmix64(seed, i))


def centrifuge_pair(seed, V, mu, s):
    return int(lib().or_centrifuge_pair(seed, V, mu, s))


def centrifuge(dims, lab, omega, seed, with_sigma=False):
    d = _dims(dims)
    lab = np.ascontiguousarray(lab, dtype=np.int8)
    V = lab.size // 4
    U = np.empty((4, V, 3, 3), dtype=np.complex128)
    sig = np.empty((4, V), dtype=np.float64) if with_sigma else None
    _check(lib().or_centrifuge(_p(d), _p(lab), omega, seed, _p(U),
                               _p(sig) if with_sigma else None), "centrifuge")
    return (U, sig) if with_sigma else U


def overimproved_coeffs(eps, u0=1.0):
    c0 = ctypes.c_double()
    c1 = ctypes.c_double()
    lib().or_overimproved_coeffs(eps, u0, ctypes.byref(c0), ctypes.byref(c1))
    return c0.value, c1.value


def staple_sum(dims, links, mu, x, c0, c1):
    d = _dims(dims)
    U = _c128(links)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
    S = np.empty((3, 3), dtype=np.complex128)
    _check(lib().or_staple_sum(_p(d), _p(U), mu, _p(xx), c0, c1, _p(S)), "staple_sum")
    return S


def expm(X):
    X = _c128(X, (3, 3))
    E = np.empty((3, 3), dtype=np.complex128)
    _check(lib().or_expm(_p(X), _p(E)), "expm")
    return E


def stout_generator(Omega):
    Om = _c128(Omega, (3, 3))
    Q = np.empty((3, 3), dtype=np.complex128)
    _check(lib().or_stout_generator(_p(Om), _p(Q)), "stout_generator")
    return Q


def colour(dims, mu, x):
    d = _dims(dims)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
    return int(lib().or_colour(_p(d), mu, _p(xx)))


def smooth(dims, links, ref_labels, n_sweeps, rho, eps=1.0, u0=1.0,
           schedule=ANNEALED, vp=True, nthreads=None, diagnostics=False, gauge=None):
    """n_sweeps of stout smoothing on a copy of ``links``; returns (links, n_reject),
    plus (candidate margins, rejected mask) of the last sweep with diagnostics=True."""
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    if np.isscalar(rho):
        rho = np.full(n_sweeps, float(rho))
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.size < n_sweeps:
        raise ValueError("rho schedule shorter than n_sweeps")
    ref = None if ref_labels is None else np.ascontiguousarray(ref_labels, dtype=np.int8)
    rej = np.zeros(max(n_sweeps, 1), dtype=np.int64)
    nt = max_threads() if nthreads is None else int(nthreads)
    V = U.size // 36
    cm = np.full((4, V), np.nan) if diagnostics else None
    rj = np.zeros((4, V), dtype=np.int8) if diagnostics else None
    G = None if gauge is None else _c128(gauge)
    _check(lib().or_smooth(_p(d), _p(U), _p(ref) if ref is not None else None, n_sweeps,
                           _p(rho), eps, u0, schedule, 1 if vp else 0, _p(rej), nt,
                           _p(cm) if diagnostics else None, _p(rj) if diagnostics else None,
                           _p(G) if G is not None else None),
           "smooth")
    if diagnostics:
        return U, rej[:n_sweeps], cm, rj
    return U, rej[:n_sweeps]


def action(dims, links, per_site=False):
    d = _dims(dims)
    U = _c128(links)
    V = U.size // 36
    m = ctypes.c_double()
    S = np.empty(V, dtype=np.float64) if per_site else None
    _check(lib().or_action(_p(d), _p(U), ctypes.byref(m), _p(S) if per_site else None), "action")
    return (m.value, S) if per_site else m.value


def centre_charges(dims, lab):
    d = _dims(dims)
    lab = np.ascontiguousarray(lab, dtype=np.int8)
    V = lab.size // 4
    ch = np.empty((6, V), dtype=np.int8)
    _check(lib().or_centre_charges(_p(d), _p(lab), _p(ch)), "centre_charges")
    return ch


def vortex_check(dims, links, ref_labels, gauge=None, near_tol=1e-5):
    """Label and centre-charge differences against ref_labels, the smallest
    angular margin of arg Tr U from a sector edge, and the number of links
    with a margin below near_tol."""
    d = _dims(dims)
    U = _c128(links)
    ref = np.ascontiguousarray(ref_labels, dtype=np.int8)
    nd = ctypes.c_int64()
    nc = ctypes.c_int64()
    nn = ctypes.c_int64()
    mm = ctypes.c_double()
    G = None if gauge is None else _c128(gauge)
    _check(lib().or_vortex_check(_p(d), _p(U), _p(ref), ctypes.byref(nd), ctypes.byref(nc),
                                 ctypes.byref(mm), _p(G) if G is not None else None,
                                 float(near_tol), ctypes.byref(nn)), "vortex_check")
    return dict(n_label_diff=nd.value, n_charge_diff=nc.value, min_margin=mm.value,
                n_near_boundary=nn.value)


def correlation(a, b):
    """C_XY of two per-site densities (Sec. VII, Eq. correlation_s)."""
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    if a.size != b.size:
        raise ValueError("densities of different sizes")
    C = ctypes.c_double()
    _check(lib().or_correlation(a.size, _p(a), _p(b), ctypes.byref(C)), "correlation")
    return C.value


def gauge_transform(dims, links, G):
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    Gc = _c128(G)
    _check(lib().or_gauge_transform(_p(d), _p(U), _p(Gc)), "gauge_transform")
    return U


def cool(dims, links, n_sweeps, n_hits=3, nthreads=None):
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    nt = max_threads() if nthreads is None else int(nthreads)
    _check(lib().or_cool(_p(d), _p(U), n_sweeps, n_hits, nt), "cool")
    return U


def aus(dims, links, ref_labels, n_sweeps, alpha, eps=1.0, u0=1.0, n_hits=3, vp=True, nthreads=None,
        gauge=None):
    """n_sweeps of annealed U-link smearing with MaxReTr; returns (links, n_reject)."""
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    ref = None if ref_labels is None else np.ascontiguousarray(ref_labels, dtype=np.int8)
    rej = np.zeros(max(n_sweeps, 1), dtype=np.int64)
    nt = max_threads() if nthreads is None else int(nthreads)
    G = None if gauge is None else _c128(gauge)
    _check(lib().or_aus(_p(d), _p(U), _p(ref) if ref is not None else None, n_sweeps, alpha, eps,
                        u0, n_hits, 1 if vp else 0, _p(rej), nt, _p(G) if G is not None else None),
           "aus")
    return U, rej[:n_sweeps]


def maxretr(U, V, n_hits=3):
    Uc = _c128(U, (3, 3))
    Vc = _c128(V, (3, 3))
    out = np.empty((3, 3), dtype=np.complex128)
    _check(lib().or_maxretr(_p(Uc), _p(Vc), n_hits, _p(out)), "maxretr")
    return out


def reunit(M):
    """Gram-Schmidt re-unitarisation of a stack of 3x3 matrices (rows 0, 1
    orthonormalised in order, row 2 = conj(r0 x r1)); any leading shape."""
    Mc = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.empty_like(Mc)
    _check(lib().or_reunit(Mc.size // 9, _p(Mc), _p(out)), "reunit")
    return out


def ucp(V):
    """Unit circle projection of one matrix (Sec. II.C); None if V is singular."""
    Vc = _c128(V, (3, 3))
    out = np.empty((3, 3), dtype=np.complex128)
    rc = lib().or_ucp(_p(Vc), _p(out))
    return None if rc == 1 else out


def ape_ucp(dims, links, ref_labels, n_sweeps, alpha, eps=1.0, u0=1.0, schedule="annealed", vp=True,
            nthreads=None, gauge=None):
    """n_sweeps of APE blocking with unit circle projection: schedule "annealed"
    (AUS+UCP) or "simultaneous" (APE smearing); returns (links, n_reject)."""
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    ref = None if ref_labels is None else np.ascontiguousarray(ref_labels, dtype=np.int8)
    rej = np.zeros(max(n_sweeps, 1), dtype=np.int64)
    nt = max_threads() if nthreads is None else int(nthreads)
    G = None if gauge is None else _c128(gauge)
    sched = {"annealed": 0, "simultaneous": 1}[schedule]
    _check(lib().or_ape_ucp(_p(d), _p(U), _p(ref) if ref is not None else None, n_sweeps, alpha, eps,
                            u0, sched, 1 if vp else 0, _p(rej), nt, _p(G) if G is not None else None),
           "ape_ucp")
    return U, rej[:n_sweeps]


def flow_rk3(dims, links, n_steps, h, eps=1.0, u0=1.0, nthreads=None):
    """n_steps of the Wilson flow (staples Sigma(eps, u0)) by third-order
    Runge-Kutta with step h; returns the links."""
    d = _dims(dims)
    U = np.array(links, dtype=np.complex128, order="C", copy=True)
    nt = max_threads() if nthreads is None else int(nthreads)
    _check(lib().or_flow_rk3(_p(d), _p(U), n_steps, h, eps, u0, nt), "flow_rk3")
    return U


def observables(dims, links, per_site=False):
    """(<S_R>/beta, Q) and, with per_site, the densities S_R(x)/beta and q(x)."""
    d = _dims(dims)
    U = _c128(links)
    V = U.size // 36
    sr = ctypes.c_double()
    q = ctypes.c_double()
    SR = np.empty(V) if per_site else None
    qs = np.empty(V) if per_site else None
    _check(lib().or_observables(_p(d), _p(U), ctypes.byref(sr), ctypes.byref(q),
                                _p(SR) if per_site else None, _p(qs) if per_site else None),
           "observables")
    if per_site:
        return sr.value, q.value, SR, qs
    return sr.value, q.value
