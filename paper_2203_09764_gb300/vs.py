"""Thin ctypes binding of libvs.so (include/vs.h), same names as the C ABI.

Only argument marshalling happens here: every step of the smoothing path runs
in the library's CUDA kernels.  Host arrays are numpy arrays; device arrays
are torch CUDA tensors (their data_ptr is passed with VS_DEVICE).  Streams are
torch.cuda.Stream objects or raw cudaStream_t integers.  The library is never
replaced by a fallback: if libvs.so is missing, importing this module raises.
"""

import ctypes
import os

import numpy as np

from . import build as _build

VS_OK, VS_EINVAL, VS_ENOMEM, VS_EBUSY, VS_EAGAIN, VS_ETIMEDOUT, VS_EDEVICE, \
    VS_EUNSUPPORTED, VS_ENOTFOUND, VS_ECANCELED = range(10)
VS_FP64, VS_FP32 = 0, 1
VS_LINK18, VS_LINK12 = 0, 1
VS_ANNEALED, VS_SIMULTANEOUS = 0, 1
VS_HOST, VS_DEVICE = 0, 1

_STATUS = {0: "VS_OK", 1: "VS_EINVAL", 2: "VS_ENOMEM", 3: "VS_EBUSY", 4: "VS_EAGAIN",
           5: "VS_ETIMEDOUT", 6: "VS_EDEVICE", 7: "VS_EUNSUPPORTED", 8: "VS_ENOTFOUND",
           9: "VS_ECANCELED"}


class VSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class vs_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("alloc", _ALLOC_FN), ("free_fn", _FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_int32), ("max_queue", ctypes.c_int32)]


class vs_anneal(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rho_per_sweep", ctypes.POINTER(ctypes.c_double)),
                ("reunit_every", ctypes.c_int32), ("action_every", ctypes.c_int32),
                ("fp64_redecide", ctypes.c_int32)]


class vs_sweep_stats(ctypes.Structure):
    _fields_ = [("n_accept", ctypes.c_int64), ("n_reject", ctypes.c_int64),
                ("n_fp64_exp", ctypes.c_int64), ("action", ctypes.c_double),
                ("has_action", ctypes.c_int32), ("n_singular", ctypes.c_int32),
                ("n_label_diff", ctypes.c_int64), ("n_undecidable", ctypes.c_int64),
                ("min_margin", ctypes.c_double), ("n_fp64_redecided", ctypes.c_int64)]


class vs_vortex_report(ctypes.Structure):
    _fields_ = [("n_links", ctypes.c_int64), ("n_label_diff", ctypes.c_int64),
                ("n_charge_diff", ctypes.c_int64), ("n_near_boundary", ctypes.c_int64),
                ("min_margin", ctypes.c_double)]


class vs_observables_out(ctypes.Structure):
    _fields_ = [("mean_S", ctypes.c_double), ("mean_SR", ctypes.c_double), ("Q", ctypes.c_double)]


class vs_field_desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("precision", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("n_sites", ctypes.c_int64),
                ("plane_stride", ctypes.c_int64), ("n_components", ctypes.c_int32),
                ("device", ctypes.c_int32), ("links", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("gauge", ctypes.c_void_p)]


class vs_job(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("precision", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("labels", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("n_cool", ctypes.c_int32),
                ("vortex_preserve", ctypes.c_int32), ("omega", ctypes.c_double),
                ("centrifuge_seed", ctypes.c_uint64), ("rho", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("u0", ctypes.c_double),
                ("n_sweeps", ctypes.c_int32), ("reunit_every", ctypes.c_int32),
                ("links_out", ctypes.c_void_p), ("fp64_redecide", ctypes.c_int32)]


class vs_result(ctypes.Structure):
    _fields_ = [("action", ctypes.c_double), ("n_reject", ctypes.c_int64),
                ("n_label_diff", ctypes.c_int64), ("t_submit_ms", ctypes.c_double),
                ("t_admit_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


class vs_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("running", ctypes.c_int64),
                ("waiting", ctypes.c_int64), ("bytes_in_use", ctypes.c_uint64),
                ("peak_bytes_in_use", ctypes.c_uint64), ("graphs_instantiated", ctypes.c_int64),
                ("graphs_reused", ctypes.c_int64)]


P = ctypes.c_void_p
_SIGS = {
    "vs_last_error": (ctypes.c_char_p, []),
    "vs_version": (ctypes.c_char_p, []),
    "vs_create": (ctypes.c_int32, [ctypes.POINTER(vs_options), ctypes.POINTER(P)]),
    "vs_destroy": (None, [P]),
    "vs_field_create": (ctypes.c_int32, [P, P, ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(P)]),
    "vs_field_destroy": (None, [P]),
    "vs_load_field": (ctypes.c_int32, [P, P, P, ctypes.c_int32]),
    "vs_load_cooled": (ctypes.c_int32, [P, ctypes.c_uint64, ctypes.c_int32]),
    "vs_centrifuge": (ctypes.c_int32, [P, ctypes.c_double, ctypes.c_uint64]),
    "vs_smooth": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.POINTER(vs_anneal), ctypes.c_int32, P]),
    "vs_smooth_aus": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]),
    "vs_smooth_ape": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]),
    "vs_flow_rk3": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int32, P]),
    "vs_subsweep": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int32]),
    "vs_vortex_check": (ctypes.c_int32, [P, ctypes.POINTER(vs_vortex_report)]),
    "vs_action": (ctypes.c_int32, [P, ctypes.POINTER(ctypes.c_double)]),
    "vs_observables": (ctypes.c_int32, [P, ctypes.POINTER(vs_observables_out), P, P, P, ctypes.c_int32]),
    "vs_correlation": (ctypes.c_int32, [P, P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "vs_read_field": (ctypes.c_int32, [P, P, ctypes.c_int32]),
    "vs_read_labels": (ctypes.c_int32, [P, P, ctypes.c_int32]),
    "vs_field_count_nonfinite": (ctypes.c_int32, [P, ctypes.POINTER(ctypes.c_int64)]),
    "vs_field_checkpoint": (ctypes.c_int32, [P, P, P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "vs_field_restore": (ctypes.c_int32, [P, P, P, ctypes.c_int64, ctypes.c_int32]),
    "vs_current_labels": (ctypes.c_int32, [P, P, ctypes.c_int32]),
    "vs_reunitarise": (ctypes.c_int32, [P]),
    "vs_gauge_transform": (ctypes.c_int32, [P, P, ctypes.c_int32]),
    "vs_synchronize": (ctypes.c_int32, [P]),
    "vs_set_profiling": (ctypes.c_int32, [P, ctypes.c_int32]),
    "vs_get_profile": (ctypes.c_int32, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "vs_field_describe": (ctypes.c_int32, [P, ctypes.POINTER(vs_field_desc)]),
    "vs_layout_index": (ctypes.c_int64, [P, P]),
    "vs_debug_expm": (ctypes.c_int32, [P, P, ctypes.c_int32, ctypes.c_int32, P]),
    "vs_submit": (ctypes.c_int32, [P, ctypes.POINTER(vs_job), ctypes.POINTER(ctypes.c_int64)]),
    "vs_poll": (ctypes.c_int32, [P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(vs_result)]),
    "vs_cancel": (ctypes.c_int32, [P, ctypes.c_int64]),
    "vs_serve_stats_get": (ctypes.c_int32, [P, ctypes.POINTER(vs_serve_stats)]),
    "vs_now_ms": (ctypes.c_double, [P]),
    "vs_kernel_launches": (ctypes.c_int64, []),
    "vs_vortex_check_noalloc": (ctypes.c_int32, [P, P, P, P, ctypes.c_int32, ctypes.c_int32, P,
                                                 ctypes.POINTER(vs_vortex_report)]),
    "vs_noalloc_prepare": (ctypes.c_int32, [ctypes.c_int32]),
}

VS_NOALLOC_MAX_LINKS = 8 * 1024 * 1024


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libvs.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_2203_09764_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
LIB_PATH = _build.LIB


def _check(st, what=""):
    if st != VS_OK:
        raise VSError(st, (lib.vs_last_error() or b"").decode() or what)


def _ptr(a):
    """Host numpy array -> (pointer, VS_HOST); torch CUDA tensor -> (pointer, VS_DEVICE)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), VS_HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (VS_DEVICE if a.is_cuda else VS_HOST)
    raise TypeError("expected a numpy array or a torch tensor")


def _host_links(a):
    """Host link or gauge input: complex128 as it is, float64 as (re, im)
    pairs, any other numeric type converted to complex128."""
    if a.dtype == np.float64:
        return np.ascontiguousarray(a)
    return np.ascontiguousarray(a, dtype=np.complex128)


def _buf(f, a, kind, n_entries, what):
    """(pointer, where) of a buffer the library reads or writes for field f,
    after checking what the C side cannot: the element type (kind "c" for
    complex128 entries, given as complex128 or as float64 (re, im) pairs, "f8"
    for float64 values, "i8" for labels), contiguity, the byte size (n_entries
    of 16, 8 or 1 bytes), and for a CUDA tensor the field's device."""
    nbytes = n_entries * {"c": 16, "f8": 8, "i8": 1}[kind]
    if isinstance(a, np.ndarray):
        ok = {"c": a.dtype in (np.complex128, np.float64), "f8": a.dtype == np.float64,
              "i8": a.dtype == np.int8}[kind]
        size, contiguous = a.nbytes, a.flags["C_CONTIGUOUS"]
    elif hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        ok = {"c": a.dtype in (torch.complex128, torch.float64), "f8": a.dtype == torch.float64,
              "i8": a.dtype == torch.int8}[kind]
        size, contiguous = a.numel() * a.element_size(), a.is_contiguous()
        if a.is_cuda and a.device.index != vs_field_describe(f)["device"]:
            raise ValueError("%s: tensor on %s, the field is on cuda:%d"
                             % (what, a.device, vs_field_describe(f)["device"]))
    else:
        raise TypeError("%s: expected a numpy array or a torch tensor" % what)
    if not ok:
        raise TypeError("%s: element type %s (expected %s)"
                        % (what, a.dtype, {"c": "complex128 or float64 pairs", "f8": "float64",
                                           "i8": "int8"}[kind]))
    if not contiguous:
        raise ValueError("%s: buffer must be contiguous" % what)
    if size != nbytes:
        raise ValueError("%s: buffer of %d bytes, the field needs %d" % (what, size, nbytes))
    return _ptr(a)


def _dims(dims):
    return (ctypes.c_int32 * 4)(*[int(d) for d in dims])


_CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the default stream, distinct from NULL


def _stream(s):
    """None -> NULL (the library creates a stream); a torch stream or handle ->
    that stream, with torch's default stream (handle 0) passed as
    cudaStreamLegacy so that work stays ordered with torch's own work."""
    if s is None:
        return None
    h = s.cuda_stream if hasattr(s, "cuda_stream") else int(s)
    return ctypes.c_void_p(h if h else _CUDA_STREAM_LEGACY)


# ---------------------------------------------------------------------------
# Context and allocator hooks
# ---------------------------------------------------------------------------

class TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device=0):
        import torch
        self._torch = torch
        self.device = device
        self.live = {}
        self.alloc_fn = _ALLOC_FN(self._alloc)
        self.free_fn = _FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8,
                                  device="cuda:%d" % self.device)
        except Exception:  # allocation failure is reported to the library as NULL
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, _user):
        self.live.pop(ptr, None)


def vs_create(device=0, allocator=None, hbm_budget_bytes=0, max_slots=0, max_queue=0):
    o = vs_options()
    o.device = device
    if allocator is not None:
        o.alloc = allocator.alloc_fn
        o.free_fn = allocator.free_fn
    o.hbm_budget_bytes = int(hbm_budget_bytes)
    o.max_slots = int(max_slots)
    o.max_queue = int(max_queue)
    h = ctypes.c_void_p()
    _check(lib.vs_create(ctypes.byref(o), ctypes.byref(h)), "vs_create")
    return h


def vs_destroy(ctx):
    lib.vs_destroy(ctx)


def vs_last_error():
    return (lib.vs_last_error() or b"").decode()


def vs_version():
    return lib.vs_version().decode()


# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------

def vs_field_create(ctx, dims, precision=VS_FP32, storage=VS_LINK18, stream=None):
    h = ctypes.c_void_p()
    _check(lib.vs_field_create(ctx, _dims(dims), precision, storage, _stream(stream), ctypes.byref(h)))
    return h


def vs_field_destroy(f):
    lib.vs_field_destroy(f)


def vs_load_field(f, links=None, labels=None):
    if (links is None) == (labels is None):
        raise ValueError("give exactly one of links / labels")
    V = _field_sites(f)
    if links is not None:
        if isinstance(links, np.ndarray):
            links = _host_links(links)
        p, where = _buf(f, links, "c", 36 * V, "vs_load_field links")
        _check(lib.vs_load_field(f, p, None, where))
    else:
        if isinstance(labels, np.ndarray):
            labels = np.ascontiguousarray(labels, dtype=np.int8)
        p, where = _buf(f, labels, "i8", 4 * V, "vs_load_field labels")
        _check(lib.vs_load_field(f, None, p, where))


def vs_load_cooled(f, seed, n_cool):
    _check(lib.vs_load_cooled(f, int(seed), int(n_cool)))


def vs_centrifuge(f, omega, seed):
    _check(lib.vs_centrifuge(f, float(omega), int(seed)))


def vs_smooth(f, n_sweeps, rho, epsilon=1.0, u0=1.0, kind=VS_ANNEALED, rho_per_sweep=None,
              reunit_every=10, action_every=0, vortex_preserve=True, stats=False, fp64_redecide=False):
    a = vs_anneal()
    a.kind = kind
    a.fp64_redecide = 1 if fp64_redecide else 0
    keep = None
    if rho_per_sweep is not None:
        keep = np.ascontiguousarray(rho_per_sweep, dtype=np.float64)
        a.rho_per_sweep = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    a.reunit_every = int(reunit_every)
    a.action_every = int(action_every)
    st = (vs_sweep_stats * max(int(n_sweeps), 1))() if stats else None
    _check(lib.vs_smooth(f, int(n_sweeps), float(rho), float(epsilon), float(u0), ctypes.byref(a),
                         1 if vortex_preserve else 0,
                         ctypes.cast(st, ctypes.c_void_p) if stats else None))
    del keep
    if not stats:
        return None
    return [dict(n_accept=s.n_accept, n_reject=s.n_reject, n_fp64_exp=s.n_fp64_exp,
                 action=(s.action if s.has_action else None), n_label_diff=s.n_label_diff,
                 n_undecidable=s.n_undecidable, min_margin=s.min_margin, n_fp64_redecided=s.n_fp64_redecided)
            for s in st[:int(n_sweeps)]]


def vs_smooth_aus(f, n_sweeps, alpha, epsilon=-0.25, u0=1.0, n_hits=3, reunit_every=10,
                  vortex_preserve=True, stats=False):
    st = (vs_sweep_stats * max(int(n_sweeps), 1))() if stats else None
    _check(lib.vs_smooth_aus(f, int(n_sweeps), float(alpha), float(epsilon), float(u0), int(n_hits),
                             int(reunit_every), 1 if vortex_preserve else 0,
                             ctypes.cast(st, ctypes.c_void_p) if stats else None))
    if not stats:
        return None
    return [dict(n_accept=s.n_accept, n_reject=s.n_reject, n_label_diff=s.n_label_diff,
                 n_undecidable=s.n_undecidable, min_margin=s.min_margin) for s in st[:int(n_sweeps)]]


def vs_smooth_ape(f, n_sweeps, alpha, epsilon=-0.25, u0=1.0, schedule=None, reunit_every=10,
                  vortex_preserve=True, stats=False):
    """APE blocking with unit circle projection: schedule VS_ANNEALED (AUS+UCP,
    the default) or VS_SIMULTANEOUS (APE smearing)."""
    sched = VS_ANNEALED if schedule is None else int(schedule)
    st = (vs_sweep_stats * max(int(n_sweeps), 1))() if stats else None
    _check(lib.vs_smooth_ape(f, int(n_sweeps), float(alpha), float(epsilon), float(u0), sched,
                             int(reunit_every), 1 if vortex_preserve else 0,
                             ctypes.cast(st, ctypes.c_void_p) if stats else None))
    if not stats:
        return None
    return [dict(n_accept=s.n_accept, n_reject=s.n_reject, n_singular=s.n_singular,
                 n_label_diff=s.n_label_diff, n_undecidable=s.n_undecidable, min_margin=s.min_margin)
            for s in st[:int(n_sweeps)]]


def vs_flow_rk3(f, n_steps, step, epsilon=1.0, u0=1.0, reunit_every=10, stats=False):
    """Wilson flow (staples Sigma(eps, u0)) by third-order Runge-Kutta."""
    st = (vs_sweep_stats * max(int(n_steps), 1))() if stats else None
    _check(lib.vs_flow_rk3(f, int(n_steps), float(step), float(epsilon), float(u0), int(reunit_every),
                           ctypes.cast(st, ctypes.c_void_p) if stats else None))
    if not stats:
        return None
    return [dict(n_fp64_exp=s.n_fp64_exp) for s in st[:int(n_steps)]]


def vs_subsweep(f, mu, colour, rho, epsilon=1.0, u0=1.0, vortex_preserve=True):
    _check(lib.vs_subsweep(f, int(mu), int(colour), float(rho), float(epsilon), float(u0),
                           1 if vortex_preserve else 0))


def vs_vortex_check(f):
    r = vs_vortex_report()
    _check(lib.vs_vortex_check(f, ctypes.byref(r)))
    return dict(n_links=r.n_links, n_label_diff=r.n_label_diff, n_charge_diff=r.n_charge_diff,
                n_near_boundary=r.n_near_boundary, min_margin=r.min_margin)


def vs_vortex_check_noalloc(links, ref_labels, dims, precision, storage, stream=None, gauge=None):
    """The vortex check on caller-owned device buffers (device pointers as
    integers, e.g. from vs_field_describe; gauge: the field's random gauge
    transformation or None), with no device allocation; see vs.h."""
    r = vs_vortex_report()
    _check(lib.vs_vortex_check_noalloc(ctypes.c_void_p(int(links)), ctypes.c_void_p(int(ref_labels)),
                                       ctypes.c_void_p(int(gauge)) if gauge else None,
                                       _dims(dims), int(precision), int(storage), _stream(stream),
                                       ctypes.byref(r)))
    return dict(n_links=r.n_links, n_label_diff=r.n_label_diff, n_charge_diff=r.n_charge_diff,
                n_near_boundary=r.n_near_boundary, min_margin=r.min_margin)


def vs_noalloc_prepare(device=0):
    """The once-per-device set-up of vs_vortex_check_noalloc (vs_create does it
    for its own device)."""
    _check(lib.vs_noalloc_prepare(int(device)))


def vs_action(f):
    v = ctypes.c_double()
    _check(lib.vs_action(f, ctypes.byref(v)))
    return v.value


def vs_observables(f, per_site=False):
    """Dict with mean_S, mean_SR, Q; with per_site also the densities S, S_R, q
    (numpy [V], lexicographic sites)."""
    o = vs_observables_out()
    if per_site:
        V = _field_sites(f)
        dens = [np.empty(V) for _ in range(3)]
        ptrs = [ctypes.c_void_p(a.ctypes.data) for a in dens]
        _check(lib.vs_observables(f, ctypes.byref(o), ptrs[0], ptrs[1], ptrs[2], VS_HOST))
    else:
        _check(lib.vs_observables(f, ctypes.byref(o), None, None, None, VS_HOST))
    r = dict(mean_S=o.mean_S, mean_SR=o.mean_SR, Q=o.Q)
    if per_site:
        r.update(S=dens[0], S_R=dens[1], q=dens[2])
    return r


def vs_correlation(f, a, b):
    """C_XY of two per-site densities over the field's V sites (Sec. VII,
    Eq. correlation_s), computed by the library: a, b float64 [V] numpy arrays
    or torch CUDA tensors (both of one kind)."""
    V = _field_sites(f)
    pa, wa = _buf(f, a, "f8", V, "vs_correlation a")
    pb, wb = _buf(f, b, "f8", V, "vs_correlation b")
    if wa != wb:
        raise ValueError("vs_correlation: a and b must both be host or both device buffers")
    C = ctypes.c_double()
    _check(lib.vs_correlation(f, pa, pb, wa, ctypes.byref(C)))
    return C.value


def _field_sites(f):
    d = vs_field_describe(f)
    return d["n_sites"]


def vs_read_field(f, out=None):
    """Current links as complex128 [4][V][3][3] (host), or into `out` (numpy or torch CUDA)."""
    V = _field_sites(f)
    if out is None:
        out = np.empty((4, V, 3, 3), dtype=np.complex128)
    p, where = _buf(f, out, "c", 36 * V, "vs_read_field out")
    _check(lib.vs_read_field(f, p, where))
    return out


def vs_field_count_nonfinite(f):
    """Number of links with a NaN or Inf entry."""
    n = ctypes.c_int64(0)
    _check(lib.vs_field_count_nonfinite(f, ctypes.byref(n)))
    return int(n.value)


def vs_field_checkpoint(f, links_out=None, labels_out=None):
    """(links, reference labels, sweeps_done) of a field: host numpy arrays, or
    the caller's buffers (both numpy or both torch CUDA)."""
    V = _field_sites(f)
    if links_out is None:
        links_out = np.empty((4, V, 3, 3), dtype=np.complex128)
    if labels_out is None:
        labels_out = np.empty((4, V), dtype=np.int8)
    pl, where = _buf(f, links_out, "c", 36 * V, "vs_field_checkpoint links_out")
    pn, where2 = _buf(f, labels_out, "i8", 4 * V, "vs_field_checkpoint labels_out")
    if where != where2:
        raise ValueError("links_out and labels_out must both be host or both device buffers")
    n = ctypes.c_int64(0)
    _check(lib.vs_field_checkpoint(f, pl, pn, ctypes.byref(n), where))
    return links_out, labels_out, int(n.value)


def vs_field_restore(f, links, labels, sweeps_done):
    """Load a checkpoint (as vs_field_checkpoint returns it) into a field of the
    same dims, precision and storage."""
    V = _field_sites(f)
    if isinstance(links, np.ndarray):
        links = _host_links(links)
    if isinstance(labels, np.ndarray):
        labels = np.ascontiguousarray(labels, dtype=np.int8)
    pl, where = _buf(f, links, "c", 36 * V, "vs_field_restore links")
    pn, where2 = _buf(f, labels, "i8", 4 * V, "vs_field_restore labels")
    if where != where2:
        raise ValueError("links and labels must both be host or both device buffers")
    _check(lib.vs_field_restore(f, pl, pn, int(sweeps_done), where))


def vs_read_labels(f, out=None):
    V = _field_sites(f)
    if out is None:
        out = np.empty((4, V), dtype=np.int8)
    p, where = _buf(f, out, "i8", 4 * V, "vs_read_labels out")
    _check(lib.vs_read_labels(f, p, where))
    return out


def vs_current_labels(f, out=None):
    V = _field_sites(f)
    if out is None:
        out = np.empty((4, V), dtype=np.int8)
    p, where = _buf(f, out, "i8", 4 * V, "vs_current_labels out")
    _check(lib.vs_current_labels(f, p, where))
    return out


def vs_gauge_transform(f, G):
    """Apply the random gauge transformation G (complex [V][3][3], numpy or torch CUDA)."""
    if isinstance(G, np.ndarray):
        G = _host_links(G)
    p, where = _buf(f, G, "c", 9 * _field_sites(f), "vs_gauge_transform G")
    _check(lib.vs_gauge_transform(f, p, where))


def vs_reunitarise(f):
    _check(lib.vs_reunitarise(f))


def vs_synchronize(f):
    _check(lib.vs_synchronize(f))


def vs_set_profiling(f, on=True):
    _check(lib.vs_set_profiling(f, 1 if on else 0))


def vs_get_profile(f):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib.vs_get_profile(f, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def vs_field_describe(f):
    d = vs_field_desc()
    _check(lib.vs_field_describe(f, ctypes.byref(d)))
    return dict(dims=tuple(d.dims), precision=d.precision, storage=d.storage, n_sites=d.n_sites,
                plane_stride=d.plane_stride, n_components=d.n_components, device=d.device,
                links=d.links, labels=d.labels, stream=d.stream, gauge=d.gauge)


def vs_layout_index(dims, x):
    xx = (ctypes.c_int32 * 4)(*[int(v) for v in x])
    return int(lib.vs_layout_index(_dims(dims), xx))


def vs_debug_expm(ctx, X, precision=VS_FP64):
    X = np.ascontiguousarray(X, dtype=np.complex128).reshape(-1, 3, 3)
    E = np.empty_like(X)
    _check(lib.vs_debug_expm(ctx, ctypes.c_void_p(X.ctypes.data), X.shape[0], precision,
                             ctypes.c_void_p(E.ctypes.data)))
    return E


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

def make_job(dims, rho, n_sweeps, epsilon=-0.25, u0=1.0, labels=None, seed=0, n_cool=20,
             omega=0.02, centrifuge_seed=1234, vortex_preserve=True, precision=VS_FP32,
             storage=VS_LINK18, reunit_every=10, links_out=None, fp64_redecide=False):
    """Build a vs_job; the returned object keeps the label / output arrays alive."""
    j = vs_job()
    for k in range(4):
        j.dims[k] = int(dims[k])
    j.precision = precision
    j.storage = storage
    keep = []
    if labels is not None:
        labels = np.ascontiguousarray(labels, dtype=np.int8)
        keep.append(labels)
        j.labels = labels.ctypes.data
    j.seed = int(seed)
    j.n_cool = int(n_cool)
    j.vortex_preserve = 1 if vortex_preserve else 0
    j.omega = float(omega)
    j.centrifuge_seed = int(centrifuge_seed)
    j.rho = float(rho)
    j.epsilon = float(epsilon)
    j.u0 = float(u0)
    j.n_sweeps = int(n_sweeps)
    j.reunit_every = int(reunit_every)
    j.fp64_redecide = 1 if fp64_redecide else 0
    if links_out is not None:
        keep.append(links_out)
        j.links_out = links_out.ctypes.data
    j._keep = keep
    return j


def vs_submit(ctx, job):
    t = ctypes.c_int64()
    _check(lib.vs_submit(ctx, ctypes.byref(job), ctypes.byref(t)))
    return t.value


def vs_poll(ctx, ticket, timeout_ms=-1):
    """Result dict, or None when not ready (EAGAIN / ETIMEDOUT)."""
    r = vs_result()
    st = lib.vs_poll(ctx, int(ticket), int(timeout_ms), ctypes.byref(r))
    if st in (VS_EAGAIN, VS_ETIMEDOUT):
        return None
    _check(st)
    return dict(action=r.action, n_reject=r.n_reject, n_label_diff=r.n_label_diff,
                t_submit_ms=r.t_submit_ms, t_admit_ms=r.t_admit_ms, t_done_ms=r.t_done_ms,
                status=r.status)


def vs_cancel(ctx, ticket):
    _check(lib.vs_cancel(ctx, int(ticket)))


def vs_serve_stats_get(ctx):
    s = vs_serve_stats()
    _check(lib.vs_serve_stats_get(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in vs_serve_stats._fields_}


def vs_now_ms(ctx):
    return float(lib.vs_now_ms(ctx))


def vs_kernel_launches():
    return int(lib.vs_kernel_launches())
