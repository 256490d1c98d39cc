"""Python binding of the B300 progressive refactor / retrieve library.

Argument marshalling only: every step of the refactor and retrieval path runs
in the CUDA kernels of ``libpcr.so`` (C ABI in ``include/pcr.h``).  PyTorch
provides device memory (its caching allocator, passed to the library as a
``pcr_allocator``) and CUDA streams.  There is no CPU fallback: importing this
package fails loudly when the library is missing.

Method: arXiv 2609.04573 (ProAICD) -- adaptive multilevel interpolation
(Sec. IV), coefficient decomposition (Sec. V), bitplane streams with error
tables (Sec. V-C), bound-driven retrieval (Sec. III-A, Alg. 2).
"""
import ctypes as C
import os
import sys
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpcr.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"{_LIB_PATH} is missing: build it with `python paper_2609_04573_b300/build.py` "
        "(nvcc, sm_103a).  There is no CPU fallback.")
_lib = C.CDLL(_LIB_PATH)

MAX_STREAMS = 64
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSAT, ERR_CORRUPT = range(8)
_STATUS = ["OK", "INVALID_ARG", "UNSUPPORTED", "OOM", "CUDA", "TIMEOUT", "UNSATISFIABLE", "CORRUPT"]


class PcrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pcr {_STATUS[status] if status < len(_STATUS) else status}: {msg}")
        self.status = status


class Unsatisfiable(PcrError):
    pass


class _Scheme(C.Structure):
    _fields_ = [("mode", C.c_int), ("interp", C.c_int), ("degree", C.c_int),
                ("order", C.c_int * 3), ("decomp_axis", C.c_int), ("encoding", C.c_int),
                ("nlevels", C.c_int), ("nplanes", C.c_int)]


class _Target(C.Structure):
    _fields_ = [("kind", C.c_int), ("value", C.c_double), ("has_box", C.c_int),
                ("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3)]


class _Info(C.Structure):
    _fields_ = [("nstreams", C.c_int), ("planes", C.c_int * MAX_STREAMS), ("bytes", C.c_uint64),
                ("bits_per_value", C.c_double), ("bound", C.c_double), ("psnr_bound", C.c_double),
                ("satisfied", C.c_int), ("plan_ms", C.c_double), ("enqueue_ms", C.c_double),
                ("want_gpu_ms", C.c_int), ("gpu_ms", C.c_double)]


class _Tables(C.Structure):
    _fields_ = [("nstreams", C.c_int), ("nplanes", C.c_int), ("exponent", C.c_int * MAX_STREAMS),
                ("maxerr", C.POINTER(C.c_double)), ("sq", C.POINTER(C.c_double)),
                ("bytes", C.POINTER(C.c_uint64))]


class _Plan(C.Structure):
    _fields_ = [("nstreams", C.c_int), ("planes", C.c_int * MAX_STREAMS), ("bound", C.c_double),
                ("psnr_bound", C.c_double), ("bytes", C.c_uint64), ("satisfied", C.c_int)]


TUNE_NTOL, TUNE_MAX = 9, 32


class _SearchInfo(C.Structure):
    _fields_ = [("expanded", C.c_int64), ("optimal", C.c_int), ("greedy_bytes", C.c_uint64), ("plan_ms", C.c_double)]


SEARCH_NODES = 4096


class _TuneInfo(C.Structure):
    _fields_ = [("ncand", C.c_int), ("winner", C.c_int), ("cand", _Scheme * TUNE_MAX), ("votes", C.c_int * TUNE_MAX),
                ("bytes", (C.c_uint64 * TUNE_NTOL) * TUNE_MAX), ("nblocks", C.c_int), ("block", C.c_int64 * 3),
                ("fraction", C.c_double), ("ms", C.c_double)]


class _StreamInfo(C.Structure):
    _fields_ = [("level", C.c_int), ("region", C.c_int), ("sub", C.c_int), ("is_fixed", C.c_int),
                ("nplanes", C.c_int), ("n_real", C.c_int64), ("n_pad", C.c_int64),
                ("words", C.c_int64), ("nseg", C.c_int64), ("exponent", C.c_int),
                ("shift", C.c_int), ("vmax", C.c_double)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


_vp, _i64p = C.c_void_p, C.POINTER(C.c_int64)
_sigs = {
    "pcr_refactor": [_vp, C.c_int, _i64p, C.c_int, C.POINTER(_Scheme), C.POINTER(_Allocator), _vp, C.POINTER(_vp)],
    "pcr_refactor_begin": [_vp, C.c_int, _i64p, C.c_int, C.POINTER(_Scheme), C.POINTER(_Allocator), _vp,
                           C.POINTER(_vp)],
    "pcr_refactor_end": [_vp, C.POINTER(_vp)],
    "pcr_refactor_batch": [C.c_int, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(_i64p), C.POINTER(C.c_int),
                           C.POINTER(_Scheme), C.POINTER(_Allocator), _vp, C.POINTER(_vp)],
    "pcr_plan": [_vp, C.POINTER(_Target), C.POINTER(_Plan)],
    "pcr_plan_more": [_vp, C.POINTER(_Target), C.POINTER(_Plan), C.POINTER(_Plan)],
    "pcr_plan_search": [_vp, C.POINTER(_Target), C.POINTER(_Plan), C.c_int64, C.POINTER(_Plan),
                        C.POINTER(_SearchInfo)],
    "pcr_plan_global": [C.c_int, C.POINTER(_vp), C.POINTER(_Target), C.POINTER(_Plan), C.POINTER(C.c_double),
                        C.POINTER(C.c_int)],
    "pcr_export_plan_state": [_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)],
    "pcr_packed_tables": [_vp, C.POINTER(C.c_uint64)],
    "pcr_debug_pack": [_vp, C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_int)],
    "pcr_serialize_packed": [_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)],
    "pcr_import_plan_state": [_vp, C.c_size_t, C.POINTER(_vp)],
    "pcr_retrieve": [_vp, C.POINTER(_Target), _vp, _vp, C.POINTER(_Info)],
    "pcr_retrieve_plan": [_vp, C.POINTER(_Plan), _vp, _vp],
    "pcr_retrieve_batch": [C.c_int, C.POINTER(_vp), C.POINTER(_Target), C.POINTER(_vp), _vp,
                           C.POINTER(_Info)],
    "pcr_retrieve_batch_plan": [C.c_int, C.POINTER(_vp), C.POINTER(_Plan), C.POINTER(_vp), _vp],
    "pcr_get_tables": [_vp, C.POINTER(_Tables)],
    "pcr_tune": [_vp, C.c_int, _i64p, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(_Allocator), _vp,
                 C.POINTER(_Scheme), C.POINTER(_TuneInfo)],
    "pcr_get_scheme": [_vp, C.POINTER(_Scheme)],
    "pcr_retrieve_static": [_vp, C.POINTER(_Plan), _vp, _vp],
    "pcr_retrieve_box": [_vp, C.POINTER(_Plan), _i64p, _i64p, _vp, _vp],
    "pcr_retrieve_scratch_bytes": [_vp, C.POINTER(C.c_size_t)],
    "pcr_num_streams": [_vp, C.POINTER(C.c_int)],
    "pcr_stream_info_get": [_vp, C.c_int, C.POINTER(_StreamInfo)],
    "pcr_stream_tables": [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_uint64)],
    "pcr_field_stats": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)],
    "pcr_stream_copy": [_vp, C.c_int, _vp, _vp, _vp, _vp],
    "pcr_max_ordering": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int)],
    "pcr_serialize": [_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)],
    "pcr_deserialize": [_vp, C.c_size_t, C.POINTER(_Allocator), _vp, C.POINTER(_vp)],
    "pcr_debug_encode": [_vp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                         C.POINTER(C.c_double)],
    "pcr_refactor_graph_create": [C.c_int, C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(_i64p),
                                  C.POINTER(C.c_int), C.POINTER(_Scheme), C.POINTER(_Allocator), _vp,
                                  C.POINTER(_vp)],
    "pcr_refactor_graph_run": [_vp, _vp],
    "pcr_refactor_graph_handle": [_vp, C.c_int, C.POINTER(_vp)],
    "pcr_refactor_graph_info": [_vp, _i64p, _i64p, _i64p],
    "pcr_refactor_graph_times": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "pcr_autotune_set": [_i64p, C.c_int],
    "pcr_device_status": [C.POINTER(C.c_int), C.c_int],
    "pcr_autotune_enable": [C.c_int],
    "pcr_autotune_read": [C.c_int, _i64p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int],
}
for _name, _args in _sigs.items():
    fn = getattr(_lib, _name)
    fn.argtypes = _args
    fn.restype = C.c_int
_lib.pcr_profile_enable.argtypes = [C.c_int]
_lib.pcr_profile_enable.restype = C.c_int
_lib.pcr_profile_read.argtypes = [C.c_int, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int), C.c_int]
_lib.pcr_profile_read.restype = C.c_int
_lib.pcr_launch_count.argtypes = []
_lib.pcr_launch_count.restype = C.c_int64
_lib.pcr_free.argtypes = [_vp]
_lib.pcr_free.restype = None
_lib.pcr_refactor_graph_free.argtypes = [_vp]
_lib.pcr_refactor_graph_free.restype = None
_lib.pcr_refactor_job_free.argtypes = [_vp]
_lib.pcr_refactor_job_free.restype = None
_lib.pcr_buffer_free.argtypes = [_vp]
_lib.pcr_buffer_free.restype = None
_lib.pcr_last_error.argtypes = []
_lib.pcr_last_error.restype = C.c_char_p

# exported symbols (checked by the CPU tests against include/pcr.h)
EXPORTS = sorted(list(_sigs) + ["pcr_free", "pcr_buffer_free", "pcr_last_error", "pcr_profile_enable",
                                "pcr_profile_read", "pcr_launch_count", "pcr_refactor_graph_free",
                                "pcr_refactor_job_free"])


def _check(st):
    if st != OK:
        msg = _lib.pcr_last_error().decode()
        raise (Unsatisfiable if st == ERR_UNSAT else PcrError)(st, msg)


# ---- torch-backed allocator (the library allocates through torch) --------
_live = {}


def _torch_alloc(ctx, nbytes, stream):
    try:
        dev = torch.cuda.current_device()
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        return ptr
    except Exception:  # out of memory -> NULL -> PCR_ERR_OOM
        return None


def _torch_free(ctx, ptr, stream):
    # at interpreter exit torch's allocator may already be gone: the process
    # releases the memory anyway
    if ptr and not sys.is_finalizing():
        torch.cuda.caching_allocator_delete(ptr)


_ALLOC_CB = _ALLOC_FN(_torch_alloc)
_FREE_CB = _FREE_FN(_torch_free)
_ALLOCATOR = _Allocator(None, _ALLOC_CB, _FREE_CB)

EB, PSNR, EXPLICIT = 0, 1, 2
AUTO, LEVEL, REGION = -1, 0, 1
LINEAR, CUBIC = 1, 3
GENERIC, NEGABINARY = 1, 2
_DT = {torch.float32: 0, torch.float64: 1}


@dataclass
class Scheme:
    """Refactoring scheme (Sec. IV-VI, tuning table of Sec. VI-A)."""
    mode: str = "eb"                 # "eb" | "psnr" | "explicit"
    interp: str = "level"            # "level" | "region" | "auto" (sampled tuner)
    degree: str = "cubic"            # "linear" | "cubic"
    order: Optional[Tuple[int, ...]] = None
    decomp_axis: int = -1
    encoding: Optional[str] = None   # None = generic (eb) / negabinary (psnr)
    nlevels: int = 0
    nplanes: int = 0

    @classmethod
    def for_target(cls, kind, **kw):
        """The paper's adaptive choice (Sec. IV, VI-A): error-bound targets use
        per-level interpolation with generic bitplanes; PSNR targets use
        per-region interpolation with negabinary + XOR."""
        if kind == "psnr":
            return cls(mode="psnr", interp="region", **kw)
        return cls(mode="eb", interp="level", **kw)

    def c(self, ndim):
        s = _Scheme()
        s.mode = {"eb": EB, "psnr": PSNR, "explicit": EXPLICIT}[self.mode]
        s.interp = {"level": LEVEL, "region": REGION, "auto": AUTO}[self.interp]
        s.degree = CUBIC if self.degree == "cubic" else LINEAR
        order = self.order or tuple(range(ndim))
        for i in range(3):
            s.order[i] = order[i] if i < len(order) else 0
        s.decomp_axis = self.decomp_axis
        s.encoding = {None: 0, "generic": GENERIC, "negabinary": NEGABINARY}[self.encoding]
        s.nlevels = self.nlevels
        s.nplanes = self.nplanes
        return s


    @classmethod
    def of(cls, s, ndim):
        """Scheme of a pcr_scheme (pass orders in user axes)."""
        interp = {LEVEL: "level", REGION: "region"}[s.interp]
        order = tuple(s.order[:ndim]) if interp == "region" else None
        enc = {GENERIC: "generic", NEGABINARY: "negabinary"}.get(s.encoding)
        mode = {EB: "eb", PSNR: "psnr", EXPLICIT: "explicit"}[s.mode]
        return cls(mode=mode, interp=interp, degree="cubic" if s.degree == CUBIC else "linear", order=order,
                   decomp_axis=s.decomp_axis, encoding=enc, nlevels=s.nlevels, nplanes=s.nplanes)


@dataclass
class Target:
    kind: str      # "abs" | "rel" | "psnr"
    value: float
    box: Optional[Tuple[Tuple[int, int], ...]] = None   # ((lo, hi) per axis) or None

    def c(self):
        t = _Target()
        t.kind = {"abs": 0, "rel": 1, "psnr": 2}[self.kind]
        t.value = float(self.value)
        if self.box is not None:
            t.has_box = 1
            for k, (lo, hi) in enumerate(self.box):
                t.lo[k], t.hi[k] = int(lo), int(hi)
        return t


@dataclass
class Plan:
    planes: list
    bound: float
    psnr_bound: float
    bytes: int
    satisfied: bool
    _c: object = field(default=None, repr=False)


@dataclass
class RetrievalInfo:
    """What one pcr_retrieve call read (pcr_retrieval_info)."""
    planes: list
    bytes: int
    bits_per_value: float
    bound: float
    psnr_bound: float
    satisfied: bool
    plan_ms: float
    enqueue_ms: float
    gpu_ms: float

    @classmethod
    def of(cls, i):
        return cls(list(i.planes[:i.nstreams]), i.bytes, i.bits_per_value, i.bound, i.psnr_bound,
                   bool(i.satisfied), i.plan_ms, i.enqueue_ms, i.gpu_ms)


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Handle:
    """Refactored field: device streams + host tables (owned by the library)."""

    def __init__(self, ptr, shape, dtype, device, owner=None, allocator=None):
        self._p = C.c_void_p(ptr)
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = device
        self._owner = owner   # a RefactorGraph owns its handles; keep it alive
        self._alloc = allocator   # a caller's allocator frees the handle's memory: keep it alive

    def __del__(self):
        # nothing is freed while the interpreter exits (the allocator
        # callbacks would run into a half torn-down torch)
        if sys.is_finalizing():
            return
        if getattr(self, "_owner", None) is None and getattr(self, "_p", None) and self._p.value:
            _lib.pcr_free(self._p)
            self._p = C.c_void_p(None)

    @property
    def nstreams(self):
        n = C.c_int()
        _check(_lib.pcr_num_streams(self._p, C.byref(n)))
        return n.value

    def stream_info(self, i):
        s = _StreamInfo()
        _check(_lib.pcr_stream_info_get(self._p, i, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _StreamInfo._fields_}

    def tables(self, i):
        B = self.stream_info(i)["nplanes"]
        me = (C.c_double * (B + 1))()
        sq = (C.c_double * (B + 1))()
        by = (C.c_uint64 * (B + 1))()
        _check(_lib.pcr_stream_tables(self._p, i, me, sq, by))
        return dict(maxerr=list(me), sq=list(sq), bytes=list(by))

    def field_stats(self):
        a, b, g = C.c_double(), C.c_double(), C.c_int()
        _check(_lib.pcr_field_stats(self._p, C.byref(a), C.byref(b), C.byref(g)))
        return a.value, b.value, g.value

    def stream_copy(self, i):
        """Plane words [B, words], sign area, sign counts [nseg, B], pairs."""
        import numpy as np
        info = self.stream_info(i)
        B, words, nseg = info["nplanes"], info["words"], info["nseg"]
        planes = np.zeros((B, words), np.uint32)
        signs = np.zeros((nseg, 128 + B), np.uint32)
        scnt = np.zeros((nseg, B), np.uint32)
        pairs = np.zeros((B, B), np.uint64)
        _check(_lib.pcr_stream_copy(self._p, i, planes.ctypes.data, signs.ctypes.data,
                                    scnt.ctypes.data, pairs.ctypes.data))
        return planes, signs, scnt, pairs

    def max_ordering(self):
        n = C.c_int()
        _check(_lib.pcr_max_ordering(self._p, None, C.byref(n)))
        if n.value == 0:
            return []
        arr = (C.c_double * n.value)()
        _check(_lib.pcr_max_ordering(self._p, arr, C.byref(n)))
        return list(arr)

    def plan(self, target, allow_unsat=False, have=None):
        """Planes per stream for `target` (pcr_plan).  `have`: a Plan whose
        planes are already fetched; the result contains it and is ranked by
        the bytes it adds (pcr_plan_more)."""
        p = _Plan()
        if have is None:
            st = _lib.pcr_plan(self._p, C.byref(target.c()), C.byref(p))
        else:
            st = _lib.pcr_plan_more(self._p, C.byref(target.c()), C.byref(have._c), C.byref(p))
        if st != OK and not (st == ERR_UNSAT and allow_unsat):
            _check(st)
        return Plan(list(p.planes[:p.nstreams]), p.bound, p.psnr_bound, p.bytes, bool(p.satisfied), p)

    def plan_search(self, target, max_nodes=SEARCH_NODES, have=None, allow_unsat=False):
        """Best-first search interpreter (pcr_plan_search): (Plan, info) with
        info = dict(expanded, optimal, greedy_bytes, plan_ms); never more
        bytes than plan(target, have=have)."""
        p, info = _Plan(), _SearchInfo()
        st = _lib.pcr_plan_search(self._p, C.byref(target.c()), C.byref(have._c) if have is not None else None,
                                  int(max_nodes), C.byref(p), C.byref(info))
        if st != OK and not (st == ERR_UNSAT and allow_unsat):
            _check(st)
        pl = Plan(list(p.planes[:p.nstreams]), p.bound, p.psnr_bound, p.bytes, bool(p.satisfied), p)
        return pl, dict(expanded=info.expanded, optimal=bool(info.optimal), greedy_bytes=info.greedy_bytes,
                        plan_ms=info.plan_ms)

    def packed_tables(self):
        """Stored bytes of each stream's first b planes with the planes
        coded losslessly: list per stream of B + 1 entries."""
        ns, B = self.nstreams, self.stream_info(0)["nplanes"]
        out = (C.c_uint64 * (ns * (B + 1)))()
        _check(_lib.pcr_packed_tables(self._p, out))
        return [list(out[i * (B + 1):(i + 1) * (B + 1)]) for i in range(ns)]

    def packed_bytes(self, plan):
        """Stored bytes of a plan's planes and signs with the planes coded."""
        t = self.packed_tables()
        return sum(t[i][b] for i, b in enumerate(plan.planes))

    def serialize_packed(self):
        """Container bytes with the planes coded losslessly."""
        buf, n = C.c_void_p(), C.c_size_t()
        _check(_lib.pcr_serialize_packed(self._p, C.byref(buf), C.byref(n)))
        try:
            return C.string_at(buf, n.value)
        finally:
            _lib.pcr_buffer_free(buf)

    def export_plan_state(self):
        """What the planner needs of this handle (no planes), as bytes."""
        buf, n = C.c_void_p(), C.c_size_t()
        _check(_lib.pcr_export_plan_state(self._p, C.byref(buf), C.byref(n)))
        try:
            return C.string_at(buf, n.value)
        finally:
            _lib.pcr_buffer_free(buf)

    def plan_from_planes(self, planes):
        p = _Plan()
        p.nstreams = len(planes)
        for i, b in enumerate(planes):
            p.planes[i] = int(b)
        return Plan(list(planes), 0.0, 0.0, 0, True, p)

    def retrieve(self, target_or_plan, out=None, stream=None, gpu_time=False):
        """Reconstruct into ``out`` (allocated when None).  A Target goes
        through the one-call pcr_retrieve (its box, if any, sets the output
        shape) and returns (out, RetrievalInfo); a Plan goes through
        pcr_retrieve_plan and returns (out, plan)."""
        if isinstance(target_or_plan, Plan):
            plan = target_or_plan
            if out is None:
                out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
            assert out.is_contiguous() and tuple(out.shape) == self.shape and out.dtype == self.dtype
            _check(_lib.pcr_retrieve_plan(self._p, C.byref(plan._c), C.c_void_p(out.data_ptr()),
                                          _stream_ptr(stream)))
            return out, plan
        t = target_or_plan
        shp = self.shape if t.box is None else tuple(hi - lo for lo, hi in t.box)
        if t.box is not None and len(t.box) != len(self.shape):
            raise ValueError("box needs one (lo, hi) pair per axis")
        if out is None:
            out = torch.empty(shp, dtype=self.dtype, device=self.device)
        assert out.is_contiguous() and tuple(out.shape) == shp and out.dtype == self.dtype
        info = _Info()
        info.want_gpu_ms = 1 if gpu_time else 0
        _check(_lib.pcr_retrieve(self._p, C.byref(t.c()), C.c_void_p(out.data_ptr()), _stream_ptr(stream),
                                 C.byref(info)))
        return out, RetrievalInfo.of(info)

    def scheme(self):
        """pcr_get_scheme: the scheme this handle was refactored with."""
        sc = _Scheme()
        _check(_lib.pcr_get_scheme(self._p, C.byref(sc)))
        return Scheme.of(sc, len(self.shape))

    def get_tables(self):
        """pcr_get_tables: per stream exponent, maxerr[B+1], sq[B+1], bytes[B+1]."""
        import numpy as np
        t = _Tables()
        _check(_lib.pcr_get_tables(self._p, C.byref(t)))
        ns, B = t.nstreams, t.nplanes
        me = np.zeros((ns, B + 1), np.float64)
        sq = np.zeros((ns, B + 1), np.float64)
        by = np.zeros((ns, B + 1), np.uint64)
        t.maxerr = me.ctypes.data_as(C.POINTER(C.c_double))
        t.sq = sq.ctypes.data_as(C.POINTER(C.c_double))
        t.bytes = by.ctypes.data_as(C.POINTER(C.c_uint64))
        _check(_lib.pcr_get_tables(self._p, C.byref(t)))
        return dict(exponent=list(t.exponent[:ns]), maxerr=me, sq=sq, bytes=by)

    def retrieve_box(self, target_or_plan, box, out=None, stream=None):
        """Reconstruct only the box ((lo, hi) per axis) of the field: the same
        values as retrieve() gives there, decoding and reconstructing only
        the box's dependency region.  Returns (out, plan)."""
        plan = target_or_plan if isinstance(target_or_plan, Plan) else self.plan(target_or_plan)
        lo = [int(a) for a, _ in box]
        hi = [int(b) for _, b in box]
        if len(lo) != len(self.shape):
            raise ValueError("box needs one (lo, hi) pair per axis")
        shp = tuple(b - a for a, b in zip(lo, hi))
        if out is None:
            out = torch.empty(shp, dtype=self.dtype, device=self.device)
        assert out.is_contiguous() and tuple(out.shape) == shp and out.dtype == self.dtype
        _check(_lib.pcr_retrieve_box(self._p, C.byref(plan._c), (C.c_int64 * len(lo))(*lo),
                                     (C.c_int64 * len(hi))(*hi), C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out, plan

    @property
    def out_bytes(self):
        n = 1
        for s in self.shape:
            n *= s
        return n * (4 if self.dtype == torch.float32 else 8)

    def retrieve_scratch_bytes(self):
        """Temporary device memory one retrieval of this handle takes."""
        v = C.c_size_t()
        _check(_lib.pcr_retrieve_scratch_bytes(self._p, C.byref(v)))
        return v.value

    def retrieve_static(self, plan, out, stream=None):
        """pcr_retrieve_static: the same result as retrieve() with every
        temporary buffer in the library's fixed device array (no device
        allocation), for callers that cannot allocate.  ``out`` must be given."""
        assert out.is_contiguous() and tuple(out.shape) == self.shape and out.dtype == self.dtype
        _check(_lib.pcr_retrieve_static(self._p, C.byref(plan._c), C.c_void_p(out.data_ptr()),
                                        _stream_ptr(stream)))
        return out

    def serialize(self):
        buf, n = C.c_void_p(), C.c_size_t()
        _check(_lib.pcr_serialize(self._p, C.byref(buf), C.byref(n)))
        data = C.string_at(buf, n.value)
        _lib.pcr_buffer_free(buf)
        return data


def tune(x, mode="eb", fraction=0.0, edge=0, stream=None):
    """pcr_tune: the target-driven sampled tuner's scheme for x (Sec. VI-A).
    Returns (Scheme, info dict: candidates, votes, bytes per tolerance (None:
    not met), blocks, block edge, sampled fraction, ms)."""
    if not (x.is_cuda and x.is_contiguous() and x.dtype in _DT and x.dim() in (2, 3)):
        raise ValueError("tune expects a contiguous 2-D/3-D float32/float64 CUDA tensor")
    dims = (C.c_int64 * x.dim())(*x.shape)
    out, info = _Scheme(), _TuneInfo()
    _check(_lib.pcr_tune(C.c_void_p(x.data_ptr()), x.dim(), dims, _DT[x.dtype], {"eb": EB, "psnr": PSNR}[mode],
                         float(fraction), int(edge), C.byref(_ALLOCATOR), _stream_ptr(stream), C.byref(out),
                         C.byref(info)))
    nd = x.dim()
    cands = [Scheme.of(info.cand[c], nd) for c in range(info.ncand)]
    table = [[None if info.bytes[c][t] == (1 << 64) - 1 else int(info.bytes[c][t]) for t in range(TUNE_NTOL)]
             for c in range(info.ncand)]
    return Scheme.of(out, nd), dict(candidates=cands, votes=list(info.votes[:info.ncand]), bytes=table,
                                    winner=info.winner, nblocks=info.nblocks, block=tuple(info.block[:nd]),
                                    fraction=info.fraction, ms=info.ms)


def _alloc_ref(allocator):
    """A caller's pcr_allocator (an object with a `.c` _Allocator, or the
    struct itself), else torch's caching allocator."""
    if allocator is None:
        return C.byref(_ALLOCATOR)
    return C.byref(getattr(allocator, "c", allocator))


def refactor(x, scheme=None, stream=None, allocator=None):
    """Refactor a contiguous CUDA float32/float64 tensor (2-D or 3-D).
    `allocator`: device memory for the handle and the call's scratch
    (default: torch's caching allocator)."""
    scheme = scheme or Scheme()
    if not (x.is_cuda and x.is_contiguous() and x.dtype in _DT and x.dim() in (2, 3)):
        raise ValueError("refactor expects a contiguous 2-D/3-D float32/float64 CUDA tensor")
    dims = (C.c_int64 * x.dim())(*x.shape)
    out = C.c_void_p()
    _check(_lib.pcr_refactor(C.c_void_p(x.data_ptr()), x.dim(), dims, _DT[x.dtype],
                             C.byref(scheme.c(x.dim())), _alloc_ref(allocator), _stream_ptr(stream),
                             C.byref(out)))
    return Handle(out.value, x.shape, x.dtype, x.device, allocator=allocator)


class RefactorJob:
    """A refactor enqueued with refactor_async; result() waits for it and
    returns the Handle.  Keeps the field tensor alive until then."""

    def __init__(self, ptr, x):
        self._p = C.c_void_p(ptr)
        self._x = x

    def result(self):
        if not self._p or not self._p.value:
            raise RuntimeError("job already consumed")
        out = C.c_void_p()
        p, self._p = self._p, C.c_void_p(None)
        _check(_lib.pcr_refactor_end(p, C.byref(out)))
        x, self._x = self._x, None
        return Handle(out.value, x.shape, x.dtype, x.device)

    def __del__(self):
        if sys.is_finalizing():
            return
        if getattr(self, "_p", None) and self._p.value:
            _lib.pcr_refactor_job_free(self._p)
            self._p = C.c_void_p(None)


def refactor_async(x, scheme=None, stream=None):
    """Enqueue the refactor of x and return a RefactorJob without waiting:
    the host can plan and retrieve other fields meanwhile.  The handle's
    buffers belong to `stream`'s allocator pool: when it is retrieved on
    another stream, keep the Handle alive until that retrieval has run."""
    scheme = scheme or Scheme()
    if not (x.is_cuda and x.is_contiguous() and x.dtype in _DT and x.dim() in (2, 3)):
        raise ValueError("refactor expects a contiguous 2-D/3-D float32/float64 CUDA tensor")
    dims = (C.c_int64 * x.dim())(*x.shape)
    out = C.c_void_p()
    _check(_lib.pcr_refactor_begin(C.c_void_p(x.data_ptr()), x.dim(), dims, _DT[x.dtype],
                                   C.byref(scheme.c(x.dim())), C.byref(_ALLOCATOR), _stream_ptr(stream),
                                   C.byref(out)))
    return RefactorJob(out.value, x)


def refactor_batch(xs: Sequence[torch.Tensor], schemes, stream=None, allocator=None):
    """Every pipeline stage in one launch (or a few) across all fields
    (batched form)."""
    n = len(xs)
    if not isinstance(schemes, (list, tuple)):
        schemes = [schemes] * n
    ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    nd = (C.c_int * n)(*[x.dim() for x in xs])
    dim_arrs = [(C.c_int64 * x.dim())(*x.shape) for x in xs]
    dims = (_i64p * n)(*[C.cast(d, _i64p) for d in dim_arrs])
    dts = (C.c_int * n)(*[_DT[x.dtype] for x in xs])
    sch = (_Scheme * n)(*[s.c(x.dim()) for s, x in zip(schemes, xs)])
    outs = (C.c_void_p * n)()
    _check(_lib.pcr_refactor_batch(n, ptrs, nd, dims, dts, sch, _alloc_ref(allocator),
                                   _stream_ptr(stream), outs))
    return [Handle(outs[i], x.shape, x.dtype, x.device, allocator=allocator) for i, x in enumerate(xs)]


def _batch_args(xs, schemes):
    n = len(xs)
    if not isinstance(schemes, (list, tuple)):
        schemes = [schemes] * n
    ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    nd = (C.c_int * n)(*[x.dim() for x in xs])
    dim_arrs = [(C.c_int64 * x.dim())(*x.shape) for x in xs]
    dims = (_i64p * n)(*[C.cast(d, _i64p) for d in dim_arrs])
    dts = (C.c_int * n)(*[_DT[x.dtype] for x in xs])
    sch = (_Scheme * n)(*[s.c(x.dim()) for s, x in zip(schemes, xs)])
    return n, ptrs, nd, dims, dim_arrs, dts, sch


class RefactorGraph:
    """A batch refactored again and again with the same shapes, captured in
    one CUDA graph (pcr_refactor_graph_*).  The tensors `xs` stay where they
    are for the graph's lifetime: refill them in place, then call run().
    Creation refactors once (autotuning the level schedule) so `handles` are
    valid right away; every run replaces their contents."""

    def __init__(self, xs: Sequence[torch.Tensor], schemes, stream=None, allocator=None):
        for x in xs:
            if not (x.is_cuda and x.is_contiguous() and x.dtype in _DT and x.dim() in (2, 3)):
                raise ValueError("RefactorGraph expects contiguous 2-D/3-D float32/float64 CUDA tensors")
        self._xs = list(xs)
        self._alloc = allocator   # kept alive: the graph frees its arena through it
        n, ptrs, nd, dims, _keep, dts, sch = _batch_args(xs, schemes)
        self._g = C.c_void_p()
        _check(_lib.pcr_refactor_graph_create(n, ptrs, nd, dims, dts, sch, _alloc_ref(allocator),
                                              _stream_ptr(stream), C.byref(self._g)))
        self.handles = []
        for i, x in enumerate(xs):
            hp = C.c_void_p()
            _check(_lib.pcr_refactor_graph_handle(self._g, i, C.byref(hp)))
            self.handles.append(Handle(hp.value, x.shape, x.dtype, x.device, owner=self))

    def run(self, stream=None):
        _check(_lib.pcr_refactor_graph_run(self._g, _stream_ptr(stream)))
        return self.handles

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(_lib.pcr_refactor_graph_info(self._g, C.byref(a), C.byref(b), C.byref(c)))
        return {"nodes": a.value, "kernels": b.value, "arena_bytes": c.value}

    def times(self):
        """Of the last run: the graph's device time and the host finish of
        the tables, in ms."""
        g, h = C.c_double(), C.c_double()
        _check(_lib.pcr_refactor_graph_times(self._g, C.byref(g), C.byref(h)))
        return {"gpu_ms": g.value, "host_ms": h.value}

    def __del__(self):
        if sys.is_finalizing():
            return
        if getattr(self, "_g", None) and self._g.value:
            _lib.pcr_refactor_graph_free(self._g)
            self._g = C.c_void_p(None)


def import_plan_state(data, shape, dtype=torch.float32):
    """A planning-only Handle from export_plan_state bytes (plans, no
    retrieval)."""
    buf = C.create_string_buffer(data, len(data))
    out = C.c_void_p()
    _check(_lib.pcr_import_plan_state(buf, len(data), C.byref(out)))
    return Handle(out.value, shape, dtype, None)


def plan_global(handles, target):
    """Plans of the blocks of one field for a whole-field target
    (pcr_plan_global): (plans, bound, satisfied)."""
    n = len(handles)
    hp = (C.c_void_p * n)(*[h._p.value for h in handles])
    pl = (_Plan * n)()
    bnd, sat = C.c_double(), C.c_int()
    st = _lib.pcr_plan_global(n, hp, C.byref(target.c()), pl, C.byref(bnd), C.byref(sat))
    if st not in (OK, ERR_UNSAT):
        _check(st)
    plans = []
    for k in range(n):
        c = _Plan.from_buffer_copy(pl[k])
        plans.append(Plan(list(c.planes[:c.nstreams]), c.bound, c.psnr_bound, c.bytes, bool(c.satisfied), c))
    return plans, bnd.value, bool(sat.value)


class Progressive:
    """A progressive retrieval session over one handle (Sec. III-A
    refinement): each refine() plans the new target from the planes fetched
    so far (pcr_plan_more), retrieves, and reports the bytes it added."""

    def __init__(self, handle):
        self.handle = handle
        self.plan = None
        self.fetched = 0

    def refine(self, target, out=None, stream=None):
        p = self.handle.plan(target, allow_unsat=True, have=self.plan)
        added = p.bytes - (self.plan.bytes if self.plan is not None else 0)
        out, _ = self.handle.retrieve(p, out=out, stream=stream)
        self.plan = p
        self.fetched += added
        return out, p, added


def autotune(enable=True):
    """Level-schedule autotuner on/off (pcr_autotune_enable)."""
    _check(_lib.pcr_autotune_enable(1 if enable else 0))


def device_status(clear=True):
    """1 when a bounded wait of a retrieval kernel gave up on the current
    device since the last clear, else 0 (pcr_device_status; synchronous)."""
    v = C.c_int()
    _check(_lib.pcr_device_status(C.byref(v), int(clear)))
    return v.value


def autotune_pin(key, choice):
    """Pin the schedule of one level grid: key = (kind, retrieve, degree,
    interp, m0, m1, m2) as autotune_table gives it (pcr_autotune_set)."""
    k = (C.c_int64 * 7)(*key)
    _check(_lib.pcr_autotune_set(k, int(choice)))


def autotune_table(reset=False):
    """Tuned entries: {(kind, retrieve, degree, interp, m0, m1, m2): (choice, ms)}."""
    n = C.c_int()
    _check(_lib.pcr_autotune_read(0, None, None, None, C.byref(n), 0))
    k = n.value
    keys = (C.c_int64 * (7 * max(k, 1)))()
    ch = (C.c_int * max(k, 1))()
    ms = (C.c_double * max(k, 1))()
    _check(_lib.pcr_autotune_read(k, keys, ch, ms, C.byref(n), 1 if reset else 0))
    return {tuple(keys[7 * i:7 * i + 7]): (ch[i], ms[i]) for i in range(min(k, n.value))}


def retrieve_batch(handles, plans, outs, stream=None):
    """pcr_retrieve_batch_plan: one work list per stage for n (handle, plan,
    output) triples."""
    n = len(handles)
    hp = (C.c_void_p * n)(*[h._p.value for h in handles])
    pl = (_Plan * n)(*[p._c for p in plans])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(_lib.pcr_retrieve_batch_plan(n, hp, pl, op, _stream_ptr(stream)))
    return outs


def retrieve_batch_targets(handles, targets, outs, stream=None):
    """pcr_retrieve_batch: each target planned, all retrieved with one work
    list per stage.  Returns [RetrievalInfo]."""
    n = len(handles)
    hp = (C.c_void_p * n)(*[h._p.value for h in handles])
    tg = (_Target * n)(*[t.c() for t in targets])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    infos = (_Info * n)()
    _check(_lib.pcr_retrieve_batch(n, hp, tg, op, _stream_ptr(stream), infos))
    return [RetrievalInfo.of(i) for i in infos]


def deserialize(data: bytes, device=None, stream=None):
    import struct
    out = C.c_void_p()
    buf = C.create_string_buffer(data, len(data))
    _check(_lib.pcr_deserialize(buf, len(data), C.byref(_ALLOCATOR), _stream_ptr(stream), C.byref(out)))
    # header: magic, hdr len, crc, then ndim, dims[3], dtype
    ndim = struct.unpack_from("<i", data, 20)[0]
    dims = struct.unpack_from("<3q", data, 24)[:ndim]
    dtype = torch.float32 if struct.unpack_from("<i", data, 48)[0] == 0 else torch.float64
    return Handle(out.value, dims, dtype, device or torch.device("cuda", torch.cuda.current_device()))


def debug_encode(vals: torch.Tensor, value_kind: int, B: int, encoding: int, want_pairs: bool, stream=None):
    """Test entry: encode already-ordered padded values (see pcr_debug_encode)."""
    import numpy as np
    n = vals.numel()
    words, nseg = n // 32, -(-n // 4096)
    planes = np.zeros((B, words), np.uint32)
    signs = np.zeros((nseg, 128 + B), np.uint32)
    scnt = np.zeros((nseg, B), np.uint32)
    pnz = np.zeros(B, np.uint32)
    pairs = np.zeros((B, B), np.uint64)
    vmax = C.c_double()
    _check(_lib.pcr_debug_encode(C.c_void_p(vals.data_ptr()), n, value_kind, B, encoding, int(want_pairs),
                                 _stream_ptr(stream), planes.ctypes.data, signs.ctypes.data,
                                 scnt.ctypes.data, pnz.ctypes.data, pairs.ctypes.data, C.byref(vmax)))
    return dict(planes=planes, signs=signs, sign_counts=scnt, plane_nz=pnz, pairs=pairs, vmax=vmax.value)


def profile_enable(on=True):
    """Per-stage CUDA-event timing inside the library (tracing)."""
    _check(_lib.pcr_profile_enable(int(on)))


def profile_read(reset=True):
    """{stage: (milliseconds, kernel launches)} since the last reset."""
    cap = 64
    names = C.create_string_buffer(48 * cap)
    ms = (C.c_double * cap)()
    ln = (C.c_int64 * cap)()
    n = C.c_int()
    _check(_lib.pcr_profile_read(cap, names, ms, ln, C.byref(n), int(reset)))
    out = {}
    for k in range(min(n.value, cap)):
        nm = names.raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (ms[k], ln[k])
    return out


def launch_count():
    """Kernels launched by libpcr since it was loaded."""
    return int(_lib.pcr_launch_count())


def library_path():
    return _LIB_PATH
