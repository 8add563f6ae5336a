"""Periodic neighbor query, RDF and Steinhardt order parameters on one GB300 GPU.

A thin ctypes binding over libfgb.so (C ABI declared in include/fgb.h).  Every step of
the computation runs in the library's CUDA kernels; this module only marshals torch
tensors (device memory and the current stream) into the C calls.  The API mirrors
freud (arXiv 1906.06317, Section "Implementation" and the usage listings):

    nq = NeighborQuery(box, points)                       # cell list on the GPU
    nl = nq.query(points, dict(r_max=2.5, exclude_ii=True)).toNeighborList()
    rdf = RDF(bins=500, r_max=5.0); rdf.compute(nq, reset=False); rdf.rdf
    q6 = Steinhardt(6); q6.compute(nq, neighbors=nl); q6.particle_order
    Q = Q6Mean.apply(points, nq, nl, 6)                   # differentiable global Q_l

There is no CPU fallback: importing works without a GPU, but every call needs the
built library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfgb.so")

OK = 0
ERR_INVALID_ARG, ERR_BOX_TOO_SMALL, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_CAPACITY = -1, -2, -3, -4, -5, -6
_ERR_NAMES = {-1: "INVALID_ARG", -2: "BOX_TOO_SMALL", -3: "OOM", -4: "CUDA", -5: "UNSUPPORTED", -6: "CAPACITY"}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_F = ctypes.c_float
_PP = ctypes.POINTER(ctypes.c_void_p)


class FGBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fgb error {_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class fgb_box(ctypes.Structure):
    _fields_ = [("Lx", _D), ("Ly", _D), ("Lz", _D), ("xy", _D), ("xz", _D), ("yz", _D)]


class fgb_query_args(ctypes.Structure):
    _fields_ = [("r_max", _D), ("num_neighbors", _I32), ("exclude_ii", _I32)]


class fgb_batch_params(ctypes.Structure):
    _fields_ = [("r_max", _D), ("l", _I32), ("rdf_bins", _I32), ("rdf_r_max", _D), ("rdf_r_min", _D),
                ("cell_div", _I32), ("block", _I32), ("hist_copies", _I32), ("tile_cells", _I32),
                ("cells_per_warp", _I32)]


_SIGS = {
    "fgb_last_error": (ctypes.c_char_p, []),
    "fgb_version": (_I32, []),
    "fgb_kernel_launches": (_I64, []),
    "fgb_trim_memory": (_I32, []),
    "fgb_set_memory_cache": (_I32, [ctypes.c_uint64]),
    "fgb_timing_enable": (_I32, [_I32]),
    "fgb_timing_read": (_I32, [ctypes.c_char_p, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "fgb_timing_reset": (_I32, []),
    "fgb_nq_create": (_I32, [ctypes.POINTER(fgb_box), _P, _I64, _D, _P, _PP]),
    "fgb_nq_destroy": (None, [_P]),
    "fgb_aabb_create": (_I32, [ctypes.POINTER(fgb_box), _P, _I64, _P, _PP]),
    "fgb_nq_create_points": (_I32, [ctypes.POINTER(fgb_box), _P, _I64, _PP]),
    "fgb_nq_dims": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "fgb_nq_cells": (_I32, [_P, _PP, _PP, _PP]),
    "fgb_nq_query": (_I32, [_P, _P, _I64, ctypes.POINTER(fgb_query_args), _P, _PP]),
    "fgb_nq_query_async": (_I32, [_P, ctypes.POINTER(fgb_query_args), _I64, _P, _PP]),
    "fgb_nlist_wait": (_I32, [_P, ctypes.POINTER(_I32)]),
    "fgb_nlist_size": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "fgb_nlist_arrays": (_I32, [_P, _PP, _PP, _PP, _PP, _PP]),
    "fgb_nlist_escalations": (_I32, [_P, ctypes.POINTER(_I64)]),
    "fgb_nlist_from_arrays": (_I32, [_I64, _I64, _P, _P, _P, _I64, _I32, _P, _PP]),
    "fgb_nlist_destroy": (None, [_P]),
    "fgb_rdf_create": (_I32, [_I32, _D, _D, _PP]),
    "fgb_rdf_destroy": (None, [_P]),
    "fgb_rdf_compute": (_I32, [_P, _P, _P, _I64, _P, _I32, _P]),
    "fgb_rdf_result": (_I32, [_P, _P, _P, _P, _P]),
    "fgb_rdf_counts_device": (_I32, [_P, _PP]),
    "fgb_rdf_escalations": (_I32, [_P, ctypes.POINTER(_I64), _P]),
    "fgb_rdf_noalloc": (_I32, [ctypes.POINTER(fgb_box), _P, _I64, _I32, _D, _D, _P, _P]),
    "fgb_rdf_params": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "fgb_nq_count_cells": (_I32, [_P, _D, _I32, _I64, _I64, _P, _P]),
    "fgb_nq_shard_segments": (_I32, [_P, _I64, _I64, _P, _P, _P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_uint32),
                                     _P]),
    "fgb_nq_write_cells": (_I32, [_P, _D, _I32, _I64, _I64, _P, _P, ctypes.c_uint32, _P, _P, _P, _P]),
    "fgb_rdf_compute_cells": (_I32, [_P, _P, _I64, _I64, _I32, _P]),
    "fgb_pmftxy_create": (_I32, [_D, _D, _I32, _I32, _PP]),
    "fgb_pmftxy_destroy": (None, [_P]),
    "fgb_pmftxy_compute": (_I32, [_P, _P, _P, _P, _I64, _P, _I32, _P]),
    "fgb_pmftxy_result": (_I32, [_P, _P, _P, _P, _P]),
    "fgb_pmftxy_counts_device": (_I32, [_P, _PP]),
    "fgb_pmftxy_escalations": (_I32, [_P, ctypes.POINTER(_I64), _P]),
    "fgb_steinhardt_create": (_I32, [_I32, _PP]),
    "fgb_steinhardt_destroy": (None, [_P]),
    "fgb_steinhardt_compute": (_I32, [_P, _P, _P, ctypes.POINTER(fgb_query_args), _P, _P]),
    "fgb_steinhardt_state": (_I32, [_P, _PP, _PP]),
    "fgb_steinhardt_backward": (_I32, [_P, _P, _P, _P, _F, _P, _P]),
    "fgb_steinhardt_wl": (_I32, [_P, _I32, _P, _P]),
    "fgb_steinhardt_average": (_I32, [_P, _P, _P, _P]),
    "fgb_local_descriptors": (_I32, [ctypes.POINTER(fgb_box), _P, _P, _P, _I32, _I32, _P, _P]),
    "fgb_cluster_compute": (_I32, [_I64, _P, _P, _P, _PP]),
    "fgb_cluster_result": (_I32, [_P, ctypes.POINTER(_I64), _PP, _PP]),
    "fgb_cluster_properties": (_I32, [_P, ctypes.POINTER(fgb_box), _P, _P, _P, _P]),
    "fgb_cluster_destroy": (None, [_P]),
    "fgb_solid_liquid": (_I32, [ctypes.POINTER(fgb_box), _P, _P, _I32, _D, _I32, _I32, _P, _P, _P, _PP]),
    "fgb_batch_create": (_I32, [_I32, _P, ctypes.POINTER(fgb_box), ctypes.POINTER(fgb_batch_params), _P, _PP]),
    "fgb_batch_destroy": (None, [_P]),
    "fgb_batch_run": (_I32, [_P, _P, _P]),
    "fgb_batch_run_graph": (_I32, [_P, _P, _P]),
    "fgb_batch_tune": (_I32, [_P, _P, _P, ctypes.POINTER(fgb_batch_params)]),
    "fgb_batch_outputs": (_I32, [_P, _PP, _PP, _PP]),
    "fgb_batch_routes": (_I32, [_P, _P, _P]),
}

_lib = None


def lib():
    """The loaded libfgb.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfgb.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                              "or python -m paper_1906_06317_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels launched by libfgb in this process so far."""
    return int(lib().fgb_kernel_launches())


def trim_memory():
    """Return the device blocks the library keeps for reuse."""
    _check(lib().fgb_trim_memory())


def set_memory_cache(nbytes: int):
    """Largest total of freed device memory the library keeps for reuse (default 4 GB)."""
    _check(lib().fgb_set_memory_cache(int(nbytes)))


def timing_enable(on: bool = True):
    _check(lib().fgb_timing_enable(int(bool(on))))


def timing_read(name: str):
    """(total device ms, launches) of the named kernel since the last reset."""
    ms, n = _D(), _I64()
    _check(lib().fgb_timing_read(name.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def timing_reset():
    _check(lib().fgb_timing_reset())


def exported_symbols():
    return [n for n in _SIGS if hasattr(lib(), n)]


def _check(code: int):
    if code != OK:
        raise FGBError(code, lib().fgb_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t: torch.Tensor, dtype=torch.float32, name="tensor") -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.contiguous()


class _DeviceArray:
    """Exposes library-owned device memory to torch without a copy; keeps its owner alive."""

    _TYPES = {torch.int32: "<i4", torch.int64: "<i8", torch.float32: "<f4", torch.uint64: "<u8",
              torch.uint32: "<u4"}

    def __init__(self, ptr: int, shape, dtype, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": self._TYPES[dtype],
                                         "data": (int(ptr or 0), False), "version": 2, "strides": None}


class _Owned:
    """Owns one library handle; tensor views of its memory keep this object (not the
    Python wrapper) alive, so wrappers and views never form a reference cycle and a
    handle is released as soon as the last of them goes."""

    def __init__(self, ptr, destroy, keep=()):
        self.ptr = ctypes.c_void_p(ptr)
        self._destroy = destroy
        self._keep = keep

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            getattr(_lib, self._destroy)(self.ptr)
            self.ptr = None


def _view(ptr, shape, dtype, owner) -> torch.Tensor:
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, shape, dtype, owner), device="cuda")


# ------------------------------------------------------------------------------ Box


@dataclass
class Box:
    """Triclinic periodic box (Lx, Ly, Lz, xy, xz, yz), centred on the origin.  Lz = 0 is
    a 2D box (xz = yz = 0, every point at z = 0)."""
    Lx: float
    Ly: float
    Lz: float
    xy: float = 0.0
    xz: float = 0.0
    yz: float = 0.0

    @classmethod
    def from_box(cls, b) -> "Box":
        if isinstance(b, Box):
            return b
        if hasattr(b, "params"):
            return cls(*[float(v) for v in b.params()])
        a = np.asarray(b, dtype=np.float64)
        if a.shape == (3, 3):
            Lx, Ly, Lz = a[0, 0], a[1, 1], a[2, 2]
            return cls(Lx, Ly, Lz, a[0, 1] / Ly, a[0, 2] / Lz, a[1, 2] / Lz)
        if a.shape == (3,):
            return cls(*a)
        if a.shape == (6,):
            return cls(*a)
        raise ValueError("box must be a Box, 3 lengths, 6 parameters or a 3x3 upper-triangular matrix")

    def _c(self) -> fgb_box:
        return fgb_box(self.Lx, self.Ly, self.Lz, self.xy, self.xz, self.yz)

    @property
    def volume(self) -> float:
        return self.Lx * self.Ly * self.Lz

    @property
    def is2D(self) -> bool:
        return self.Lz == 0.0

    @property
    def area(self) -> float:
        return self.Lx * self.Ly


# ------------------------------------------------------------------- NeighborQuery


class NeighborList:
    """Query results, sorted by (query index, point index) (ball) or by distance (kNN).

    A list from NeighborQuery.query_async is pending until wait() (or the first read of
    its sizes or arrays, which waits)."""

    _LAZY = frozenset(("n_pairs", "n_query", "query_point_indices", "point_indices", "distances", "segments",
                       "neighbor_counts", "escalations", "rewritten"))

    def __init__(self, handle, keep, pending=False, on_complete=None):
        self._o = _Owned(handle, "fgb_nlist_destroy", keep)
        self._h = self._o.ptr
        self._pending = pending
        self._on_complete = on_complete
        if not pending:
            self.rewritten = False
            self._fill()

    def __getattr__(self, name):
        if name in NeighborList._LAZY and self.__dict__.get("_pending"):
            self.wait()
            return self.__dict__[name]
        raise AttributeError(name)

    def wait(self) -> "NeighborList":
        """Completes a pending list (fgb_nlist_wait); no-op for a complete one."""
        if self.__dict__.get("_pending"):
            r = _I32()
            _check(lib().fgb_nlist_wait(self._h, ctypes.byref(r)))
            self._pending = False
            self.rewritten = bool(r.value)
            self._fill()
            if self._on_complete is not None:
                self._on_complete(self.n_pairs)
        return self

    def _fill(self):
        L = lib()
        m, nq = _I64(), _I64()
        _check(L.fgb_nlist_size(self._h, ctypes.byref(m), ctypes.byref(nq)))
        self.n_pairs, self.n_query = m.value, nq.value
        p = [ctypes.c_void_p() for _ in range(5)]
        _check(L.fgb_nlist_arrays(self._h, *[ctypes.byref(x) for x in p]))
        o = self._o
        self.query_point_indices = _view(p[0].value, (self.n_pairs,), torch.int32, o)
        self.point_indices = _view(p[1].value, (self.n_pairs,), torch.int32, o)
        self.distances = _view(p[2].value, (self.n_pairs,), torch.float32, o)
        self.segments = _view(p[3].value, (self.n_query + 1,), torch.int64, o)
        self.neighbor_counts = _view(p[4].value, (self.n_query,), torch.int32, o)
        e = _I64()
        _check(L.fgb_nlist_escalations(self._h, ctypes.byref(e)))
        self.escalations = e.value

    @classmethod
    def from_arrays(cls, num_query_points, num_points, query_point_indices, point_indices, distances=None,
                    symmetric=False):
        qi = _need_cuda(query_point_indices, torch.int32, "query_point_indices")
        pj = _need_cuda(point_indices, torch.int32, "point_indices")
        d = None if distances is None else _need_cuda(distances, torch.float32, "distances")
        h = ctypes.c_void_p()
        _check(lib().fgb_nlist_from_arrays(num_query_points, num_points, qi.data_ptr(), pj.data_ptr(),
                                           None if d is None else d.data_ptr(), qi.numel(), int(bool(symmetric)),
                                           _stream(), ctypes.byref(h)))
        return cls(h.value, None)

    def __len__(self):
        return self.n_pairs


class _QueryResult:
    def __init__(self, nq, query_points, args):
        self._nq, self._qp, self._args = nq, query_points, args

    def toNeighborList(self) -> NeighborList:
        return self._nq._run_query(self._qp, self._args)


class NeighborQuery:
    """Cell-list NeighborQuery over device points (N, 3) float32.

    r_cell sets the cell width (default: the r_max it will mostly be queried with);
    queries with a larger r_max widen the stencil automatically."""

    def __init__(self, box, points: torch.Tensor, r_cell: float = None):
        self.box = Box.from_box(box)
        self.points = _need_cuda(points, name="points")
        if self.points.ndim != 2 or self.points.shape[1] != 3:
            raise ValueError("points must have shape (N, 3)")
        if r_cell is None:
            n = max(1, self.points.shape[0])
            if self.box.is2D:
                r_cell = 1.5 * (self.box.area / n) ** 0.5
            else:
                r_cell = 1.5 * (self.box.volume / n) ** (1.0 / 3.0)
        self.r_cell = float(r_cell)
        h = ctypes.c_void_p()
        b = self.box._c()
        _check(lib().fgb_nq_create(ctypes.byref(b), self.points.data_ptr(), self.points.shape[0], self.r_cell,
                                   _stream(), ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_nq_destroy", (self.points,))
        self._h = self._o.ptr

    @property
    def n_points(self) -> int:
        return int(self.points.shape[0])

    def cell_dims(self):
        nc = (_I32 * 3)()
        n = _I64()
        _check(lib().fgb_nq_dims(self._h, nc, ctypes.byref(n)))
        return tuple(nc)

    def cells(self):
        """(sorted (N,4) float32 view, sorted cell ids uint32, cell_start uint32)."""
        p = [ctypes.c_void_p() for _ in range(3)]
        _check(lib().fgb_nq_cells(self._h, *[ctypes.byref(x) for x in p]))
        nx, ny, nz = self.cell_dims()
        n = self.n_points
        o = self._o
        return (_view(p[0].value, (n, 4), torch.float32, o), _view(p[1].value, (n,), torch.int32, o),
                _view(p[2].value, (nx * ny * nz + 1,), torch.int32, o))

    def query(self, query_points=None, query_args=None) -> _QueryResult:
        args = dict(query_args or {})
        return _QueryResult(self, query_points, args)

    def _run_query(self, query_points, args) -> NeighborList:
        qa = fgb_query_args(float(args.get("r_max", 0.0) or 0.0), int(args.get("num_neighbors", 0) or 0),
                            int(bool(args.get("exclude_ii", query_points is None or query_points is self.points))))
        keep = [self._o]
        if query_points is None or query_points is self.points:
            qp, nq = None, 0
        else:
            qpt = _need_cuda(query_points, name="query_points")
            keep.append(qpt)
            qp, nq = qpt.data_ptr(), qpt.shape[0]
        h = ctypes.c_void_p()
        _check(lib().fgb_nq_query(self._h, qp, nq, ctypes.byref(qa), _stream(), ctypes.byref(h)))
        return NeighborList(h.value, keep)

    def query_async(self, r_max: float, exclude_ii: bool = True, capacity: int = None) -> NeighborList:
        """Self ball query queued on the current stream without a host synchronisation
        (fgb_nq_query_async).  The list is pending until wait() or the first read of its
        sizes or arrays.  capacity (pairs) defaults to 5 % above the last list of the
        same r_max from this NeighborQuery, else to the library's estimate for uniformly
        spread points; a list that does not fit is written again when completed."""
        key = (float(r_max), bool(exclude_ii))
        hints = self.__dict__.setdefault("_capacity_hints", {})
        if capacity is None:
            capacity = int(hints[key] * 1.05) + 1024 if key in hints else 0
        qa = fgb_query_args(float(r_max), 0, int(bool(exclude_ii)))
        h = ctypes.c_void_p()
        _check(lib().fgb_nq_query_async(self._h, ctypes.byref(qa), int(capacity), _stream(), ctypes.byref(h)))

        def remember(n_pairs, hints=hints, key=key):
            hints[key] = n_pairs
        return NeighborList(h.value, [self._o], pending=True, on_complete=remember)


class AABBQuery(NeighborQuery):
    """Tree NeighborQuery (freud locality.AABBQuery): a bounding-volume hierarchy over the
    device points, answering ball (r_max) and k-nearest queries with the same NeighborList
    as the cell list.  RDF and Steinhardt take it together with a NeighborList."""

    def __init__(self, box, points: torch.Tensor):
        self.box = Box.from_box(box)
        self.points = _need_cuda(points, name="points")
        if self.points.ndim != 2 or self.points.shape[1] != 3:
            raise ValueError("points must have shape (N, 3)")
        self.r_cell = None
        h = ctypes.c_void_p()
        b = self.box._c()
        _check(lib().fgb_aabb_create(ctypes.byref(b), self.points.data_ptr(), self.points.shape[0], _stream(),
                                     ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_nq_destroy", (self.points,))
        self._h = self._o.ptr

    def cells(self):
        raise FGBError(ERR_UNSUPPORTED, "a tree NeighborQuery has no cell list")



class PointsQuery(NeighborQuery):
    """The box and the points only, for computes given a NeighborList (no search
    structure is built; querying it raises)."""

    def __init__(self, box, points: torch.Tensor):
        self.box = Box.from_box(box)
        self.points = _need_cuda(points, name="points")
        if self.points.ndim != 2 or self.points.shape[1] != 3:
            raise ValueError("points must have shape (N, 3)")
        self.r_cell = None
        h = ctypes.c_void_p()
        b = self.box._c()
        _check(lib().fgb_nq_create_points(ctypes.byref(b), self.points.data_ptr(), self.points.shape[0],
                                          ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_nq_destroy", (self.points,))
        self._h = self._o.ptr

    def cells(self):
        raise FGBError(ERR_UNSUPPORTED, "a NeighborQuery of points only has no cell list")


def _as_nq(system, r_cell=None) -> NeighborQuery:
    if isinstance(system, NeighborQuery):
        return system
    box, pts = system
    return NeighborQuery(box, pts, r_cell)


# ------------------------------------------------------------------------------- RDF


class RDF:
    """Radial distribution function g(r) accumulated over frames (freud density.RDF)."""

    def __init__(self, bins: int, r_max: float, r_min: float = 0.0):
        self.bins, self.r_max, self.r_min = int(bins), float(r_max), float(r_min)
        h = ctypes.c_void_p()
        _check(lib().fgb_rdf_create(self.bins, self.r_max, self.r_min, ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_rdf_destroy")
        self._h = self._o.ptr

    def compute(self, system, neighbors=None, query_points=None, reset=True):
        nq = _as_nq(system, self.r_max)
        nl = neighbors if isinstance(neighbors, NeighborList) else None
        qp, n_q = None, 0
        if query_points is not None:
            qpt = _need_cuda(query_points, name="query_points")
            qp, n_q = qpt.data_ptr(), qpt.shape[0]
        _check(lib().fgb_rdf_compute(self._h, nq._h, qp, n_q, nl._h if nl is not None else None, int(bool(reset)), _stream()))
        self._nq = nq
        return self

    def _result(self):
        c = np.zeros(self.bins, np.uint64)
        g = np.zeros(self.bins, np.float64)
        r = np.zeros(self.bins, np.float64)
        _check(lib().fgb_rdf_result(self._h, c.ctypes.data, g.ctypes.data, r.ctypes.data, _stream()))
        return c, g, r

    @property
    def bin_counts(self) -> np.ndarray:
        return self._result()[0]

    @property
    def rdf(self) -> np.ndarray:
        return self._result()[1]

    @property
    def bin_centers(self) -> np.ndarray:
        return self._result()[2]

    def counts_device(self) -> torch.Tensor:
        p = ctypes.c_void_p()
        _check(lib().fgb_rdf_counts_device(self._h, ctypes.byref(p)))
        return _view(p.value, (self.bins,), torch.int64, self._o)

    def escalations(self) -> int:
        n = _I64()
        _check(lib().fgb_rdf_escalations(self._h, ctypes.byref(n), _stream()))
        return n.value


# ------------------------------------------------------------------------------ PMFT


class PMFTXY:
    """PMFT(x, y) of a 2D system accumulated over frames (freud pmft.PMFTXY): every bond
    in the frame of its query particle (orientation angle about z), binned on
    [-x_max, x_max) x [-y_max, y_max); `bins` is one count or (bins_x, bins_y)."""

    def __init__(self, x_max: float, y_max: float, bins):
        bx, by = (bins, bins) if np.isscalar(bins) else bins
        self.x_max, self.y_max, self.bins = float(x_max), float(y_max), (int(bx), int(by))
        h = ctypes.c_void_p()
        _check(lib().fgb_pmftxy_create(self.x_max, self.y_max, self.bins[0], self.bins[1], ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_pmftxy_destroy")
        self._h = self._o.ptr

    def compute(self, system, query_orientations, query_points=None, neighbors=None, reset=True):
        reach = (self.x_max ** 2 + self.y_max ** 2) ** 0.5 * (1.0 + 1e-6)
        nq = _as_nq(system, reach)
        nl = neighbors if isinstance(neighbors, NeighborList) else None
        th = _need_cuda(query_orientations, name="query_orientations")
        qp, n_q = None, nq.n_points
        if query_points is not None:
            qpt = _need_cuda(query_points, name="query_points")
            qp, n_q = qpt.data_ptr(), qpt.shape[0]
        if th.numel() != n_q:
            raise ValueError("one orientation per query point")
        _check(lib().fgb_pmftxy_compute(self._h, nq._h, qp, th.data_ptr(), n_q, nl._h if nl is not None else None,
                                        int(bool(reset)), _stream()))
        self._nq = nq
        return self

    def _result(self):
        shape = self.bins
        c = np.zeros(shape, np.uint64)
        g = np.zeros(shape, np.float64)
        f = np.zeros(shape, np.float64)
        _check(lib().fgb_pmftxy_result(self._h, c.ctypes.data, g.ctypes.data, f.ctypes.data, _stream()))
        return c, g, f

    @property
    def bin_counts(self) -> np.ndarray:
        return self._result()[0]

    @property
    def pcf(self) -> np.ndarray:
        return self._result()[1]

    @property
    def pmft(self) -> np.ndarray:
        return self._result()[2]

    @property
    def bin_centers(self):
        bx, by = self.bins
        dx, dy = 2 * self.x_max / bx, 2 * self.y_max / by
        return (-self.x_max + (np.arange(bx) + 0.5) * dx, -self.y_max + (np.arange(by) + 0.5) * dy)

    def counts_device(self) -> torch.Tensor:
        p = ctypes.c_void_p()
        _check(lib().fgb_pmftxy_counts_device(self._h, ctypes.byref(p)))
        return _view(p.value, self.bins, torch.int64, self._o)

    def escalations(self) -> int:
        n = _I64()
        _check(lib().fgb_pmftxy_escalations(self._h, ctypes.byref(n), _stream()))
        return n.value


# ------------------------------------------------------------------------ Steinhardt


class Steinhardt:
    """Steinhardt q_l per particle (freud order.Steinhardt); wl() gives W_l and average()
    the neighbor-averaged q_l from the same Q_lm."""

    def __init__(self, l: int):
        self.l = int(l)
        h = ctypes.c_void_p()
        _check(lib().fgb_steinhardt_create(self.l, ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_steinhardt_destroy")
        self._h = self._o.ptr
        self.particle_order = None

    def compute(self, system, neighbors=None):
        nq = _as_nq(system)
        nl = neighbors if isinstance(neighbors, NeighborList) else None
        qa = None
        if nl is None:
            d = dict(neighbors or {})
            if "num_neighbors" in d:
                nl = nq.query(None, d).toNeighborList()
            else:
                qa = fgb_query_args(float(d.get("r_max", 0.0)), 0, int(bool(d.get("exclude_ii", True))))
        q = torch.empty(nq.n_points, dtype=torch.float32, device="cuda")
        _check(lib().fgb_steinhardt_compute(self._h, nq._h, nl._h if nl is not None else None,
                                            ctypes.byref(qa) if qa is not None else None, q.data_ptr(), _stream()))
        self.particle_order = q
        self._nq, self._nl = nq, nl
        return self

    def qlm(self) -> torch.Tensor:
        p, c = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgb_steinhardt_state(self._h, ctypes.byref(p), ctypes.byref(c)))
        return torch.view_as_complex(_view(p.value, (self._nq.n_points, self.l + 1, 2), torch.float32, self._o))

    def neighbor_counts(self) -> torch.Tensor:
        p, c = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgb_steinhardt_state(self._h, ctypes.byref(p), ctypes.byref(c)))
        return _view(c.value, (self._nq.n_points,), torch.int32, self._o)

    def wl(self, normalize: bool = True) -> torch.Tensor:
        """W_l per particle from the current Q_lm (normalised by |Q_l|^3 unless normalize=False)."""
        w = torch.empty(self._nq.n_points, dtype=torch.float32, device="cuda")
        _check(lib().fgb_steinhardt_wl(self._h, int(bool(normalize)), w.data_ptr(), _stream()))
        return w

    def average(self, neighbors: "NeighborList" = None) -> torch.Tensor:
        """Neighbor-averaged q_l (Lechner-Dellago); the state then holds the averaged Q_lm."""
        nl = neighbors if neighbors is not None else self._nl
        if nl is None:
            raise FGBError(ERR_UNSUPPORTED, "averaging needs the neighbors as a NeighborList")
        q = torch.empty(self._nq.n_points, dtype=torch.float32, device="cuda")
        _check(lib().fgb_steinhardt_average(self._h, nl._h, q.data_ptr(), _stream()))
        self.particle_order = q
        return q

    def backward(self, upstream: float = 1.0) -> torch.Tensor:
        """d(upstream * mean_i q_l(i)) / d positions, neighbor list of the last compute fixed."""
        if self._nl is None:
            raise FGBError(ERR_UNSUPPORTED, "backward needs the neighbors as a NeighborList")
        g = torch.empty((self._nq.n_points, 3), dtype=torch.float32, device="cuda")
        _check(lib().fgb_steinhardt_backward(self._h, self._nq._h, self._nl._h, self.particle_order.data_ptr(),
                                             float(upstream), g.data_ptr(), _stream()))
        return g



class LocalDescriptors:
    """Spherical harmonics Y_lm (l <= l_max) of every bond of a NeighborList (freud
    environment.LocalDescriptors, global orientation): sph is (n_pairs, n_sph) complex64,
    m = -l..l per l when negative_m (else m = 0..l)."""

    def __init__(self, l_max: int, negative_m: bool = True):
        self.l_max, self.negative_m = int(l_max), bool(negative_m)
        self.sph = None

    @property
    def num_sphs(self) -> int:
        return (self.l_max + 1) ** 2 if self.negative_m else (self.l_max + 1) * (self.l_max + 2) // 2

    def compute(self, system, neighbors: NeighborList, query_points=None):
        nq = _as_nq(system)
        out = torch.empty((neighbors.n_pairs, self.num_sphs, 2), dtype=torch.float32, device="cuda")
        qp = None if query_points is None else _need_cuda(query_points, name="query_points")
        b = nq.box._c()
        _check(lib().fgb_local_descriptors(ctypes.byref(b), nq.points.data_ptr(), None if qp is None else qp.data_ptr(),
                                           neighbors._h, self.l_max, int(self.negative_m), out.data_ptr(), _stream()))
        self.sph = torch.view_as_complex(out)
        return self


class Cluster:
    """Clusters of points joined by neighbor bonds (freud cluster.Cluster): cluster_idx per
    point, clusters numbered by decreasing size (ties: smallest member first).  bond_mask
    (uint8 per pair of the list) selects the bonds that join."""

    def __init__(self):
        self.cluster_idx = None
        self.cluster_sizes = None
        self.num_clusters = 0
        self._o = None

    def compute(self, system, neighbors: NeighborList, bond_mask: torch.Tensor = None):
        nq = _as_nq(system)
        m = None if bond_mask is None else _need_cuda(bond_mask, torch.uint8, "bond_mask")
        h = ctypes.c_void_p()
        _check(lib().fgb_cluster_compute(nq.n_points, neighbors._h, None if m is None else m.data_ptr(), _stream(),
                                         ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_cluster_destroy")
        nc, ci, sz = _I64(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgb_cluster_result(self._o.ptr, ctypes.byref(nc), ctypes.byref(ci), ctypes.byref(sz)))
        self.num_clusters = nc.value
        self.cluster_idx = _view(ci.value, (nq.n_points,), torch.int32, self._o)
        self.cluster_sizes = _view(sz.value, (nc.value,), torch.int32, self._o)
        self._nq = nq
        return self

    def properties(self):
        """(centers (num_clusters, 3), gyration tensors (num_clusters, 3, 3)) on the device."""
        c = torch.empty((self.num_clusters, 3), dtype=torch.float32, device="cuda")
        g = torch.empty((self.num_clusters, 3, 3), dtype=torch.float32, device="cuda")
        b = self._nq.box._c()
        _check(lib().fgb_cluster_properties(self._o.ptr, ctypes.byref(b), self._nq.points.data_ptr(), c.data_ptr(),
                                            g.data_ptr(), _stream()))
        return c, g


class SolidLiquid:
    """Solid-liquid order parameter (freud order.SolidLiquid): per bond the normalised
    q_lm dot product ql_ij, per particle the number of solid-like bonds (ql_ij >
    q_threshold), and clusters of solid particles (>= solid_threshold solid-like bonds)
    joined by solid-like bonds."""

    def __init__(self, l: int, q_threshold: float, solid_threshold: int, normalize_q: bool = True):
        self.l, self.q_threshold = int(l), float(q_threshold)
        self.solid_threshold, self.normalize_q = int(solid_threshold), bool(normalize_q)

    def compute(self, system, neighbors: NeighborList):
        nq = _as_nq(system)
        self.ql_ij = torch.empty(neighbors.n_pairs, dtype=torch.float32, device="cuda")
        self.num_connections = torch.empty(nq.n_points, dtype=torch.int32, device="cuda")
        b = nq.box._c()
        h = ctypes.c_void_p()
        _check(lib().fgb_solid_liquid(ctypes.byref(b), nq.points.data_ptr(), neighbors._h, self.l, self.q_threshold,
                                      self.solid_threshold, int(self.normalize_q), self.ql_ij.data_ptr(),
                                      self.num_connections.data_ptr(), _stream(), ctypes.byref(h)))
        c = Cluster()
        c._o = _Owned(h.value, "fgb_cluster_destroy")
        nc, ci, sz = _I64(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgb_cluster_result(c._o.ptr, ctypes.byref(nc), ctypes.byref(ci), ctypes.byref(sz)))
        c.num_clusters = nc.value
        c.cluster_idx = _view(ci.value, (nq.n_points,), torch.int32, c._o)
        c.cluster_sizes = _view(sz.value, (nc.value,), torch.int32, c._o)
        c._nq = nq
        self.clusters = c
        self.cluster_idx = c.cluster_idx
        self.largest_cluster_size = int(c.cluster_sizes[0]) if nc.value > 0 else 0
        return self


class Q6Mean(torch.autograd.Function):
    """Q_l = mean_i q_l(i) as a differentiable function of the positions (neighbor list
    fixed), with the hand-written backward kernel.  Usage: Q6Mean.apply(points, box, nl, 6)."""

    @staticmethod
    def forward(ctx, points, box, nlist, l=6):
        nq = PointsQuery(box, points.detach())  # the list is fixed: no cell list needed
        st = Steinhardt(l)
        st.compute(nq, neighbors=nlist)
        ctx.st = st
        return st.particle_order.mean()

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.st.backward(1.0)
        return g * grad_out, None, None, None


# ---------------------------------------------------------------------------- batches


class Batch:
    """Many frames of uneven size analysed in one pass (RDF counts per frame and q_l per
    particle), replayable from a CUDA graph."""

    def __init__(self, frame_sizes, boxes, r_max=1.5, l=6, rdf_bins=200, rdf_r_max=3.0, rdf_r_min=0.0,
                 cell_div=0, block=0, hist_copies=0, tile_cells=0, cells_per_warp=0):
        sizes = np.asarray(frame_sizes, dtype=np.int64)
        self.offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=self.offsets[1:])
        bx = (fgb_box * len(sizes))(*[Box.from_box(b)._c() for b in boxes])
        self.params = fgb_batch_params(r_max, l, rdf_bins, rdf_r_max, rdf_r_min, cell_div, block, hist_copies,
                                       tile_cells, cells_per_warp)
        h = ctypes.c_void_p()
        _check(lib().fgb_batch_create(len(sizes), self.offsets.ctypes.data, bx, ctypes.byref(self.params), _stream(),
                                      ctypes.byref(h)))
        self._o = _Owned(h.value, "fgb_batch_destroy")
        self._h = self._o.ptr
        self.n_frames, self.rdf_bins = len(sizes), rdf_bins
        self.total = int(self.offsets[-1])

    def run(self, points: torch.Tensor, graph: bool = False):
        p = _need_cuda(points, name="points")
        self._points = p
        fn = lib().fgb_batch_run_graph if graph else lib().fgb_batch_run
        _check(fn(self._h, p.data_ptr(), _stream()))
        return self

    def tune(self, points: torch.Tensor):
        p = _need_cuda(points, name="points")
        chosen = fgb_batch_params()
        _check(lib().fgb_batch_tune(self._h, p.data_ptr(), _stream(), ctypes.byref(chosen)))
        return dict(cell_div=chosen.cell_div, block=chosen.block, hist_copies=chosen.hist_copies,
                    tile_cells=chosen.tile_cells, cells_per_warp=chosen.cells_per_warp)

    def routes(self):
        """Frames on the cell-tile kernels and on the per-point kernel (current settings)."""
        t, p = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fgb_batch_routes(self._h, ctypes.byref(t), ctypes.byref(p)))
        return dict(tile=t.value, per_point=p.value)

    def outputs(self):
        r, q, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgb_batch_outputs(self._h, ctypes.byref(r), ctypes.byref(q), ctypes.byref(n)))
        o = self._o
        return (_view(r.value, (self.n_frames, self.rdf_bins), torch.int64, o),
                _view(q.value, (self.total,), torch.float32, o), _view(n.value, (self.total,), torch.int32, o))
