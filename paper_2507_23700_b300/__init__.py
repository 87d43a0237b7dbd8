"""B300-native linear-BVH geometric search: the Python binding of libarbx.

A thin ctypes layer over the C ABI in ``include/arbx.h`` (same entry points,
same names).  It only marshals arguments: torch tensors supply device memory
and the current CUDA stream; every step of building and querying runs in the
CUDA kernels of ``libarbx.so``.  There is no CPU fallback: importing this
package fails if the library has not been built
(``python paper_2507_23700_b300/_build.py``).

    import torch, paper_2507_23700_b300 as arbx
    pts = torch.rand(1_000_000, 3, device="cuda")
    tree = arbx.Tree(pts)                          # BVH(space, values)
    off, idx, d2 = tree.radius(queries, 0.01)      # storage query, CRS
    idx, d2 = tree.knn(queries, 16)                # nearest(point, k)
    cnt = tree.count(queries, 0.01)                # pure callback: count
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import torch

_PKG = Path(__file__).resolve().parent
# ARBX_CHECKED=1 loads the bounds-checked build of the same library
CHECKED = os.environ.get("ARBX_CHECKED", "0") == "1"
LIB_PATH = _PKG / ("libarbx_checked.so" if CHECKED else "libarbx.so")

if not LIB_PATH.exists():
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2507_23700_b300/_build.py"
                      f"{' --checked' if CHECKED else ''}`")

_lib = ctypes.CDLL(str(LIB_PATH))

# ------------------------------------------------------------------ constants (arbx.h)
(OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STACK_OVERFLOW, ERR_UNSUPPORTED, ERR_NONFINITE, ERR_CAPACITY,
 ERR_BOUNDS) = range(10)
LIB_CHECKED = 1
POINT, BOX, TRIANGLE = 0, 1, 2
SPHERE, BOX_PRED, NEAREST, RAY_NEAREST, RAY_INTERSECT, RAY_ORDERED = 0, 1, 2, 3, 4, 5
RAY_KINDS = (RAY_NEAREST, RAY_INTERSECT, RAY_ORDERED)
CB_COUNT, CB_COUNT_UP_TO, CB_FIRST_HIT = 0, 1, 2
QUANTIZED_NODES = 1
WIDE_NODES = 2
PARENT_RELATIVE = 4

_KINDS = {"point": POINT, "box": BOX, "triangle": TRIANGLE}


class arbx_primitives(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("n", ctypes.c_int64),
                ("data_dev", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class arbx_predicates(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("m", ctypes.c_int64),
                ("data_dev", ctypes.c_void_p), ("radii_dev", ctypes.c_void_p),
                ("radius", ctypes.c_float), ("k", ctypes.c_int32), ("order_dev", ctypes.c_void_p)]


class arbx_crs(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets_dev", ctypes.c_void_p),
                ("indices_dev", ctypes.c_void_p), ("d2_dev", ctypes.c_void_p)]


class arbx_tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("sort_queries", ctypes.c_int32),
                ("top_levels", ctypes.c_int32), ("grid_per_sm", ctypes.c_int32),
                ("warp_refill", ctypes.c_int32), ("stackless", ctypes.c_int32),
                ("single_pass", ctypes.c_int32), ("lanes_per_query", ctypes.c_int32),
                ("wide_nodes", ctypes.c_int32), ("warp_packets", ctypes.c_int32), ("query_runs", ctypes.c_int32)]


class arbx_forest_tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("chunk", ctypes.c_int32), ("sort_queries", ctypes.c_int32 * 3)]


_P = ctypes.c_void_p
_S = ctypes.c_int32
_SIGS = {
    "arbx_status_string": ([_S], ctypes.c_char_p),
    "arbx_abi_version": ([], ctypes.c_int32),
    "arbx_library_flags": ([], ctypes.c_uint32),
    "arbx_build": ([ctypes.POINTER(_P), ctypes.POINTER(arbx_primitives), _P], _S),
    "arbx_tree_info": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), _P], _S),
    "arbx_tree_destroy": ([_P], _S),
    "arbx_query_crs": ([_P, ctypes.POINTER(arbx_predicates), ctypes.c_int32, ctypes.POINTER(arbx_tuning),
                        ctypes.POINTER(arbx_crs), _P], _S),
    "arbx_crs_free": ([ctypes.POINTER(arbx_crs), _P], _S),
    "arbx_query_crs_host": ([_P, ctypes.POINTER(arbx_predicates), ctypes.c_int32, ctypes.POINTER(arbx_tuning), _P, _P,
                             _P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P], _S),
    "arbx_query_callback": ([_P, ctypes.POINTER(arbx_predicates), ctypes.c_int32, ctypes.c_int32, _P,
                             ctypes.POINTER(arbx_tuning), _P], _S),
    "arbx_query_offsets": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P], _S),
    "arbx_query_fill": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P, _P, _P], _S),
    "arbx_query_knn": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P, _P], _S),
    "arbx_query_ray_nearest": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P, _P], _S),
    "arbx_query_stats": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P], _S),
    "arbx_query_count_stats": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P], _S),
    "arbx_query_stats_r2": ([_P, ctypes.POINTER(arbx_predicates), ctypes.POINTER(arbx_tuning), _P, _P, _P], _S),
    "arbx_query_order": ([_P, ctypes.POINTER(arbx_predicates), _P, _P], _S),
    "arbx_query_offsets_noalloc": ([_P, ctypes.POINTER(arbx_predicates), _P, _P, _P], _S),
    "arbx_stream_check": ([_P], _S),
    "arbx_tree_export": ([_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P], _S),
    "arbx_profile_enable": ([ctypes.c_int32], _S),
    "arbx_profile_read": ([_P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], _S),
    "arbx_profile_reset": ([], _S),
    "arbx_launch_count": ([], ctypes.c_int64),
    "arbx_memory_trim": ([ctypes.c_int64], _S),
    "arbx_debug_fail_allocs": ([ctypes.c_int64, ctypes.c_int64], _S),
    "arbx_autotune": ([_P, ctypes.POINTER(arbx_predicates), ctypes.c_int64, ctypes.POINTER(arbx_tuning),
                       ctypes.POINTER(ctypes.c_double), _P], _S),
    "arbx_autotune_save": ([ctypes.c_char_p], _S),
    "arbx_dbscan": ([_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_int32, _P,
                     ctypes.POINTER(ctypes.c_int64), _P], _S),
    "arbx_autotune_load": ([ctypes.c_char_p], _S),
    "arbx_autotune_clear": ([], _S),
    "arbx_forest_build": ([ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _P, _P], _S),
    "arbx_forest_destroy": ([_P], _S),
    "arbx_forest_info": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)], _S),
    "arbx_forest_batch_create": ([ctypes.POINTER(_P), _P, _P, _P, _P], _S),
    "arbx_forest_batch_destroy": ([_P], _S),
    "arbx_forest_batch_total": ([_P, ctypes.POINTER(ctypes.c_int64)], _S),
    "arbx_forest_query_radius": ([_P, _P, _P, _P, _P, ctypes.c_int64, _P, _P], _S),
    "arbx_forest_query_knn": ([_P, _P, ctypes.c_int32, _P, _P, _P], _S),
    "arbx_forest_graph_create": ([ctypes.POINTER(_P), _P, _P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int32, _P, _P,
                                  _P], _S),
    "arbx_graph_launch": ([_P, _P], _S),
    "arbx_forest_batch_set_tuning": ([_P, ctypes.POINTER(arbx_forest_tuning)], _S),
    "arbx_forest_batch_get_tuning": ([_P, ctypes.POINTER(arbx_forest_tuning)], _S),
    "arbx_forest_autotune": ([_P, _P, ctypes.c_int32, ctypes.POINTER(arbx_forest_tuning),
                              ctypes.POINTER(ctypes.c_double), _P], _S),
    "arbx_graph_destroy": ([_P], _S),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class ArbxError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib.arbx_status_string(status).decode()} (status {status})")


def _check(status: int, what: str) -> None:
    if status != OK:
        raise ArbxError(status, what)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    return t.contiguous()


def _tuning(tuning) -> ctypes.POINTER(arbx_tuning) | None:
    if tuning is None:
        return None
    if isinstance(tuning, dict):
        t = arbx_tuning(tuning.get("block", 0), tuning.get("sort_queries", -1),
                        tuning.get("top_levels", -1), tuning.get("grid_per_sm", 0),
                        tuning.get("warp_refill", -1), tuning.get("stackless", -1),
                        tuning.get("single_pass", -1), tuning.get("lanes_per_query", 0),
                        tuning.get("wide_nodes", -1), tuning.get("warp_packets", -1), tuning.get("query_runs", 0))
    else:
        t = tuning
    return ctypes.pointer(t)


def abi_version() -> int:
    return _lib.arbx_abi_version()


def library_flags() -> int:
    """LIB_CHECKED when the bounds-checked build is loaded, else 0."""
    return int(_lib.arbx_library_flags())


def launch_count() -> int:
    """Kernels launched by libarbx since it was loaded."""
    return _lib.arbx_launch_count()


def profile_enable(on: bool = True) -> None:
    _check(_lib.arbx_profile_enable(1 if on else 0), "arbx_profile_enable")


def profile_reset() -> None:
    _check(_lib.arbx_profile_reset(), "arbx_profile_reset")


def profile_read() -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total device ms)} recorded since the last reset."""
    cap = 64
    names = ctypes.create_string_buffer(64 * cap)
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = ctypes.c_int32(0)
    _check(_lib.arbx_profile_read(names, launches, ms, cap, ctypes.byref(cnt)), "arbx_profile_read")
    out = {}
    for i in range(min(cnt.value, cap)):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def autotune_save(path: str) -> None:
    """Write the recorded launch settings (arbx_autotune_save)."""
    _check(_lib.arbx_autotune_save(str(path).encode()), "arbx_autotune_save")


def autotune_load(path: str) -> None:
    """Merge launch settings from a file written by autotune_save."""
    _check(_lib.arbx_autotune_load(str(path).encode()), "arbx_autotune_load")


def autotune_clear() -> None:
    """Forget every recorded launch setting."""
    _check(_lib.arbx_autotune_clear(), "arbx_autotune_clear")


def dbscan(points: torch.Tensor, eps: float, min_pts: int, stream=None) -> tuple[torch.Tensor, int]:
    """DBSCAN of CUDA float32 points (n, dim) (arbx_dbscan): (labels int32[n],
    -1 for noise, else the smallest core index of the cluster; number of
    clusters)."""
    pts = _dev_f32(points, "points")
    n, dim = pts.shape
    labels = torch.empty(n, dtype=torch.int32, device=pts.device)
    nc = ctypes.c_int64(0)
    _check(_lib.arbx_dbscan(pts.data_ptr() if n else None, n, dim, float(eps), int(min_pts),
                            labels.data_ptr() if n else None, ctypes.byref(nc), _stream(stream)), "arbx_dbscan")
    return labels, nc.value


def debug_fail_allocs(after: int, count: int) -> None:
    """Fault injection for tests (arbx_debug_fail_allocs): the next `count`
    device allocations after `after` successful ones fail with ERR_OOM."""
    _check(_lib.arbx_debug_fail_allocs(int(after), int(count)), "arbx_debug_fail_allocs")


def memory_trim(keep_bytes: int = 0) -> None:
    """Return the library's cached device memory to the driver (arbx_memory_trim)."""
    _check(_lib.arbx_memory_trim(int(keep_bytes)), "arbx_memory_trim")


def stream_check(stream=None) -> None:
    """Synchronise the stream and raise if a kernel reported an error."""
    _check(_lib.arbx_stream_check(_stream(stream)), "arbx_stream_check")


class _CRSOwner:
    """Owns the device buffers of one library CRS and frees them when the last
    reference goes (the CRS object and every tensor view hold one).  It holds
    no reference back, so no cycle delays the free to a garbage collection."""

    def __init__(self, crs: arbx_crs, stream: int):
        self.crs = crs
        self.stream = stream

    def __del__(self):
        try:
            _lib.arbx_crs_free(ctypes.byref(self.crs), self.stream)
        except Exception:  # interpreter shutdown
            pass


class _LibBuffer:
    """Device array owned by a library CRS, exposed to torch through the CUDA
    array interface; it keeps the owner alive."""

    def __init__(self, owner: _CRSOwner, ptr: int, n: int, typestr: str):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "stream": None}


class LibraryCRS:
    """CRS result allocated by ``arbx_query_crs``; freed when this object and
    every tensor view of it are gone."""

    def __init__(self, crs: arbx_crs, stream: int, want_d2: bool = False):
        self._owner = owner = _CRSOwner(crs, stream)
        m, nnz = crs.m, crs.nnz
        dev = torch.device("cuda", torch.cuda.current_device())

        def view(ptr, n, typestr, dtype):
            if n == 0 or not ptr:
                return torch.empty(0, dtype=dtype, device=dev)
            return torch.as_tensor(_LibBuffer(owner, ptr, n, typestr), device=dev)

        self.offsets = view(crs.offsets_dev, m + 1, "<i8", torch.int64)
        self.indices = view(crs.indices_dev, nnz, "<i4", torch.int32)
        self.d2 = view(crs.d2_dev, nnz, "<f4", torch.float32) if (crs.d2_dev or (want_d2 and nnz == 0)) else None


class Tree:
    """A linear BVH over primitives (ArborX 2.0, section 2.1: BVH(space, values)).

    data: CUDA float32 tensor; points (n, dim), boxes (n, 2*dim) as lo then hi,
    or triangles (n, 3, 3).  dim in {2, 3, 6} (triangles: 3).  quantized=True
    stores 16-bit child boxes in 48-byte nodes that keep their own box origin,
    quantized="parent" in 32-byte nodes coded relative to the box their parent
    decodes for them (triangles only); wide=True also builds the four-wide
    records of the nearest and counting traversals (points, boxes).
    """

    def __init__(self, data: torch.Tensor, kind: str = "point", quantized: bool | str = False, stream=None,
                 wide: bool = False):
        if quantized not in (False, True, "parent"):
            raise ValueError("quantized must be False, True or 'parent'")
        if kind not in _KINDS:
            raise ValueError(f"kind must be one of {sorted(_KINDS)}")
        data = _dev_f32(data, "data")
        self.kind = _KINDS[kind]
        if self.kind == TRIANGLE:
            n, dim = data.shape[0], 3
        elif self.kind == BOX:
            n, dim = data.shape[0], data.shape[1] // 2
        else:
            n, dim = data.shape[0], data.shape[1]
        self._data_keepalive = data
        prim = arbx_primitives(self.kind, dim, n, data.data_ptr() if n else None,
                               (QUANTIZED_NODES if quantized else 0) | (PARENT_RELATIVE if quantized == "parent" else 0)
                               | (WIDE_NODES if wide else 0))
        h = _P()
        self._stream = _stream(stream)
        self.device = data.device
        self._h = None
        _check(_lib.arbx_build(ctypes.byref(h), ctypes.byref(prim), self._stream), "arbx_build")
        self._h = h
        self._data_keepalive = None
        self.dim = dim
        self.n = n

    # ---- metadata (size(), empty(), bounds())
    def size(self) -> int:
        s = ctypes.c_int64(0)
        _check(_lib.arbx_tree_info(self._h, ctypes.byref(s), None, None), "arbx_tree_info")
        return s.value

    def empty(self) -> bool:
        return self.size() == 0

    def bounds(self) -> tuple[list[float], list[float]]:
        b = (ctypes.c_float * (2 * self.dim))()
        _check(_lib.arbx_tree_info(self._h, None, None, b), "arbx_tree_info")
        return list(b[:self.dim]), list(b[self.dim:])

    def close(self) -> None:
        if self._h:
            _lib.arbx_tree_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- predicates
    def _pred(self, kind: int, data: torch.Tensor, radius=None, k: int = 0, order=None):
        data = _dev_f32(data, "queries")
        m = data.shape[0]
        radii = None
        r = 0.0
        if kind == SPHERE:
            if isinstance(radius, torch.Tensor):
                radii = _dev_f32(radius, "radii")
                if radii.numel() != m:
                    raise ValueError("one radius per query")
            else:
                r = float(radius)
        cols = data.shape[1] if data.dim() > 1 else 0
        qdim = cols // 2 if kind == BOX_PRED else (3 if kind in RAY_KINDS and cols == 6 else
                                                   -1 if kind in RAY_KINDS else cols)
        if order is not None:
            if not isinstance(order, torch.Tensor) or not order.is_cuda or order.dtype not in (torch.int32,) \
                    or order.numel() != m:
                raise TypeError("order must be a CUDA int32 tensor of m entries (from query_order)")
            order = order.contiguous()
        p = arbx_predicates(kind, qdim, m, data.data_ptr() if m else None,
                            radii.data_ptr() if radii is not None else None, r, int(k),
                            order.data_ptr() if order is not None and m else None)
        return p, (data, radii, order)

    def query_order(self, kind: int, data: torch.Tensor, radius=None, k: int = 0, stream=None) -> torch.Tensor:
        """The Morton processing order of these predicates (arbx_query_order),
        as an int32 tensor of m entries holding uint32 indices; pass it as
        `order=` to later calls over the same queries to sort them once."""
        p, keep = self._pred(kind, data, radius, k)
        out = torch.empty(p.m, dtype=torch.int32, device=data.device)
        _check(_lib.arbx_query_order(self._h, ctypes.byref(p), out.data_ptr() if p.m else None, _stream(stream)),
               "arbx_query_order")
        del keep
        return out

    def query_crs(self, kind: int, data: torch.Tensor, radius=None, k: int = 0, want_d2: bool = True,
                  tuning=None, stream=None, order=None) -> LibraryCRS:
        """Storage query with library-allocated CRS buffers (arbx_query_crs)."""
        p, keep = self._pred(kind, data, radius, k, order)
        out = arbx_crs()
        st = _stream(stream)
        _check(_lib.arbx_query_crs(self._h, ctypes.byref(p), 1 if want_d2 else 0, _tuning(tuning),
                                   ctypes.byref(out), st), "arbx_query_crs")
        del keep
        return LibraryCRS(out, st, want_d2 and kind in (SPHERE, NEAREST, *RAY_KINDS))

    def query_crs_host(self, kind: int, data: torch.Tensor, radius=None, want_d2: bool = True, tuning=None,
                       chunk_bytes: int = 0, stream=None):
        """Storage query with the results in host memory, filled in query
        ranges that fit the device (arbx_query_crs_host): numpy (offsets
        int64[m+1], indices int32[nnz], d2 float32[nnz] or None)."""
        import numpy as np
        p, keep = self._pred(kind, data, radius)
        off = np.empty(p.m + 1, np.int64)
        nnz = ctypes.c_int64(0)
        st = _stream(stream)
        status = _lib.arbx_query_crs_host(self._h, ctypes.byref(p), 1 if want_d2 else 0, _tuning(tuning),
                                          off.ctypes.data, None, None, 0, int(chunk_bytes), ctypes.byref(nnz), st)
        if status not in (OK, ERR_CAPACITY):
            _check(status, "arbx_query_crs_host")
        idx = np.empty(nnz.value, np.int32)
        d2 = np.empty(nnz.value, np.float32) if want_d2 and kind in (SPHERE, RAY_INTERSECT, RAY_ORDERED) else None
        if nnz.value > 0:
            _check(_lib.arbx_query_crs_host(self._h, ctypes.byref(p), 1 if want_d2 else 0, _tuning(tuning),
                                            off.ctypes.data, idx.ctypes.data, None if d2 is None else d2.ctypes.data,
                                            nnz.value, int(chunk_bytes), None, st), "arbx_query_crs_host")
        del keep
        return off, idx, d2

    def radius(self, queries: torch.Tensor, radius, want_d2: bool = True, tuning=None, stream=None, order=None):
        """All primitives within `radius` (inclusive) of each query: (offsets
        int64[m+1], indices int32[nnz], d2 float32[nnz] or None), each
        segment in left-to-right leaf order."""
        crs = self.query_crs(SPHERE, queries, radius, want_d2=want_d2, tuning=tuning, stream=stream, order=order)
        return crs.offsets, crs.indices, crs.d2

    def box(self, boxes: torch.Tensor, tuning=None, stream=None):
        """All primitives whose bounding box overlaps each query box: (offsets, indices)."""
        crs = self.query_crs(BOX_PRED, boxes, want_d2=False, tuning=tuning, stream=stream)
        return crs.offsets, crs.indices

    def knn(self, queries: torch.Tensor, k: int, want_d2: bool = True, tuning=None, stream=None, order=None):
        """The min(k, n) nearest primitives of each query, ascending by (d2,
        index): (indices int32[m, kk], d2 float32[m, kk] or None)."""
        p, keep = self._pred(NEAREST, queries, k=k, order=order)
        kk = min(int(k), self.n)
        dev = queries.device
        idx = torch.empty((p.m, kk), dtype=torch.int32, device=dev)
        d2 = torch.empty((p.m, kk), dtype=torch.float32, device=dev) if want_d2 else None
        _check(_lib.arbx_query_knn(self._h, ctypes.byref(p), _tuning(tuning), idx.data_ptr() if idx.numel() else None,
                                   d2.data_ptr() if d2 is not None and d2.numel() else None, _stream(stream)),
               "arbx_query_knn")
        del keep
        return idx, d2

    def ray_nearest(self, rays: torch.Tensor, k: int = 1, tuning=None, stream=None):
        """First k triangle hits of each ray (origin, direction), ascending by
        (t, index): k == 1 gives (hit int32[m], t float32[m]); k > 1 gives
        [m, k] arrays; -1 / +inf past the last hit."""
        p, keep = self._pred(RAY_NEAREST, rays, k=k)
        kk = max(1, int(k))
        shape = (p.m,) if k <= 1 else (p.m, kk)
        hit = torch.empty(shape, dtype=torch.int32, device=rays.device)
        t = torch.empty(shape, dtype=torch.float32, device=rays.device)
        _check(_lib.arbx_query_ray_nearest(self._h, ctypes.byref(p), _tuning(tuning),
                                           hit.data_ptr() if p.m else None, t.data_ptr() if p.m else None,
                                           _stream(stream)), "arbx_query_ray_nearest")
        del keep
        return hit, t

    def ray_intersect(self, rays: torch.Tensor, ordered: bool = False, want_t: bool = True, tuning=None,
                      stream=None):
        """Every triangle hit of each ray: (offsets int64[m+1], indices int32[nnz],
        t float32[nnz] or None); in leaf order, or ascending by (t, index) when
        `ordered` (ordered_intersect)."""
        crs = self.query_crs(RAY_ORDERED if ordered else RAY_INTERSECT, rays, want_d2=want_t, tuning=tuning,
                             stream=stream)
        return crs.offsets, crs.indices, crs.d2

    def callback(self, kind: int, data: torch.Tensor, cb: int, radius=None, limit: int = 0, tuning=None,
                 stream=None, order=None) -> torch.Tensor:
        """Pure-callback query (arbx_query_callback): int32[m] per-query results."""
        p, keep = self._pred(kind, data, radius, order=order)
        out = torch.empty(p.m, dtype=torch.int32, device=data.device)
        _check(_lib.arbx_query_callback(self._h, ctypes.byref(p), cb, int(limit), out.data_ptr() if p.m else None,
                                        _tuning(tuning), _stream(stream)), "arbx_query_callback")
        del keep
        return out

    def count(self, queries: torch.Tensor, radius, tuning=None, stream=None) -> torch.Tensor:
        return self.callback(SPHERE, queries, CB_COUNT, radius, tuning=tuning, stream=stream)

    def count_up_to(self, queries: torch.Tensor, radius, limit: int, tuning=None, stream=None) -> torch.Tensor:
        return self.callback(SPHERE, queries, CB_COUNT_UP_TO, radius, limit, tuning=tuning, stream=stream)

    def first_hit(self, queries: torch.Tensor, radius, tuning=None, stream=None) -> torch.Tensor:
        return self.callback(SPHERE, queries, CB_FIRST_HIT, radius, tuning=tuning, stream=stream)

    def offsets_fill(self, kind: int, data: torch.Tensor, radius=None, want_d2: bool = True, tuning=None,
                     stream=None):
        """Two-phase storage query into torch-allocated buffers
        (arbx_query_offsets then arbx_query_fill)."""
        p, keep = self._pred(kind, data, radius)
        st = _stream(stream)
        off = torch.empty(p.m + 1, dtype=torch.int64, device=data.device)
        _check(_lib.arbx_query_offsets(self._h, ctypes.byref(p), _tuning(tuning), off.data_ptr(), st),
               "arbx_query_offsets")
        nnz = int(off[-1].item())
        idx = torch.empty(nnz, dtype=torch.int32, device=data.device)
        d2 = (torch.empty(nnz, dtype=torch.float32, device=data.device)
              if want_d2 and kind in (SPHERE, RAY_INTERSECT, RAY_ORDERED) else None)
        _check(_lib.arbx_query_fill(self._h, ctypes.byref(p), _tuning(tuning), off.data_ptr(),
                                    idx.data_ptr() if nnz else None,
                                    d2.data_ptr() if d2 is not None and nnz else None, st), "arbx_query_fill")
        del keep
        return off, idx, d2

    def stats(self, kind: int, data: torch.Tensor, radius=None, k: int = 0, tuning=None, stream=None,
              counting: bool = False) -> dict:
        """Instrumented traversal (arbx_query_stats): totals over all queries of
        node records fetched, leaf records fetched and matches.  counting=True
        (arbx_query_count_stats): the counting traversal of a spatial predicate."""
        p, keep = self._pred(kind, data, radius, k)
        out = (ctypes.c_int64 * 3)()
        fn, name = ((_lib.arbx_query_count_stats, "arbx_query_count_stats") if counting
                    else (_lib.arbx_query_stats, "arbx_query_stats"))
        _check(fn(self._h, ctypes.byref(p), _tuning(tuning), out, _stream(stream)), name)
        del keep
        return {"nodes": int(out[0]), "leaves": int(out[1]), "matches": int(out[2]), "queries": int(p.m)}

    def stats_r2(self, queries: torch.Tensor, r2: torch.Tensor, stream=None, tuning=None) -> dict:
        """Visit counters of the sphere walk with per-query squared radii r2
        used as given (arbx_query_stats_r2): with the final k-th squared
        distances of a nearest query, the nodes any exact best-first search
        opens."""
        p, keep = self._pred(SPHERE, queries, 0.0)
        r2 = _dev_f32(r2, "r2")
        if r2.numel() != p.m:
            raise ValueError("one squared radius per query")
        out = (ctypes.c_int64 * 3)()
        _check(_lib.arbx_query_stats_r2(self._h, ctypes.byref(p), _tuning(tuning), r2.data_ptr() if p.m else None,
                                        out, _stream(stream)), "arbx_query_stats_r2")
        del keep
        return {"nodes": int(out[0]), "leaves": int(out[1]), "matches": int(out[2]), "queries": int(p.m)}

    def autotune(self, kind: int, data: torch.Tensor, radius=None, k: int = 0, sample: int = 0,
                 stream=None) -> tuple[dict, float]:
        """Time the candidate launch settings on (a sample of) these predicates
        and record the fastest for later calls given no tuning
        (arbx_autotune): (setting as a tuning dict, its time in ms)."""
        p, keep = self._pred(kind, data, radius, k)
        best = arbx_tuning()
        ms = ctypes.c_double(0.0)
        _check(_lib.arbx_autotune(self._h, ctypes.byref(p), int(sample), ctypes.byref(best), ctypes.byref(ms),
                                  _stream(stream)), "arbx_autotune")
        del keep
        return ({"block": best.block, "sort_queries": best.sort_queries, "top_levels": best.top_levels,
                 "grid_per_sm": best.grid_per_sm, "warp_refill": best.warp_refill, "stackless": best.stackless,
                 "single_pass": best.single_pass, "lanes_per_query": best.lanes_per_query,
                 "wide_nodes": best.wide_nodes, "warp_packets": best.warp_packets, "query_runs": best.query_runs},
                ms.value)

    def layout(self) -> dict:
        """Sizes of the internal arrays: {'node_bytes', 'leaf_bytes',
        'node_stride', 'leaf_stride', 'root'} (no copy)."""
        b = (ctypes.c_int64 * 5)()
        _check(_lib.arbx_tree_export(self._h, None, 0, None, 0, b), "arbx_tree_export")
        return {"node_bytes": int(b[0]), "leaf_bytes": int(b[1]), "node_stride": int(b[2]),
                "leaf_stride": int(b[3]), "root": int(b[4])}

    def export(self) -> dict:
        """Host copies of the internal arrays: {'nodes': uint8, 'leaves': uint8,
        'node_stride', 'leaf_stride', 'root'}."""
        import numpy as np
        b = (ctypes.c_int64 * 5)()
        _check(_lib.arbx_tree_export(self._h, None, 0, None, 0, b), "arbx_tree_export")
        nodes = np.empty(b[0], np.uint8)
        leaves = np.empty(b[1], np.uint8)
        _check(_lib.arbx_tree_export(self._h, nodes.ctypes.data if b[0] else None, b[0],
                                     leaves.ctypes.data if b[1] else None, b[1], None), "arbx_tree_export")
        return {"nodes": nodes, "leaves": leaves, "node_stride": int(b[2]), "leaf_stride": int(b[3]),
                "root": int(b[4])}


def _ptr(t):
    return t.data_ptr() if t is not None and t.numel() else None


class Forest:
    """Many independent point sets, one BVH each, built together
    (arbx_forest_build).  sets: CUDA float32 tensors of shape (n_s, d_s) with
    d_s in {2, 3, 6}; results use set-local indices."""

    def __init__(self, sets: list | None = None, stream=None, packed=None, dims=None, counts=None):
        """Either `sets`, or `packed` (one CUDA float32 tensor holding the sets
        one after another) with `dims` and `counts` per set."""
        import numpy as np
        if sets is not None:
            self.dims = np.array([int(s.shape[1]) for s in sets], np.int32)
            self.counts = np.array([int(s.shape[0]) for s in sets], np.int64)
            packed = torch.cat([_dev_f32(s, "set").reshape(-1) for s in sets]) if sets else None
        else:
            self.dims = np.ascontiguousarray(dims, np.int32)
            self.counts = np.ascontiguousarray(counts, np.int64)
            packed = _dev_f32(packed, "packed")
        nsets = len(self.dims)
        h = _P()
        self._h = None
        _check(_lib.arbx_forest_build(ctypes.byref(h), nsets, self.dims.ctypes.data, self.counts.ctypes.data,
                                      _ptr(packed), _stream(stream)), "arbx_forest_build")
        self._h = h

    def info(self) -> tuple[int, int]:
        ns, npts = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(_lib.arbx_forest_info(self._h, ctypes.byref(ns), ctypes.byref(npts)), "arbx_forest_info")
        return ns.value, npts.value

    def close(self):
        if self._h:
            _lib.arbx_forest_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ForestBatch:
    """Query layout of a forest (arbx_forest_batch_create): qcounts[s] queries
    for set s, packed set after set; radii[s] per set (or None)."""

    def __init__(self, forest: Forest, qcounts, radii=None, stream=None):
        import numpy as np
        self.forest = forest
        self.qcounts = np.ascontiguousarray(qcounts, np.int64)
        r = None if radii is None else np.ascontiguousarray(radii, np.float32)
        h = _P()
        self._h = None
        _check(_lib.arbx_forest_batch_create(ctypes.byref(h), forest._h, self.qcounts.ctypes.data,
                                             None if r is None else r.ctypes.data, _stream(stream)),
               "arbx_forest_batch_create")
        self._h = h
        t = ctypes.c_int64(0)
        _check(_lib.arbx_forest_batch_total(self._h, ctypes.byref(t)), "arbx_forest_batch_total")
        self.total = t.value

    def radius_into(self, queries, offsets, indices, d2, capacity: int, nnz, stream=None):
        _check(_lib.arbx_forest_query_radius(self._h, _ptr(queries), offsets.data_ptr(), _ptr(indices), _ptr(d2),
                                             int(capacity), _ptr(nnz), _stream(stream)), "arbx_forest_query_radius")

    def radius(self, queries: torch.Tensor, stream=None):
        """(offsets int64[M+1], indices int32[nnz], d2 float32[nnz]) over all
        sets' queries in packed order: a count pass sizes the output, then the
        full query fills it."""
        dev = queries.device
        off = torch.empty(self.total + 1, dtype=torch.int64, device=dev)
        self.radius_into(queries, off, None, None, 0, None, stream)
        nnz = int(off[-1].item())
        idx = torch.empty(nnz, dtype=torch.int32, device=dev)
        d2 = torch.empty(nnz, dtype=torch.float32, device=dev)
        self.radius_into(queries, off, idx, d2, nnz, None, stream)
        return off, idx, d2

    def knn(self, queries: torch.Tensor, k: int, stream=None):
        dev = queries.device
        idx = torch.empty((self.total, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((self.total, k), dtype=torch.float32, device=dev)
        _check(_lib.arbx_forest_query_knn(self._h, _ptr(queries), int(k), _ptr(idx), _ptr(d2), _stream(stream)),
               "arbx_forest_query_knn")
        return idx, d2

    def set_tuning(self, tuning: dict | None) -> None:
        """Launch settings of the batch's query kernels
        (arbx_forest_batch_set_tuning): {'block', 'chunk', 'sort_queries':
        [dims 2, 3, 6]}; None restores the defaults."""
        if tuning is None:
            _check(_lib.arbx_forest_batch_set_tuning(self._h, None), "arbx_forest_batch_set_tuning")
            return
        t = arbx_forest_tuning(int(tuning.get("block", 0)), int(tuning.get("chunk", 0)),
                               (ctypes.c_int32 * 3)(*tuning.get("sort_queries", [-1, -1, -1])))
        _check(_lib.arbx_forest_batch_set_tuning(self._h, ctypes.byref(t)), "arbx_forest_batch_set_tuning")

    def tuning(self) -> dict:
        t = arbx_forest_tuning()
        _check(_lib.arbx_forest_batch_get_tuning(self._h, ctypes.byref(t)), "arbx_forest_batch_get_tuning")
        return {"block": t.block, "chunk": t.chunk, "sort_queries": list(t.sort_queries)}

    def autotune(self, queries: torch.Tensor, k: int, stream=None) -> tuple[dict, float]:
        """Search the batch's launch settings on its queries (arbx_forest_autotune):
        (the chosen setting, now the batch's, and its time in ms)."""
        t = arbx_forest_tuning()
        ms = ctypes.c_double(0.0)
        _check(_lib.arbx_forest_autotune(self._h, _ptr(queries), int(k), ctypes.byref(t), ctypes.byref(ms),
                                         _stream(stream)), "arbx_forest_autotune")
        return {"block": t.block, "chunk": t.chunk, "sort_queries": list(t.sort_queries)}, ms.value

    def graph(self, queries, offsets, indices, d2, capacity, nnz, k, knn_idx, knn_d2, stream) -> "Graph":
        """Capture radius (count, scan, fill) + kNN into one CUDA graph on `stream`."""
        h = _P()
        _check(_lib.arbx_forest_graph_create(ctypes.byref(h), self._h, _ptr(queries), offsets.data_ptr(),
                                             _ptr(indices), _ptr(d2), int(capacity), _ptr(nnz), int(k),
                                             _ptr(knn_idx), _ptr(knn_d2), _stream(stream)),
               "arbx_forest_graph_create")
        return Graph(h)

    def close(self):
        if self._h:
            _lib.arbx_forest_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, h):
        self._h = h

    def launch(self, stream=None):
        _check(_lib.arbx_graph_launch(self._h, _stream(stream)), "arbx_graph_launch")

    def close(self):
        if self._h:
            _lib.arbx_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class arbx_request(ctypes.Structure):
    _fields_ = [("tree_id", ctypes.c_int32), ("kind", ctypes.c_int32), ("callback", ctypes.c_int32),
                ("limit", ctypes.c_int32), ("k", ctypes.c_int32), ("radius", ctypes.c_float),
                ("m", ctypes.c_int64), ("queries_dev", ctypes.c_void_p), ("arrival_s", ctypes.c_double)]


class arbx_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("offsets_dev", ctypes.c_void_p), ("indices_dev", ctypes.c_void_p), ("d2_dev", ctypes.c_void_p),
                ("counts_dev", ctypes.c_void_p), ("latency_s", ctypes.c_double)]


_SIGS2 = {
    "arbx_server_create": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64], _S),
    "arbx_server_add_tree": ([_P, _P, ctypes.POINTER(ctypes.c_int32)], _S),
    "arbx_server_now": ([_P], ctypes.c_double),
    "arbx_server_submit": ([_P, ctypes.POINTER(arbx_request), ctypes.POINTER(ctypes.c_uint64)], _S),
    "arbx_server_wait": ([_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(arbx_result)], _S),
    "arbx_server_release": ([_P, ctypes.POINTER(arbx_result)], _S),
    "arbx_server_stats": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)], _S),
    "arbx_server_reset_stats": ([_P], _S),
    "arbx_server_destroy": ([_P], _S),
}
for _name, (_args, _res) in _SIGS2.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
_SIGS.update(_SIGS2)


class _ResultOwner:
    """Owns the device buffers of one served result (no reference back to
    the views, so they are released as soon as the last view goes)."""

    def __init__(self, server: "Server", res: arbx_result):
        self.server = server
        self.res = res

    def __del__(self):
        try:
            if self.server._h:
                _lib.arbx_server_release(self.server._h, ctypes.byref(self.res))
        except Exception:
            pass


class ServerResult:
    """Result of one served request; its device buffers are released when
    this object and every tensor view of it are gone."""

    def __init__(self, server: "Server", res: arbx_result):
        self._owner = owner = _ResultOwner(server, res)
        self.latency_s = res.latency_s
        self.m, self.nnz = res.m, res.nnz
        dev = torch.device("cuda", torch.cuda.current_device())

        def view(ptr, n, typestr, dtype):
            if not ptr or n == 0:
                return torch.empty(0, dtype=dtype, device=dev)
            return torch.as_tensor(_LibBuffer(owner, ptr, n, typestr), device=dev)

        self.offsets = view(res.offsets_dev, res.m + 1, "<i8", torch.int64) if res.offsets_dev else None
        self.indices = view(res.indices_dev, res.nnz, "<i4", torch.int32) if res.offsets_dev else None
        self.d2 = view(res.d2_dev, res.nnz, "<f4", torch.float32) if res.d2_dev else None
        self.counts = view(res.counts_dev, res.m, "<i4", torch.int32) if res.counts_dev else None


class Server:
    """Serving runtime (arbx_server_*): resident trees, `slots` concurrent
    request slots, admission by a device-memory budget."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 64 << 30):
        h = _P()
        self._h = None
        _check(_lib.arbx_server_create(ctypes.byref(h), int(slots), int(hbm_budget_bytes)), "arbx_server_create")
        self._h = h
        self._keep = {}

    def add_tree(self, tree: Tree) -> int:
        tid = ctypes.c_int32(0)
        _check(_lib.arbx_server_add_tree(self._h, tree._h, ctypes.byref(tid)), "arbx_server_add_tree")
        tree._h = None  # owned by the server now
        return tid.value

    def now(self) -> float:
        return _lib.arbx_server_now(self._h)

    def submit(self, tree_id: int, kind: int, queries: torch.Tensor, radius: float = 0.0, k: int = 0,
               callback: int = -1, limit: int = 0, arrival_s: float = -1.0) -> int:
        q = _dev_f32(queries, "queries")
        req = arbx_request(int(tree_id), int(kind), int(callback), int(limit), int(k), float(radius),
                           q.shape[0], q.data_ptr() if q.shape[0] else None, float(arrival_s))
        t = ctypes.c_uint64(0)
        _check(_lib.arbx_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "arbx_server_submit")
        self._keep[t.value] = q  # the queries must outlive the request
        return t.value

    def wait(self, ticket: int, timeout_s: float | None = None) -> ServerResult:
        res = arbx_result()
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = _lib.arbx_server_wait(self._h, ticket, us, ctypes.byref(res))
        if st == ERR_TIMEOUT and not res.offsets_dev and not res.counts_dev:
            raise ArbxError(st, "arbx_server_wait")
        self._keep.pop(ticket, None)
        out = ServerResult(self, res)
        _check(st, "arbx_server_wait")
        return out

    def stats(self) -> dict:
        p50, p99, mq = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(_lib.arbx_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(mq),
                                      ctypes.byref(n)), "arbx_server_stats")
        return {"p50_s": p50.value, "p99_s": p99.value, "mqps": mq.value, "completed": n.value}

    def reset_stats(self) -> None:
        _check(_lib.arbx_server_reset_stats(self._h), "arbx_server_reset_stats")

    def close(self):
        if self._h:
            _lib.arbx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exported_symbols() -> list[str]:
    return sorted(_SIGS)
