"""FP64 CPU oracle for the Voronoi pipeline -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package. The product path (the
``paper_2412_04514_gb300`` package and its CUDA library) never imports, links
or runs it, and this package imports nothing from the product.

Contents
--------
* :func:`grid_sort` -- the grid counting sort written out in NumPy (paper,
  Summary: the generators are first binned into a uniform grid).
* :func:`morisita_index` -- the clustering statistic the autotuner keys on:
  the Morisita index of the generators on that grid.
* :func:`knn` -- exact k nearest neighbours (C kd-tree), ordered by
  ``(d2, index)`` with ``d2`` in double from the float32 inputs.
* :func:`tessellate` -- Voronoi cells by nearest-first bisector clipping of
  the box with the security-radius stop and k doubling (paper, Summary), or
  by clipping with every generator (``mode="brute"``) for the pins.
* :func:`knn_periodic` / ``tessellate(..., periodic=True)`` -- the same in a
  periodic box: every generator repeats at p + t (hi - lo), each cell starts
  as the cube of one period around its generator (the Voronoi definition of
  the Statement of need applied to all images).
* :func:`moments_adjoint` -- gradients of cell volume, first moment and
  second moment with respect to the generators, from face integrals.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines (SciPy's Qhull and periodic kd-tree),
brute force and invariants; the periodic mode also against the non-periodic
oracle on replicated clouds. None is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvto.so")
_SOURCES = [os.path.join(_HERE, "vt_oracle.c")]
_lock = threading.Lock()
_lib = None

VTO_OK, VTO_ERR_ARG, VTO_ERR_DUPLICATE, VTO_ERR_CAPACITY = 0, 1, 2, 3
MODE_SECURITY, MODE_BRUTE = 0, 1


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build/libvto.so``.

    ``-ffp-contract=off`` keeps every double operation separately rounded
    (no fused multiply-add), so x86-64 and aarch64 hosts agree bit for bit.
    """
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in _SOURCES if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "vt_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp",
           "-shared", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Result(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int64),
        ("status", ctypes.c_int),
        ("vol", ctypes.POINTER(ctypes.c_double)),
        ("cen", ctypes.POINTER(ctypes.c_double)),
        ("m2", ctypes.POINTER(ctypes.c_double)),
        ("nbr_off", ctypes.POINTER(ctypes.c_int64)),
        ("nbr", ctypes.POINTER(ctypes.c_int32)),
        ("n_nbr", ctypes.c_int64),
        ("k_used", ctypes.POINTER(ctypes.c_int32)),
        ("n_clips", ctypes.POINTER(ctypes.c_int32)),
        ("euler", ctypes.POINTER(ctypes.c_int32)),
        ("nvert", ctypes.POINTER(ctypes.c_int32)),
        ("face_off", ctypes.POINTER(ctypes.c_int64)),
        ("face_tag", ctypes.POINTER(ctypes.c_int32)),
        ("face_area", ctypes.POINTER(ctypes.c_double)),
        ("face_cen", ctypes.POINTER(ctypes.c_double)),
        ("face_plane", ctypes.POINTER(ctypes.c_double)),
        ("face_size", ctypes.POINTER(ctypes.c_int32)),
        ("face_vtx", ctypes.POINTER(ctypes.c_double)),
        ("n_faces", ctypes.c_int64),
        ("n_face_vtx", ctypes.c_int64),
        ("work_sign", ctypes.POINTER(ctypes.c_int64)),
        ("work_newv", ctypes.POINTER(ctypes.c_int64)),
        ("work_nbrs", ctypes.POINTER(ctypes.c_int64)),
        ("face_img", ctypes.POINTER(ctypes.c_int32)),
        ("periodic", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.vto_knn.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, P, P, ctypes.c_int]
            lib.vto_knn.restype = ctypes.c_int
            lib.vto_tessellate.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, P, P,
                                           ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.POINTER(_Result))]
            lib.vto_tessellate.restype = ctypes.c_int
            lib.vto_tessellate_periodic.argtypes = lib.vto_tessellate.argtypes
            lib.vto_tessellate_periodic.restype = ctypes.c_int
            lib.vto_knn_periodic.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int64, ctypes.c_int, P, P, P,
                                             ctypes.c_int]
            lib.vto_knn_periodic.restype = ctypes.c_int
            lib.vto_result_free.argtypes = [ctypes.POINTER(_Result)]
            lib.vto_result_free.restype = None
            if hasattr(lib, "vto_moments_adjoint"):
                lib.vto_moments_adjoint.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int, P, P, P, P, ctypes.c_int]
                lib.vto_moments_adjoint.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pts(points) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("points must be float32[n, 3]")
    return p


def _arr(ptr, n, dtype, shape=None):
    if n == 0 or not ptr:
        out = np.zeros(0 if shape is None else (0,) + tuple(shape[1:]), dtype=dtype)
        return out
    a = np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------------------
# grid counting sort (paper, Summary: points are sorted into a grid)
# ---------------------------------------------------------------------------

def grid_cell_ids(points, G: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Grid cell of each point, ``cid = (ix*G + iy)*G + iz`` (z fastest).

    ``ix = min(G-1, floor((x - lo) * s))`` with ``s = float32(G) / (hi - lo)``,
    every operation a separately rounded float32 operation (the grid is a
    float32 construct: it only needs to be consistent, not exact).
    """
    p = _pts(points)
    lo32 = np.asarray(lo, dtype=np.float32)
    hi32 = np.asarray(hi, dtype=np.float32)
    scale = (np.float32(G) / (hi32 - lo32)).astype(np.float32)
    t = ((p - lo32).astype(np.float32) * scale).astype(np.float32)
    ijk = np.clip(np.floor(t).astype(np.int64), 0, G - 1)
    return ((ijk[:, 0] * G + ijk[:, 1]) * G + ijk[:, 2]).astype(np.int64)


def grid_sort(points, G: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> dict:
    """Stable counting sort of the points by grid cell.

    Returns ``cid`` (per input point), ``cell_off`` (``int64[G^3 + 1]``,
    exclusive prefix sum of the per-cell counts), ``perm`` (sorted position ->
    input index; stable, i.e. input order within a cell) and ``sorted``
    (``float32[n, 3]`` points in sorted order).
    """
    p = _pts(points)
    cid = grid_cell_ids(p, G, lo, hi)
    counts = np.bincount(cid, minlength=G**3)
    off = np.zeros(G**3 + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    perm = np.argsort(cid, kind="stable")
    return {"cid": cid, "cell_off": off, "perm": perm.astype(np.int64), "sorted": p[perm]}


def morisita_index(points, G: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> float:
    """Morisita's index of dispersion of the points over the G^3 grid cells:
    I = Q * sum_c n_c (n_c - 1) / (n (n - 1)) with Q = G^3 cells holding n_c
    points each (Morisita 1959). It is the ratio of the observed probability
    that two distinct points share a cell to the one under a uniform
    distribution: 1 in expectation for i.i.d. uniform points, 0 when no cell
    holds two points, Q when all points share one cell. 0 for n < 2."""
    p = _pts(points)
    n = len(p)
    if n < 2:
        return 0.0
    counts = np.bincount(grid_cell_ids(p, G, lo, hi), minlength=G**3).astype(np.int64)
    pairs = int(np.sum(counts * (counts - 1)))
    return float(G**3) * float(pairs) / (float(n) * (float(n) - 1.0))


def grid_resolution(n: int, rho: float) -> int:
    """``G = max(1, ceil(cbrt(n / rho)))``: about ``rho`` points per grid cell."""
    if n <= 0:
        return 1
    g = int(np.ceil(np.cbrt(n / rho) - 1e-9))
    return max(1, g)


# ---------------------------------------------------------------------------
# kNN and tessellation
# ---------------------------------------------------------------------------

def knn(points, k: int, queries=None, threads: int | None = None):
    """Exact k nearest neighbours of ``queries`` (default all points), self excluded.

    Returns ``(nbr int32[q, k], d2 float64[q, k])`` ordered by ``(d2, index)``
    with ``d2 = ((dx*dx + dy*dy) + dz*dz)`` in double, ``dx = double(x_j) -
    double(x_i)``. Slots beyond ``n - 1`` neighbours hold -1 / inf.
    """
    p = _pts(points)
    n = len(p)
    q = np.arange(n, dtype=np.int64) if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nbr = np.empty((len(q), k), dtype=np.int32)
    d2 = np.empty((len(q), k), dtype=np.float64)
    st = _load().vto_knn(_ptr(p), n, _ptr(q), len(q), k, _ptr(nbr), _ptr(d2), threads or default_threads())
    if st != VTO_OK:
        raise OracleError(f"vto_knn failed with status {st}")
    return nbr, d2


def img_shift(code):
    """Image shift t [..., 3] (integers in [-2, 2]) of shift codes (tx+2)*25 + (ty+2)*5 + (tz+2)."""
    c = np.asarray(code, dtype=np.int64)
    return np.stack([c // 25 - 2, (c // 5) % 5 - 2, c % 5 - 2], axis=-1)


def img_code(t):
    """Shift code of image shifts t [..., 3]."""
    t = np.asarray(t, dtype=np.int64)
    return (t[..., 0] + 2) * 25 + (t[..., 1] + 2) * 5 + (t[..., 2] + 2)


def knn_periodic(points, k: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), queries=None, threads: int | None = None):
    """Exact k nearest images in the periodic box [lo, hi), own images excluded.

    Returns ``(nbr, img, d2)`` [q, k]: generator, shift code and key, ordered
    by ``(d2, generator, code)`` with ``d2`` from the offsets
    ``(x_j - x_i) + t L`` in double (L = hi - lo).
    """
    p = _pts(points)
    n = len(p)
    q = np.arange(n, dtype=np.int64) if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    lo32 = np.ascontiguousarray(lo, dtype=np.float32)
    hi32 = np.ascontiguousarray(hi, dtype=np.float32)
    nbr = np.empty((len(q), k), dtype=np.int32)
    img = np.empty((len(q), k), dtype=np.int32)
    d2 = np.empty((len(q), k), dtype=np.float64)
    st = _load().vto_knn_periodic(_ptr(p), n, _ptr(lo32), _ptr(hi32), _ptr(q), len(q), k, _ptr(nbr), _ptr(img),
                                  _ptr(d2), threads or default_threads())
    if st != VTO_OK:
        raise OracleError(f"vto_knn_periodic failed with status {st}")
    return nbr, img, d2


def tessellate(points, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), k0: int = 16, mode: str = "security",
               order=None, cells=None, geometry: bool = False, threads: int | None = None,
               periodic: bool = False) -> dict:
    """FP64 Voronoi cells of ``cells`` (default every generator) in the box ``[lo, hi)``.

    ``mode="security"``: k nearest neighbours nearest first with the
    security-radius stop, k doubling until the cell validates.
    ``mode="brute"``: clip by every other generator in index order, or in
    ``order`` (a permutation of all indices), with no stop test.

    Returns a dict of NumPy arrays: ``vol``, ``cen`` [c,3], ``m2``,
    ``nbr_off``/``nbr`` (CSR, neighbour indices ascending), ``k_used``,
    ``n_clips``, ``euler``, ``nvert``, ``face_off``/``face_tag``/``face_area``/
    ``face_cen``/``face_plane``/``face_size``/``face_img`` and, with
    ``geometry=True``, ``face_vtx`` (CCW loops seen from outside, global
    coordinates).

    ``periodic=True``: the box is periodic (every generator repeats at
    p + t (hi - lo)); each cell starts as the cube of one period around its
    generator and is cut by the images of the others. ``face_tag`` is then the
    generator of each face (the cell's own index for the cube's faces),
    ``face_img`` its image shift code, and ``nbr`` lists the generator of every
    face above the area threshold, repeats included. Requires
    ``|L|^2 <= 4 min L_a^2`` and ``n < 2^24``.
    """
    p = _pts(points)
    n = len(p)
    lo32 = np.ascontiguousarray(lo, dtype=np.float32)
    hi32 = np.ascontiguousarray(hi, dtype=np.float32)
    m = {"security": MODE_SECURITY, "brute": MODE_BRUTE}[mode]
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    c = None if cells is None else np.ascontiguousarray(cells, dtype=np.int64)
    res = ctypes.POINTER(_Result)()
    lib = _load()
    fn = lib.vto_tessellate_periodic if periodic else lib.vto_tessellate
    st = fn(_ptr(p), n, _ptr(lo32), _ptr(hi32), k0, m, _ptr(o), _ptr(c), 0 if c is None else len(c),
            int(geometry), threads or default_threads(), ctypes.byref(res))
    if not res:
        raise OracleError(f"vto_tessellate failed with status {st}")
    try:
        r = res.contents
        nc = r.n_cells
        nf = r.n_faces
        out = {
            "status": r.status,
            "vol": _arr(r.vol, nc, np.float64),
            "cen": _arr(r.cen, 3 * nc, np.float64, (nc, 3)),
            "m2": _arr(r.m2, nc, np.float64),
            "nbr_off": _arr(r.nbr_off, nc + 1, np.int64),
            "nbr": _arr(r.nbr, r.n_nbr, np.int32),
            "k_used": _arr(r.k_used, nc, np.int32),
            "n_clips": _arr(r.n_clips, nc, np.int32),
            "euler": _arr(r.euler, nc, np.int32),
            "nvert": _arr(r.nvert, nc, np.int32),
            "face_off": _arr(r.face_off, nc + 1, np.int64),
            "face_tag": _arr(r.face_tag, nf, np.int32),
            "face_area": _arr(r.face_area, nf, np.float64),
            "face_cen": _arr(r.face_cen, 3 * nf, np.float64, (nf, 3)),
            "face_plane": _arr(r.face_plane, 4 * nf, np.float64, (nf, 4)),
            "face_size": _arr(r.face_size, nf, np.int32),
            "face_img": _arr(r.face_img, nf, np.int32),
            "work_sign": _arr(r.work_sign, nc, np.int64),
            "work_newv": _arr(r.work_newv, nc, np.int64),
            "work_nbrs": _arr(r.work_nbrs, nc, np.int64),
        }
        if geometry:
            out["face_vtx"] = _arr(r.face_vtx, 3 * r.n_face_vtx, np.float64, (r.n_face_vtx, 3))
    finally:
        lib.vto_result_free(res)
    if st != VTO_OK:
        raise OracleError(f"vto_tessellate failed with status {st}")
    return out


# FP32 operations of one validated cell, an FMA counted as 2 (the clipper's
# minimal work: no re-queue repeats): per bisector tested, the plane and the
# security-radius test (12); per vertex-plane sign test, one 3-term dot product
# minus the offset (6); per vertex created, a 3x3 solve by Cramer's rule plus
# its squared radius (60); per final vertex, its three (vertex, face) moment
# terms (3 x 60).
FLOPS_PER_NBR, FLOPS_PER_SIGN, FLOPS_PER_NEWV, FLOPS_PER_FINAL_VERTEX = 12, 6, 60, 180


def clip_flops(res: dict) -> np.ndarray:
    """Algorithmic FP32 flops of each cell's validated clipping (see constants)."""
    return (FLOPS_PER_NBR * res["work_nbrs"] + FLOPS_PER_SIGN * res["work_sign"]
            + FLOPS_PER_NEWV * res["work_newv"] + FLOPS_PER_FINAL_VERTEX * res["nvert"].astype(np.int64))


def neighbour_lists(res: dict) -> list[np.ndarray]:
    """Per-cell neighbour arrays from a CSR result."""
    off, nbr = res["nbr_off"], res["nbr"]
    return [nbr[off[i]:off[i + 1]] for i in range(len(off) - 1)]
