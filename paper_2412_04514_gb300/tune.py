"""Binding of the autotuner (vt_autotune, vt_autotune_batch) and its JSON cache.

The timing itself runs in libvt.so (host code around CUDA events); this module
marshals arguments and keeps tuned parameters in a JSON file keyed by the
precision, the outputs, the size bucket ``round(log4 n)`` and the clustering
class of the input (Morisita index on the grid, see :func:`cluster_index`),
so that later runs of the same kind of input reuse them without timing.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import _lib as L
from .api import Batch, Params, Workspace, _alloc, _check_points, _out_struct, _ptr, _stream, batch_plan

_TUNED = ("threads_per_cell", "k0", "k_max", "grid_density")


def default_space(**over) -> dict:
    """The default search space as a dict (tpc, k0, kmax_mult, rho, reps)."""
    s = L.VtTuneSpace()
    L.load().vt_tune_space_default(ctypes.byref(s))
    d = {"tpc": list(s.tpc[: s.n_tpc]), "k0": list(s.k0[: s.n_k0]), "kmax_mult": list(s.kmax_mult[: s.n_kmax]),
         "rho": [float(x) for x in s.rho[: s.n_rho]], "reps": s.reps}
    d.update(over)
    return d


def _space(d: dict | None) -> L.VtTuneSpace:
    d = default_space(**(d or {}))
    s = L.VtTuneSpace()
    s.n_tpc = len(d["tpc"])
    s.n_k0 = len(d["k0"])
    s.n_kmax = len(d["kmax_mult"])
    s.n_rho = len(d["rho"])
    if s.n_tpc > 4 or s.n_k0 > 8 or s.n_kmax > 4 or s.n_rho > 8:
        raise ValueError("tune space too large (at most 4 tpc, 8 k0, 4 multiples, 8 densities)")
    for i, v in enumerate(d["tpc"]):
        s.tpc[i] = v
    for i, v in enumerate(d["k0"]):
        s.k0[i] = v
    for i, v in enumerate(d["kmax_mult"]):
        s.kmax_mult[i] = v
    for i, v in enumerate(d["rho"]):
        s.rho[i] = v
    s.reps = d["reps"]
    return s


def _report(r: L.VtTuneResult) -> dict:
    m = min(r.n_tried, L.VT_TUNE_MAX_TRIED)
    tried = [{"threads_per_cell": t.threads_per_cell, "k0": t.k0, "k_max": t.k_max, "cls": t.cls,
              "grid_density": round(float(t.grid_density), 6), "ms": t.ms, "status": L.STATUS_NAMES.get(t.status)}
             for t in r.tried[:m]]
    return {"best_ms": r.best_ms, "n_tried": r.n_tried, "tried": tried,
            "density_of_class": [round(float(x), 6) for x in r.density_of_class]}


def _with(params: Params, best: L.VtParams) -> Params:
    return Params(**{**params.__dict__, "threads_per_cell": best.threads_per_cell, "k0": best.k0,
                     "k_max": best.k_max, "grid_density": round(float(best.grid_density), 6), "grid_res": 0})


# ---------------------------------------------------------------------------
# clustering statistic
# ---------------------------------------------------------------------------

def cluster_index(points: torch.Tensor, params: Params | None = None, workspace: Workspace | None = None) -> float:
    """Morisita index of the points on the grid of ``params`` (vt_cluster_index)."""
    params = params or Params()
    pts = _check_points(points)
    n = pts.shape[0]
    ws = workspace if workspace is not None and workspace.fits(params, n) else Workspace(params, n, pts.device)
    out = (ctypes.c_double * 1)()
    L.check(L.load().vt_cluster_index(_ptr(pts), n, None, None, 1, 0, ctypes.byref(params.c()), out, _ptr(ws.buf),
                                      ws.buf.numel(), _stream(pts.device)))
    return float(out[0])


def batch_cluster_index(points: torch.Tensor, set_off, params: Params | None = None) -> np.ndarray:
    """Morisita index of every set of a batch, each on its own grid."""
    params = params or Params()
    pts = _check_points(points)
    off = [int(x) for x in set_off]
    ns = len(off) - 1
    plan, cells = batch_plan(off, params)
    dev = pts.device
    plan_d = torch.frombuffer(bytearray(bytes(plan)), dtype=torch.uint8).to(dev)
    off_d = torch.tensor(off, dtype=torch.int64, device=dev)
    b = ctypes.c_size_t()
    L.check(L.load().vt_batch_workspace_size(ctypes.byref(params.c()), pts.shape[0], cells, ctypes.byref(b)))
    ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
    out = (ctypes.c_double * ns)()
    L.check(L.load().vt_cluster_index(_ptr(pts), pts.shape[0], _ptr(plan_d), _ptr(off_d), ns, cells,
                                      ctypes.byref(params.c()), out, _ptr(ws), ws.numel(), _stream(dev)))
    return np.array(out[:], dtype=np.float64)


def cluster_class(index: float) -> int:
    return int(L.load().vt_cluster_class(float(index)))


def size_bucket(n: int) -> int:
    return int(round(math.log(max(n, 1), 4)))


# ---------------------------------------------------------------------------
# JSON cache
# ---------------------------------------------------------------------------

def cache_key(params: Params, n: int, cls: int) -> str:
    emit = "+".join(sorted(params.emit))
    flags = ("nosync" if params.no_sync else "sync") + ("+periodic" if params.periodic else "")
    return f"{params.precision}|{emit}|{flags}|n4^{size_bucket(n)}|c{cls}"


def _device_name(dev) -> str:
    try:
        return torch.cuda.get_device_name(dev)
    except Exception:  # pragma: no cover - no device
        return "unknown"


def load_cache(path: str) -> dict:
    if not path or not os.path.exists(path):
        return {"version": 1, "entries": {}}
    with open(path) as f:
        d = json.load(f)
    if d.get("version") != 1 or not isinstance(d.get("entries"), dict):
        raise ValueError(f"{path}: not a tuning cache of version 1")
    return d


def store_cache(path: str, d: dict) -> None:
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(path: str, params: Params, n: int, cls: int, device_name: str) -> Params | None:
    e = load_cache(path)["entries"].get(cache_key(params, n, cls))
    if not e or e.get("device") != device_name:
        return None
    return Params(**{**params.__dict__, **{k: e[k] for k in _TUNED}, "grid_res": 0})


# ---------------------------------------------------------------------------
# tuning
# ---------------------------------------------------------------------------

def autotune(points: torch.Tensor, params: Params | None = None, space: dict | None = None,
             cache: str | None = None, sample: int | None = None, seed: int = 0):
    """Fastest (threads_per_cell, k0, k_max, grid_density) for points like these.

    With ``cache`` the result is read from / written to that JSON file under
    the key of (precision, outputs, schedule, size bucket, clustering class).
    ``sample`` tunes on a seeded random subset of that many points (its size
    bucket then keys the cache). Returns (tuned Params, report dict)."""
    params = params or Params()
    pts = _check_points(points)
    if sample is not None and sample < pts.shape[0]:
        g = torch.Generator(device="cpu").manual_seed(seed)
        idx = torch.randperm(pts.shape[0], generator=g)[:sample].to(pts.device)
        pts = pts[idx].contiguous()
    n = pts.shape[0]
    dev = pts.device
    cls = cluster_class(cluster_index(pts, params))
    name = _device_name(dev)
    if cache:
        hit = lookup(cache, params, n, cls, name)
        if hit is not None:
            return hit, {"cached": True, "key": cache_key(params, n, cls), "cls": cls}
    sp = _space(space)
    pc = Params(**{**params.__dict__, "stage_times": False}).c()
    lib = L.load()
    b = ctypes.c_size_t()
    L.check(lib.vt_autotune_workspace_size(ctypes.byref(pc), ctypes.byref(sp), n, ctypes.byref(b)))
    ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
    cells = _alloc(params, n, dev, False)
    o = _out_struct(cells)
    r = L.VtTuneResult()
    L.check(lib.vt_autotune(_ptr(pts), n, ctypes.byref(pc), ctypes.byref(sp), ctypes.byref(o), ctypes.byref(r),
                            _ptr(ws), ws.numel(), _stream(dev)))
    tuned = _with(params, r.best)
    rep = {"cached": False, "key": cache_key(params, n, cls), "cls": cls, **_report(r)}
    if cache:
        d = load_cache(cache)
        d["entries"][rep["key"]] = {**{k: getattr(tuned, k) for k in _TUNED}, "ms": r.best_ms, "device": name,
                                    "n": n}
        store_cache(cache, d)
    return tuned, rep


def autotune_batch(points: torch.Tensor, set_off, params: Params | None = None, space: dict | None = None,
                   sample_sets: int | None = None, seed: int = 0):
    """Tunes a batch: grid density per clustering class of the sets, and k0,
    k_max, threads per cell for the whole batch, timed on the schedule the
    batch runs (no-sync). ``sample_sets`` tunes on that many seeded randomly
    chosen sets. Returns (Params, density per class, class of every set,
    report)."""
    params = Params(**{**(params or Params()).__dict__, "no_sync": True, "stage_times": False})
    pts = _check_points(points)
    dev = pts.device
    off = np.asarray([int(x) for x in set_off], dtype=np.int64)
    classes = np.array([cluster_class(x) for x in batch_cluster_index(pts, off, params)], dtype=np.int32)
    ns = len(off) - 1
    if sample_sets is not None and sample_sets < ns:
        pick = np.sort(np.random.default_rng(seed).choice(ns, sample_sets, replace=False))
        parts = [pts[off[s]:off[s + 1]] for s in pick]
        t_pts = torch.cat(parts).contiguous()
        t_off = np.zeros(len(pick) + 1, dtype=np.int64)
        t_off[1:] = np.cumsum([off[s + 1] - off[s] for s in pick])
        t_cls = classes[pick]
    else:
        t_pts, t_off, t_cls = pts, off, classes
    lib = L.load()
    sp = _space(space)
    pc = params.c()
    nt = len(t_off) - 1
    offs_h = (ctypes.c_int64 * len(t_off))(*t_off.tolist())
    cls_h = (ctypes.c_int * nt)(*t_cls.tolist())
    b = ctypes.c_size_t()
    L.check(lib.vt_autotune_batch_workspace_size(offs_h, nt, ctypes.byref(pc), ctypes.byref(sp), ctypes.byref(b)))
    ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
    off_d = torch.tensor(t_off, dtype=torch.int64, device=dev)
    plan_d = torch.empty(nt * ctypes.sizeof(L.VtSetDesc), dtype=torch.uint8, device=dev)
    n = t_pts.shape[0]
    cells = _alloc(params, n, dev, False)
    o = _out_struct(cells)
    r = L.VtTuneResult()
    L.check(lib.vt_autotune_batch(_ptr(t_pts), offs_h, _ptr(off_d), nt, cls_h, ctypes.byref(pc), ctypes.byref(sp),
                                  _ptr(plan_d), ctypes.byref(o), ctypes.byref(r), _ptr(ws), ws.numel(), _stream(dev)))
    del ws, cells
    tuned = _with(params, r.best)
    dens = [float(x) for x in r.density_of_class]
    return tuned, dens, classes, {"sets_timed": nt, **_report(r)}


def tuned_batch(points: torch.Tensor, set_off, params: Params | None = None, space: dict | None = None,
                sample_sets: int | None = None, seed: int = 0):
    """A :class:`Batch` with tuned parameters and per-set grid resolutions
    (each set's G from the density tuned for its clustering class)."""
    tuned, dens, classes, rep = autotune_batch(points, set_off, params, space, sample_sets, seed)
    lib = L.load()
    off = [int(x) for x in set_off]
    G = []
    for s in range(len(off) - 1):
        p = Params(**{**tuned.__dict__, "grid_density": dens[classes[s]], "grid_res": 0})
        G.append(int(lib.vt_grid_resolution(ctypes.byref(p.c()), off[s + 1] - off[s])))
    b = Batch(points, off, tuned, grid_res=G)
    b.tune_report = {**rep, "density_of_class": dens, "class_counts": np.bincount(classes, minlength=4).tolist()}
    return b
