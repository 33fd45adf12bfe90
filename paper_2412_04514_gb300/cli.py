"""numpy and command-line front-ends over the same C ABI.

The method is reachable three ways (Features section of the paper): the
library call, a Python wrapper taking and returning numpy arrays, and a
command-line program. Here the library call is ``vt_tessellate`` (through
:func:`.api.tessellate`), the numpy wrapper is :func:`tessellate_numpy` and
the command line is ``python -m paper_2412_04514_gb300``. Both front-ends
only convert arrays and files; every step of the tessellation runs in the
CUDA library, and neither has a CPU path.

Files: points are read from ``.npy`` (float array [n, 3]), ``.npz`` (array
``points``) or text (``.txt``/``.csv``/``.xyz``: three columns separated by
whitespace or commas, ``#`` comments). Cells are written to ``.npz`` (every
emitted array under its own name, plus ``points``) or to text (``.txt``: one
line per cell, the cell's neighbour ids in ascending order; with volumes
emitted the line starts with the volume).
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

_OUTPUTS = ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
            "face_vtx", "perm")


def read_points(path: str) -> np.ndarray:
    """Points [n, 3] as float32 from a .npy, .npz or text file."""
    low = path.lower()
    if low.endswith(".npy"):
        a = np.load(path)
    elif low.endswith(".npz"):
        with np.load(path) as z:
            if "points" not in z:
                raise ValueError(f"{path}: no array named 'points'")
            a = z["points"]
    else:
        with open(path) as f:
            rows = []
            for line in f:
                line = line.split("#", 1)[0].strip()
                if not line:
                    continue
                parts = line.replace(",", " ").split()
                if len(parts) != 3:
                    raise ValueError(f"{path}: expected 3 columns, got {len(parts)}: {line!r}")
                rows.append([float(x) for x in parts])
        a = np.asarray(rows, dtype=np.float64).reshape(-1, 3)
    a = np.asarray(a)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError(f"{path}: points must have shape (n, 3), got {a.shape}")
    if not np.issubdtype(a.dtype, np.floating):
        raise ValueError(f"{path}: points must be floating point, got {a.dtype}")
    return np.ascontiguousarray(a, dtype=np.float32)


def neighbour_lists(nbr_off: np.ndarray, nbr: np.ndarray) -> list:
    """The jagged neighbour array as one int32 array per cell."""
    off = np.asarray(nbr_off, dtype=np.int64)
    return np.split(np.asarray(nbr), off[1:-1]) if off.size > 1 else []


def write_cells(path: str, cells: dict, points: np.ndarray | None = None) -> None:
    """Write the numpy cells of :func:`tessellate_numpy` to .npz or text."""
    if path.lower().endswith(".npz"):
        arrays = {k: v for k, v in cells.items() if isinstance(v, np.ndarray)}
        if points is not None:
            arrays["points"] = points
        np.savez(path, **arrays)
        return
    if cells.get("nbr") is None:
        raise ValueError("text output lists the neighbours: emit must include 'nbr'")
    vol = cells.get("vol")
    with open(path, "w") as f:
        for i, row in enumerate(neighbour_lists(cells["nbr_off"], cells["nbr"])):
            ids = " ".join(str(int(x)) for x in row)
            f.write(f"{vol[i]:.17g} {ids}\n" if vol is not None else ids + "\n")


def make_params(precision="fp32", emit=("nbr", "vol", "cen"), k0=16, k_max=32, grid_density=2.0, grid_res=0,
                threads_per_cell=0, index_space="original", box=None, periodic=False, fused=False):
    """:class:`.api.Params` from plain values (``box`` = (lo[3], hi[3]))."""
    from .api import Params

    p = Params(precision=precision, emit=tuple(emit), k0=k0, k_max=k_max, grid_density=grid_density,
               grid_res=grid_res, threads_per_cell=threads_per_cell, index_space=index_space, periodic=periodic,
               fused=fused)
    if box is not None:
        lo, hi = box
        p.box_lo, p.box_hi = tuple(float(x) for x in lo), tuple(float(x) for x in hi)
    return p


def tessellate_numpy(points, params=None, device="cuda", tune: bool = False, tune_cache: str | None = None,
                     **kw) -> dict:
    """Voronoi cells of a numpy array of points [n, 3].

    ``params`` is an :class:`.api.Params`; otherwise the keyword arguments of
    :func:`make_params` build one. The points are converted to float32 (the
    method's input type), copied to ``device``, tessellated there and every
    output comes back as a numpy array in a dict (keys as in
    :class:`.api.Cells`, plus ``stats``). ``tune=True`` first picks the
    run-time parameters with the autotuner (cached in ``tune_cache``)."""
    import torch

    from .api import tessellate_host
    from .tune import autotune

    pts = np.ascontiguousarray(np.asarray(points), dtype=np.float32)
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("points must have shape (n, 3)")
    p = params if params is not None else make_params(**kw)
    tuning = None
    if tune:
        p, tuning = autotune(torch.from_numpy(pts).to(device), p, cache=tune_cache)
    c = tessellate_host(pts, p, device=device)
    out = {k: (None if getattr(c, k) is None else getattr(c, k).numpy()) for k in _OUTPUTS}
    out["stats"] = dict(c.stats)
    if tuning is not None:
        out["stats"]["tuned"] = {k: getattr(p, k) for k in ("threads_per_cell", "k0", "k_max", "grid_density")}
    return out


def parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(prog="python -m paper_2412_04514_gb300",
                                 description="3D Voronoi tessellation of a point file on the GPU.")
    ap.add_argument("input", help="points: .npy, .npz (array 'points') or text with 3 columns")
    ap.add_argument("-o", "--output", required=True, help="cells: .npz (all outputs) or .txt (neighbour lists)")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--emit", default="nbr,vol,cen", help="comma list of nbr, vol, cen, m2, geom")
    ap.add_argument("--k0", type=int, default=16)
    ap.add_argument("--k-max", type=int, default=32)
    ap.add_argument("--rho", type=float, default=2.0, help="mean generators per grid cell")
    ap.add_argument("--grid-res", type=int, default=0, help="grid cells per axis (0: from --rho)")
    ap.add_argument("--threads-per-cell", type=int, default=0, choices=(0, 8, 16, 32))
    ap.add_argument("--index-space", choices=("original", "sorted"), default="original")
    ap.add_argument("--box", type=float, nargs=6, metavar=("X0", "Y0", "Z0", "X1", "Y1", "Z1"),
                    help="bounding box (default the unit cube)")
    ap.add_argument("--periodic", action="store_true", help="the box is periodic")
    ap.add_argument("--fused", action="store_true",
                    help="no neighbour lists: every cell clips straight from its grid walk (smaller workspace)")
    ap.add_argument("--tune", action="store_true", help="autotune the run-time parameters first")
    ap.add_argument("--tune-cache", default=None, help="JSON cache of tuned parameters")
    ap.add_argument("--device", default="cuda")
    ap.add_argument("--stats", action="store_true", help="print the run statistics as JSON on stdout")
    return ap


def params_from_args(a: argparse.Namespace):
    emit = tuple(x.strip() for x in a.emit.split(",") if x.strip())
    bad = [x for x in emit if x not in ("nbr", "vol", "cen", "m2", "geom")]
    if bad:
        raise ValueError(f"unknown output(s) in --emit: {', '.join(bad)}")
    box = None if a.box is None else (a.box[:3], a.box[3:])
    return make_params(precision=a.precision, emit=emit, k0=a.k0, k_max=a.k_max, grid_density=a.rho,
                       grid_res=a.grid_res, threads_per_cell=a.threads_per_cell, index_space=a.index_space,
                       box=box, periodic=a.periodic, fused=a.fused)


def main(argv=None) -> int:
    a = parser().parse_args(argv)
    p = params_from_args(a)
    pts = read_points(a.input)
    cells = tessellate_numpy(pts, p, device=a.device, tune=a.tune, tune_cache=a.tune_cache)
    write_cells(a.output, cells, pts)
    if a.stats:
        print(json.dumps(cells["stats"], sort_keys=True, default=str))
    return 0


if __name__ == "__main__":  # pragma: no cover
    sys.exit(main())
