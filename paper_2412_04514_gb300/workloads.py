"""Seeded synthetic point clouds for the Voronoi pipeline.

This module only draws inputs; it holds none of the tessellation arithmetic, so
both the CUDA path's tests and the CPU oracle's tests can share it.

The paper (Summary, Performance) names no dataset: its Figure 1 inputs are not
given. The workloads below are synthetic stand-ins shaped like the
astrophysical point sets the Statement of need mentions (uniform background
plus Gaussian clumps), drawn with NumPy's PCG64 in float64 and cast to float32.

Every generator returns a C-contiguous ``float32[n, 3]`` array whose points lie
in the half-open box ``[lo, hi)`` (default the unit cube) and are pairwise
distinct (a duplicate generator has no Voronoi cell of its own).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform",
    "clustered",
    "mixed",
    "cubic_lattice",
    "bcc_lattice",
    "batch_sets",
    "sub_box_cells",
]


def _in_box_f32(x64: np.ndarray, lo: float, hi: float) -> tuple[np.ndarray, np.ndarray]:
    """Cast to float32 and flag rows that left ``[lo, hi)`` after rounding."""
    x32 = x64.astype(np.float32)
    ok = np.all((x32 >= np.float32(lo)) & (x32 < np.float32(hi)), axis=1)
    return x32, ok


def _dedupe(pts: np.ndarray) -> np.ndarray:
    """Boolean mask of rows that duplicate an earlier row (exact float32 bits)."""
    view = np.ascontiguousarray(pts).view(np.dtype((np.void, 12))).ravel()
    _, first = np.unique(view, return_index=True)
    dup = np.ones(len(pts), dtype=bool)
    dup[first] = False
    return dup


def uniform(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` points i.i.d. uniform in ``[lo, hi)^3``.

    Rows that round to ``hi`` in float32, or that repeat an earlier row, are
    redrawn from the same generator stream.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3), dtype=np.float32)
    filled = 0
    while filled < n:
        need = n - filled
        x64 = lo + (hi - lo) * rng.random((need, 3))
        x32, ok = _in_box_f32(x64, lo, hi)
        x32 = x32[ok]
        out[filled : filled + len(x32)] = x32
        filled += len(x32)
        if filled == n:
            dup = _dedupe(out)
            if dup.any():
                keep = out[~dup]
                out[: len(keep)] = keep
                filled = len(keep)
    return out


def clustered(
    n: int,
    n_clumps: int,
    rng: np.random.Generator,
    lo: float = 0.0,
    hi: float = 1.0,
    log10_sigma: tuple[float, float] = (-3.0, -2.0),
    periodic: bool = False,
) -> np.ndarray:
    """``n`` points from ``n_clumps`` isotropic Gaussian clumps.

    Clump centres are uniform in the box; each clump's sigma is log-uniform in
    ``10**log10_sigma`` (times the box edge); each point picks a clump
    uniformly. Draws that land outside the box are redrawn from the same clump
    (resampling, not clamping: clamping would pile points onto the walls and
    create coplanar or duplicate generators). With ``periodic`` they are
    wrapped by whole periods instead, so clumps continue across the faces of a
    periodic box.
    """
    span = hi - lo
    centres = lo + span * rng.random((n_clumps, 3))
    sigmas = span * 10.0 ** rng.uniform(log10_sigma[0], log10_sigma[1], size=n_clumps)
    which = rng.integers(0, n_clumps, size=n)
    out = np.empty((n, 3), dtype=np.float32)
    todo = np.arange(n)
    while len(todo):
        c = which[todo]
        x64 = centres[c] + sigmas[c, None] * rng.standard_normal((len(todo), 3))
        if periodic:
            x64 = x64 - np.floor((x64 - lo) / span) * span
        x32, ok = _in_box_f32(x64, lo, hi)
        out[todo[ok]] = x32[ok]
        todo = todo[~ok]
    return out


def mixed(
    n: int,
    seed: int,
    n_clumps: int = 1000,
    clustered_fraction: float = 0.5,
    lo: float = 0.0,
    hi: float = 1.0,
    periodic: bool = False,
) -> np.ndarray:
    """Half uniform, half clustered cloud (the 1M / 8M benchmark recipe).

    ``n_uniform = n - round(n * clustered_fraction)`` uniform points plus the
    rest drawn by :func:`clustered` with ``n_clumps`` clumps, then shuffled so
    the input order carries no spatial structure. Duplicate rows (possible in
    very tight clumps at float32 resolution) are redrawn uniformly.
    ``periodic``: clumps wrap across the faces of the box (see :func:`clustered`).
    """
    rng = np.random.default_rng(seed)
    n_cl = int(round(n * clustered_fraction))
    n_un = n - n_cl
    parts = []
    if n_un:
        parts.append((lo + (hi - lo) * rng.random((n_un, 3))))
    pts = np.concatenate(
        [p.astype(np.float32) for p in parts]
        + ([clustered(n_cl, n_clumps, rng, lo, hi, periodic=periodic)] if n_cl else []),
        axis=0,
    )
    # uniform draws that rounded up to hi in float32
    bad = ~np.all((pts >= np.float32(lo)) & (pts < np.float32(hi)), axis=1)
    while True:
        bad |= _dedupe(pts)
        if not bad.any():
            break
        x32, ok = _in_box_f32(lo + (hi - lo) * rng.random((int(bad.sum()), 3)), lo, hi)
        idx = np.flatnonzero(bad)
        pts[idx[ok]] = x32[ok]
        bad[:] = False
        bad[idx[~ok]] = True
    perm = rng.permutation(n)
    return np.ascontiguousarray(pts[perm])


def cubic_lattice(m: int = 16) -> np.ndarray:
    """Simple cubic lattice ``((a+1/2)/m, (b+1/2)/m, (c+1/2)/m)``, exact in float32 for m = 2^j."""
    g = (np.arange(m, dtype=np.float64) + 0.5) / m
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32))


def bcc_lattice(m: int = 16) -> np.ndarray:
    """Body-centred cubic lattice of spacing ``h = 1/m`` in the unit cube.

    Sub-lattice A at ``(a+1/2)h`` (m^3 points) and sub-lattice B at ``(a+1)h``
    for ``a < m-1`` ((m-1)^3 points, so no point sits on the wall ``x = 1``).
    """
    h = 1.0 / m
    ga = (np.arange(m) + 0.5) * h
    gb = (np.arange(m - 1) + 1.0) * h
    a = np.stack(np.meshgrid(ga, ga, ga, indexing="ij"), -1).reshape(-1, 3)
    b = np.stack(np.meshgrid(gb, gb, gb, indexing="ij"), -1).reshape(-1, 3)
    return np.ascontiguousarray(np.concatenate([a, b]).astype(np.float32))


def batch_sets(
    n_sets: int = 512,
    seed: int = 3,
    size_range: tuple[int, int] = (1000, 200_000),
    clustered_per_clump: int = 524,
) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Many independent point sets of uneven sizes, each in the unit cube.

    Sizes are ``floor(10**U(log10 a, log10 b))``; a seeded coin flip makes a
    set uniform or clustered (the mixed recipe with ``ceil(n / 1048)`` clumps,
    about ``clustered_per_clump`` clustered points per clump). Set ``s`` draws
    from seed ``seed * 10**6 + s``.

    Returns ``(points float32[sum n, 3], set_off int64[n_sets + 1],
    is_clustered bool[n_sets])``.
    """
    rng = np.random.default_rng(seed)
    sizes = np.floor(10.0 ** rng.uniform(np.log10(size_range[0]), np.log10(size_range[1]), n_sets)).astype(np.int64)
    coin = rng.random(n_sets) < 0.5
    parts = []
    for s in range(n_sets):
        n = int(sizes[s])
        if coin[s]:
            n_clumps = max(1, -(-n // (2 * clustered_per_clump)))
            parts.append(mixed(n, seed * 10**6 + s, n_clumps=n_clumps))
        else:
            parts.append(uniform(n, seed * 10**6 + s))
    off = np.zeros(n_sets + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return np.ascontiguousarray(np.concatenate(parts)), off, coin


def sub_box_cells(pts: np.ndarray, target: int, seed: int) -> np.ndarray:
    """Indices of the generators inside a seeded axis-aligned sub-box.

    The sub-box is a cube placed uniformly at random in the unit box and grown
    (by bisection on its edge) until it holds about ``target`` generators.
    Returns sorted int64 indices into ``pts``.
    """
    rng = np.random.default_rng(seed)
    corner = rng.random(3) * 0.5
    lo_e, hi_e = 0.0, 0.5
    sel = np.zeros(0, dtype=np.int64)
    for _ in range(40):
        e = 0.5 * (lo_e + hi_e)
        inside = np.all((pts >= corner) & (pts < corner + e), axis=1)
        cnt = int(inside.sum())
        sel = np.flatnonzero(inside)
        if abs(cnt - target) <= max(1, target // 100):
            break
        if cnt < target:
            lo_e = e
        else:
            hi_e = e
    return sel.astype(np.int64)
