"""Vertex-by-vertex comparison of one cell's geometry with the oracle's.

A Voronoi cell's geometry (paper, Summary: the output is each cell's
polyhedron) is a set of vertices and, per face, the counter-clockwise loop of
its vertices. Two cells are the same when there is a one-to-one pairing of
their vertices within a tolerance (found as the minimum-cost assignment on
squared distances, so that a vertex is never paired twice and a coordinate
moved from one vertex to another is caught) and every face of one is a face
of the other with the same neighbour id and the same cyclic sequence of
vertex positions, in the same orientation.

Test helper only: no test is collected from this module.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def oracle_cell(want: dict, a: int):
    """Vertices (unique rows) and faces [(tag, loop of vertex indices)] of
    cell a of an oracle result computed with ``geometry=True``."""
    start = np.concatenate([[0], np.cumsum(want["face_size"])])
    f0, f1 = int(want["face_off"][a]), int(want["face_off"][a + 1])
    rows = np.concatenate([want["face_vtx"][start[f]:start[f + 1]] for f in range(f0, f1)])
    verts, inv = np.unique(rows, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    faces, k = [], 0
    for f in range(f0, f1):
        m = int(want["face_size"][f])
        faces.append((int(want["face_tag"][f]), inv[k:k + m]))
        k += m
    return verts, faces


def emitted_cell(geo, i: int):
    """Vertices and faces of cell i from emitted CSR arrays
    (vtx_off, vtx, face_off, face_nbr, face_vtx_off, face_vtx)."""
    vo, v, fo, fn, fvo, fv = geo
    verts = np.asarray(v[vo[i]:vo[i + 1]], dtype=np.float64)
    faces = [(int(fn[f]), np.asarray(fv[fvo[f]:fvo[f + 1]])) for f in range(fo[i], fo[i + 1])]
    return verts, faces


def match_cell(V, faces_v, W, faces_w, atol: float) -> None:
    """Asserts that (V, faces_v) and (W, faces_w) are the same polyhedron."""
    V = np.asarray(V, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    assert V.shape == W.shape, f"vertex counts differ: {len(V)} vs {len(W)}"
    d2 = ((V[:, None, :] - W[None, :, :]) ** 2).sum(-1)
    r, c = linear_sum_assignment(d2)
    worst = float(np.sqrt(d2[r, c].max())) if len(r) else 0.0
    assert worst <= atol, f"no one-to-one vertex pairing within {atol:.3g} (worst pair {worst:.3g})"
    assert len(faces_v) == len(faces_w), f"face counts differ: {len(faces_v)} vs {len(faces_w)}"
    used = [False] * len(faces_w)
    for tag, loop in faces_v:
        P = V[loop]
        hit = -1
        for b, (tw, lw) in enumerate(faces_w):
            if used[b] or tw != tag or len(lw) != len(loop):
                continue
            Q = W[lw]
            for rot in range(len(lw)):
                if np.abs(P - np.roll(Q, -rot, axis=0)).max() <= atol:
                    hit = b
                    break
            if hit >= 0:
                break
        assert hit >= 0, f"face {tag} (loop of {len(loop)}) has no counterpart with the same cyclic order"
        used[hit] = True
