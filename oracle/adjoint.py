"""FP64 oracle of the moments adjoint -- TEST INFRASTRUCTURE ONLY.

Vector-Jacobian product of the per-cell volume V_i, centroid c_i and second
moment M2_i = integral over C_i of |x - p_i|^2, with respect to every
generator p_k, for upstream gradients (gV_i, gC_i, gM_i):

    grad_k = sum_i gV_i dV_i/dp_k + gC_i . dc_i/dp_k + gM_i dM2_i/dp_k.

Derivation (Reynolds transport; the paper gives no formula).
The face f_ij of cell i lies on the bisector n.x = (|p_j|^2 - |p_i|^2)/2,
n = p_j - p_i, d = |n|. Moving p_j moves the face along its outward normal
with speed (p_j - x).dp_j / d; moving p_i, with speed (x - p_i).dp_i / d.
Walls do not move. For Q_i = integral over C_i of g_i:

    dQ_i/dp_j = (1/d) integral_f g_i(x) (p_j - x) dA            (j a neighbour)
    dQ_i/dp_i = sum_j (1/d) integral_f g_i(x) (x - p_i) dA + integral_C dg_i/dp_i.

Combining the three outputs, cell i contributes the density
h_i(x) = gV_i + gC_i.(x - c_i) / V_i + gM_i |x - p_i|^2 (the centroid term
from c = S/V with S the first moment), and the interior term
2 gM_i V_i (p_i - c_i) to grad_i. Face integrals of h times an affine vector
are polynomials of degree <= 3 in x, integrated exactly on a triangle fan of
each face with the 7-point degree-3 rule (weights 1/20 at the vertices, 2/15
at the edge midpoints, 9/20 at the centroid, times the area).

In a periodic box the neighbour across a face is the image p_j + t L that the
face's shift code names (the cell's own image for the faces of its starting
cube); moving p_j moves every image with it, so the same formulas hold with
that image in place of p_j.

This implementation scatters each face term to both generators; it shares no
code with the CUDA kernel. Pins: tests/test_oracle_adjoint.py (the Lloyd
closed form, conservation of total volume and first moment, central finite
differences, exactness of the quadrature rule).
"""
from __future__ import annotations

import numpy as np

from . import img_shift, tessellate

# 7-point rule on a triangle (barycentric coordinates, weights relative to the area)
_BARY = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1],
                  [0.5, 0.5, 0], [0, 0.5, 0.5], [0.5, 0, 0.5],
                  [1 / 3, 1 / 3, 1 / 3]], dtype=np.float64)
_W = np.array([1 / 20, 1 / 20, 1 / 20, 2 / 15, 2 / 15, 2 / 15, 9 / 20], dtype=np.float64)


def triangle_rule(a: np.ndarray, b: np.ndarray, c: np.ndarray):
    """Quadrature points [T, 7, 3] and weights [T, 7] for triangles (a, b, c) [T, 3]."""
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    pts = _BARY[None, :, 0, None] * a[:, None, :] + _BARY[None, :, 1, None] * b[:, None, :] \
        + _BARY[None, :, 2, None] * c[:, None, :]
    return pts, area[:, None] * _W[None, :]


def face_triangles(res: dict, pts64: np.ndarray, cells=None):
    """Fan triangles of every neighbour face: (cell, neighbour, shift code, a, b, c)."""
    foff, tag, size, vtx = res["face_off"], res["face_tag"], res["face_size"], res["face_vtx"]
    img = res["face_img"]
    vstart = np.concatenate([[0], np.cumsum(size)])
    nc = len(foff) - 1
    cell_of_face = np.repeat(np.arange(nc), np.diff(foff))
    if cells is not None:
        cell_of_face = np.asarray(cells)[cell_of_face]
    ci, nj, im, A, B, C = [], [], [], [], [], []
    for f in range(len(tag)):
        if tag[f] < 0:
            continue
        loop = vtx[vstart[f]:vstart[f + 1]]
        m = len(loop)
        for t in range(1, m - 1):
            ci.append(cell_of_face[f])
            nj.append(tag[f])
            im.append(img[f])
            A.append(loop[0])
            B.append(loop[t])
            C.append(loop[t + 1])
    return (np.array(ci, dtype=np.int64), np.array(nj, dtype=np.int64), np.array(im, dtype=np.int64),
            np.array(A).reshape(-1, 3), np.array(B).reshape(-1, 3), np.array(C).reshape(-1, 3))


def moments_adjoint(points, gV=None, gC=None, gM=None, res: dict | None = None, lo=(0.0, 0.0, 0.0),
                    hi=(1.0, 1.0, 1.0), k0: int = 16, periodic: bool = False) -> np.ndarray:
    """Gradient [n, 3] (float64) of sum_i gV_i V_i + gC_i . c_i + gM_i M2_i.

    ``res`` may pass an oracle tessellation made with ``geometry=True`` (and
    the same ``periodic``). Missing upstream gradients count as zero.
    """
    p = np.ascontiguousarray(points, dtype=np.float32)
    n = len(p)
    p64 = p.astype(np.float64)
    if res is None:
        res = tessellate(p, lo=lo, hi=hi, k0=k0, geometry=True, periodic=periodic)
    gV = np.zeros(n) if gV is None else np.asarray(gV, dtype=np.float64)
    gC = np.zeros((n, 3)) if gC is None else np.asarray(gC, dtype=np.float64)
    gM = np.zeros(n) if gM is None else np.asarray(gM, dtype=np.float64)
    V, c = res["vol"], res["cen"]
    # h_i(x) = alpha_i + beta_i . x + gamma_i |x - p_i|^2
    beta = gC / V[:, None]
    alpha = gV - np.einsum("ij,ij->i", beta, c)
    gamma = gM
    grad = 2.0 * (gamma * V)[:, None] * (p64 - c)  # interior term of M2

    ci, nj, im, a, b, cc = face_triangles(res, p64)
    if len(ci):
        qp, qw = triangle_rule(a, b, cc)  # [T, 7, 3], [T, 7]
        L = np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)
        pi, pj = p64[ci], p64[nj] + img_shift(im) * L  # the neighbour's image across the face
        hq = (alpha[ci][:, None] + np.einsum("tk,tqk->tq", beta[ci], qp)
              + gamma[ci][:, None] * np.sum((qp - pi[:, None, :]) ** 2, axis=2))
        d = np.linalg.norm(pj - pi, axis=1)
        # integral of h (x - p_i) and of h (p_j - x) over each triangle
        own = np.einsum("tq,tqk->tk", hq * qw, qp - pi[:, None, :]) / d[:, None]
        other = np.einsum("tq,tqk->tk", hq * qw, pj[:, None, :] - qp) / d[:, None]
        np.add.at(grad, ci, own)
        np.add.at(grad, nj, other)
    return grad


def loss(points, gV, gC, gM, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), cells=None, periodic: bool = False) -> float:
    """sum over `cells` (default all) of gV_i V_i + gC_i . c_i + gM_i M2_i, in FP64."""
    r = tessellate(points, lo=lo, hi=hi, cells=cells, periodic=periodic)
    idx = np.arange(len(points)) if cells is None else np.asarray(cells)
    return float(np.sum(gV[idx] * r["vol"]) + np.sum(gC[idx] * r["cen"]) + np.sum(gM[idx] * r["m2"]))
