"""Exact rational geometry of an oracle cell, for pinning the oracle's FP64
arithmetic: every vertex is re-solved from three of its face planes in
rational arithmetic (the generators are float32, hence exact rationals), and
the volume is summed exactly over the faces' fans from the generator."""
from fractions import Fraction as F

import numpy as np


def _det3(a, b, c):
    return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
            + a[2] * (b[0] * c[1] - b[1] * c[0]))


def _solve(planes):
    (n1, b1), (n2, b2), (n3, b3) = planes
    D = _det3(n1, n2, n3)
    if D == 0:
        return None
    out = []
    for k in range(3):
        rows = [list(n1), list(n2), list(n3)]
        for row, bb in zip(rows, (b1, b2, b3)):
            row[k] = bb
        out.append(_det3(*rows) / D)
    return out


def cell_planes(pts, i, res, a, lo=(0, 0, 0), hi=(1, 1, 1)):
    """Exact planes n.x <= b (global frame) of the faces of sampled cell a (generator i)."""
    p = [F(float(x)) for x in pts[i]]
    f0, f1 = res["face_off"][a], res["face_off"][a + 1]
    planes = []
    for t in res["face_tag"][f0:f1]:
        if t >= 0:
            q = [F(float(x)) for x in pts[t]]
            n = [q[k] - p[k] for k in range(3)]
            b = sum(n[k] * (q[k] + p[k]) for k in range(3)) / 2
        else:
            w = -int(t) - 1
            ax, upper = w // 2, w % 2
            n = [F(0)] * 3
            n[ax] = F(1) if upper else F(-1)
            b = F(float(np.float32(hi[ax]))) if upper else -F(float(np.float32(lo[ax])))
        planes.append((n, b))
    return p, planes


def exact_cell(pts, i, res, a, lo=(0, 0, 0), hi=(1, 1, 1)):
    """(exact volume, exact vertices of every face loop) of sampled cell a.
    ``res`` must come from oracle.tessellate(..., geometry=True)."""
    p, planes = cell_planes(pts, i, res, a, lo, hi)
    fl = [(np.array([float(x) for x in n]), float(b)) for n, b in planes]
    sizes = res["face_size"]
    f0, f1 = res["face_off"][a], res["face_off"][a + 1]
    start = int(np.sum(sizes[:f0]))
    vol = F(0)
    loops = []
    for fi in range(f1 - f0):
        sz = int(sizes[f0 + fi])
        loop = res["face_vtx"][start:start + sz]
        start += sz
        ex = []
        for v in loop:
            r = [abs(n @ v - b) / np.linalg.norm(n) for n, b in fl]
            order = [fi] + [j for j in np.argsort(r) if j != fi]
            sol = None
            for jj in range(1, 6):
                for kk in range(jj + 1, 8):
                    if kk >= len(order):
                        break
                    sol = _solve([planes[fi], planes[order[jj]], planes[order[kk]]])
                    if sol is not None:
                        break
                if sol is not None:
                    break
            assert sol is not None
            ex.append(sol)
        for t in range(1, sz - 1):
            d = [[ex[s][k] - p[k] for k in range(3)] for s in (0, t, t + 1)]
            vol += _det3(*d) / 6
        loops.append(ex)
    return vol, loops, planes
