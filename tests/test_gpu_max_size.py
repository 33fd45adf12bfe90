"""The largest periodic input, 2^24 - 1 points, walled and periodic, against the oracle.

Entries of the periodic lists pack a sorted index in 24 bits beside a 7-bit
image code, and tie keys hold original index x 128 + code, so n = 2^24 - 1 is
the edge of that encoding (``vt_tessellate`` refuses n >= 2^24 in a periodic
box). At this size the oracle computes sampled cells from their local
clouds. A cell is the box cut by its generator's bisectors (Summary of the
paper), and only generators within twice the cell's radius can cut it. So
the oracle's cell of generator i among the generators within a ball B of
radius r around it is its cell in the whole set whenever that cell's radius
stays below r / 2, which each sampled cell checks. Periodic images are
unwrapped by whole periods on the side that lies in [0.5, 1), where float32
subtraction of 1 is exact (Sterbenz), so the local offsets are the ones the
periodic box defines. The sample: random cells, cells on the box faces and the
cells of the corner [0.98, 1)^3, whose grid-sorted indices are the largest.
Tolerances as in the other parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = (1 << 24) - 1
RADIUS = 6.0 * N ** (-1.0 / 3.0)  # six mean spacings


def local_oracle(pts, tree, i, periodic):
    """The oracle's cell of generator i from the generators within RADIUS."""
    p64 = pts.astype(np.float64)
    near = np.asarray(tree.query_ball_point(p64[i], RADIUS), dtype=np.int64)
    ids = np.concatenate([[i], near[near != i]])
    q = p64[ids].copy()
    if periodic:
        wrap = np.concatenate([[False] * 3, (np.abs(q[1:] - q[0]) > 0.5).ravel()]).reshape(-1, 3)
        for a in range(3):
            if wrap[:, a].any():
                side = wrap[:, a] if q[0, a] < 0.5 else ~wrap[:, a]
                assert np.all(q[side, a] >= 0.5)
                q[side, a] -= 1.0
    q32 = q.astype(np.float32)
    assert np.array_equal(q32.astype(np.float64), q)
    lo, hi = q[0] - 2 * RADIUS, q[0] + 2 * RADIUS
    if not periodic:
        lo, hi = np.maximum(lo, 0.0), np.minimum(hi, 1.0)
    r = oracle.tessellate(q32, lo=tuple(lo), hi=tuple(hi), cells=np.array([0]), geometry=True)
    f0, f1 = r["face_off"][0], r["face_off"][1]
    radius = np.sqrt(((r["face_vtx"] - q[0]) ** 2).sum(1).max())
    assert 2 * radius < RADIUS, (i, radius)
    return dict(vol=r["vol"][0], cen=r["cen"][0], nbr=np.sort(ids[r["nbr"][r["nbr_off"][0]:r["nbr_off"][1]]]),
                face_ids=ids[np.maximum(r["face_tag"][f0:f1], 0)] * (r["face_tag"][f0:f1] >= 0)
                + r["face_tag"][f0:f1] * (r["face_tag"][f0:f1] < 0),
                face_area=r["face_area"][f0:f1])


@pytest.fixture(scope="module")
def cloud():
    from scipy.spatial import cKDTree

    pts = W.uniform(N, 91)
    rng = np.random.default_rng(92)
    faces = np.flatnonzero((pts < 0.002).any(1) | (pts > 0.998).any(1))
    corner = np.flatnonzero((pts >= 0.98).all(1))
    sample = np.unique(np.concatenate([rng.choice(N, 200, replace=False), rng.choice(faces, 100, replace=False),
                                       corner]))
    p64 = pts.astype(np.float64)
    trees = {False: cKDTree(p64), True: cKDTree(p64, boxsize=1.0)}
    want = {per: [local_oracle(pts, trees[per], i, per) for i in sample] for per in (False, True)}
    return pts, sample, want


@pytest.mark.parametrize("periodic", [False, True], ids=["walls", "periodic"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_largest_periodic_size(cloud, periodic, precision):
    pts, sample, want = cloud
    p = vt.Params(precision=precision, k0=16, k_max=32, threads_per_cell=32, emit=("nbr", "vol", "cen"),
                  periodic=periodic)
    cells = vt.tessellate(torch.from_numpy(pts).cuda(), p)
    assert cells.stats["status"] == "VT_OK"
    vol, cen = cells.vol.cpu().numpy(), cells.cen.cpu().numpy()
    off, nb = cells.nbr_off.cpu().numpy(), cells.nbr.cpu().numpy()
    del cells
    torch.cuda.empty_cache()
    fp64 = precision == "fp64"
    assert abs(vol.sum() - 1.0) < (1e-9 if fp64 else 1e-6)
    bad = 0
    for i, w in zip(sample, want[periodic]):
        dc = cen[i] - w["cen"]
        if periodic:  # the local frame may sit whole periods away
            dc -= np.round(dc)
        got = np.sort(nb[off[i]:off[i + 1]])
        if fp64:
            np.testing.assert_allclose(vol[i], w["vol"], rtol=1e-12)
            assert np.abs(dc).max() < 1e-12, (i, dc)
            assert np.array_equal(got, w["nbr"]), i
        else:
            np.testing.assert_allclose(vol[i], w["vol"], rtol=1e-5)
            assert np.linalg.norm(dc) < 1e-5 * np.linalg.norm(w["cen"] - np.floor(w["cen"])) + 1e-12, (i, dc)
            if not np.array_equal(got, w["nbr"]):
                bad += 1
                for j in set(got.tolist()) ^ set(w["nbr"].tolist()):
                    areas = w["face_area"][w["face_ids"] == j]
                    assert len(areas) == 0 or areas.min() < 1e-6 * w["vol"] ** (2 / 3), (i, j, areas)
    assert bad <= 2
