"""The benchmark's own launch configuration at full size, against the oracle.

``bench.py`` times 32 lanes per cell, k0 = 16 doubled to k_max = 32, two
points per grid cell and full geometry on 1,048,576 points, walled (mixed
recipe, seed 1) and periodic (mixed recipe with wrapped clumps, seed 5), in
the list schedule and in the fused one (VT_FLAG_FUSED, the bench's fused_form). At
that size the oracle computes sampled cells one by one (its cells are
independent, Summary of the paper); on the whole output the tests check
what holds at any size: the cells fill the box (volumes and first moments),
every cell is a simple polyhedron (V = 2F - 4), its faces are its neighbours,
its walls and faces below the neighbour threshold, and a neighbour relation
seen from one side only is such a tiny face (areas from the emitted geometry).
Tolerances as elsewhere: the FP64 form's sampled neighbour multisets are
exact and its moments agree to 1e-12; the FP32 form's volumes agree to 1e-5
relative, centroids to 1e-5 of |c|, and neighbours differ only by faces the
oracle measures below 1e-6 V^(2/3).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from geometry_match import emitted_cell, match_cell, oracle_cell
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 1 << 20
EMIT = ("nbr", "vol", "cen", "geom")


def bench_params(precision, periodic, fused=False):
    return vt.Params(precision=precision, k0=16, k_max=32, threads_per_cell=32, grid_density=2.0, emit=EMIT,
                     periodic=periodic, fused=fused)


def np_(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module", params=[False, True], ids=["mixed-1m", "periodic-1m"])
def workload(request):
    periodic = request.param
    pts = W.mixed(N, 5 if periodic else 1, n_clumps=1000, periodic=periodic)
    sample = np.sort(np.random.default_rng(17).choice(N, 2000, replace=False))
    want = oracle.tessellate(pts, periodic=periodic, cells=sample, geometry=True)
    return pts, periodic, sample, want


def ragged(off, val, rows):
    return [np.sort(val[off[i]:off[i + 1]]) for i in rows]


def tiny_face(want, a, j):
    f0, f1 = want["face_off"][a], want["face_off"][a + 1]
    areas = want["face_area"][f0:f1][want["face_tag"][f0:f1] == j]
    return len(areas) == 0 or areas.min() < 1e-6 * want["vol"][a] ** (2 / 3)


def face_areas(cells_np, i):
    """Areas of cell i's faces from the emitted geometry (Newell's formula) and their ids."""
    vo, v, fo, fn, fvo, fv = cells_np
    V = v[vo[i]:vo[i + 1]].astype(np.float64)
    areas = []
    for f in range(fo[i], fo[i + 1]):
        P = V[fv[fvo[f]:fvo[f + 1]]]
        P = P - P[0]
        areas.append(0.5 * np.linalg.norm(np.cross(P, np.roll(P, -1, axis=0)).sum(0)))
    return np.asarray(areas), fn[fo[i]:fo[i + 1]]


def whole_output_properties(cells, periodic, fp64):
    vol, cen = np_(cells.vol), np_(cells.cen)
    tol = 1e-9 if fp64 else 1e-6
    assert abs(vol.sum() - 1.0) < tol
    if not periodic:  # the box's first moment (a periodic cell's centroid may lie across a face)
        np.testing.assert_allclose((vol[:, None] * cen).sum(0), 0.5, atol=tol)
    geo = tuple(np_(t) for t in (cells.vtx_off, cells.vtx, cells.face_off, cells.face_nbr, cells.face_vtx_off,
                                 cells.face_vtx))
    off, nb = np_(cells.nbr_off), np_(cells.nbr)
    nf, nv = np.diff(geo[2]), np.diff(geo[0])
    tiny = lambda i, j: 1e-6 * max(vol[i], vol[j]) ** (2 / 3)  # noqa: E731
    # simple polyhedra: three faces at every vertex
    assert np.count_nonzero(nv != 2 * nf - 4) <= (10 if fp64 else 1e-4 * N)
    # every neighbour is a face; the other faces are walls or below the
    # neighbour threshold (a face counts as a neighbour only above a small
    # fraction of V^(2/3))
    walls = np.bincount(np.repeat(np.arange(N), nf)[geo[3] < 0], minlength=N)
    extra = nf - np.diff(off) - walls
    assert extra.min() >= 0
    for i in np.flatnonzero(extra):
        areas, ids = face_areas(geo, i)
        listed = list(nb[off[i]:off[i + 1]])
        for a, t in sorted(zip(areas, ids), key=lambda x: -x[0]):
            if t < 0:
                continue
            if t in listed:
                listed.remove(t)
            else:
                assert a < tiny(i, t), (i, t, a)
        assert not listed
    # mutual neighbours: a pair listed on one side only is a face below the
    # threshold of the larger cell (the threshold is relative to each cell's
    # own volume; the oracle's own mixed-1m output has four such pairs)
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(off))
    fwd, bwd = rows * N + nb, nb.astype(np.int64) * N + rows
    uf, cf = np.unique(fwd, return_counts=True)
    ub, cb = np.unique(bwd, return_counts=True)
    keys = np.union1d(uf, ub)
    kf = np.zeros(len(keys), np.int64)
    kb = np.zeros(len(keys), np.int64)
    kf[np.searchsorted(keys, uf)] = cf
    kb[np.searchsorted(keys, ub)] = cb
    one_sided = keys[kf > kb]
    assert len(one_sided) <= 1e-4 * len(nb), len(one_sided)
    for key in one_sided:
        i, j = divmod(int(key), N)
        areas, ids = face_areas(geo, i)
        assert areas[ids == j].min() < tiny(i, j), (i, j, areas[ids == j], vol[i], vol[j])


@pytest.mark.parametrize("fused", [False, True], ids=["lists", "fused"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bench_configuration_sampled_and_whole(workload, precision, fused):
    # the list schedule (the bench line) and the fused schedule (its fused_form)
    pts, periodic, sample, want = workload
    cells = vt.tessellate(torch.from_numpy(pts).cuda(), bench_params(precision, periodic, fused))
    assert cells.stats["status"] == "VT_OK"
    fp64 = precision == "fp64"
    vol, cen = np_(cells.vol)[sample], np_(cells.cen)[sample]
    got = ragged(np_(cells.nbr_off), np_(cells.nbr), sample)
    ref = ragged(want["nbr_off"], want["nbr"], range(len(sample)))
    if fp64:
        np.testing.assert_allclose(vol, want["vol"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(cen, want["cen"], rtol=0, atol=1e-12)
        assert all(np.array_equal(g, w) for g, w in zip(got, ref))
    else:
        np.testing.assert_allclose(vol, want["vol"], rtol=1e-5, atol=0)
        rel_c = np.linalg.norm(cen - want["cen"], axis=1) / np.linalg.norm(want["cen"], axis=1)
        assert rel_c.max() < 1e-5, rel_c.max()
        bad = [a for a, (g, w) in enumerate(zip(got, ref)) if not np.array_equal(g, w)]
        for a in bad:
            for j in set(got[a].tolist()) ^ set(ref[a].tolist()):
                assert tiny_face(want, a, j), (sample[a], j)
        assert len(bad) <= max(2, 1e-3 * len(sample))
    # geometry of the sampled cells whose neighbours match: a one-to-one
    # pairing of the vertices (FP64 to 1e-12, FP32 to 1e-5 of the cell's
    # size) and every face the same cyclic loop with the same neighbour id
    geo = tuple(np_(t) for t in (cells.vtx_off, cells.vtx, cells.face_off, cells.face_nbr, cells.face_vtx_off,
                                 cells.face_vtx))
    for a, i in enumerate(sample):
        if not np.array_equal(got[a], ref[a]):
            continue
        V, fv = emitted_cell(geo, i)
        assert len(V) == want["nvert"][a], (i, len(V), want["nvert"][a])
        W_, fw = oracle_cell(want, a)
        scale = np.cbrt(want["vol"][a])
        # (FP32 vertices are float32 coordinates: a few ulps of |x| on top)
        amax = np.abs(W_).max()
        atol = 1e-12 * max(1.0, amax) if fp64 else 1e-5 * scale + 4 * np.finfo(np.float32).eps * amax
        match_cell(V, fv, W_, fw, atol)
    whole_output_properties(cells, periodic, fp64)
