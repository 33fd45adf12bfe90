"""The fused schedule (VT_FLAG_FUSED): kNN and clipping in one kernel, no
neighbour lists. Every cell starts from the box and clips the generators its
grid-shell walk meets, nearest first within each batch, until the security
radius concludes it (paper, Summary: the kNN of a grid sort bounds what can
cut a cell; the fused walk visits the same generators without storing them).

A validated cell is the exact cell whatever the order of its cuts, so the
fused schedule must meet the oracle with the list schedules' tolerances:
FP64 neighbours exact and moments 1e-12 relative, FP32 moments 1e-5 relative
with neighbour differences only on faces below 1e-6 V^(2/3).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from geometry_match import emitted_cell, match_cell, oracle_cell
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMIT = ("nbr", "vol", "cen", "m2")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def np_(t):
    return None if t is None else t.cpu().numpy()


def lists(off, val):
    return [sorted(val[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def check(cells, want, prec, max_bad=1e-3):
    assert cells.stats["status"] == "VT_OK"
    vol, cen = np_(cells.vol), np_(cells.cen)
    got = lists(np_(cells.nbr_off), np_(cells.nbr))
    ref = lists(want["nbr_off"], want["nbr"])
    scale = np.cbrt(want["vol"])[:, None]
    if prec == "fp64":
        np.testing.assert_allclose(vol, want["vol"], rtol=1e-12, atol=0)
        assert (np.abs(cen - want["cen"]) / scale).max() < 1e-12
        np.testing.assert_allclose(np_(cells.m2), want["m2"], rtol=1e-11, atol=0)
        assert got == ref
        return
    np.testing.assert_allclose(vol, want["vol"], rtol=1e-5, atol=0)
    assert (np.abs(cen - want["cen"]) / scale).max() < 1e-5
    bad = 0
    for i, (g, w) in enumerate(zip(got, ref)):
        if g == w:
            continue
        bad += 1
        f0, f1 = want["face_off"][i], want["face_off"][i + 1]
        tiny = 1e-6 * want["vol"][i] ** (2 / 3)
        for j in set(g) ^ set(w):
            areas = want["face_area"][f0:f1][want["face_tag"][f0:f1] == j]
            assert len(areas) == 0 or areas.min() < tiny, (i, j, areas)
    assert bad <= max(2, max_bad * len(got))


@pytest.fixture(scope="module")
def uniform():
    pts = W.uniform(4096, 0)
    return pts, oracle.tessellate(pts)


@pytest.fixture(scope="module")
def clustered():
    # clumps of sigma 1e-3 put hundreds of generators into one grid cell
    pts = W.mixed(40_000, 3, n_clumps=40)
    return pts, oracle.tessellate(pts)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("no_sync", [False, True])
def test_fused_uniform_matches_the_oracle(uniform, prec, no_sync):
    pts, want = uniform
    cells = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=EMIT, fused=True, no_sync=no_sync))
    check(cells, want, prec)
    assert abs(np_(cells.vol).sum() - 1.0) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_clustered_matches_the_oracle(clustered, prec):
    pts, want = clustered
    cells = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=EMIT, fused=True, stage_times=True))
    check(cells, want, prec)
    st = cells.stats
    # one pass, no lists: the walk is the whole clip
    assert st["passes"] == 1 and st["k_of_pass"][0] == 0 and st["exhaustive_cells"] == len(pts)
    assert st["unvalidated"] == 0


@pytest.mark.parametrize("tpc", [8, 16])
def test_fused_threads_per_cell(uniform, tpc):
    pts, want = uniform
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=EMIT, fused=True, threads_per_cell=tpc))
    check(cells, want, "fp64")


def test_fused_lattices_fp64():
    # every bisector plane of a lattice cell passes through vertices of others
    for pts in (W.cubic_lattice(12), W.bcc_lattice(8)):
        want = oracle.tessellate(pts)
        cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=EMIT, fused=True))
        check(cells, want, "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_periodic_matches_the_oracle(prec):
    pts = W.mixed(30_000, 61, n_clumps=25, periodic=True)
    want = oracle.tessellate(pts, periodic=True)
    cells = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=EMIT, fused=True, periodic=True))
    check(cells, want, prec)


@pytest.mark.parametrize("n", [1, 2, 5, 20])
def test_fused_periodic_tiny_sets(n):
    # shells wider than the box: the walk meets several images of one generator
    pts = W.uniform(n, 70 + n)
    want = oracle.tessellate(pts, periodic=True)
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=EMIT, fused=True, periodic=True))
    check(cells, want, "fp64")


def test_fused_geometry_fp64_matches_oracle(uniform):
    pts, _ = uniform
    want = oracle.tessellate(pts, geometry=True)
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "geom"), fused=True))
    geo = tuple(np_(t) for t in (cells.vtx_off, cells.vtx, cells.face_off, cells.face_nbr, cells.face_vtx_off,
                                 cells.face_vtx))
    for i in range(0, len(pts), 7):
        V, faces = emitted_cell(geo, i)
        Wv, wfaces = oracle_cell(want, i)
        match_cell(V, faces, Wv, wfaces, 1e-13)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_batch_matches_the_oracle_per_set(prec):
    parts = [W.uniform(3000, 1), np.zeros((0, 3), np.float32), W.mixed(5000, 2, n_clumps=5), W.uniform(1, 3),
             W.uniform(17, 4)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    pts = np.concatenate(parts).astype(np.float32)
    cells = vt.tessellate_batch(dev(pts), off, vt.Params(precision=prec, emit=EMIT, fused=True))
    assert cells.stats["status"] == "VT_OK"
    nbr_off, nbr = np_(cells.nbr_off), np_(cells.nbr)
    for s, p in enumerate(parts):
        if not len(p):
            continue
        w = oracle.tessellate(p)
        a, b = off[s], off[s + 1]
        rtol = 1e-12 if prec == "fp64" else 1e-5
        np.testing.assert_allclose(np_(cells.vol)[a:b], w["vol"], rtol=rtol)
        got = [nbr[nbr_off[i]:nbr_off[i + 1]] - a for i in range(a, b)]
        bad = sum(not np.array_equal(g, x) for g, x in zip(got, oracle.neighbour_lists(w)))
        assert bad == 0 if prec == "fp64" else bad <= max(2, 1e-3 * len(p))



def test_fused_no_sync_equals_sync_with_geometry():
    # both schedules run the same single walk pass
    pts = W.mixed(60000, 8, n_clumps=60)
    emit = EMIT + ("geom",)
    a = vt.tessellate(dev(pts), vt.Params(precision="fp32", emit=emit, fused=True))
    b = vt.tessellate(dev(pts), vt.Params(precision="fp32", emit=emit, fused=True, no_sync=True))
    for name in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                 "face_vtx"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name


def test_fused_batch_graph_replay_matches_eager_and_the_oracle():
    # a CUDA graph of the fused schedule over a batch, replayed on new points
    parts = [W.uniform(2000, 11), W.mixed(6000, 12, n_clumps=6), W.uniform(1, 13), W.uniform(40, 14)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    pts = np.concatenate(parts).astype(np.float32)
    prm = vt.Params(precision="fp32", emit=EMIT, fused=True)
    b = vt.Batch(dev(pts), off, prm)
    b.capture()
    other_parts = [W.uniform(len(p), 90 + i) for i, p in enumerate(parts)]
    other = np.concatenate(other_parts).astype(np.float32)
    b.points.copy_(dev(other))
    b.replay()
    got = b.result()
    want = vt.tessellate_batch(dev(other), off, prm)
    for name in ("vol", "cen", "m2", "nbr_off", "nbr"):
        assert torch.equal(getattr(got, name), getattr(want, name)), name
    vol = np_(got.vol)
    for s, p in enumerate(other_parts):
        w = oracle.tessellate(p)
        np.testing.assert_allclose(vol[off[s]:off[s + 1]], w["vol"], rtol=1e-5)
