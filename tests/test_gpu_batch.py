"""Batches of independent point sets (vt_tessellate_batch) and the no-sync,
graph-capturable schedule.

Every set of a batch is its own tessellation, so the batch must reproduce,
cell by cell, what a single-set run on that set gives (bit for bit when both
use the same grid resolution: same grid, same neighbour lists, same
arithmetic), and therefore the oracle on that set with the single-set
tolerances: FP64 neighbours exact and moments 1e-12 relative; FP32 moments
1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import _lib as L
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMIT = ("nbr", "vol", "cen", "m2")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def np_(t):
    return None if t is None else t.cpu().numpy()


def small_batch():
    # uneven sizes, an empty set and a one-point set, uniform and clustered
    parts = [W.uniform(3000, 1), np.zeros((0, 3), np.float32), W.mixed(5000, 2, n_clumps=5), W.uniform(1, 3),
             W.uniform(17, 4), W.mixed(12000, 5, n_clumps=12), W.uniform(700, 6), W.uniform(2, 7)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    return np.concatenate(parts).astype(np.float32), off, parts


@pytest.fixture(scope="module")
def batch():
    pts, off, parts = small_batch()
    return pts, off, parts, [oracle.tessellate(p) if len(p) else None for p in parts]


def split(cells, off, s):
    a, b = off[s], off[s + 1]
    nbr_off = np_(cells.nbr_off)
    nbr = np_(cells.nbr)
    lists = [nbr[nbr_off[i]:nbr_off[i + 1]] for i in range(a, b)]
    return np_(cells.vol)[a:b], np_(cells.cen)[a:b], np_(cells.m2)[a:b], lists


@pytest.mark.parametrize("prec,no_sync", [("fp64", False), ("fp64", True), ("fp32", False), ("fp32", True)])
def test_batch_matches_the_oracle_per_set(batch, prec, no_sync):
    pts, off, parts, want = batch
    cells = vt.tessellate_batch(dev(pts), off, vt.Params(precision=prec, emit=EMIT, no_sync=no_sync))
    assert cells.stats["status"] == "VT_OK"
    for s, w in enumerate(want):
        if w is None:
            continue
        vol, cen, m2, lists = split(cells, off, s)
        rtol = 1e-12 if prec == "fp64" else 1e-5
        np.testing.assert_allclose(vol, w["vol"], rtol=rtol)
        np.testing.assert_allclose(cen, w["cen"], rtol=rtol, atol=1e-15)
        wl = oracle.neighbour_lists(w)
        bad = sum(not np.array_equal(g - off[s], x) for g, x in zip(lists, wl))
        if prec == "fp64":
            np.testing.assert_allclose(m2, w["m2"], rtol=1e-11)
            assert bad == 0
        else:
            assert bad <= max(2, 1e-3 * len(wl))
        for g in lists:  # neighbours never leave the set
            assert len(g) == 0 or (g.min() >= off[s] and g.max() < off[s + 1])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_is_bit_identical_to_single_set_runs(batch, prec):
    pts, off, parts, _ = batch
    G = [vt.grid_resolution(vt.Params(), max(len(p), 1)) for p in parts]
    prm = vt.Params(precision=prec, emit=EMIT)
    cells = vt.tessellate_batch(dev(pts), off, vt.Params(precision=prec, emit=EMIT, no_sync=True), grid_res=G)
    for s, p in enumerate(parts):
        if not len(p):
            continue
        one = vt.tessellate(dev(p), prm)
        vol, cen, m2, lists = split(cells, off, s)
        assert np.array_equal(vol, np_(one.vol))
        assert np.array_equal(cen, np_(one.cen))
        assert np.array_equal(m2, np_(one.m2))
        ol = np_(one.nbr_off)
        for i, g in enumerate(lists):
            assert np.array_equal(g - off[s], np_(one.nbr)[ol[i]:ol[i + 1]])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_no_sync_schedule_equals_the_synchronising_one(prec):
    pts = W.mixed(60000, 8, n_clumps=60)
    a = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=EMIT + ("geom",)))
    b = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=EMIT + ("geom",), no_sync=True))
    for name in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                 "face_vtx"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name


def test_graph_replay_equals_eager_runs(batch):
    pts, off, parts, _ = batch
    b = vt.Batch(dev(pts), off, vt.Params(precision="fp32", emit=EMIT))
    b.capture()
    other = W.uniform(len(pts), 77)  # new coordinates, same set sizes
    b.points.copy_(dev(other))
    b.replay()
    got = b.result()
    want = vt.tessellate_batch(dev(other), off, vt.Params(precision="fp32", emit=EMIT))  # synchronising schedule
    for name in ("vol", "cen", "m2", "nbr_off", "nbr"):
        assert torch.equal(getattr(got, name), getattr(want, name)), name
    snap = {k: getattr(got, k).clone() for k in ("vol", "nbr")}
    b.replay()
    again = b.result()
    assert torch.equal(again.vol, snap["vol"]) and torch.equal(again.nbr, snap["nbr"])


def test_no_sync_capacity_overflow_is_reported_then_grown(batch):
    pts, off, parts, want = batch
    b = vt.Batch(dev(pts), off, vt.Params(precision="fp64", emit=EMIT), nbr_per_cell=1)
    b.run()
    with pytest.raises(L.VtError) as e:
        b.result()
    assert e.value.code == L.VT_ERR_CAPACITY
    assert b.needed["nbr"] > len(pts)
    b.grow()
    b.run()
    cells = b.result()
    vol, cen, m2, lists = split(cells, off, 0)
    np.testing.assert_allclose(vol, want[0]["vol"], rtol=1e-12)


def test_no_sync_reports_bad_points():
    pts, off, _ = small_batch()
    pts = pts.copy()
    pts[5, 1] = np.float32(1.5)
    b = vt.Batch(dev(pts), off, vt.Params(precision="fp32"))
    b.run()
    with pytest.raises(L.VtError) as e:
        b.result()
    assert e.value.code == L.VT_ERR_INVALID_ARG


def test_sync_batch_grows_small_outputs_and_reports_passes(batch):
    pts, off, parts, want = batch
    cells = vt.tessellate_batch(dev(pts), off, vt.Params(precision="fp64", emit=EMIT + ("geom",), stage_times=True))
    assert cells.stats["passes"] >= 2 and cells.stats["ms_clip"] > 0
    vol, cen, m2, lists = split(cells, off, 5)
    np.testing.assert_allclose(vol, want[5]["vol"], rtol=1e-12)
    nv = np.diff(cells.vtx_off.cpu().numpy())
    assert nv.sum() == cells.vtx.shape[0]


def test_batch_plan_grids():
    off = [0, 1000, 1000, 9000]
    plan, cells = vt.batch_plan(off, vt.Params(), grid_res=[0, 0, 5])
    assert [plan[i].G for i in range(3)] == [vt.grid_resolution(vt.Params(), 1000), 1, 5]
    assert [plan[i].cell_base for i in range(3)] == [0, plan[0].G ** 3, plan[0].G ** 3 + 1]
    assert cells == plan[0].G ** 3 + 1 + 125


# --------------------------------------------------------------------------
# the 512-set workload (about 18M points), as the benchmark launches it
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big_batch():
    pts, off, coin = W.batch_sets()
    return pts, off, coin


def test_512_sets_graph_sampled_against_the_oracle(big_batch):
    pts, off, coin = big_batch
    b = vt.Batch(dev(pts), off, vt.Params(precision="fp32", emit=("nbr", "vol", "cen")))
    b.capture()
    b.replay()
    cells = b.result()
    vol = np_(cells.vol)
    # every set fills the unit box
    sums = np.add.reduceat(vol, off[:-1])
    assert np.abs(sums - 1.0).max() < 1e-6
    nbr_off, nbr = np_(cells.nbr_off), np_(cells.nbr)
    set_of = np.repeat(np.arange(len(off) - 1), np.diff(off))
    owner = np.repeat(np.arange(len(pts)), np.diff(nbr_off))
    assert np.array_equal(set_of[owner], set_of[nbr])  # neighbours stay in their set
    rng = np.random.default_rng(21)
    for s in rng.choice(len(off) - 1, 6, replace=False):
        a, z = off[s], off[s + 1]
        sample = np.sort(rng.choice(z - a, min(200, z - a), replace=False))
        w = oracle.tessellate(pts[a:z], cells=sample)
        np.testing.assert_allclose(vol[a + sample], w["vol"], rtol=1e-5)
        bad = 0
        for t, i in enumerate(sample):
            g = nbr[nbr_off[a + i]:nbr_off[a + i + 1]] - a
            bad += not np.array_equal(g, w["nbr"][w["nbr_off"][t]:w["nbr_off"][t + 1]])
        assert bad <= 2, (s, bad)
