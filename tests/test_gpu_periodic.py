"""Periodic boxes on the GPU (VT_FLAG_PERIODIC) against the oracle's periodic mode.

Tolerances as for the non-periodic box: the FP64 form's neighbour multisets
are exact and its moments agree to 1e-12 relative; the FP32 form's moments
agree to 1e-5 relative, and its neighbours differ only by faces the oracle
measures below 1e-6 V^(2/3). Cases: uniform and wrapped-clump clouds, sets of
one to twenty points (shells wider than the box, faces on the cell's own
images), offset lattices whose every cell is a closed form, a box that is
neither the unit cube nor at the origin, the kNN lists, batches, the no-sync
schedule, the geometry, the adjoint and Lloyd's iteration.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from oracle import adjoint as oadj
from paper_2412_04514_gb300 import _lib as L
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMIT = ("nbr", "vol", "cen", "m2")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def np_(t):
    return None if t is None else t.cpu().numpy()


def lists(off, val):
    return [sorted(val[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def run(pts, prec, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), emit=EMIT, **kw):
    return vt.tessellate(dev(pts), vt.Params(precision=prec, emit=emit, periodic=True, box_lo=lo, box_hi=hi, **kw))


def check_fp64(cells, want):
    np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(np_(cells.cen), want["cen"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(np_(cells.m2), want["m2"], rtol=1e-11, atol=0)
    assert lists(np_(cells.nbr_off), np_(cells.nbr)) == lists(want["nbr_off"], want["nbr"])


def check_fp32(cells, want, max_bad=1e-3):
    vol, cen = np_(cells.vol), np_(cells.cen)
    np.testing.assert_allclose(vol, want["vol"], rtol=1e-5, atol=0)
    scale = np.cbrt(want["vol"])[:, None]
    assert (np.abs(cen - want["cen"]) / scale).max() < 1e-5
    got = lists(np_(cells.nbr_off), np_(cells.nbr))
    ref = lists(want["nbr_off"], want["nbr"])
    bad = 0
    for i, (g, w) in enumerate(zip(got, ref)):
        if g == w:
            continue
        bad += 1
        # every differing neighbour is a face the oracle measures as tiny
        f0, f1 = want["face_off"][i], want["face_off"][i + 1]
        tiny = 1e-6 * want["vol"][i] ** (2 / 3)
        for j in set(g) ^ set(w) or set(g):
            areas = want["face_area"][f0:f1][want["face_tag"][f0:f1] == j]
            assert len(areas) == 0 or areas.min() < tiny, (i, j, areas)
    assert bad <= max(2, max_bad * len(got))


# --------------------------------------------------------------------------
# parity with the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("cloud", ["uniform", "clumps"])
def test_periodic_matches_the_oracle(prec, cloud):
    pts = W.uniform(4096, 60) if cloud == "uniform" else W.mixed(30_000, 61, n_clumps=25, periodic=True)
    want = oracle.tessellate(pts, periodic=True)
    cells = run(pts, prec)
    assert cells.stats["status"] == "VT_OK"
    (check_fp64 if prec == "fp64" else check_fp32)(cells, want)
    assert abs(np_(cells.vol).sum() - 1.0) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 20, 60])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_tiny_sets(n, prec):
    # a handful of points: shells wider than the box, several images of one
    # generator as faces, and (n = 1) the cube of the cell's own images
    pts = W.uniform(n, 70 + n)
    want = oracle.tessellate(pts, periodic=True)
    cells = run(pts, prec)
    assert cells.stats["status"] == "VT_OK"
    if prec == "fp64":
        check_fp64(cells, want)
    else:
        np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-5)
        assert lists(np_(cells.nbr_off), np_(cells.nbr)) == lists(want["nbr_off"], want["nbr"])
    if n == 1:
        assert np_(cells.nbr).tolist() == [0] * 6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_offset_lattices(prec):
    m = 8
    a = (np.arange(m) * 4 + 1) / (4.0 * m)
    cubic = np.array(np.meshgrid(a, a, a, indexing="ij")).reshape(3, -1).T.astype(np.float32)
    cells = run(cubic, prec)
    tol = 1e-12 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(np_(cells.vol), 1.0 / m ** 3, rtol=tol)
    np.testing.assert_allclose(np_(cells.cen), cubic.astype(np.float64), atol=tol / m)
    assert np.all(np.diff(np_(cells.nbr_off)) == 6)
    h = 1.0 / m
    b = (np.arange(m) + 0.25) * h
    c = (np.arange(m) + 0.75) * h
    bcc = np.concatenate([np.array(np.meshgrid(b, b, b, indexing="ij")).reshape(3, -1).T,
                          np.array(np.meshgrid(c, c, c, indexing="ij")).reshape(3, -1).T]).astype(np.float32)
    cells = run(bcc, prec)
    np.testing.assert_allclose(np_(cells.vol), h ** 3 / 2, rtol=tol)
    assert np.all(np.diff(np_(cells.nbr_off)) == 14)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_box_off_the_origin(prec):
    lo, hi = (-1.0, 0.0, 2.0), (0.0, 1.0, 2.875)
    L_ = np.subtract(hi, lo)
    pts = (W.uniform(5000, 80).astype(np.float64) * L_ + lo).astype(np.float32)
    pts = np.minimum(pts, np.nextafter(np.asarray(hi, np.float32), -np.inf))
    want = oracle.tessellate(pts, lo=lo, hi=hi, periodic=True)
    cells = run(pts, prec, lo=lo, hi=hi)
    (check_fp64 if prec == "fp64" else check_fp32)(cells, want)


def test_periodic_geometry_and_sorted_index_space():
    pts = W.mixed(6000, 81, n_clumps=6, periodic=True)
    want = oracle.tessellate(pts, periodic=True, geometry=True)
    cells = run(pts, "fp64", emit=("nbr", "vol", "geom"))
    vo, v = np_(cells.vtx_off), np_(cells.vtx)
    fo, fn = np_(cells.face_off), np_(cells.face_nbr)
    p64 = pts.astype(np.float64)
    for i in range(0, len(pts), 97):
        # unwrapped vertices around the generator, one for each of the oracle's
        got = v[vo[i]:vo[i + 1]]
        wv = want["face_vtx"][np.sum(want["face_size"][:want["face_off"][i]]):
                              np.sum(want["face_size"][:want["face_off"][i + 1]])]
        ref = np.unique(wv, axis=0)  # the oracle repeats each vertex once per face, bit-identical
        assert len(got) == len(ref)
        dist = np.linalg.norm(got[:, None, :] - ref[None, :, :], axis=2)
        assert dist.min(axis=1).max() < 1e-10 and dist.min(axis=0).max() < 1e-10
        assert np.abs(got - p64[i]).max() <= 0.5 + 1e-12  # inside the cube of one period around p_i
        assert sorted(fn[fo[i]:fo[i + 1]].tolist()) == sorted(want["face_tag"][want["face_off"][i]:want["face_off"][i + 1]].tolist())
    # the sorted index space maps back through perm to the same neighbours
    s = vt.tessellate(dev(pts), vt.Params(precision="fp64", periodic=True, index_space="sorted"), want_perm=True)
    perm = np_(s.perm)
    ref = lists(want["nbr_off"], want["nbr"])
    got = lists(np_(s.nbr_off), np_(s.nbr))
    for si in range(0, len(pts), 53):
        assert sorted(perm[got[si]].tolist()) == ref[perm[si]]


# --------------------------------------------------------------------------
# kNN lists: packed image codes, exact FP64 keys
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [16, 64])
def test_periodic_knn_fp64_is_exact(k):
    pts = W.mixed(8000, 82, n_clumps=8, periodic=True)
    p = vt.Params(precision="fp64", periodic=True)
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    nbr, d2 = vt.knn(sorted_, off, G, k, p, workspace=ws)
    perm_ = np_(perm)
    e = np_(nbr)
    got_j = perm_[e & ((1 << 24) - 1)]
    got_c = (e.astype(np.int64) >> 24) & 127
    want, wimg, wd2 = oracle.knn_periodic(pts, k, queries=perm_)
    assert np.array_equal(got_j, want)
    assert np.array_equal(got_c, wimg)
    assert np.array_equal(np_(d2), wd2)


# --------------------------------------------------------------------------
# batches and the no-sync schedule
# --------------------------------------------------------------------------

@pytest.mark.parametrize("no_sync", [False, True])
def test_periodic_batch_matches_the_oracle_per_set(no_sync):
    parts = [W.uniform(2000, 90), W.uniform(1, 91), W.mixed(6000, 92, n_clumps=6, periodic=True), W.uniform(7, 93)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    pts = np.concatenate(parts).astype(np.float32)
    cells = vt.tessellate_batch(dev(pts), off, vt.Params(precision="fp64", emit=EMIT, periodic=True, no_sync=no_sync))
    vol, nbo, nb = np_(cells.vol), np_(cells.nbr_off), np_(cells.nbr)
    for s, part in enumerate(parts):
        want = oracle.tessellate(part, periodic=True)
        a, b = off[s], off[s + 1]
        np.testing.assert_allclose(vol[a:b], want["vol"], rtol=1e-12)
        got = [sorted((nb[nbo[i]:nbo[i + 1]] - a).tolist()) for i in range(a, b)]
        assert got == lists(want["nbr_off"], want["nbr"])


def test_periodic_no_sync_fp32():
    pts = W.mixed(20_000, 94, n_clumps=20, periodic=True)
    want = oracle.tessellate(pts, periodic=True)
    cells = run(pts, "fp32", no_sync=True)
    check_fp32(cells, want)


# --------------------------------------------------------------------------
# adjoint and Lloyd
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_adjoint_matches_the_oracle(prec):
    pts = W.mixed(3000, 95, n_clumps=5, periodic=True)
    rng = np.random.default_rng(96)
    n = len(pts)
    gV, gC, gM = rng.standard_normal(n), rng.standard_normal((n, 3)), rng.standard_normal(n)
    want = oadj.moments_adjoint(pts, gV, gC, gM, periodic=True)
    p = vt.Params(precision=prec, emit=("vol", "cen", "m2", "geom"), periodic=True)
    d = dev(pts)
    cells = vt.tessellate(d, p)
    got = vt.moments_adjoint(d, cells, dev(gV), dev(gC), dev(gM), precision=prec, params=p).cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= (1e-9 if prec == "fp64" else 2e-4) * scale


def test_periodic_lloyd_decreases_energy_and_stays_in_the_box():
    pts = W.mixed(20_000, 97, n_clumps=30, periodic=True)
    p = vt.Params(precision="fp32", periodic=True)
    energies = []
    out = vt.lloyd(dev(pts), 8, p, callback=lambda it, e: energies.append(e))
    q = np_(out)
    assert np.all(q >= 0.0) and np.all(q < 1.0)
    assert all(b < a for a, b in zip(energies, energies[1:]))
    # the relaxed cloud is a valid periodic tessellation with the oracle's cells
    want = oracle.tessellate(q, periodic=True)
    check_fp32(run(q, "fp32"), want)


def test_periodic_rejects_an_elongated_box():
    pts = (W.uniform(100, 98) * np.float32(0.5)).astype(np.float32)
    with pytest.raises(L.VtError):
        run(pts, "fp32", hi=(1.0, 1.0, 0.5))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_lattice_on_the_box_faces(prec):
    # points exactly on the faces and on grid-cell boundaries (a / m, a = 0..m-1):
    # images land exactly on the other faces, ties everywhere; every cell is a cube
    m = 8
    a = np.arange(m) / m
    pts = np.array(np.meshgrid(a, a, a, indexing="ij")).reshape(3, -1).T.astype(np.float32)
    want = oracle.tessellate(pts, periodic=True)
    np.testing.assert_allclose(want["vol"], 1.0 / m ** 3, rtol=1e-13)
    cells = run(pts, prec, grid_res=m)
    tol = 1e-12 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(np_(cells.vol), 1.0 / m ** 3, rtol=tol)
    np.testing.assert_allclose(np_(cells.cen), pts.astype(np.float64), atol=tol / m)
    assert lists(np_(cells.nbr_off), np_(cells.nbr)) == lists(want["nbr_off"], want["nbr"])
