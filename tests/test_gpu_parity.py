"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (from the FP64 form's rounding and the stated FP32 target):
  * grid sort, FP64 kNN lists, FP64 neighbour sets: bit-exact;
  * FP64 volumes / centroids / second moments: 1e-12 relative;
  * FP32+FP64-recheck form: 1e-5 relative on volumes and centroids;
    neighbour sets equal except faces the oracle measures below 1e-6 V^(2/3)
    (a face that small is below float32 resolution of the cell).
"""
import ctypes
import warnings

import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from geometry_match import emitted_cell, match_cell, oracle_cell
from paper_2412_04514_gb300 import _lib as L
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def np_(t):
    return None if t is None else t.cpu().numpy()


def csr_lists(off, val):
    return [val[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def oracle_face_area(res, i, j):
    f0, f1 = res["face_off"][i], res["face_off"][i + 1]
    tags = res["face_tag"][f0:f1]
    w = np.flatnonzero(tags == j)
    return float(res["face_area"][f0 + w[0]]) if len(w) else 0.0


def check_fp64(cells, want, n_sample=None):
    np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(np_(cells.cen), want["cen"], rtol=1e-12, atol=1e-15)
    if cells.m2 is not None:
        np.testing.assert_allclose(np_(cells.m2), want["m2"], rtol=1e-11, atol=0)
    assert np.array_equal(np_(cells.nbr_off), want["nbr_off"])
    assert np.array_equal(np_(cells.nbr), want["nbr"])


def check_fp32(vol, cen, nbr_lists, want, cells_idx=None, max_bad_frac=1e-3):
    np.testing.assert_allclose(vol, want["vol"], rtol=1e-5, atol=0)
    rel_c = np.linalg.norm(cen - want["cen"], axis=1) / np.linalg.norm(want["cen"], axis=1)
    assert rel_c.max() < 1e-5, rel_c.max()
    wl = oracle.neighbour_lists(want)
    bad = 0
    for a, (g, w) in enumerate(zip(nbr_lists, wl)):
        if not np.array_equal(g, w):
            bad += 1
            i = a
            V = want["vol"][a]
            for j in set(w.tolist()) ^ set(g.tolist()):
                assert oracle_face_area(want, i, j) < 1e-6 * V ** (2 / 3), (i, j)
    assert bad <= max(2, max_bad_frac * len(wl)), bad


# --------------------------------------------------------------------------
# stage 1: grid sort
# --------------------------------------------------------------------------

@pytest.mark.parametrize("maker", [lambda: W.uniform(4096, 0), lambda: W.mixed(300_000, 1), lambda: W.uniform(7, 3)])
def test_grid_build_is_bit_exact(maker):
    pts = maker()
    sorted_, perm, off, G, _ = vt.grid_build(dev(pts))
    g = oracle.grid_sort(pts, G)
    assert np.array_equal(np_(perm), g["perm"])
    assert np.array_equal(np_(off).astype(np.int64), g["cell_off"])
    s = np_(sorted_)
    assert np.array_equal(s[:, :3], g["sorted"])
    assert np.array_equal(s[:, 3].view(np.int32), g["perm"].astype(np.int32))


def test_grid_build_with_huge_cells():
    # one grid cell holds thousands of points: the block-wide fix-up sort
    rng = np.random.default_rng(9)
    pts = (0.5 + 1e-4 * rng.standard_normal((20000, 3))).astype(np.float32)
    pts = np.unique(pts, axis=0)
    pts = pts[rng.permutation(len(pts))]
    sorted_, perm, off, G, _ = vt.grid_build(dev(pts), vt.Params(grid_res=8))
    g = oracle.grid_sort(pts, G)
    assert np.array_equal(np_(perm), g["perm"])
    assert np.array_equal(np_(off).astype(np.int64), g["cell_off"])


# --------------------------------------------------------------------------
# stage 2: kNN
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 16, 32, 50, 128, 256])
def test_knn_fp64_is_exact(k):
    pts = W.uniform(4096, 0)
    p = vt.Params(precision="fp64")
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    nbr, d2 = vt.knn(sorted_, off, G, k, p, workspace=ws)
    perm_ = np_(perm)
    got = perm_[np_(nbr)]
    want, wd2 = oracle.knn(pts, k, queries=perm_)
    assert np.array_equal(got, want)
    assert np.array_equal(np_(d2), wd2)


@pytest.mark.parametrize("k", [6, 26, 64])
def test_knn_fp64_exact_with_exact_ties(k):
    # lattice points: many candidates at exactly equal FP64 distances, so the
    # list order rests on the FP64 keys and the index tie-break, not on the
    # float32 keys the kNN orders by first
    pts = W.bcc_lattice(8)
    p = vt.Params(precision="fp64")
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    nbr, d2 = vt.knn(sorted_, off, G, k, p, workspace=ws)
    perm_ = np_(perm)
    want, wd2 = oracle.knn(pts, k, queries=perm_)
    assert np.array_equal(perm_[np_(nbr)], want)
    assert np.array_equal(np_(d2), wd2)


def test_knn_fp64_exact_on_clustered_points_with_query_list():
    pts = W.mixed(50_000, 2, n_clumps=50)
    p = vt.Params(precision="fp64")
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    q = torch.arange(0, len(pts), 7, dtype=torch.int32, device="cuda")
    nbr, d2 = vt.knn(sorted_, off, G, 64, p, queries=q, workspace=ws)
    perm_ = np_(perm)
    want, wd2 = oracle.knn(pts, 64, queries=perm_[np_(q)])
    assert np.array_equal(perm_[np_(nbr)], want)
    assert np.array_equal(np_(d2), wd2)


def test_knn_fp32_matches_fp64_up_to_near_ties():
    pts = W.uniform(20000, 4)
    p = vt.Params(precision="fp32")
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    nbr, d2 = vt.knn(sorted_, off, G, 16, p, workspace=ws)
    perm_ = np_(perm)
    want, wd2 = oracle.knn(pts, 16, queries=perm_)
    np.testing.assert_allclose(np_(d2), wd2, rtol=2e-6)
    same = np.all(perm_[np_(nbr)] == want, axis=1)
    assert same.mean() > 0.999


def test_knn_fewer_points_than_k():
    pts = W.uniform(5, 1)
    p = vt.Params(precision="fp64")
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    nbr, d2 = vt.knn(sorted_, off, G, 8, p, workspace=ws)
    nb = np_(nbr)
    assert np.all(nb[:, 4:] == -1) and np.all(np.isinf(np_(d2)[:, 4:]))
    assert np.all(nb[:, :4] >= 0)


# --------------------------------------------------------------------------
# whole path, FP64 form: bit-exact neighbours, 1e-12 moments
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg0():
    pts = W.uniform(4096, 0)
    return pts, oracle.tessellate(pts, k0=16, geometry=True)


def test_fp64_uniform_4096(cfg0):
    pts, want = cfg0
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "cen", "m2")))
    check_fp64(cells, want)
    st = cells.stats
    assert st["k_of_pass"][0] == 16 and st["unvalidated"] == 0


@pytest.mark.parametrize("tpc", [8, 16, 32])
def test_fp32_uniform_4096(cfg0, tpc):
    pts, want = cfg0
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp32", threads_per_cell=tpc, emit=("nbr", "vol", "cen")))
    check_fp32(np_(cells.vol), np_(cells.cen), csr_lists(np_(cells.nbr_off), np_(cells.nbr)), want)


@pytest.mark.parametrize("tpc", [8, 32])
def test_fp64_threads_per_cell(cfg0, tpc):
    pts, want = cfg0
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", threads_per_cell=tpc, emit=("nbr", "vol", "cen")))
    check_fp64(cells, want)


@pytest.fixture(scope="module")
def clustered():
    pts = W.mixed(40_000, 3, n_clumps=40)
    return pts, oracle.tessellate(pts, k0=16)


def test_fp64_clustered_runs_every_pass(clustered):
    pts, want = clustered
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", k_max=256, emit=("nbr", "vol", "cen", "m2")))
    check_fp64(cells, want)
    st = cells.stats
    assert st["k_of_pass"][:5] == [16, 32, 64, 128, 256]
    assert st["exhaustive_cells"] > 0 and st["k_of_pass"][-1] == 0


@pytest.mark.parametrize("k0,k_max", [(16, 16), (16, 32), (32, 64)])
def test_pass_policies_agree(clustered, k0, k_max):
    pts, want = clustered
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", k0=k0, k_max=k_max, emit=("nbr", "vol", "cen")))
    check_fp64(cells, want)


def test_fp32_clustered(clustered):
    pts, want = clustered
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp32", emit=("nbr", "vol", "cen")))
    check_fp32(np_(cells.vol), np_(cells.cen), csr_lists(np_(cells.nbr_off), np_(cells.nbr)), want)


def test_lattices_fp64():
    for pts in (W.cubic_lattice(16), W.bcc_lattice(12)):
        want = oracle.tessellate(pts)
        cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "cen")))
        check_fp64(cells, want)


def test_lattices_fp32():
    pts = W.cubic_lattice(16)
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp32", emit=("nbr", "vol", "cen")))
    np.testing.assert_allclose(np_(cells.vol), 16.0**-3, rtol=1e-5)
    np.testing.assert_allclose(np_(cells.cen), pts, rtol=1e-5)


def test_geometry_fp64_matches_oracle(cfg0):
    pts, want = cfg0
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "geom")))
    geo = tuple(np_(t) for t in (cells.vtx_off, cells.vtx, cells.face_off, cells.face_nbr, cells.face_vtx_off,
                                 cells.face_vtx))
    p64 = pts.astype(np.float64)
    for i in range(0, len(pts), 5):
        V, faces = emitted_cell(geo, i)
        assert len(V) == want["nvert"][i]
        # one-to-one vertex pairing and the same cyclic loop per face, by id
        W_, wfaces = oracle_cell(want, i)
        match_cell(V, faces, W_, wfaces, 1e-13)
        for tag, loop in faces:
            P = V[loop]
            # counter-clockwise seen from outside: Newell normal points away from the generator
            nrm = np.cross(P - p64[i], np.roll(P, -1, axis=0) - p64[i]).sum(0)
            assert nrm @ (P.mean(0) - p64[i]) > 0


def test_sorted_index_space(cfg0):
    pts, want = cfg0
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", index_space="sorted", emit=("nbr", "vol")),
                          want_perm=True)
    perm = np_(cells.perm)
    np.testing.assert_allclose(np_(cells.vol), want["vol"][perm], rtol=1e-12)
    lists = csr_lists(np_(cells.nbr_off), np_(cells.nbr))
    wl = oracle.neighbour_lists(want)
    for a in range(0, len(pts), 11):
        assert sorted(perm[lists[a]].tolist()) == wl[perm[a]].tolist()
        assert np.all(np.diff(lists[a]) > 0)


def test_stage_calls_and_exhaustive_mode(cfg0):
    pts, want = cfg0
    p = vt.Params(precision="fp64", emit=("vol", "cen"))
    sorted_, perm, off, G, ws = vt.grid_build(dev(pts), p)
    # exhaustive mode (no list) gives every cell directly
    cells, failed, _ = vt.clip_cells(sorted_, off, G, None, None, p, workspace=ws)
    assert failed.numel() == 0
    np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-12)
    # list mode with k = 64: the cells that fail are exactly those the oracle needed k > 64 for
    nbr, d2 = vt.knn(sorted_, off, G, 64, p, workspace=ws)
    cells, failed, _ = vt.clip_cells(sorted_, off, G, nbr, d2, p, workspace=ws)
    failed_orig = np.sort(np_(perm)[np_(failed)])
    assert np.array_equal(failed_orig, np.flatnonzero(want["k_used"] > 64))
    ok = np.isfinite(np_(cells.vol))
    np.testing.assert_allclose(np_(cells.vol)[ok], want["vol"][ok], rtol=1e-12)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_empty_and_tiny_inputs():
    for n in (0, 1, 2, 3, 9):
        pts = W.uniform(n, 50 + n) if n else np.zeros((0, 3), np.float32)
        for prec in ("fp64", "fp32"):
            cells = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=("nbr", "vol", "cen")))
            assert np_(cells.nbr_off).shape == (n + 1,)
            if n:
                want = oracle.tessellate(pts, k0=16)
                np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-5 if prec == "fp32" else 1e-12)
                assert np.array_equal(np_(cells.nbr), want["nbr"])


def test_general_box():
    lo, hi = (-2.0, 0.5, 1.0), (1.0, 0.75, 3.0)
    u = W.uniform(3000, 8).astype(np.float64)
    pts = (np.array(lo) + (np.array(hi) - np.array(lo)) * u).astype(np.float32)
    pts = pts[np.all((pts >= np.float32(lo)) & (pts < np.float32(hi)), axis=1)]
    want = oracle.tessellate(pts, lo=lo, hi=hi)
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", box_lo=lo, box_hi=hi, emit=("nbr", "vol", "cen")))
    check_fp64(cells, want)


@pytest.mark.parametrize("bad", ["nan", "outside", "upper"])
def test_invalid_points_are_rejected(bad):
    pts = W.uniform(100, 2)
    pts[37] = {"nan": [np.nan, 0.5, 0.5], "outside": [0.5, -0.1, 0.5], "upper": [0.5, 0.5, 1.0]}[bad]
    with pytest.raises(L.VtError) as e:
        vt.tessellate(dev(pts))
    assert e.value.code == L.VT_ERR_INVALID_ARG
    assert "37" in str(e.value)


def test_duplicate_points_are_rejected():
    pts = W.uniform(100, 2)
    pts[50] = pts[10]
    for prec in ("fp64", "fp32"):
        with pytest.raises(L.VtError) as e:
            vt.tessellate(dev(pts), vt.Params(precision=prec))
        assert e.value.code == L.VT_ERR_DUPLICATE_POINTS


def test_small_output_capacity_goes_through_emit(cfg0):
    pts, want = cfg0
    p = vt.Params(precision="fp64", emit=("nbr", "vol"))
    ws = vt.Workspace(p, len(pts))
    cells = vt.tessellate(dev(pts), p, workspace=ws)
    again = vt.emit(len(pts), p, ws, guess={"nbr": 10})
    assert np.array_equal(np_(again.nbr), want["nbr"])
    assert np.array_equal(np_(cells.nbr), want["nbr"])


# --------------------------------------------------------------------------
# the benchmark workload (1M half uniform, half clustered) on sampled cells
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def bench_1m():
    pts = W.mixed(1 << 20, 1)
    sample = np.sort(np.random.default_rng(11).choice(len(pts), 3000, replace=False))
    return pts, sample, oracle.tessellate(pts, k0=16, cells=sample)


def test_bench_workload_fp64_sampled(bench_1m):
    pts, sample, want = bench_1m
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "cen", "m2")))
    np.testing.assert_allclose(np_(cells.vol)[sample], want["vol"], rtol=1e-12)
    np.testing.assert_allclose(np_(cells.cen)[sample], want["cen"], rtol=1e-12)
    np.testing.assert_allclose(np_(cells.m2)[sample], want["m2"], rtol=1e-11)
    lists = csr_lists(np_(cells.nbr_off), np_(cells.nbr))
    for a, i in enumerate(sample):
        assert np.array_equal(lists[i], want["nbr"][want["nbr_off"][a]:want["nbr_off"][a + 1]])
    assert abs(np_(cells.vol).sum() - 1.0) < 1e-9


def test_bench_workload_fp32_sampled(bench_1m):
    pts, sample, want = bench_1m
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp32", emit=("nbr", "vol", "cen")))
    lists = csr_lists(np_(cells.nbr_off), np_(cells.nbr))
    check_fp32(np_(cells.vol)[sample], np_(cells.cen)[sample], [lists[i] for i in sample], want)
    assert abs(np_(cells.vol).sum() - 1.0) < 1e-6


# --------------------------------------------------------------------------
# sparse cells next to a dense clump: thousands of generators lie within
# twice their radius, so they reach the exhaustive pass, and clipped in walk
# order the clump's bisectors would overflow the polyhedron; the robust
# variant clips by a nearest-first list before its walk
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def clump_cloud():
    rng = np.random.default_rng(31)
    sparse = rng.random((6000, 3))
    dense = 0.5 + 1e-3 * rng.standard_normal((8000, 3))
    pts = np.unique(np.concatenate([sparse, dense]).astype(np.float32), axis=0)
    pts = pts[rng.permutation(len(pts))]
    return pts, oracle.tessellate(pts)


@pytest.mark.parametrize("no_sync", [False, True])
def test_sparse_cells_next_to_a_dense_clump_fp64(clump_cloud, no_sync):
    pts, want = clump_cloud
    assert want["k_used"].max() >= 1024  # the workload has the hard cells
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp64", emit=("nbr", "vol", "cen", "m2"), no_sync=no_sync))
    assert cells.stats["unvalidated"] == 0
    check_fp64(cells, want)


def test_sparse_cells_next_to_a_dense_clump_fp32(clump_cloud):
    pts, want = clump_cloud
    cells = vt.tessellate(dev(pts), vt.Params(precision="fp32"))
    check_fp32(np_(cells.vol), np_(cells.cen), csr_lists(np_(cells.nbr_off), np_(cells.nbr)), want)


def test_host_outputs_written_directly_equal_device_outputs():
    # the neighbour and geometry arrays written by the emit kernel straight
    # into pinned host memory are the same bytes as the device-emitted copies
    pts = W.mixed(30_000, 33, n_clumps=20)
    p = vt.Params(precision="fp32", emit=("nbr", "vol", "cen", "m2", "geom"))
    direct = vt.tessellate_host(pts, p, direct=True)
    copied = vt.tessellate_host(pts, p, direct=False)
    for name in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                 "face_vtx"):
        a, b = getattr(direct, name), getattr(copied, name)
        assert not a.is_cuda and not b.is_cuda
        assert torch.equal(a, b), name
    host = vt.tessellate(dev(pts), p, host_csr=True)
    assert not host.nbr.is_cuda and host.nbr.is_pinned() and host.vol.is_cuda
    assert torch.equal(host.nbr, copied.nbr) and torch.equal(host.vol.cpu(), copied.vol)


def test_pageable_host_outputs_are_refused_before_any_launch():
    # a plain (pageable) host array is not memory device code can use on every
    # system: the library checks the output pointers first and returns an
    # argument error without launching; where the system does map such memory
    # for the device, the call must give the same cells as device outputs
    pts = W.uniform(2000, 34)
    d = dev(pts)
    p = vt.Params(precision="fp64", emit=("nbr", "vol"))
    want = vt.tessellate(d, p)
    lib = L.load()
    ws = vt.Workspace(p, len(pts))
    vol = torch.zeros(len(pts), dtype=torch.float64)  # pageable host memory
    nbr_off = torch.zeros(len(pts) + 1, dtype=torch.int64, device="cuda")
    nbr = torch.zeros(40 * len(pts), dtype=torch.int32, device="cuda")
    o = L.VtCellsOut()
    o.vol, o.nbr_off, o.nbr, o.nbr_cap = vol.data_ptr(), nbr_off.data_ptr(), nbr.data_ptr(), nbr.numel()
    st = L.VtStats()
    code = lib.vt_tessellate(d.data_ptr(), len(pts), ctypes.byref(p.c()), ctypes.byref(o), ctypes.byref(st),
                             ws.buf.data_ptr(), ws.buf.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if code == L.VT_ERR_INVALID_ARG:
        assert "device-accessible" in lib.vt_last_error().decode()
        assert torch.count_nonzero(vol) == 0
    else:
        assert code == L.VT_OK
        assert torch.equal(vol, want.vol.cpu())


def test_tessellate_stream_equals_one_call_at_a_time():
    # the pipelined stream (copy in / tessellate / copy back on three streams)
    # yields, in order, the cells of every cloud, bit-identical to single calls;
    # a change of cloud size re-sizes the workspace on the way
    clouds = [W.mixed(20_000, 35, n_clumps=10), W.uniform(20_000, 36), W.uniform(5_000, 37),
              W.mixed(20_000, 38, n_clumps=4)]
    p = vt.Params(precision="fp32", emit=("nbr", "vol", "cen", "geom"))
    got = list(vt.tessellate_stream(clouds, p))
    assert len(got) == len(clouds)
    for cloud, g in zip(clouds, got):
        want = vt.tessellate_host(cloud, p)
        for name in ("vol", "cen", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx"):
            assert torch.equal(getattr(g, name), getattr(want, name)), name
    assert list(vt.tessellate_stream([], p)) == []


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["plane", "line"])
def test_coplanar_and_collinear_generators(prec, shape):
    # every cell reaches the box walls (prisms over the plane's 2D cells, or
    # slabs along the line), so every security radius is large and the cells
    # are finished by the exhaustive walk
    rng = np.random.default_rng(39)
    n = 1500 if shape == "plane" else 300
    pts = np.full((n, 3), 0.5, dtype=np.float64)
    pts[:, 0] = rng.random(n)
    if shape == "plane":
        pts[:, 1] = rng.random(n)
    pts = np.unique(pts.astype(np.float32), axis=0)
    want = oracle.tessellate(pts)
    with warnings.catch_warnings(record=True) as caught:
        warnings.simplefilter("always")
        cells = vt.tessellate(dev(pts), vt.Params(precision=prec, emit=("nbr", "vol", "cen")))
    assert cells.stats["status"] == "VT_OK"
    # every cell walks the shells within 2R in the last pass (range lists, and
    # the clipper's walk when they overflow), examining about every generator:
    # reported (above a floor of 1,000 per walk, so the 300-point line is not)
    assert cells.stats["walk_cells"] > 0.9 * len(pts)
    assert cells.stats["walk_candidates"] > 0.25 * len(pts) * cells.stats["walk_cells"]
    warned = [w for w in caught if issubclass(w.category, RuntimeWarning) and "degenerate" in str(w.message)]
    assert len(warned) == (1 if shape == "plane" else 0)
    assert abs(np_(cells.vol).sum() - 1.0) < (1e-12 if prec == "fp64" else 1e-5)
    if prec == "fp64":
        np.testing.assert_allclose(np_(cells.vol), want["vol"], rtol=1e-12)
        assert np.array_equal(np_(cells.nbr_off), want["nbr_off"]) and np.array_equal(np_(cells.nbr), want["nbr"])
    else:
        check_fp32(np_(cells.vol), np_(cells.cen), csr_lists(np_(cells.nbr_off), np_(cells.nbr)), want)
    if shape == "line":  # slabs: two neighbours each, one at the ends
        counts = np.diff(np_(cells.nbr_off))
        assert counts.max() == 2 and (counts == 1).sum() == 2
