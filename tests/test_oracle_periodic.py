"""Pins of the oracle's periodic mode against things other than itself.

In a periodic box every generator repeats at p + t L (L = hi - lo). The
periodic cell of p_i is therefore the non-periodic cell of p_i among all
images. The strongest pin computes exactly that with the (separately pinned)
non-periodic oracle on a cloud replicated 5 x 5 x 5 times. Dyadic coordinates
make the replication exact in float32. The other pins are closed forms on
lattices, the volume of the torus, the symmetry of two generators,
translation invariance, matching faces seen from both sides, SciPy's periodic
kd-tree as the owner of random samples, a brute-force image kNN, and the
Poisson-Voronoi mean face and vertex counts.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2412_04514_gb300 import workloads as W


def dyadic(n, seed, L=(1.0, 1.0, 1.0), bits=20):
    """n distinct points of [0, L) whose coordinates are multiples of 2^-bits."""
    rng = np.random.default_rng(seed)
    scale = float(1 << bits)
    pts = np.floor(rng.random((4 * n + 16, 3)) * np.asarray(L) * scale) / scale
    pts = np.unique(pts.astype(np.float32), axis=0)
    return pts[rng.permutation(len(pts))[:n]]


def replicate(p, L, reach=2):
    """Copies p + t L for t in [-reach, reach]^3; copy c of point j is row c * n + j,
    the unshifted copy is c0."""
    shifts = list(itertools.product(range(-reach, reach + 1), repeat=3))
    Lv = np.asarray(L, dtype=np.float32)
    reps = [p + np.asarray(t, dtype=np.float32) * Lv for t in shifts]
    c0 = shifts.index((0, 0, 0))
    return np.concatenate(reps).astype(np.float32), c0


def multisets(res):
    return [sorted(map(int, s)) for s in oracle.neighbour_lists(res)]


# --------------------------------------------------------------------------
# the periodic cell is the non-periodic cell among the replicated images
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed,L", [(1, 0, (1, 1, 1)), (2, 1, (1, 1, 1)), (3, 2, (1, 1, 1)), (7, 3, (1, 1, 1)),
                                      (20, 4, (1, 1, 1)), (60, 5, (1, 1, 1)), (9, 6, (1.0, 1.0, 0.875)),
                                      (40, 7, (1.0, 0.875, 1.0))])
def test_periodic_equals_replicated_non_periodic(n, seed, L):
    p = dyadic(n, seed, L)
    n = len(p)
    rep, c0 = replicate(p, L)
    lo = tuple(-2.0 * a for a in L)
    hi = tuple(3.0 * a for a in L)
    central = np.arange(c0 * n, (c0 + 1) * n)
    want = oracle.tessellate(rep, lo=lo, hi=hi, cells=central)
    got = oracle.tessellate(p, hi=L, periodic=True)
    np.testing.assert_allclose(got["vol"], want["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["cen"], want["cen"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(got["m2"], want["m2"], rtol=1e-11, atol=0)
    assert multisets(got) == [sorted(int(j) % n for j in s) for s in oracle.neighbour_lists(want)]
    # the face of image (j, t) is the face of copy (t, j) in the replicated cloud
    shifts = list(itertools.product(range(-2, 3), repeat=3))
    for i in range(n):
        f0, f1 = got["face_off"][i], got["face_off"][i + 1]
        g0, g1 = want["face_off"][i], want["face_off"][i + 1]
        t = oracle.img_shift(got["face_img"][f0:f1])
        copy = [shifts.index(tuple(int(a) for a in row)) for row in t]
        tags = sorted(zip((np.asarray(copy) * n + got["face_tag"][f0:f1]).tolist(), got["face_area"][f0:f1]))
        ref = sorted(zip(want["face_tag"][g0:g1].tolist(), want["face_area"][g0:g1]))
        assert [a for a, _ in tags] == [a for a, _ in ref]
        np.testing.assert_allclose([b for _, b in tags], [b for _, b in ref], rtol=1e-10, atol=1e-14)


def test_brute_force_equals_security_radius_path():
    p = W.uniform(40, 11)
    a = oracle.tessellate(p, periodic=True)
    b = oracle.tessellate(p, periodic=True, mode="brute")
    c = oracle.tessellate(p, periodic=True, mode="brute", order=np.random.default_rng(3).permutation(len(p)))
    for r in (b, c):
        np.testing.assert_allclose(a["vol"], r["vol"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(a["cen"], r["cen"], rtol=0, atol=1e-13)
        assert multisets(a) == multisets(r)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lo,hi", [((0, 0, 0), (1, 1, 1)), ((-1.0, 0.0, 2.0), (0.5, 1.25, 3.375))])
def test_cells_fill_the_torus(lo, hi):
    L = np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)
    p = W.uniform(3000, 12, lo=0.0, hi=1.0).astype(np.float64) * L + np.asarray(lo)
    p = np.minimum(p.astype(np.float32), np.nextafter(np.asarray(hi, dtype=np.float32), -np.inf))
    r = oracle.tessellate(p, lo=lo, hi=hi, periodic=True)
    assert abs(r["vol"].sum() - np.prod(L)) <= 1e-12 * np.prod(L)
    assert np.all(r["euler"] == 2)
    assert np.all(r["vol"] > 0)


def test_single_generator_is_the_cube_around_it():
    p = np.array([[0.1, 0.7, 0.25]], dtype=np.float32)
    r = oracle.tessellate(p, periodic=True, geometry=True)
    assert r["vol"][0] == pytest.approx(1.0, rel=1e-15)
    np.testing.assert_allclose(r["cen"][0], p[0].astype(np.float64), atol=1e-15)
    assert r["nbr"].tolist() == [0] * 6
    assert sorted(r["face_img"].tolist()) == sorted(oracle.img_code(np.vstack([np.eye(3), -np.eye(3)])).tolist())
    v = r["face_vtx"]
    np.testing.assert_allclose(v.min(0), p[0] - 0.5, atol=1e-15)
    np.testing.assert_allclose(v.max(0), p[0] + 0.5, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_two_generators_split_the_torus_in_halves(seed):
    # x -> p + q - x maps the periodic pattern onto itself and swaps the two
    # generators, so both cells have volume 1/2
    p = W.uniform(2, 20 + seed)
    r = oracle.tessellate(p, periodic=True)
    np.testing.assert_allclose(r["vol"], [0.5, 0.5], rtol=1e-13)
    assert r["euler"].tolist() == [2, 2]


def test_offset_cubic_lattice_cells_are_cubes():
    m = 8
    a = (np.arange(m) * 4 + 1) / (4.0 * m)  # (a + 1/4) / m, exact in float32
    p = np.array(list(itertools.product(a, a, a)), dtype=np.float32)
    r = oracle.tessellate(p, periodic=True)
    np.testing.assert_allclose(r["vol"], 1.0 / m ** 3, rtol=1e-13)
    np.testing.assert_allclose(r["cen"], p.astype(np.float64), atol=1e-15)
    counts = np.diff(r["nbr_off"])
    assert np.all(counts == 6)
    # the six neighbours are the lattice neighbours across the wrap
    idx = {tuple(np.round(q * 4 * m).astype(int)): i for i, q in enumerate(p)}
    for i, q in enumerate(p):
        c = np.round(q * 4 * m).astype(int)
        want = sorted(idx[tuple((c + 4 * d) % (4 * m))] for d in np.vstack([np.eye(3, dtype=int), -np.eye(3, dtype=int)]))
        assert r["nbr"][r["nbr_off"][i]:r["nbr_off"][i + 1]].tolist() == want


def test_bcc_lattice_every_cell_is_a_truncated_octahedron():
    m = 8
    h = 1.0 / m
    a = (np.arange(m) + 0.25) * h
    b = (np.arange(m) + 0.75) * h
    p = np.array(list(itertools.product(a, a, a)) + list(itertools.product(b, b, b)), dtype=np.float32)
    r = oracle.tessellate(p, periodic=True)
    np.testing.assert_allclose(r["vol"], h ** 3 / 2, rtol=1e-13)
    np.testing.assert_allclose(r["cen"], p.astype(np.float64), atol=1e-15)
    off = r["face_off"]
    tau = 1e-12 * (h ** 3 / 2) ** (2 / 3)
    for i in range(len(p)):
        sizes = r["face_size"][off[i]:off[i + 1]][r["face_area"][off[i]:off[i + 1]] > tau]
        assert sorted(sizes.tolist()) == [4] * 6 + [6] * 8


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_translation_invariance():
    p = dyadic(400, 30)
    r = oracle.tessellate(p, periodic=True)
    s = np.array([0.3125, 0.8671875, 0.5], dtype=np.float64)
    q = np.mod(p.astype(np.float64) + s, 1.0).astype(np.float32)  # exact: dyadic coordinates
    rq = oracle.tessellate(q, periodic=True)
    np.testing.assert_allclose(rq["vol"], r["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(rq["cen"] - q.astype(np.float64), r["cen"] - p.astype(np.float64), atol=1e-13)
    assert multisets(rq) == multisets(r)


def test_faces_match_from_both_sides():
    p = W.mixed(1500, 31, n_clumps=6)
    r = oracle.tessellate(p, periodic=True)
    off = r["face_off"]
    faces = {}
    for i in range(len(p)):
        for f in range(off[i], off[i + 1]):
            faces[(i, int(r["face_tag"][f]), int(r["face_img"][f]))] = r["face_area"][f]
    for (i, j, c), area in faces.items():
        back = faces.get((j, i, int(oracle.img_code(-oracle.img_shift(c)))))
        if back is None:
            assert area < 1e-12 * r["vol"][i] ** (2 / 3)
        else:
            assert abs(back - area) <= 1e-10 * max(area, 1e-30) + 1e-18


def test_random_samples_fall_in_nearest_image_cell():
    from scipy.spatial import cKDTree

    p = W.mixed(2000, 32, n_clumps=8)
    r = oracle.tessellate(p, periodic=True)
    x = np.random.default_rng(33).random((100_000, 3))
    p64 = p.astype(np.float64)
    _, owner = cKDTree(p64, boxsize=1.0).query(x)
    off, plane = r["face_off"], r["face_plane"]
    for i in np.unique(owner):
        d = x[owner == i] - p64[i]
        d -= np.round(d)  # the image of p_i nearest to the sample
        pl = plane[off[i]:off[i + 1]]
        assert np.all(d @ pl[:, :3].T - pl[:, 3] <= 1e-12)
    counts = np.bincount(owner, minlength=len(p))
    expect = r["vol"] * len(x)
    big = expect >= 100
    assert big.sum() > 200
    z = (counts[big] - expect[big]) / np.sqrt(expect[big] * (1 - r["vol"][big]))
    assert np.abs(z).max() < 6.0


# --------------------------------------------------------------------------
# periodic kNN vs brute force over every image
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,k,L", [(3, 20, (1, 1, 1)), (300, 32, (1, 1, 1)), (500, 16, (1.0, 0.875, 1.0))])
def test_knn_periodic_matches_brute_force(n, k, L):
    p = dyadic(n, 40 + n, L) if n < 10 else (W.uniform(n, 40 + n) * np.asarray(L, dtype=np.float32))
    p = np.minimum(p, np.nextafter(np.asarray(L, dtype=np.float32), -np.inf))
    nbr, img, d2 = oracle.knn_periodic(p, k, hi=L)
    p64 = p.astype(np.float64)
    Lv = np.asarray(L, dtype=np.float64)
    t = oracle.img_shift(np.arange(125))
    for i in range(len(p)):
        # offsets ((x_j - x_i) + t L), keys ((dx dx + dy dy) + dz dz), all images but i's own
        off = (p64[None, :, :] - p64[i]) + (t[:, None, :] * Lv)
        dd = (off[..., 0] * off[..., 0] + off[..., 1] * off[..., 1]) + off[..., 2] * off[..., 2]
        code = np.repeat(np.arange(125), len(p))
        gen = np.tile(np.arange(len(p)), 125)
        dd = dd.reshape(-1)
        keep = gen != i
        order = np.lexsort((code[keep], gen[keep], dd[keep]))[:k]
        assert np.array_equal(nbr[i], gen[keep][order])
        assert np.array_equal(img[i], code[keep][order])
        assert np.array_equal(d2[i], dd[keep][order])


def test_rejects_boxes_too_elongated_for_two_periods():
    p = W.uniform(10, 50) * np.float32(0.5)
    with pytest.raises(oracle.OracleError):
        oracle.tessellate(p, hi=(1.0, 1.0, 0.5), periodic=True)  # |L|^2 = 2.25 > 4 * 0.25
    r = oracle.tessellate(p, hi=(0.5, 0.5, 0.5), periodic=True)
    assert abs(r["vol"].sum() - 0.125) < 1e-14


def test_non_periodic_faces_have_no_shift():
    r = oracle.tessellate(W.uniform(200, 51))
    assert np.all(r["face_img"] == 62)


def test_every_periodic_cell_is_a_typical_poisson_voronoi_cell():
    """On the torus a uniform cloud has no boundary, so every cell counts
    towards the typical cell's statistics (Meijering: mean faces
    2 + 48 pi^2 / 35, mean vertices 96 pi^2 / 35), and every cell is simple,
    V = 2F - 4."""
    p = W.uniform(300_000, 43)
    r = oracle.tessellate(p, periodic=True)
    faces, verts = np.diff(r["face_off"]), r["nvert"]
    assert np.all(r["face_tag"] >= 0)
    assert abs(faces.mean() - (2.0 + 48.0 * np.pi ** 2 / 35.0)) < 0.02, faces.mean()
    assert abs(verts.mean() - 96.0 * np.pi ** 2 / 35.0) < 0.04, verts.mean()
    np.testing.assert_array_equal(verts, 2 * faces - 4)
