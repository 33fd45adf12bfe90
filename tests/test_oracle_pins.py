"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks the oracle against mathematics the paper fixes (the Voronoi
cell is the box intersected with the bisector half-spaces, Statement of need
and Summary) by a route that does not reuse the oracle's code: closed forms
on lattices, a library routine (SciPy's Qhull), brute force, and invariants.
A plausible bug anywhere in the oracle -- a dropped clip, a wrong sign in the
bisector offset, a mis-oriented face, a bad security-radius stop, a broken
kNN tie order -- fails at least one of them.
"""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from paper_2412_04514_gb300 import workloads as W

UNIT_LO = (0.0, 0.0, 0.0)
UNIT_HI = (1.0, 1.0, 1.0)


def _nbr_sets(res):
    return [set(map(int, s)) for s in oracle.neighbour_lists(res)]


# --------------------------------------------------------------------------
# kNN (the oracle's own kd-tree) vs brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,k,seed", [(2, 1, 0), (7, 6, 1), (500, 16, 2), (1500, 40, 3)])
def test_knn_matches_brute_force(n, k, seed):
    p = W.uniform(n, seed)
    nbr, d2 = oracle.knn(p, k)
    p64 = p.astype(np.float64)
    for i in range(n):
        dx = p64[:, 0] - p64[i, 0]
        dy = p64[:, 1] - p64[i, 1]
        dz = p64[:, 2] - p64[i, 2]
        dd = (dx * dx + dy * dy) + dz * dz
        idx = np.arange(n)
        keep = idx != i
        order = np.lexsort((idx[keep], dd[keep]))
        want = idx[keep][order][:k]
        assert np.array_equal(nbr[i, : len(want)], want)
        assert np.array_equal(d2[i, : len(want)], dd[keep][order][:k])


def test_knn_tie_order_by_index():
    # points on a lattice have many exactly equal distances: ties must go by index
    p = W.cubic_lattice(4)
    nbr, d2 = oracle.knn(p, 12)
    for i in range(len(p)):
        for a in range(11):
            assert d2[i, a] < d2[i, a + 1] or (d2[i, a] == d2[i, a + 1] and nbr[i, a] < nbr[i, a + 1])


# --------------------------------------------------------------------------
# P1: security-radius path == clipping with every generator (any order)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 50, 500, 2000])
def test_security_radius_equals_brute_force(n):
    p = W.uniform(n, 100 + n)
    a = oracle.tessellate(p, k0=4 if n < 50 else 16)
    b = oracle.tessellate(p, mode="brute")
    order = np.random.default_rng(n).permutation(n)
    c = oracle.tessellate(p, mode="brute", order=order)
    for other in (b, c):
        np.testing.assert_allclose(a["vol"], other["vol"], rtol=1e-13, atol=0)
        np.testing.assert_allclose(a["cen"], other["cen"], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(a["m2"], other["m2"], rtol=1e-12, atol=0)
        assert _nbr_sets(a) == _nbr_sets(other)


def test_security_radius_on_clustered_input():
    p = W.mixed(3000, 7, n_clumps=5)
    a = oracle.tessellate(p)
    b = oracle.tessellate(p, mode="brute")
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-12, atol=0)
    assert _nbr_sets(a) == _nbr_sets(b)
    assert a["k_used"].max() > 16  # clump-edge cells needed k doubling


# --------------------------------------------------------------------------
# SciPy's Qhull with the points mirrored across the six walls
# --------------------------------------------------------------------------

def _qhull_cells(p):
    """Bounded Voronoi cells via scipy.spatial.Voronoi (Qhull).

    Mirroring every generator across each wall makes each wall the bisector
    of a generator and its image, so the Voronoi cell of an original
    generator in the augmented set is exactly its cell clipped to the box.
    Volume and centroid come from scipy.spatial.ConvexHull of the cell's
    vertices (a triangulated hull, integrated here by a fan from the hull's
    mean vertex).
    """
    from scipy.spatial import ConvexHull, Voronoi

    n = len(p)
    p64 = p.astype(np.float64)
    imgs = [p64]
    for axis in range(3):
        for wall in (0.0, 1.0):
            q = p64.copy()
            q[:, axis] = 2 * wall - q[:, axis]
            imgs.append(q)
    allp = np.concatenate(imgs)
    vor = Voronoi(allp)
    vols, cens, nbrs = np.zeros(n), np.zeros((n, 3)), [set() for _ in range(n)]
    for i in range(n):
        reg = vor.regions[vor.point_region[i]]
        assert -1 not in reg
        verts = vor.vertices[reg]
        hull = ConvexHull(verts)
        o = verts.mean(axis=0)
        tri = verts[hull.simplices]
        a, b, c = tri[:, 0] - o, tri[:, 1] - o, tri[:, 2] - o
        dv = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0
        vols[i] = dv.sum()
        cens[i] = o + (dv[:, None] * (a + b + c) / 4.0).sum(0) / vols[i]
    for (u, v) in vor.ridge_points:
        if u < n and v < n:
            nbrs[u].add(int(v))
            nbrs[v].add(int(u))
    return vols, cens, nbrs


@pytest.mark.parametrize("n,seed", [(300, 11), (1000, 12)])
def test_matches_qhull(n, seed):
    p = W.uniform(n, seed)
    r = oracle.tessellate(p)
    qv, qc, qn = _qhull_cells(p)
    np.testing.assert_allclose(r["vol"], qv, rtol=1e-9)
    np.testing.assert_allclose(r["cen"], qc, rtol=0, atol=1e-11)
    assert _nbr_sets(r) == qn


# --------------------------------------------------------------------------
# P2-P4: partition of the box, symmetry, Euler
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lo,hi", [(UNIT_LO, UNIT_HI), ((-2.0, 0.5, 1.0), (1.0, 0.75, 3.0))])
def test_cells_partition_the_box(lo, hi):
    lo_, hi_ = np.array(lo), np.array(hi)
    u = W.uniform(5000, 21)
    p = (lo_ + (hi_ - lo_) * u.astype(np.float64)).astype(np.float32)
    p = p[np.all((p >= lo_.astype(np.float32)) & (p < hi_.astype(np.float32)), axis=1)]
    r = oracle.tessellate(p, lo=lo, hi=hi)
    box_v = np.prod(hi_ - lo_)
    assert abs(r["vol"].sum() - box_v) <= 1e-12 * box_v
    first = (r["vol"][:, None] * r["cen"]).sum(0)
    np.testing.assert_allclose(first, box_v * (lo_ + hi_) / 2, rtol=1e-12)
    # every cell contains its generator's own position in its centroid's box
    assert np.all(r["vol"] > 0)


def test_neighbour_symmetry_and_shared_faces():
    p = W.mixed(4000, 5, n_clumps=20)
    r = oracle.tessellate(p)
    off, tag = r["face_off"], r["face_tag"]
    faces = {}
    for i in range(len(p)):
        for f in range(off[i], off[i + 1]):
            if tag[f] >= 0:
                faces[(i, int(tag[f]))] = (r["face_area"][f], r["face_cen"][f])
    sets = _nbr_sets(r)
    for i, s in enumerate(sets):
        for j in s:
            assert i in sets[j]
            ai, ci = faces[(i, j)]
            aj, cj = faces[(j, i)]
            assert abs(ai - aj) <= 1e-11 * max(ai, 1e-300) + 1e-18
            np.testing.assert_allclose(ci, cj, rtol=0, atol=1e-12)


def test_euler_characteristic():
    for p in (W.uniform(3000, 9), W.mixed(3000, 10, n_clumps=10), W.cubic_lattice(8), W.bcc_lattice(8)):
        r = oracle.tessellate(p)
        assert np.all(r["euler"] == 2)


# --------------------------------------------------------------------------
# P5-P7: closed forms
# --------------------------------------------------------------------------

def test_cubic_lattice_cells_are_cubes():
    m = 16
    p = W.cubic_lattice(m)
    r = oracle.tessellate(p)
    a = 1.0 / m
    np.testing.assert_allclose(r["vol"], a**3, rtol=0, atol=1e-14 * a**3)
    np.testing.assert_allclose(r["cen"], p.astype(np.float64), rtol=0, atol=1e-14)
    # second moment of a cube of side a about its centre: a^5 / 4
    np.testing.assert_allclose(r["m2"], a**5 / 4, rtol=1e-12)
    assert np.all(np.diff(r["face_off"]) == 6)
    np.testing.assert_allclose(r["face_area"], a * a, rtol=1e-13)
    # interior cells have exactly their 6 axis neighbours
    deg = np.diff(r["nbr_off"])
    ijk = np.rint(p.astype(np.float64) * m - 0.5).astype(int)
    interior = np.all((ijk > 0) & (ijk < m - 1), axis=1)
    assert np.all(deg[interior] == 6)


def test_bcc_lattice_interior_cells_are_truncated_octahedra():
    m = 16
    h = 1.0 / m
    p = W.bcc_lattice(m)
    r = oracle.tessellate(p)
    p64 = p.astype(np.float64)
    interior = np.all((p64 >= 1.5 * h) & (p64 <= 1 - 1.5 * h), axis=1)
    assert interior.sum() > 1000
    idx = np.flatnonzero(interior)
    np.testing.assert_allclose(r["vol"][idx], h**3 / 2, rtol=1e-13)
    np.testing.assert_allclose(r["cen"][idx], p64[idx], rtol=0, atol=1e-14)
    # dimensionless second moment of the truncated octahedron (the BCC
    # lattice quantiser constant, Conway & Sloane): 19 / (192 * 2^(1/3))
    G = r["m2"][idx] / (3 * r["vol"][idx] ** (5.0 / 3.0))
    np.testing.assert_allclose(G, 19.0 / (192.0 * 2.0 ** (1.0 / 3.0)), rtol=1e-12)
    off = r["face_off"]
    for i in idx[:200]:
        sizes = np.sort(r["face_size"][off[i]:off[i + 1]])
        assert list(sizes) == [4] * 6 + [6] * 8
    assert np.all(np.diff(r["nbr_off"])[idx] == 14)


def test_single_generator_is_the_box():
    p = np.array([[0.3, 0.6, 0.1]], dtype=np.float32)
    r = oracle.tessellate(p)
    assert r["vol"][0] == 1.0
    np.testing.assert_allclose(r["cen"][0], [0.5, 0.5, 0.5], atol=1e-15)
    assert len(r["nbr"]) == 0
    # second moment of the unit box about p: sum over axes of 1/3 - p + p^2
    pp = p[0].astype(np.float64)
    np.testing.assert_allclose(r["m2"][0], np.sum(1 / 3 - pp + pp * pp), rtol=1e-14)


def test_two_generators_axis_split():
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = np.sort(rng.random(2)).astype(np.float32)
        if x[0] == x[1]:
            continue
        y, z = rng.random(2).astype(np.float32)
        p = np.array([[x[0], y, z], [x[1], y, z]], dtype=np.float32)
        r = oracle.tessellate(p)
        mid = (np.float64(x[0]) + np.float64(x[1])) / 2
        np.testing.assert_allclose(r["vol"], [mid, 1 - mid], rtol=1e-14)
        np.testing.assert_allclose(r["cen"][0], [mid / 2, 0.5, 0.5], rtol=1e-13)
        np.testing.assert_allclose(r["cen"][1], [(1 + mid) / 2, 0.5, 0.5], rtol=1e-13)
        assert list(r["nbr"]) == [1, 0]


def test_two_generators_oblique_split():
    d = np.float32(0.125)
    p = np.array([[0.5 - d, 0.5 - d, 0.5], [0.5 + d, 0.5 + d, 0.5]], dtype=np.float32)
    r = oracle.tessellate(p)
    # plane x + y = 1: each half is a triangular prism with centroid (1/3, 1/3, 1/2)
    np.testing.assert_allclose(r["vol"], [0.5, 0.5], rtol=1e-15)
    np.testing.assert_allclose(r["cen"][0], [1 / 3, 1 / 3, 0.5], rtol=1e-14)
    np.testing.assert_allclose(r["cen"][1], [2 / 3, 2 / 3, 0.5], rtol=1e-14)


# --------------------------------------------------------------------------
# P8: every vertex is a Voronoi vertex (empty sphere), brute force
# --------------------------------------------------------------------------

def test_vertices_satisfy_the_empty_sphere_property():
    p = W.uniform(800, 31)
    r = oracle.tessellate(p, geometry=True)
    p64 = p.astype(np.float64)
    foff, fsize, tag, vtx = r["face_off"], r["face_size"], r["face_tag"], r["face_vtx"]
    vstart = np.concatenate([[0], np.cumsum(fsize)])
    for i in range(0, len(p), 7):
        for f in range(foff[i], foff[i + 1]):
            loop = vtx[vstart[f]:vstart[f + 1]]
            di = np.linalg.norm(loop - p64[i], axis=1)
            if tag[f] >= 0:  # the vertex is equidistant from p_i and p_j
                dj = np.linalg.norm(loop - p64[tag[f]], axis=1)
                np.testing.assert_allclose(dj, di, rtol=1e-11, atol=1e-14)
            dall = np.linalg.norm(loop[:, None, :] - p64[None, :, :], axis=2)
            assert np.all(dall.min(axis=1) >= di * (1 - 1e-11) - 1e-14)


# --------------------------------------------------------------------------
# P9: Poisson-Voronoi statistics (Meijering's closed forms)
# --------------------------------------------------------------------------

MEAN_FACES = 2.0 + 48.0 * np.pi ** 2 / 35.0  # 15.5355: mean faces of the typical Poisson-Voronoi cell
MEAN_VERTICES = 96.0 * np.pi ** 2 / 35.0  # 27.0709


def test_poisson_voronoi_mean_face_and_vertex_counts():
    """Uniform points are a Poisson-like process: the cells of generators
    4 mean spacings or more from every wall (chosen by position only, so the
    choice does not depend on the cells) are typical cells, whose mean face
    and vertex counts have Meijering's closed forms. Over ~360k such cells
    the standard error of the mean face count is about 0.005; each cell is
    also simple (three faces at every vertex), so V = 2F - 4 holds per cell."""
    n = 500_000
    p = W.uniform(n, 41)
    r = oracle.tessellate(p)
    h = n ** (-1.0 / 3.0)
    p64 = p.astype(np.float64)
    deep = np.all((p64 >= 4 * h) & (p64 <= 1 - 4 * h), axis=1)
    assert deep.sum() > 350_000
    nf = np.diff(r["face_off"])
    assert not np.any(r["face_tag"][np.repeat(deep, nf)] < 0)  # no deep cell reaches a wall
    faces, verts = nf[deep], r["nvert"][deep]
    assert abs(faces.mean() - MEAN_FACES) < 0.02, faces.mean()
    assert abs(verts.mean() - MEAN_VERTICES) < 0.04, verts.mean()
    np.testing.assert_array_equal(verts, 2 * faces - 4)


# --------------------------------------------------------------------------
# membership: random samples lie in the cell of their nearest generator
# --------------------------------------------------------------------------

def test_random_samples_fall_in_nearest_generators_cell():
    from scipy.spatial import cKDTree

    p = W.mixed(2000, 41, n_clumps=8)
    r = oracle.tessellate(p)
    x = np.random.default_rng(42).random((100_000, 3))
    _, owner = cKDTree(p.astype(np.float64)).query(x)
    off, plane = r["face_off"], r["face_plane"]
    p64 = p.astype(np.float64)
    counts = np.bincount(owner, minlength=len(p))
    for i in range(len(p)):
        xs = x[owner == i] - p64[i]
        pl = plane[off[i]:off[i + 1]]
        s = xs @ pl[:, :3].T - pl[:, 3]
        assert np.all(s <= 1e-12)
    # volume fractions agree with the sample counts (binomial error), for the
    # cells big enough to expect at least 100 samples
    expect = r["vol"] * len(x)
    big = expect >= 100
    assert big.sum() > 200
    z = (counts[big] - expect[big]) / np.sqrt(expect[big] * (1 - r["vol"][big]))
    assert np.abs(z).max() < 6.0


# --------------------------------------------------------------------------
# exact rational arithmetic: the oracle's FP64 volumes against the same
# cells solved exactly (vertices from three face planes, rational fan sums),
# on uniform cells and on tiny cells inside a dense clump, where rounding
# relative to the cell size matters most; every exact vertex also satisfies
# every face half-space of its cell
# --------------------------------------------------------------------------

def _clump_cloud():
    rng = np.random.default_rng(31)
    sparse = rng.random((6000, 3))
    dense = 0.5 + 1e-3 * rng.standard_normal((8000, 3))
    pts = np.unique(np.concatenate([sparse, dense]).astype(np.float32), axis=0)
    return pts[rng.permutation(len(pts))]


@pytest.mark.parametrize("which", ["uniform", "clump"])
def test_volumes_match_exact_rational_arithmetic(which):
    from exact_cells import exact_cell

    if which == "uniform":
        pts = W.uniform(3000, 12)
        cells = [3, 100, 2999]
    else:
        pts = _clump_cloud()
        cells = [419, 1048, 1088, 5]
    res = oracle.tessellate(pts, cells=cells, geometry=True)
    for a, i in enumerate(cells):
        vol, loops, planes = exact_cell(pts, i, res, a)
        assert abs(float((F(res["vol"][a]) - vol) / vol)) < 1e-14
        for loop in loops:
            for v in loop:
                assert all(sum(n[k] * v[k] for k in range(3)) <= b for n, b in planes)
