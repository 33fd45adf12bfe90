"""Pins of the oracle's moments adjoint (oracle/adjoint.py).

Each pin comes from outside the adjoint code: the exact integrals of
barycentric monomials, the Lloyd identity d(sum M2)/dp_k = 2 V_k (p_k - c_k)
(face terms of neighbouring cells cancel because |x - p_i| = |x - p_j| on a
shared face), conservation of total volume and first moment (the box does not
move), and central finite differences of the oracle's own tessellation.
"""
from math import factorial

import numpy as np
import pytest

import oracle
from oracle import adjoint as adj
from paper_2412_04514_gb300 import workloads as W


def _bary_monomial_exact(area, a, b, c):
    # integral over a triangle of l1^a l2^b l3^c dA = 2 A a! b! c! / (a + b + c + 2)!
    return 2 * area * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)


def test_triangle_rule_is_exact_to_degree_three_only():
    rng = np.random.default_rng(3)
    A, B, C = rng.random((3, 1, 3))
    pts, w = adj.triangle_rule(A, B, C)
    area = w.sum()
    # barycentric coordinates of the quadrature points
    M = np.stack([A[0], B[0], C[0]], axis=1)
    lam = np.linalg.lstsq(M, pts[0].T, rcond=None)[0].T
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                got = np.sum(w[0] * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c)
                assert abs(got - _bary_monomial_exact(area, a, b, c)) < 1e-14
    got4 = np.sum(w[0] * lam[:, 0] ** 4)
    assert abs(got4 - _bary_monomial_exact(area, 4, 0, 0)) > 1e-6 * area


@pytest.fixture(scope="module")
def cloud():
    p = W.uniform(600, 5)
    return p, oracle.tessellate(p, geometry=True)


def test_lloyd_gradient_closed_form(cloud):
    p, res = cloud
    g = adj.moments_adjoint(p, gM=np.ones(len(p)), res=res)
    want = 2 * res["vol"][:, None] * (p.astype(np.float64) - res["cen"])
    np.testing.assert_allclose(g, want, rtol=1e-9, atol=1e-15)


def test_total_volume_and_first_moment_are_conserved(cloud):
    p, res = cloud
    n = len(p)
    g = adj.moments_adjoint(p, gV=np.ones(n), res=res)
    assert np.abs(g).max() < 1e-13
    for a in range(3):
        e = np.zeros((n, 3))
        e[:, a] = res["vol"]
        g = adj.moments_adjoint(p, gV=res["cen"][:, a], gC=e, res=res)
        assert np.abs(g).max() < 1e-13


def test_matches_central_finite_differences():
    n = 256
    p = W.uniform(n, 5)
    rng = np.random.default_rng(55)
    gV, gC, gM = rng.standard_normal(n), rng.standard_normal((n, 3)), rng.standard_normal(n)
    res = oracle.tessellate(p, geometry=True)
    g = adj.moments_adjoint(p, gV, gC, gM, res=res)
    nbrs = oracle.neighbour_lists(res)
    h = 1e-4

    def central(k, a, hh, cells):
        pp, pm = p.copy(), p.copy()
        pp[k, a] = np.float32(p[k, a] + hh)
        pm[k, a] = np.float32(p[k, a] - hh)
        step = np.float64(pp[k, a]) - np.float64(pm[k, a])
        return (adj.loss(pp, gV, gC, gM, cells=cells) - adj.loss(pm, gV, gC, gM, cells=cells)) / step

    for k in rng.choice(n, 8, replace=False):
        cells = np.unique(np.concatenate([[k], nbrs[k]]))  # the cells that move with p_k
        for a in range(3):
            # central differences with h = 1e-4 and h/2, one Richardson step to
            # cancel the h^2 truncation term (small cells curve fast)
            d1, d2 = central(k, a, h, cells), central(k, a, h / 2, cells)
            fd = (4 * d2 - d1) / 3
            assert abs(fd - g[k, a]) <= 1e-6 * max(1.0, abs(g[k, a])), (k, a, fd, g[k, a])
            assert abs(d1 - g[k, a]) <= 1e-4 * max(1.0, abs(g[k, a]))


# --------------------------------------------------------------------------
# periodic box: the same identities, the neighbour across a face being the
# image its shift names
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def periodic_cloud():
    p = W.mixed(500, 6, n_clumps=4)
    return p, oracle.tessellate(p, geometry=True, periodic=True)


def test_periodic_lloyd_gradient_closed_form(periodic_cloud):
    p, res = periodic_cloud
    g = adj.moments_adjoint(p, gM=np.ones(len(p)), res=res, periodic=True)
    want = 2 * res["vol"][:, None] * (p.astype(np.float64) - res["cen"])
    np.testing.assert_allclose(g, want, rtol=1e-9, atol=1e-15)


def test_periodic_total_volume_is_conserved(periodic_cloud):
    p, res = periodic_cloud
    g = adj.moments_adjoint(p, gV=np.ones(len(p)), res=res, periodic=True)
    assert np.abs(g).max() < 1e-13


def test_periodic_matches_central_finite_differences():
    n = 200
    p = W.uniform(n, 7)
    rng = np.random.default_rng(56)
    gV, gC, gM = rng.standard_normal(n), rng.standard_normal((n, 3)), rng.standard_normal(n)
    res = oracle.tessellate(p, geometry=True, periodic=True)
    g = adj.moments_adjoint(p, gV, gC, gM, res=res, periodic=True)
    nbrs = oracle.neighbour_lists(res)
    h = 1e-4
    # generators whose cells reach across the box's faces (the wrapped images matter)
    near_wall = np.flatnonzero(np.any((p < 0.15) | (p > 0.85), axis=1) & np.all((p > 2 * h) & (p < 1 - 2 * h), axis=1))

    def central(k, a, hh, cells):
        pp, pm = p.copy(), p.copy()
        pp[k, a] = np.float32(p[k, a] + hh)
        pm[k, a] = np.float32(p[k, a] - hh)
        step = np.float64(pp[k, a]) - np.float64(pm[k, a])
        return (adj.loss(pp, gV, gC, gM, cells=cells, periodic=True)
                - adj.loss(pm, gV, gC, gM, cells=cells, periodic=True)) / step

    for k in rng.choice(near_wall, 8, replace=False):
        cells = np.unique(np.concatenate([[k], nbrs[k]]))
        for a in range(3):
            d1, d2 = central(k, a, h, cells), central(k, a, h / 2, cells)
            fd = (4 * d2 - d1) / 3
            assert abs(fd - g[k, a]) <= 1e-6 * max(1.0, abs(g[k, a])), (k, a, fd, g[k, a])
