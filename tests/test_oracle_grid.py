"""Pins of the oracle's grid counting sort (paper, Summary: the points are
sorted into a grid before the neighbour search).

The grid sort's definition: cell id from a float32 floor of the scaled
coordinate (z fastest), per-cell counts, exclusive prefix sum, stable order.
These tests check it against exact rational arithmetic away from cell
boundaries and against a pure-Python stable bucket sort.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2412_04514_gb300 import workloads as W


@pytest.mark.parametrize("G", [1, 3, 7, 16])
def test_cell_ids_match_exact_floor_away_from_boundaries(G):
    p = W.uniform(3000, G)
    cid = oracle.grid_cell_ids(p, G)
    for i in range(len(p)):
        ijk = []
        near = False
        for a in range(3):
            t = Fraction(float(p[i, a])) * G
            f = int(t)  # floor for t >= 0
            if abs(t - round(t)) < Fraction(1, 10**5):
                near = True
            ijk.append(min(G - 1, f))
        if not near:
            assert cid[i] == (ijk[0] * G + ijk[1]) * G + ijk[2]


def test_cell_ids_general_box_and_clamp():
    lo, hi = (-1.0, 2.0, 0.0), (1.0, 3.0, 0.5)
    p = np.array([[-1.0, 2.0, 0.0], [0.999999, 2.999999, 0.4999999], [0.0, 2.5, 0.25]], dtype=np.float32)
    cid = oracle.grid_cell_ids(p, 4, lo, hi)
    assert list(cid) == [0, 63, (2 * 4 + 2) * 4 + 2]


@pytest.mark.parametrize("n,G", [(0, 3), (1, 1), (50, 2), (777, 5)])
def test_stable_counting_sort_matches_bucket_sort(n, G):
    p = W.uniform(n, 7) if n else np.zeros((0, 3), np.float32)
    g = oracle.grid_sort(p, G)
    cid = g["cid"]
    buckets = [[] for _ in range(G**3)]
    for i in range(n):  # pure-Python stable bucket sort
        buckets[int(cid[i])].append(i)
    perm = [i for b in buckets for i in b]
    off = [0]
    for b in buckets:
        off.append(off[-1] + len(b))
    assert list(g["perm"]) == perm
    assert list(g["cell_off"]) == off
    assert np.array_equal(g["sorted"], p[perm] if n else p)


def test_clustered_sort_invariants():
    p = W.mixed(20000, 3, n_clumps=30)
    G = oracle.grid_resolution(len(p), 2.0)
    g = oracle.grid_sort(p, G)
    cs = g["cid"][g["perm"]]
    assert np.all(np.diff(cs) >= 0)
    same = np.diff(cs) == 0
    assert np.all(np.diff(g["perm"])[same] > 0)  # stable inside a cell
    assert np.array_equal(np.sort(g["perm"]), np.arange(len(p)))
    assert g["cell_off"][-1] == len(p)


def test_grid_resolution():
    assert oracle.grid_resolution(0, 2.0) == 1
    assert oracle.grid_resolution(1, 2.0) == 1
    assert oracle.grid_resolution(16, 2.0) == 2
    assert oracle.grid_resolution(1 << 20, 2.0) == 81
    assert oracle.grid_resolution(1 << 23, 2.0) == 162
