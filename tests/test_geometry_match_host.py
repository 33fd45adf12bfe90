"""The vertex-matching geometry check used by the GPU parity tests, on the CPU.

The cells are the oracle's own (FP64, paper Summary: each cell is the box cut
by bisector planes), re-indexed the way the library emits them (a vertex
array and per-face loops of indices into it). The check must accept the same
polyhedron under any vertex order and loop start, and reject what a
per-coordinate sorted comparison lets through: a coordinate moved from one
vertex to another, a face loop in the wrong orientation, a face with another
neighbour's id, a vertex moved by more than the tolerance.
"""
import numpy as np
import pytest

import oracle
from geometry_match import match_cell, oracle_cell
from paper_2412_04514_gb300 import workloads as W


@pytest.fixture(scope="module")
def cells():
    pts = W.uniform(400, 9)
    want = oracle.tessellate(pts, geometry=True)
    return [oracle_cell(want, a) for a in range(0, 400, 7)]


def relabel(V, faces, rng):
    """The same polyhedron with shuffled vertex indices and rotated loops."""
    perm = rng.permutation(len(V))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(V))
    out = []
    for tag, loop in faces:
        k = int(rng.integers(len(loop)))
        out.append((tag, np.roll(inv[loop], -k)))
    order = rng.permutation(len(out))
    return V[perm], [out[i] for i in order]


def test_accepts_the_same_cell_in_any_order(cells):
    rng = np.random.default_rng(0)
    for V, faces in cells:
        Vr, fr = relabel(V, faces, rng)
        match_cell(Vr, fr, V, faces, 1e-12)


def test_rejects_a_coordinate_moved_between_vertices(cells):
    rng = np.random.default_rng(1)
    for V, faces in cells:
        Vr, fr = relabel(V, faces, rng)
        bad = Vr.copy()
        j = int(np.argmax(np.abs(bad[:, 0] - bad[0, 0])))  # a vertex with another x
        bad[[0, j], 0] = bad[[j, 0], 0]
        # a per-axis sorted comparison cannot tell the difference
        np.testing.assert_array_equal(np.sort(bad, axis=0), np.sort(V, axis=0))
        with pytest.raises(AssertionError):
            match_cell(bad, fr, V, faces, 1e-12)


def test_rejects_a_reversed_face_loop(cells):
    rng = np.random.default_rng(2)
    for V, faces in cells:
        Vr, fr = relabel(V, faces, rng)
        fr = list(fr)
        tag, loop = fr[0]
        fr[0] = (tag, loop[::-1])
        with pytest.raises(AssertionError):
            match_cell(Vr, fr, V, faces, 1e-12)


def test_rejects_a_face_with_another_id(cells):
    rng = np.random.default_rng(3)
    for V, faces in cells:
        Vr, fr = relabel(V, faces, rng)
        fr = list(fr)
        (t0, l0), (t1, l1) = fr[0], fr[1]
        fr[0], fr[1] = (t1, l0), (t0, l1)
        with pytest.raises(AssertionError):
            match_cell(Vr, fr, V, faces, 1e-12)


def test_rejects_a_vertex_beyond_the_tolerance(cells):
    rng = np.random.default_rng(4)
    for V, faces in cells:
        Vr, fr = relabel(V, faces, rng)
        bad = Vr.copy()
        bad[3, 2] += 1e-9
        match_cell(bad, fr, V, faces, 1e-8)
        with pytest.raises(AssertionError):
            match_cell(bad, fr, V, faces, 1e-10)
