"""Property search over small degenerate and near-degenerate inputs for the oracle.

Generators on coarse dyadic lattices (exact in float32) give many co-spherical
and coplanar configurations -- the degenerate cases of the method -- and
moving their coordinates by a few float32 ulps gives nearly degenerate ones.
For every drawn set, walled or periodic: the cells fill the box (volumes, and
first moment with walls), every cell has volume and Euler characteristic 2,
a neighbour pair listed on one side only is a face below the neighbour
threshold of the larger cell, and (walls) each centroid lies in its own
generator's cell by the nearest-generator rule. The search is derandomized,
so the cases are the same on every run.
"""
from collections import Counter

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies


@hyp.settings(max_examples=400, deadline=None, suppress_health_check=list(hyp.HealthCheck), derandomize=True)
@hyp.given(st.integers(2, 80), st.sampled_from([2, 3, 4, 8, 16]), st.integers(0, 2**31 - 1), st.booleans(),
           st.sampled_from([0, 1, 4, 64]))
def test_lattice_subsets_and_their_ulp_neighbours(n, m, seed, periodic, ulps):
    rng = np.random.default_rng(seed)
    cells = rng.choice(m ** 3, size=min(n, m ** 3), replace=False)
    pts = ((np.stack(np.unravel_index(cells, (m, m, m)), 1) + 0.5) / m).astype(np.float32)
    if ulps:
        k = rng.integers(-ulps, ulps + 1, size=pts.shape).astype(np.int32)
        pts = (pts.view(np.int32) + k).view(np.float32)
        pts = np.unique(np.clip(pts, 0, np.nextafter(np.float32(1), np.float32(0))), axis=0)
    r = oracle.tessellate(pts, periodic=periodic)
    vol = r["vol"]
    assert abs(vol.sum() - 1.0) < 1e-12
    assert np.all(vol > 0)
    assert np.all(r["euler"] == 2)
    if not periodic:
        np.testing.assert_allclose((vol[:, None] * r["cen"]).sum(0), 0.5, atol=1e-12)
    lists = oracle.neighbour_lists(r)
    fwd = Counter((i, int(j)) for i, lst in enumerate(lists) for j in lst)
    bwd = Counter((int(j), i) for i, lst in enumerate(lists) for j in lst)
    for i, j in (fwd - bwd) + (bwd - fwd):
        f0, f1 = r["face_off"][i], r["face_off"][i + 1]
        area = r["face_area"][f0:f1][r["face_tag"][f0:f1] == j]
        assert len(area) == 0 or area.min() < 1e-6 * max(vol[i], vol[j]) ** (2 / 3)
    if not periodic:
        p64 = pts.astype(np.float64)
        d = ((r["cen"][:, None, :] - p64[None, :, :]) ** 2).sum(2)
        assert np.all(np.diag(d) <= d.min(1) + 1e-12)
