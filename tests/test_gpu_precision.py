"""The precision workload at full size: 8,388,608 points of the mixed recipe
(half uniform, half in 1,000 clumps), the FP32 form (float32 kNN and
clipping, FP64 security radius, near-zero sign rechecks and accumulation)
and the plain FP64 form, each against the FP64 oracle on the cells of a
seeded sub-box holding about 65,536 generators, in the launch configuration
the benchmark times (32 lanes per cell, k0 16 doubled to k_max 32, two
points per grid cell, geometry emitted).

Tolerances: FP64 form -- neighbours exact, volumes and centroids 1e-12
relative; FP32 form -- volumes and centroids 1e-5 relative, neighbour lists
equal except faces the oracle measures below 1e-6 V^(2/3).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def bench_params(precision):
    return vt.Params(precision=precision, k0=16, k_max=32, threads_per_cell=32, grid_density=2.0,
                     emit=("nbr", "vol", "cen", "geom"))


@pytest.fixture(scope="module")
def cloud8m():
    pts = W.mixed(1 << 23, 2)
    idx = W.sub_box_cells(pts, 65536, 17)
    assert abs(len(idx) - 65536) <= 656
    return pts, idx, oracle.tessellate(pts, cells=idx)


def _lists(cells, idx):
    off, nbr = cells.nbr_off.cpu().numpy(), cells.nbr.cpu().numpy()
    return [nbr[off[i]:off[i + 1]] for i in idx]


def _face_area(w, a, j):
    f0, f1 = w["face_off"][a], w["face_off"][a + 1]
    hit = np.flatnonzero(w["face_tag"][f0:f1] == j)
    return float(w["face_area"][f0 + hit[0]]) if len(hit) else 0.0


def test_fp64_form_on_the_sub_box(cloud8m):
    pts, idx, w = cloud8m
    cells = vt.tessellate(torch.from_numpy(pts).cuda(), bench_params("fp64"))
    np.testing.assert_allclose(cells.vol.cpu().numpy()[idx], w["vol"], rtol=1e-12)
    np.testing.assert_allclose(cells.cen.cpu().numpy()[idx], w["cen"], rtol=1e-12)
    for a, g in enumerate(_lists(cells, idx)):
        assert np.array_equal(g, w["nbr"][w["nbr_off"][a]:w["nbr_off"][a + 1]])
    assert abs(float(cells.vol.sum()) - 1.0) < 1e-9


def test_fp32_form_on_the_sub_box(cloud8m):
    pts, idx, w = cloud8m
    cells = vt.tessellate(torch.from_numpy(pts).cuda(), bench_params("fp32"))
    vol = cells.vol.cpu().numpy()[idx]
    cen = cells.cen.cpu().numpy()[idx]
    np.testing.assert_allclose(vol, w["vol"], rtol=1e-5)
    rc = np.linalg.norm(cen - w["cen"], axis=1) / np.linalg.norm(w["cen"], axis=1)
    assert rc.max() < 1e-5
    bad = 0
    for a, g in enumerate(_lists(cells, idx)):
        ww = w["nbr"][w["nbr_off"][a]:w["nbr_off"][a + 1]]
        if not np.array_equal(g, ww):
            bad += 1
            for j in set(g.tolist()) ^ set(ww.tolist()):
                assert _face_area(w, a, j) < 1e-6 * w["vol"][a] ** (2 / 3)
    assert bad <= 1e-3 * len(idx)
    assert cells.stats["unvalidated"] == 0
