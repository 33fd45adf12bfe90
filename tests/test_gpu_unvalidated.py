"""Cells the device cannot finish are reported, marked and listed, never wrong.

A generator at the centre of the box surrounded by 100 generators on a sphere
has a cell with 100 faces and 196 vertices (V = 2F - 4), more than the
largest clipping variant holds (128 vertex slots). Every other cell is
ordinary. Both forms and both schedules must return VT_ERR_UNVALIDATED for
that one cell, give its id through vt_unvalidated_cells, write NaN into its
volume, centroid and second moment, leave it without neighbours, and match
the FP64 oracle on every other cell (paper, Summary: a validated cell is the
exact cell).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import workloads as W
from paper_2412_04514_gb300._lib import VtError

pytestmark = pytest.mark.gpu


def sphere_cloud():
    m = 100
    i = np.arange(m) + 0.5
    phi = np.arccos(1 - 2 * i / m)
    th = np.pi * (1 + 5 ** 0.5) * i
    shell = 0.5 + 0.08 * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    rest = W.uniform(4000, 7).astype(np.float64)
    rest = rest[np.linalg.norm(rest - 0.5, axis=1) > 0.2][:1500]
    pts = np.concatenate([[[0.5, 0.5, 0.5]], shell, rest]).astype(np.float32)
    return pts


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("no_sync", [False, True])
def test_oversized_cell_is_reported_and_marked(precision, no_sync):
    pts = sphere_cloud()
    n = len(pts)
    want = oracle.tessellate(pts)
    assert want["nbr_off"][1] - want["nbr_off"][0] == 100  # the centre cell has a face per shell point
    d = torch.from_numpy(pts).cuda()
    p = vt.Params(precision=precision, emit=("nbr", "vol", "cen", "m2"), no_sync=no_sync)
    with pytest.raises(VtError, match="VT_ERR_UNVALIDATED"):
        vt.tessellate(d, p)
    cells = vt.tessellate(d, p, strict=False)
    assert cells.stats["status"] == "VT_ERR_UNVALIDATED"
    assert cells.stats["unvalidated"] == 1
    assert cells.unvalidated.cpu().tolist() == [0]
    vol, cen, m2 = cells.vol.cpu().numpy(), cells.cen.cpu().numpy(), cells.m2.cpu().numpy()
    assert np.isnan(vol[0]) and np.isnan(cen[0]).all() and np.isnan(m2[0])
    off = cells.nbr_off.cpu().numpy()
    assert off[1] == off[0]
    tol = 1e-12 if precision == "fp64" else 1e-5
    np.testing.assert_allclose(vol[1:], want["vol"][1:], rtol=tol)
    np.testing.assert_allclose(cen[1:], want["cen"][1:], rtol=tol)
    np.testing.assert_allclose(m2[1:], want["m2"][1:], rtol=10 * tol)
    nbr = cells.nbr.cpu().numpy()
    for i in range(1, n):
        got = nbr[off[i]:off[i + 1]]
        ref = want["nbr"][want["nbr_off"][i]:want["nbr_off"][i + 1]]
        if precision == "fp64":
            assert np.array_equal(got, ref), i
    # the validated cells and the oracle's centre cell fill the box
    assert abs(vol[1:].sum() + want["vol"][0] - 1.0) < tol


def test_sorted_index_space_lists_sorted_ids():
    pts = sphere_cloud()
    d = torch.from_numpy(pts).cuda()
    cells = vt.tessellate(d, vt.Params(precision="fp64", index_space="sorted"), strict=False, want_perm=True)
    ids = cells.unvalidated.cpu().numpy()
    perm = cells.perm.cpu().numpy()
    assert len(ids) == 1 and perm[ids[0]] == 0
    assert np.isnan(cells.vol.cpu().numpy()[ids[0]])


def test_validated_run_lists_nothing():
    d = torch.from_numpy(W.uniform(2048, 3)).cuda()
    cells = vt.tessellate(d, vt.Params(precision="fp32"))
    assert cells.stats["status"] == "VT_OK" and cells.unvalidated.numel() == 0
    assert not torch.isnan(cells.vol).any()
