"""The autotuner on the GPU: the clustering statistic it keys on against the
oracle (bit-exact: integer pair counts, then the same FP64 formula), the tuner
returning a candidate of its space that is no slower than the starting point,
the cache, and tuned runs that still match the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("maker", [lambda: W.uniform(100_000, 3), lambda: W.mixed(300_000, 1),
                                   lambda: W.cubic_lattice(20), lambda: W.uniform(1, 0)])
def test_cluster_index_matches_the_oracle(maker):
    p = maker()
    prm = vt.Params()
    G = vt.grid_resolution(prm, len(p))
    assert vt.cluster_index(dev(p), prm) == oracle.morisita_index(p, G)


def test_batch_cluster_index_matches_the_oracle_per_set():
    pts, off, coin = W.batch_sets(n_sets=12, seed=5, size_range=(500, 20_000))
    idx = vt.batch_cluster_index(dev(pts), off)
    for s in range(12):
        q = pts[off[s]:off[s + 1]]
        G = vt.grid_resolution(vt.Params(), len(q))
        assert idx[s] == oracle.morisita_index(q, G)
    # clustered sets sit in a higher class than uniform ones
    cls = [vt.cluster_class(x) for x in idx]
    assert all(c == 0 for c, k in zip(cls, coin) if not k)
    assert all(c >= 1 for c, k in zip(cls, coin) if k)


SMALL_SPACE = {"tpc": [16, 32], "k0": [12, 16], "kmax_mult": [1, 2], "rho": [1.0, 2.0, 4.0], "reps": 2}


def test_autotune_picks_a_candidate_no_slower_than_the_start(tmp_path):
    p = W.mixed(200_000, 4)
    prm = vt.Params(precision="fp64", emit=("nbr", "vol", "cen"))
    cache = str(tmp_path / "tune.json")
    tuned, rep = vt.autotune(dev(p), prm, SMALL_SPACE, cache=cache)
    assert not rep["cached"] and rep["cls"] == vt.cluster_class(oracle.morisita_index(p, vt.grid_resolution(prm, len(p))))
    assert tuned.threads_per_cell in SMALL_SPACE["tpc"] + [32]
    assert tuned.k0 in SMALL_SPACE["k0"] + [prm.k0]
    assert tuned.grid_density in SMALL_SPACE["rho"] + [prm.grid_density]
    start = rep["tried"][0]
    assert start["status"] == "VT_OK" and rep["best_ms"] <= start["ms"]
    assert all(t["status"] == "VT_OK" for t in rep["tried"])
    again, rep2 = vt.autotune(dev(p), prm, SMALL_SPACE, cache=cache)
    assert rep2["cached"] and again == tuned
    # tuned parameters change speed, not results
    sample = np.sort(np.random.default_rng(2).choice(len(p), 500, replace=False))
    want = oracle.tessellate(p, cells=sample)
    cells = vt.tessellate(dev(p), tuned)
    np.testing.assert_allclose(cells.vol.cpu().numpy()[sample], want["vol"], rtol=1e-12)
    lists = cells.nbr.cpu().numpy(), cells.nbr_off.cpu().numpy()
    for a, i in enumerate(sample):
        assert np.array_equal(lists[0][lists[1][i]:lists[1][i + 1]],
                              want["nbr"][want["nbr_off"][a]:want["nbr_off"][a + 1]])


def test_tuned_batch_matches_the_oracle_per_set():
    pts, off, coin = W.batch_sets(n_sets=16, seed=6, size_range=(500, 30_000))
    b = vt.tuned_batch(dev(pts), off, vt.Params(precision="fp64", emit=("nbr", "vol", "cen")),
                       space={"tpc": [16, 32], "k0": [16], "kmax_mult": [2], "rho": [1.0, 3.0], "reps": 1},
                       sample_sets=8)
    rep = b.tune_report
    assert rep["sets_timed"] == 8 and sum(rep["class_counts"]) == 16
    b.capture()
    b.replay()
    cells = b.result()
    vol = cells.vol.cpu().numpy()
    nbr, nbr_off = cells.nbr.cpu().numpy(), cells.nbr_off.cpu().numpy()
    for s in (0, 5, 11):
        q = pts[off[s]:off[s + 1]]
        w = oracle.tessellate(q)
        np.testing.assert_allclose(vol[off[s]:off[s + 1]], w["vol"], rtol=1e-12)
        for i in range(len(q)):
            g = nbr[nbr_off[off[s] + i]:nbr_off[off[s] + i + 1]] - off[s]
            assert np.array_equal(g, w["nbr"][w["nbr_off"][i]:w["nbr_off"][i + 1]])
