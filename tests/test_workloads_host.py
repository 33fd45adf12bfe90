"""The seeded input generators follow the stated recipes.

Every parity test and the benchmark draw their points from
``paper_2412_04514_gb300.workloads``; these tests pin the recipes there: float32
points inside the half-open box, no repeated rows, the same cloud for the same
seed, clumps whose spread matches their log-uniform sigma range, draws outside
the box resampled (walls) or wrapped by whole periods (periodic), the
half-uniform / half-clustered split of the mixed cloud, the sizes of the batch
sets, and the sub-box sample of the precision case.
"""
import numpy as np
import pytest

from paper_2412_04514_gb300 import workloads as W


def distinct(p):
    return len(np.unique(p.view(np.dtype((np.void, 12))))) == len(p)


@pytest.mark.parametrize("make", [lambda s: W.uniform(50_000, s), lambda s: W.mixed(50_000, s, n_clumps=50),
                                  lambda s: W.mixed(50_000, s, n_clumps=50, periodic=True)])
def test_points_are_float32_inside_distinct_and_seeded(make):
    p = make(4)
    assert p.dtype == np.float32 and p.shape == (50_000, 3) and p.flags.c_contiguous
    assert np.all((p >= 0) & (p < 1))
    assert distinct(p)
    assert np.array_equal(p, make(4))
    assert not np.array_equal(p, make(5))


def test_uniform_points_are_uniform():
    p = W.uniform(200_000, 7).astype(np.float64)
    # the largest gap between the empirical and the uniform CDF, per axis
    # (Kolmogorov-Smirnov: 1.95 / sqrt(n) at the 0.1% level)
    for a in range(3):
        x = np.sort(p[:, a])
        i = np.arange(1, len(x) + 1) / len(x)
        assert max(np.abs(i - x).max(), np.abs(i - 1 / len(x) - x).max()) < 1.95 / np.sqrt(len(x))


def test_a_clump_spread_is_its_sigma_and_stays_in_the_box():
    # one clump at a time: its sample spread is the drawn sigma, which lies in
    # [1e-3, 1e-2]; a clump near a wall is resampled, not clamped onto it
    for seed in range(8):
        rng = np.random.default_rng(seed)
        p = W.clustered(20_000, 1, rng).astype(np.float64)
        assert np.all((p >= 0) & (p < 1))
        centre = np.median(p, axis=0)
        if np.all((centre > 0.05) & (centre < 0.95)):
            s = p.std(axis=0).mean()
            assert 0.95e-3 < s < 1.05e-2, s
        assert not np.any(np.isin(p, [0.0]))  # nothing piled onto the lower walls


def test_periodic_clumps_wrap_across_the_faces():
    # a clump centred on a face: its points appear on both sides, none outside
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = W.clustered(5000, 1, np.random.default_rng(rng.integers(1 << 30)), periodic=True).astype(np.float64)
        assert np.all((p >= 0) & (p < 1))
        near_lo, near_hi = (p < 0.02).any(axis=1).sum(), (p > 0.98).any(axis=1).sum()
        if near_lo > 100 and near_hi > 100:
            return
    pytest.fail("no clump of 50 straddled a face")


def test_mixed_cloud_is_half_uniform_half_clumps():
    n = 100_000
    p = W.mixed(n, 3, n_clumps=20).astype(np.float64)
    # clumps are at most a few 1e-2 across: cells of a 10^3 grid far from
    # every clump hold only the uniform half, n / 2 / 1000 points on average
    G = 10
    cid = np.minimum((p * G).astype(int), G - 1)
    counts = np.bincount((cid[:, 0] * G + cid[:, 1]) * G + cid[:, 2], minlength=G ** 3)
    assert abs(np.median(counts) - n / 2 / G ** 3) < 0.15 * n / 2 / G ** 3
    assert counts.sum() == n
    # and the input order carries no spatial structure (shuffled)
    assert abs(np.corrcoef(np.arange(n), p[:, 0])[0, 1]) < 0.02


def test_batch_sets_follow_the_size_recipe():
    pts, off, coin = W.batch_sets(n_sets=40, seed=9, size_range=(1000, 20_000))
    sizes = np.diff(off)
    assert len(sizes) == 40 and off[0] == 0 and off[-1] == len(pts)
    assert sizes.min() >= 1000 and sizes.max() < 20_000
    assert 0 < coin.sum() < 40
    for s in range(40):
        q = pts[off[s]:off[s + 1]]
        assert np.all((q >= 0) & (q < 1)) and distinct(q)


def test_sub_box_holds_about_the_target():
    p = W.uniform(300_000, 11)
    idx = W.sub_box_cells(p, 5000, 3)
    assert abs(len(idx) - 5000) <= 50
    assert np.all(np.diff(idx) > 0)
    q = p[idx]
    # a cube: equal extents, and no other point inside its bounding box
    ext = q.max(0) - q.min(0)
    assert ext.max() - ext.min() < 0.05 * ext.max()
    inside = np.all((p >= q.min(0)) & (p <= q.max(0)), axis=1)
    assert inside.sum() == len(idx)


def test_lattices_are_exact_in_float32():
    c = W.cubic_lattice(8)
    assert len(c) == 512 and np.array_equal(c.astype(np.float64) * 16 % 2, np.ones_like(c, dtype=np.float64))
    b = W.bcc_lattice(4)
    assert len(b) == 64 + 27 and distinct(b) and np.all((b > 0) & (b < 1))
