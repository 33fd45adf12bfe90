"""Host side of the autotuner: the oracle's clustering statistic against its
closed forms, the clustering classes, the tune space checks and the JSON
cache (no GPU needed)."""
import ctypes
import json

import numpy as np
import pytest

import oracle
from paper_2412_04514_gb300 import _lib as L
from paper_2412_04514_gb300 import tune as T
from paper_2412_04514_gb300 import workloads as W
from paper_2412_04514_gb300.api import Params


def test_morisita_is_zero_when_no_cell_holds_two_points():
    m = 12
    assert oracle.morisita_index(W.cubic_lattice(m), m) == 0.0


def test_morisita_of_one_full_cell_is_the_cell_count():
    rng = np.random.default_rng(1)
    p = (0.01 + 0.02 * rng.random((500, 3))).astype(np.float32)  # all in cell 0 of a 10^3 grid
    assert oracle.morisita_index(p, 10) == 1000.0


def test_morisita_of_two_equal_cells():
    rng = np.random.default_rng(2)
    m = 300
    a = 0.05 * rng.random((m, 3))
    b = 0.55 + 0.05 * rng.random((m, 3))
    p = np.concatenate([a, b]).astype(np.float32)
    G = 4
    want = G**3 * 2 * m * (m - 1) / (2 * m * (2 * m - 1))
    assert abs(oracle.morisita_index(p, G) - want) < 1e-12 * want


def test_morisita_of_uniform_points_is_one():
    # E[n_c (n_c - 1)] = n (n - 1) / Q for a multinomial with equal cells
    vals = [oracle.morisita_index(W.uniform(100_000, s), 37) for s in range(4)]
    assert abs(np.mean(vals) - 1.0) < 0.02


def test_morisita_separates_the_mixed_cloud():
    assert oracle.morisita_index(W.mixed(200_000, 1), 46) > 8.0
    assert oracle.morisita_index(W.uniform(1, 0), 1) == 0.0


@pytest.mark.parametrize("index,cls", [(0.0, 0), (1.0, 0), (1.99, 0), (2.0, 1), (7.9, 1), (8.0, 2), (31.0, 2),
                                       (32.0, 3), (1e9, 3), (float("nan"), 3)])
def test_cluster_classes(index, cls):
    assert T.cluster_class(index) == cls


def test_default_space_and_workspace():
    d = T.default_space()
    assert d["tpc"] == [8, 16, 32] and d["k0"] == [8, 12, 16, 24, 32] and d["rho"] == [1, 2, 3, 4, 6]
    lib = L.load()
    sp = T._space(None)
    p = Params().c()
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.vt_autotune_workspace_size(ctypes.byref(p), ctypes.byref(sp), 100_000, ctypes.byref(a)) == 0
    assert lib.vt_workspace_size(ctypes.byref(p), 100_000, ctypes.byref(b)) == 0
    assert a.value >= b.value  # the widest candidate (rho 1, k0 32) needs at least the base's workspace
    off = (ctypes.c_int64 * 3)(0, 1000, 5000)
    assert lib.vt_autotune_batch_workspace_size(off, 2, ctypes.byref(p), ctypes.byref(sp), ctypes.byref(a)) == 0


@pytest.mark.parametrize("field,value", [("tpc", [12]), ("k0", [0]), ("kmax_mult", [0]), ("rho", [-1.0]),
                                         ("reps", 0), ("k0", list(range(1, 10)))])
def test_bad_tune_spaces_are_rejected(field, value):
    lib = L.load()
    p = Params().c()
    b = ctypes.c_size_t()
    try:
        sp = T._space({field: value})
    except ValueError:
        return
    assert lib.vt_autotune_workspace_size(ctypes.byref(p), ctypes.byref(sp), 10, ctypes.byref(b)) == \
        L.VT_ERR_INVALID_ARG


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    prm = Params(precision="fp32")
    assert T.lookup(path, prm, 1 << 20, 3, "dev") is None
    d = T.load_cache(path)
    key = T.cache_key(prm, 1 << 20, 3)
    assert key == "fp32|cen+nbr+vol|sync|n4^10|c3"
    d["entries"][key] = {"threads_per_cell": 16, "k0": 24, "k_max": 48, "grid_density": 3.0, "ms": 1.0,
                         "device": "dev", "n": 1 << 20}
    T.store_cache(path, d)
    got = T.lookup(path, prm, 1 << 20, 3, "dev")
    assert (got.threads_per_cell, got.k0, got.k_max, got.grid_density) == (16, 24, 48, 3.0)
    assert got.precision == "fp32" and got.emit == prm.emit
    assert T.lookup(path, prm, 1 << 20, 3, "other device") is None
    assert T.lookup(path, prm, 1 << 16, 3, "dev") is None  # other size bucket
    per = Params(precision="fp32", periodic=True)
    assert T.cache_key(per, 1 << 20, 3) == "fp32|cen+nbr+vol|sync+periodic|n4^10|c3"
    assert T.lookup(path, per, 1 << 20, 3, "dev") is None  # a periodic box is tuned on its own
    with open(path, "w") as f:
        json.dump({"version": 99}, f)
    with pytest.raises(ValueError):
        T.load_cache(path)
