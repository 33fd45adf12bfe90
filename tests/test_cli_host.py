"""The numpy / command-line front-ends: file formats and argument handling (CPU only)."""
import numpy as np
import pytest

from paper_2412_04514_gb300 import cli


def test_read_points_formats(tmp_path):
    p = np.array([[0.1, 0.2, 0.3], [0.5, 0.25, 0.125], [0.9, 0.8, 0.7]], dtype=np.float64)
    np.save(tmp_path / "a.npy", p)
    np.savez(tmp_path / "a.npz", points=p)
    (tmp_path / "a.txt").write_text("# x y z\n0.1 0.2 0.3\n\n0.5\t0.25 0.125  # second\n0.9 0.8 0.7\n")
    (tmp_path / "a.csv").write_text("0.1,0.2,0.3\n0.5,0.25,0.125\n0.9,0.8,0.7\n")
    for name in ("a.npy", "a.npz", "a.txt", "a.csv"):
        a = cli.read_points(str(tmp_path / name))
        assert a.dtype == np.float32 and a.shape == (3, 3) and a.flags.c_contiguous
        np.testing.assert_array_equal(a, p.astype(np.float32))


def test_read_points_rejects_bad_files(tmp_path):
    (tmp_path / "b.txt").write_text("0.1 0.2\n")
    with pytest.raises(ValueError, match="3 columns"):
        cli.read_points(str(tmp_path / "b.txt"))
    np.save(tmp_path / "b.npy", np.zeros((4, 2)))
    with pytest.raises(ValueError, match=r"shape \(n, 3\)"):
        cli.read_points(str(tmp_path / "b.npy"))
    np.save(tmp_path / "c.npy", np.zeros((4, 3), dtype=np.int32))
    with pytest.raises(ValueError, match="floating point"):
        cli.read_points(str(tmp_path / "c.npy"))
    np.savez(tmp_path / "d.npz", pts=np.zeros((4, 3)))
    with pytest.raises(ValueError, match="'points'"):
        cli.read_points(str(tmp_path / "d.npz"))


def test_neighbour_lists_split():
    off = np.array([0, 2, 2, 5], dtype=np.int64)
    nbr = np.array([4, 7, 1, 2, 3], dtype=np.int32)
    rows = cli.neighbour_lists(off, nbr)
    assert [r.tolist() for r in rows] == [[4, 7], [], [1, 2, 3]]
    assert cli.neighbour_lists(np.array([0]), np.array([], dtype=np.int32)) == []


def test_write_cells_text_and_npz(tmp_path):
    cells = {"vol": np.array([0.25, 0.75]), "nbr_off": np.array([0, 1, 2], dtype=np.int64),
             "nbr": np.array([1, 0], dtype=np.int32), "cen": None, "stats": {"x": 1}}
    cli.write_cells(str(tmp_path / "o.txt"), cells)
    lines = (tmp_path / "o.txt").read_text().splitlines()
    assert lines == ["0.25 1", "0.75 0"]
    pts = np.zeros((2, 3), dtype=np.float32)
    cli.write_cells(str(tmp_path / "o.npz"), cells, pts)
    with np.load(tmp_path / "o.npz") as z:
        assert sorted(z.files) == ["nbr", "nbr_off", "points", "vol"]
        np.testing.assert_array_equal(z["nbr"], cells["nbr"])
    with pytest.raises(ValueError, match="nbr"):
        cli.write_cells(str(tmp_path / "p.txt"), {"vol": cells["vol"], "nbr": None})


def test_params_from_args():
    a = cli.parser().parse_args(["in.npy", "-o", "out.npz", "--precision", "fp64", "--emit", "nbr, vol,m2",
                                 "--k0", "8", "--k-max", "64", "--rho", "3", "--threads-per-cell", "16",
                                 "--index-space", "sorted", "--box", "-1", "-2", "-3", "1", "2", "3"])
    p = cli.params_from_args(a)
    assert p.precision == "fp64" and p.emit == ("nbr", "vol", "m2")
    assert (p.k0, p.k_max, p.grid_density, p.threads_per_cell) == (8, 64, 3.0, 16)
    assert p.index_space == "sorted"
    assert p.box_lo == (-1.0, -2.0, -3.0) and p.box_hi == (1.0, 2.0, 3.0)
    assert not p.periodic
    assert cli.params_from_args(cli.parser().parse_args(["i", "-o", "o.npz", "--periodic"])).periodic
    assert not p.fused and p.c().flags == 0
    pf = cli.params_from_args(cli.parser().parse_args(["i", "-o", "o.npz", "--fused"]))
    assert pf.fused and pf.c().flags == 8  # VT_FLAG_FUSED
    with pytest.raises(ValueError, match="unknown output"):
        cli.params_from_args(cli.parser().parse_args(["i", "-o", "o.npz", "--emit", "nbr,area"]))
    with pytest.raises(SystemExit):
        cli.parser().parse_args(["i", "-o", "o.npz", "--threads-per-cell", "4"])
