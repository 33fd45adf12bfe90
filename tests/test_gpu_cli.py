"""The numpy and command-line front-ends on the GPU, against the FP64 oracle."""
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2412_04514_gb300 import cli
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tessellate_numpy_fp64_matches_oracle():
    pts = W.uniform(3000, seed=41)
    got = cli.tessellate_numpy(pts, precision="fp64", emit=("nbr", "vol", "cen", "m2"))
    want = oracle.tessellate(pts)
    np.testing.assert_allclose(got["vol"], want["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["cen"], want["cen"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got["m2"], want["m2"], rtol=1e-11, atol=0)
    assert np.array_equal(got["nbr_off"], want["nbr_off"]) and np.array_equal(got["nbr"], want["nbr"])
    assert got["stats"]["status"] == "VT_OK"


def test_command_line_round_trip(tmp_path):
    pts = W.mixed(4000, seed=42, n_clumps=8)
    np.savetxt(tmp_path / "p.txt", pts.astype(np.float64), fmt="%.9g")
    out_npz, out_txt = tmp_path / "c.npz", tmp_path / "c.txt"
    for out in (out_npz, out_txt):
        r = subprocess.run([sys.executable, "-m", "paper_2412_04514_gb300", str(tmp_path / "p.txt"), "-o", str(out),
                            "--precision", "fp64", "--emit", "nbr,vol,cen", "--stats"],
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
    want = oracle.tessellate(pts)
    with np.load(out_npz) as z:
        np.testing.assert_array_equal(z["points"], pts)
        np.testing.assert_allclose(z["vol"], want["vol"], rtol=1e-12, atol=0)
        assert np.array_equal(z["nbr_off"], want["nbr_off"]) and np.array_equal(z["nbr"], want["nbr"])
    lines = out_txt.read_text().splitlines()
    assert len(lines) == len(pts)
    for i in (0, 1, len(pts) // 2, len(pts) - 1):
        f = lines[i].split()
        assert float(f[0]) == pytest.approx(want["vol"][i], rel=1e-12)
        assert [int(x) for x in f[1:]] == want["nbr"][want["nbr_off"][i]:want["nbr_off"][i + 1]].tolist()
