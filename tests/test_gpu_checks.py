"""The bounds-checked debug build (-DVT_CHECKS) on the small and degenerate cases.

The debug build checks every shared-memory plane and vertex-slot index that
comes from data, every output-record index and every CSR write, and turns a
bad one into VT_ERR_INTERNAL instead of an out-of-bounds access. It is built
into a directory of its own and run in a child process (the regular library
stays loaded in this one) on the 4,096-point configuration in both forms and
both schedules (and the fused schedule on the first three clouds),
clustered, periodic and batched input with geometry, and
subsets of degenerate and ulp-moved lattices; every call must return VT_OK
with cells that fill the box.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    import numpy as np, torch
    import paper_2412_04514_gb300 as vt
    from paper_2412_04514_gb300 import workloads as W
    from test_gpu_degenerate_sweep import draw
    cases = [(W.uniform(4096, 0), False), (W.mixed(30000, 3, n_clumps=20), False),
             (W.mixed(20000, 5, n_clumps=10, periodic=True), True)]
    cases += [draw(seed) for seed in range(32)]
    n_calls = 0
    for ci, (pts, periodic) in enumerate(cases):
        d = torch.from_numpy(pts).cuda()
        for prec in ("fp32", "fp64"):
            for no_sync in (False, True):
                # the fused schedule (one walk from the box) on the first three clouds
                for fused in ((False, True) if ci < 3 else (False,)):
                    p = vt.Params(precision=prec, emit=("nbr", "vol", "cen", "geom"), periodic=periodic,
                                  no_sync=no_sync, fused=fused)
                    c = vt.tessellate(d, p)
                    assert c.stats["status"] == "VT_OK", c.stats["status"]
                    assert abs(float(c.vol.sum()) - 1.0) < 1e-5
                    n_calls += 1
    sets = [W.uniform(3000, 7), W.uniform(1, 8), W.mixed(6000, 9, n_clumps=5), W.uniform(3000, 10)]
    off = [0] + list(np.cumsum([len(x) for x in sets]))
    pts = np.concatenate(sets)
    b = vt.tessellate_batch(torch.from_numpy(pts).cuda(), off, vt.Params(emit=("nbr", "vol", "cen")))
    assert b.stats["status"] == "VT_OK"
    print("checked calls:", n_calls + 1)
""")


def test_debug_build_finds_no_bad_index(tmp_path):
    env = dict(os.environ, VT_NVCC_FLAGS="-DVT_CHECKS", VT_BUILD_DIR=str(tmp_path / "checks"))
    script = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked calls: 153" in r.stdout
