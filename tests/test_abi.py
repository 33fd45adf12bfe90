"""The C-ABI library builds, loads and exports every entry point that
include/vt.h declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2412_04514_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vt.h")).read()
    return re.findall(r"VT_API\s+[\w\s\*]+?\b(vt_\w+)\s*\(", txt)


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("vt_grid_build", "vt_knn", "vt_clip_cells", "vt_tessellate"):
        assert want in names
    assert sorted(names) == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = L.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_sizes_match_the_header():
    # vt_params: 8 ints/floats + 6 floats; vt_cells_out: pointers and int64s
    assert ctypes.sizeof(L.VtParams) == 4 * 8 + 4 * 6 + 4
    assert ctypes.sizeof(L.VtCellsOut) == 8 * 20


def test_host_only_calls():
    lib = L.load()
    p = L.VtParams()
    lib.vt_params_default(ctypes.byref(p))
    assert (p.k0, p.k_max, p.precision) == (16, 32, L.VT_FP32_RECHECK)
    assert lib.vt_grid_resolution(ctypes.byref(p), 1 << 20) == 81
    assert lib.vt_grid_resolution(ctypes.byref(p), 1 << 23) == 162
    b = ctypes.c_size_t()
    assert lib.vt_workspace_size(ctypes.byref(p), 4096, ctypes.byref(b)) == L.VT_OK
    assert b.value > 4096 * 16
    assert lib.vt_version().decode().startswith("vt ")


@pytest.mark.parametrize("field,value", [("k0", 0), ("k_max", 512), ("threads_per_cell", 12), ("precision", 7)])
def test_bad_params_are_rejected_on_the_host(field, value):
    lib = L.load()
    p = L.VtParams()
    lib.vt_params_default(ctypes.byref(p))
    setattr(p, field, value)
    b = ctypes.c_size_t()
    assert lib.vt_workspace_size(ctypes.byref(p), 10, ctypes.byref(b)) == L.VT_ERR_INVALID_ARG
    assert lib.vt_last_error().decode()


def test_bad_box_and_small_workspace_are_rejected_before_any_cuda_call():
    lib = L.load()
    p = L.VtParams()
    lib.vt_params_default(ctypes.byref(p))
    p.box_hi[1] = p.box_lo[1]
    b = ctypes.c_size_t()
    assert lib.vt_workspace_size(ctypes.byref(p), 10, ctypes.byref(b)) == L.VT_ERR_INVALID_ARG
    lib.vt_params_default(ctypes.byref(p))
    o = L.VtCellsOut()
    st = L.VtStats()
    code = lib.vt_tessellate(None, 0, ctypes.byref(p), ctypes.byref(o), ctypes.byref(st), None, 0, None)
    assert code == L.VT_ERR_WORKSPACE


def test_grid_resolution_agrees_with_the_oracle_reading():
    import oracle

    lib = L.load()
    p = L.VtParams()
    lib.vt_params_default(ctypes.byref(p))
    for n in (1, 2, 16, 4096, 1 << 20, 3_000_000):
        for rho in (1.0, 2.0, 3.0):
            p.grid_density = rho
            assert lib.vt_grid_resolution(ctypes.byref(p), n) == oracle.grid_resolution(n, rho)


def test_periodic_limits_are_checked_on_the_host():
    lib = L.load()
    p = L.VtParams()
    lib.vt_params_default(ctypes.byref(p))
    p.flags = L.VT_FLAG_PERIODIC
    b = ctypes.c_size_t()
    assert lib.vt_workspace_size(ctypes.byref(p), 4096, ctypes.byref(b)) == L.VT_OK
    # sorted indices of periodic lists have 24 bits
    assert lib.vt_workspace_size(ctypes.byref(p), 1 << 24, ctypes.byref(b)) == L.VT_ERR_INVALID_ARG
    assert lib.vt_workspace_size(ctypes.byref(p), (1 << 24) - 1, ctypes.byref(b)) == L.VT_OK
    # |L|^2 <= 4 min L_a^2: (1, 1, 0.85) passes, (1, 1, 0.8) does not
    p.box_hi[2] = 0.85
    assert lib.vt_workspace_size(ctypes.byref(p), 4096, ctypes.byref(b)) == L.VT_OK
    p.box_hi[2] = 0.8
    assert lib.vt_workspace_size(ctypes.byref(p), 4096, ctypes.byref(b)) == L.VT_ERR_INVALID_ARG
    p.flags = 0
    assert lib.vt_workspace_size(ctypes.byref(p), 4096, ctypes.byref(b)) == L.VT_OK


def test_fused_schedule_workspace_holds_no_lists():
    # VT_FLAG_FUSED clips from the grid walk: neither the n x 2 k0 list (ids
    # and float keys) nor the saved polyhedra are in the workspace
    lib = L.load()
    n = 1 << 20
    sizes = {}
    for flags in (0, L.VT_FLAG_FUSED, L.VT_FLAG_FUSED | L.VT_FLAG_NO_SYNC):
        p = L.VtParams()
        lib.vt_params_default(ctypes.byref(p))
        p.flags = flags
        b = ctypes.c_size_t()
        assert lib.vt_workspace_size(ctypes.byref(p), n, ctypes.byref(b)) == L.VT_OK
        sizes[flags] = b.value
    assert sizes[0] - sizes[L.VT_FLAG_FUSED] >= n * (32 * 8 + 1024)
    assert sizes[L.VT_FLAG_FUSED | L.VT_FLAG_NO_SYNC] == sizes[L.VT_FLAG_FUSED]
    # a batch (the no-sync schedule of a CUDA graph) saves the same per point
    batch = {}
    for flags in (L.VT_FLAG_NO_SYNC, L.VT_FLAG_FUSED | L.VT_FLAG_NO_SYNC):
        p.flags = flags
        assert lib.vt_batch_workspace_size(ctypes.byref(p), n, 512 * 4096, ctypes.byref(b)) == L.VT_OK
        batch[flags] = b.value
    assert batch[L.VT_FLAG_NO_SYNC] - batch[L.VT_FLAG_FUSED | L.VT_FLAG_NO_SYNC] >= n * (64 * 8 + 1024) - 4096
    p.flags = 16
    assert lib.vt_workspace_size(ctypes.byref(p), n, ctypes.byref(b)) == L.VT_ERR_INVALID_ARG


def test_degenerate_input_warning_threshold():
    # the walks' counts of a coplanar cloud (every cell, about n generators
    # each) warn; a clumped 1M cloud (about 150 per walk), a dense clump whose
    # few sparse neighbours walk long, a small line and a run without walks
    # do not
    import warnings

    from paper_2412_04514_gb300.api import _warn_degenerate

    with pytest.warns(RuntimeWarning, match="degenerate"):
        _warn_degenerate({"walk_cells": 1500, "walk_candidates": 1500 * 1500}, 1500)
    with pytest.warns(RuntimeWarning, match="O\\(n\\^2\\)"):
        _warn_degenerate({"walk_cells": 10**6, "walk_candidates": 10**6 * 300_000}, 10**6)
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        _warn_degenerate({"walk_cells": 1_003_534, "walk_candidates": 1_003_534 * 150}, 1 << 20)
        _warn_degenerate({"walk_cells": 164, "walk_candidates": 164 * 7356}, 14_000)
        _warn_degenerate({"walk_cells": 300, "walk_candidates": 300 * 300}, 300)
        _warn_degenerate({"walk_cells": 0, "walk_candidates": 0}, 10)
        _warn_degenerate({}, 10)


def test_binding_structs_match_the_header_layout(tmp_path):
    # every ctypes mirror of a vt.h struct has the C compiler's size and field
    # offsets (a field added to one side only would shift the other's)
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"vt_params": L.VtParams, "vt_cells_out": L.VtCellsOut, "vt_set_desc": L.VtSetDesc,
               "vt_tune_space": L.VtTuneSpace, "vt_tune_trial": L.VtTuneTrial, "vt_tune_result": L.VtTuneResult,
               "vt_stats": L.VtStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vt.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, what, value = line.split()
            got[(cname, what)] = int(value)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
