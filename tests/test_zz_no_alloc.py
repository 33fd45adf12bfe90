"""vt_grid_build_static: the grid sort for callers that cannot allocate device
memory (a fixed arena handed out up front, no cudaMalloc allowed while they
run). Its scratch is a device array inside libvt.so instead of a workspace.

Checked through the C ABI against vt_grid_build (which takes a caller-allocated
workspace) on two calls in a row: the grid sort is integer work, so the
outputs must be identical.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2412_04514_gb300 as vt
from paper_2412_04514_gb300 import _lib as L
from paper_2412_04514_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static_sort(lib, pts: torch.Tensor, params: L.VtParams):
    n = pts.shape[0]
    G = lib.vt_grid_resolution(ctypes.byref(params), n)
    sorted_ = torch.empty((max(n, 1), 4), dtype=torch.float32, device=pts.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=pts.device)
    cell_off = torch.empty(G**3 + 1, dtype=torch.int32, device=pts.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.vt_grid_build_static(ctypes.c_void_p(pts.data_ptr()), n, ctypes.byref(params), G,
                                    ctypes.c_void_p(sorted_.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                    ctypes.c_void_p(cell_off.data_ptr()), stream)
    return code, sorted_[:n], perm[:n], cell_off


def test_static_grid_sort_matches_the_workspace_entry_point_on_two_calls():
    lib = L.load()
    params = vt.Params().c()
    clouds = [W.mixed(300_000, 1, n_clumps=300), W.uniform(4096, 0)]
    for pts_np in clouds:  # two calls in a row share the library's scratch array
        pts = torch.from_numpy(pts_np).cuda()
        code, s_sorted, s_perm, s_off = _static_sort(lib, pts, params)
        assert code == L.VT_OK, lib.vt_last_error()
        w_sorted, w_perm, w_off, G, _ = vt.grid_build(pts)
        torch.cuda.synchronize()
        assert torch.equal(s_perm, w_perm)
        assert torch.equal(s_off, w_off)
        assert torch.equal(s_sorted.view(torch.int32), w_sorted.view(torch.int32))


def test_static_grid_sort_rejects_requests_beyond_its_limit_and_recovers():
    lib = L.load()
    params = vt.Params().c()
    big = torch.from_numpy(W.uniform((1 << 20) + 1, 5)).cuda()
    code, *_ = _static_sort(lib, big, params)
    assert code == L.VT_ERR_INVALID_ARG
    assert b"limited to" in lib.vt_last_error()
    bad = W.uniform(1000, 6)
    bad[10] = [np.nan, 0.5, 0.5]
    code, *_ = _static_sort(lib, torch.from_numpy(bad).cuda(), params)
    assert code == L.VT_ERR_INVALID_ARG
    ok = torch.from_numpy(W.uniform(1000, 7)).cuda()
    code, s_sorted, s_perm, s_off = _static_sort(lib, ok, params)
    assert code == L.VT_OK
    w_sorted, w_perm, w_off, _, _ = vt.grid_build(ok)
    assert torch.equal(s_perm, w_perm) and torch.equal(s_off, w_off)
