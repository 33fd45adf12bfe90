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


def test_static_grid_sort_refuses_pageable_host_buffers():
    # plain (pageable) host memory is not memory device code can use on every
    # system: the call checks its buffers first and returns an argument error
    # without launching; where the system maps such memory for the device
    # (coherent host memory), the call must give the same sort instead
    lib = L.load()
    params = vt.Params().c()
    pts_h = W.uniform(1000, 8)
    n = len(pts_h)
    G = lib.vt_grid_resolution(ctypes.byref(params), n)
    d_pts = torch.from_numpy(pts_h).cuda()
    sorted_ = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    cell_off = torch.empty(G**3 + 1, dtype=torch.int32, device="cuda")
    host_sorted = np.zeros((n, 4), np.float32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    code, w_sorted, w_perm, w_off = _static_sort(lib, d_pts, params)
    assert code == L.VT_OK
    w_sorted = w_sorted.cpu().numpy()
    code = lib.vt_grid_build_static(ctypes.c_void_p(pts_h.ctypes.data), n, ctypes.byref(params), G, ptr(sorted_),
                                    ptr(perm), ptr(cell_off), stream)
    if code == L.VT_ERR_INVALID_ARG:
        assert b"pts is not device-accessible" in lib.vt_last_error()
    else:
        assert code == L.VT_OK
        assert np.array_equal(sorted_.cpu().numpy().view(np.int32), w_sorted.view(np.int32))
    code = lib.vt_grid_build_static(ptr(d_pts), n, ctypes.byref(params), G, ctypes.c_void_p(host_sorted.ctypes.data),
                                    ptr(perm), ptr(cell_off), stream)
    if code == L.VT_ERR_INVALID_ARG:
        assert b"sorted is not device-accessible" in lib.vt_last_error()
        assert not host_sorted.any()
    else:
        assert code == L.VT_OK
        assert np.array_equal(host_sorted.view(np.int32), w_sorted.view(np.int32))


def test_static_grid_sort_allocates_no_device_memory():
    lib = L.load()
    params = vt.Params().c()
    pts = torch.from_numpy(W.mixed(200_000, 4, n_clumps=200)).cuda()
    n = pts.shape[0]
    G = lib.vt_grid_resolution(ctypes.byref(params), n)
    sorted_ = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    cell_off = torch.empty(G**3 + 1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (ctypes.c_void_p(pts.data_ptr()), n, ctypes.byref(params), G, ctypes.c_void_p(sorted_.data_ptr()),
            ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(cell_off.data_ptr()), stream)
    assert lib.vt_grid_build_static(*args) == L.VT_OK  # warm-up: the same kernels as the call measured
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert lib.vt_grid_build_static(*args) == L.VT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
