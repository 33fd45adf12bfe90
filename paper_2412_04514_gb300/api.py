"""PyTorch binding of the Voronoi library: argument marshalling only.

Every computation happens in libvt.so's CUDA kernels; these functions only
allocate torch tensors (device memory), pass their pointers and the current
CUDA stream through the C ABI of include/vt.h, and wrap the results.
The library runs on the current CUDA device, so with several GPUs make the
tensors' device current first (``torch.cuda.set_device`` or
``with torch.cuda.device(...)``).
"""
from __future__ import annotations

import ctypes
import warnings
from dataclasses import dataclass, field

import torch

from . import _lib as L

_EMIT_BITS = {"nbr": L.VT_EMIT_NBR, "vol": L.VT_EMIT_VOL, "cen": L.VT_EMIT_CEN, "m2": L.VT_EMIT_M2,
              "geom": L.VT_EMIT_GEOM}
_PREC = {"fp64": L.VT_FP64, "fp32": L.VT_FP32_RECHECK}


@dataclass
class Params:
    """Run-time parameters (vt_params). ``precision`` is ``"fp32"`` (float32
    clipping with FP64 rechecks) or ``"fp64"`` (plain FP64). ``periodic``:
    the box [box_lo, box_hi) is periodic (VT_FLAG_PERIODIC). ``fused``: no
    neighbour lists, every cell clips straight from its grid-shell walk
    (VT_FLAG_FUSED)."""

    k0: int = 16
    k_max: int = 32
    grid_density: float = 2.0
    grid_res: int = 0
    threads_per_cell: int = 0
    precision: str = "fp32"
    emit: tuple = ("nbr", "vol", "cen")
    index_space: str = "original"
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    stage_times: bool = False
    no_sync: bool = False
    periodic: bool = False
    fused: bool = False

    def c(self) -> L.VtParams:
        p = L.VtParams()
        p.k0, p.k_max = self.k0, self.k_max
        p.grid_density, p.grid_res = self.grid_density, self.grid_res
        p.threads_per_cell = self.threads_per_cell
        p.precision = _PREC[self.precision]
        bits = 0
        for e in self.emit:
            bits |= _EMIT_BITS[e]
        p.emit = bits
        p.index_space = {"original": L.VT_INDEX_ORIGINAL, "sorted": L.VT_INDEX_SORTED}[self.index_space]
        for a in range(3):
            p.box_lo[a] = self.box_lo[a]
            p.box_hi[a] = self.box_hi[a]
        p.flags = ((L.VT_FLAG_STAGE_TIMES if self.stage_times else 0) | (L.VT_FLAG_NO_SYNC if self.no_sync else 0)
                   | (L.VT_FLAG_PERIODIC if self.periodic else 0) | (L.VT_FLAG_FUSED if self.fused else 0))
        return p


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_points(points: torch.Tensor) -> torch.Tensor:
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must have shape (n, 3)")
    if points.dtype != torch.float32:
        raise ValueError("points must be float32")
    if not points.is_cuda:
        raise ValueError("points must be a CUDA tensor (use tessellate_host for host arrays)")
    return points.contiguous()


def workspace_size(params: Params, n: int) -> int:
    lib = L.load()
    b = ctypes.c_size_t()
    L.check(lib.vt_workspace_size(ctypes.byref(params.c()), n, ctypes.byref(b)))
    return b.value


def grid_resolution(params: Params, n: int) -> int:
    g = L.load().vt_grid_resolution(ctypes.byref(params.c()), n)
    if g < 1:
        raise ValueError("invalid parameters")
    return g


class Workspace:
    """Device scratch memory for (params, n), reused across calls."""

    def __init__(self, params: Params, n: int, device="cuda"):
        self.nbytes = workspace_size(params, n)
        self.buf = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=device)

    def fits(self, params: Params, n: int) -> bool:
        return workspace_size(params, n) <= self.buf.numel()


@dataclass
class Cells:
    vol: torch.Tensor | None = None
    cen: torch.Tensor | None = None
    m2: torch.Tensor | None = None
    nbr_off: torch.Tensor | None = None
    nbr: torch.Tensor | None = None
    vtx_off: torch.Tensor | None = None
    vtx: torch.Tensor | None = None
    face_off: torch.Tensor | None = None
    face_nbr: torch.Tensor | None = None
    face_vtx_off: torch.Tensor | None = None
    face_vtx: torch.Tensor | None = None
    perm: torch.Tensor | None = None
    stats: dict = field(default_factory=dict)
    # ids (in the call's index space) of the cells left unvalidated, whose
    # vol / cen / m2 are NaN; empty when every cell was validated
    unvalidated: torch.Tensor | None = None


def _out_struct(cells: Cells) -> L.VtCellsOut:
    o = L.VtCellsOut()
    for name in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                 "face_vtx", "perm"):
        t = getattr(cells, name)
        setattr(o, name, None if t is None else t.data_ptr())
    o.nbr_cap = 0 if cells.nbr is None else cells.nbr.numel()
    o.vtx_cap = 0 if cells.vtx is None else cells.vtx.shape[0]
    o.face_cap = 0 if cells.face_nbr is None else cells.face_nbr.numel()
    o.face_vtx_cap = 0 if cells.face_vtx is None else cells.face_vtx.numel()
    return o


def _alloc(params: Params, n: int, dev, want_perm: bool, guess: dict | None = None, host_csr: bool = False) -> Cells:
    """Output tensors on ``dev``; with ``host_csr`` the variable-length (CSR)
    outputs are pinned host memory instead, which the emit kernel writes
    directly (pinned memory is device-addressable)."""
    e = set(params.emit)
    g = guess or {}
    c = Cells()
    f64 = dict(dtype=torch.float64, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    where = dict(device="cpu", pin_memory=True) if host_csr else dict(device=dev)
    cf64 = dict(dtype=torch.float64, **where)
    ci64 = dict(dtype=torch.int64, **where)
    ci32 = dict(dtype=torch.int32, **where)
    if "vol" in e:
        c.vol = torch.empty(n, **f64)
    if "cen" in e:
        c.cen = torch.empty((n, 3), **f64)
    if "m2" in e:
        c.m2 = torch.empty(n, **f64)
    if "nbr" in e:
        c.nbr_off = torch.empty(n + 1, **ci64)
        c.nbr = torch.empty(max(g.get("nbr", 20 * n + 64), 1), **ci32)
    if "geom" in e:
        c.vtx_off = torch.empty(n + 1, **ci64)
        c.vtx = torch.empty((max(g.get("vtx", 34 * n + 64), 1), 3), **cf64)
        c.face_off = torch.empty(n + 1, **ci64)
        nf = max(g.get("face", 20 * n + 64), 1)
        c.face_nbr = torch.empty(nf, **ci32)
        c.face_vtx_off = torch.empty(nf + 1, **ci64)
        c.face_vtx = torch.empty(max(g.get("face_vtx", 100 * n + 64), 1), **ci32)
    if want_perm:
        c.perm = torch.empty(max(n, 1), **i32)
    return c


def _trim(c: Cells, o: L.VtCellsOut) -> None:
    if c.nbr is not None:
        c.nbr = c.nbr[: o.needed_nbr]
    if c.vtx is not None:
        c.vtx = c.vtx[: o.needed_vtx]
        c.face_nbr = c.face_nbr[: o.needed_face]
        c.face_vtx_off = c.face_vtx_off[: o.needed_face + 1]
        c.face_vtx = c.face_vtx[: o.needed_face_vtx]


def _unvalidated_ids(params: Params, n: int, ws: torch.Tensor, dev, s, code: int, cells: Cells) -> int:
    """Fills cells.unvalidated (vt_unvalidated_cells) and returns the call's
    status, VT_ERR_UNVALIDATED whenever cells were left unvalidated."""
    if code != L.VT_ERR_UNVALIDATED and not cells.stats.get("unvalidated"):
        cells.unvalidated = torch.empty(0, dtype=torch.int32, device=dev)  # nothing to read back
        return code
    lib = L.load()
    cnt = ctypes.c_int64()
    pc = params.c()
    L.check(lib.vt_unvalidated_cells(ctypes.byref(pc), n, None, 0, ctypes.byref(cnt), _ptr(ws), ws.numel(), s))
    ids = torch.empty(max(cnt.value, 1), dtype=torch.int32, device=dev)
    if cnt.value:
        L.check(lib.vt_unvalidated_cells(ctypes.byref(pc), n, _ptr(ids), ids.numel(), ctypes.byref(cnt), _ptr(ws),
                                         ws.numel(), s))
        if code == L.VT_OK:
            code = L.VT_ERR_UNVALIDATED
    cells.unvalidated = ids[: cnt.value]
    return code


def tessellate(points: torch.Tensor, params: Params | None = None, workspace: Workspace | None = None,
               want_perm: bool = False, strict: bool = True, host_csr: bool = False) -> Cells:
    """Voronoi cells of the generators ``points`` (float32 CUDA tensor (n, 3)).

    Runs vt_tessellate on the current CUDA stream. Variable-length outputs are
    sized from a first guess; if too small they are reallocated from the
    library's exact counts and written by vt_emit. ``strict=False`` returns
    the cells even when some could not be validated (status in
    ``stats["status"]``). ``host_csr=True`` places the neighbour and geometry
    arrays in pinned host memory, written there by the emit kernel itself
    (the moments stay on the device).
    """
    params = params or Params()
    pts = _check_points(points)
    n = pts.shape[0]
    dev = pts.device
    lib = L.load()
    ws = workspace if workspace is not None and workspace.fits(params, n) else Workspace(params, n, dev)
    cells = _alloc(params, n, dev, want_perm, host_csr=host_csr)
    o = _out_struct(cells)
    st = L.VtStats()
    pc = params.c()
    s = _stream(dev)
    code = lib.vt_tessellate(_ptr(pts), n, ctypes.byref(pc), ctypes.byref(o), ctypes.byref(st), _ptr(ws.buf),
                             ws.buf.numel(), s)
    if code == L.VT_OK and params.no_sync:  # the call only enqueued: read status and sizes now
        code = lib.vt_read_stats(_ptr(ws.buf), ws.buf.numel(), ctypes.byref(st), ctypes.byref(o), s)
        if code == L.VT_ERR_CAPACITY:
            pc = Params(**{**params.__dict__, "no_sync": False}).c()
    if code == L.VT_ERR_CAPACITY and o.needed_nbr >= 0:
        guess = {"nbr": o.needed_nbr, "vtx": o.needed_vtx, "face": o.needed_face, "face_vtx": o.needed_face_vtx}
        fresh = _alloc(Params(**{**params.__dict__, "emit": tuple(x for x in params.emit if x in ("nbr", "geom"))}),
                       n, dev, False, guess, host_csr=host_csr)
        for name in ("nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off", "face_vtx"):
            setattr(cells, name, getattr(fresh, name))
        o = _out_struct(cells)
        code = lib.vt_emit(n, ctypes.byref(pc), ctypes.byref(o), _ptr(ws.buf), ws.buf.numel(), s)
    cells.stats = st.as_dict()
    if code in (L.VT_OK, L.VT_ERR_UNVALIDATED):
        code = _unvalidated_ids(params, n, ws.buf, dev, s, code, cells)
        cells.stats["unvalidated"] = cells.unvalidated.numel()
    cells.stats["status"] = L.STATUS_NAMES.get(code, code)
    if code not in (L.VT_OK, L.VT_ERR_UNVALIDATED) or (strict and code != L.VT_OK):
        L.check(code)
    _warn_degenerate(cells.stats, n)
    _trim(cells, o)
    return cells


def _warn_degenerate(stats: dict, n: int) -> None:
    """RuntimeWarning when at least half the cells walked the grid shells
    within twice their radius in the last pass and those walks examined at
    least max(1000, n / 4) generators each on average: coplanar or collinear
    input, whose cells all reach the walls, so that the run costs O(n^2). The
    cells are exact; only the time grows. (A dense clump makes the few sparse
    cells next to it walk long, which this does not report.)"""
    wc = stats.get("walk_cells", 0)
    if wc > 0 and 2 * wc >= n and stats.get("walk_candidates", 0) >= wc * max(1000, n // 4):
        warnings.warn(f"near-degenerate input (coplanar or collinear generators?): the exhaustive walk examined "
                      f"{stats['walk_candidates'] / wc:.0f} generators per walked cell over {wc} cells of {n}; "
                      f"the run costs O(n^2)", RuntimeWarning, stacklevel=3)


def tessellate_host(points, params: Params | None = None, device="cuda", direct: bool = False) -> Cells:
    """End-to-end call on host arrays: copies the points to the device (from
    pinned memory), tessellates and returns every output in host memory.

    By default every output is emitted on the device and copied back by the
    copy engines (measured faster: 41.6 ms against 45.6 ms per 1M-cell step
    with geometry). ``direct=True`` lets the emit kernel write the neighbour
    and geometry arrays straight into pinned host memory instead (no device
    copy of them: for outputs larger than free device memory)."""
    t = torch.as_tensor(points, dtype=torch.float32)
    if not t.is_pinned():
        t = t.pin_memory()
    d = t.to(device, non_blocking=True)
    try:
        cells = tessellate(d, params, host_csr=direct)
    except L.VtError as err:
        # pinned memory that device code cannot address here: the library
        # refused it before any launch; emit on the device and copy instead
        if not direct or "device-accessible" not in str(err):
            raise
        cells = tessellate(d, params, host_csr=False)
    out = Cells(stats=cells.stats)
    # device-to-host copies into pinned buffers (torch caches the pinned
    # allocations across calls), all queued before one synchronisation
    for name in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
                 "face_vtx", "perm"):
        v = getattr(cells, name)
        if v is None or not v.is_cuda:
            setattr(out, name, v)
            continue
        h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
        h.copy_(v, non_blocking=True)
        setattr(out, name, h)
    torch.cuda.current_stream(d.device).synchronize()
    return out


_OUT_NAMES = ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off",
              "face_vtx", "perm")


def tessellate_stream(clouds, params: Params | None = None, device="cuda"):
    """Pipelined end-to-end tessellation of a sequence of host point clouds.

    Yields, in order, one :class:`Cells` in host memory per cloud of
    ``clouds`` (an iterable of float32 host arrays or tensors of shape (n, 3)).
    Three CUDA streams overlap the work: while cloud i is tessellated, cloud
    i+1 is copied to the device and the outputs of cloud i-1 are copied back
    (the copy engines run beside the SMs), so a long sequence costs about the
    tessellation time per cloud instead of tessellation plus both copies. Every
    cloud still makes its own host-to-device and device-to-host round trip.
    The workspace is reused while the clouds keep their size."""
    params = params or Params()
    dev = torch.device(device)
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def stage_in(points):
        t = torch.as_tensor(points, dtype=torch.float32)
        if not t.is_pinned():
            t = t.pin_memory()
        with torch.cuda.stream(s_in):
            d = t.to(dev, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_in)
        return d, ev, t

    it = iter(clouds)
    first = next(it, None)
    if first is None:
        return
    nxt = stage_in(first)
    ws = None
    pending = None  # (host cells, copy-back event) of the previous cloud
    while nxt is not None:
        d, ev_in, _keep = nxt
        follow = next(it, None)
        # the next cloud's copy in is queued before this cloud's compute starts
        nxt = stage_in(follow) if follow is not None else None
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev_in)
            d.record_stream(s_cmp)
            n = d.shape[0]
            if ws is None or not ws.fits(params, n):
                ws = Workspace(params, n, dev)
            cells = tessellate(d, params, workspace=ws)
            done = torch.cuda.Event()
            done.record(s_cmp)
        out = Cells(stats=cells.stats)
        with torch.cuda.stream(s_out):
            s_out.wait_event(done)
            for name in _OUT_NAMES:
                v = getattr(cells, name)
                if v is None:
                    continue
                v.record_stream(s_out)  # the caching allocator keeps it until the copy is done
                h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                h.copy_(v, non_blocking=True)
                setattr(out, name, h)
            copied = torch.cuda.Event()
            copied.record(s_out)
        if pending is not None:
            pending[1].synchronize()
            yield pending[0]
        pending = (out, copied)
    pending[1].synchronize()
    yield pending[0]


# ---------------------------------------------------------------------------
# batches of independent point sets (vt_batch_plan, vt_tessellate_batch)
# ---------------------------------------------------------------------------

def batch_plan(set_off, params: Params | None = None, grid_res=None):
    """Host plan of a batch: (plan as a list of L.VtSetDesc, total grid cells).
    ``set_off`` holds the n_sets + 1 point offsets of the sets in the
    concatenated input; ``grid_res`` optionally fixes G per set (0 = derive)."""
    params = params or Params()
    off = [int(x) for x in set_off]
    ns = len(off) - 1
    if ns < 1:
        raise ValueError("a batch needs at least one set")
    offs = (ctypes.c_int64 * len(off))(*off)
    gr = None if grid_res is None else (ctypes.c_int * ns)(*[int(g) for g in grid_res])
    plan = (L.VtSetDesc * ns)()
    cells = ctypes.c_int64()
    L.check(L.load().vt_batch_plan(offs, ns, ctypes.byref(params.c()), gr, plan, ctypes.byref(cells)))
    return plan, cells.value


class Batch:
    """A batch of independent point sets tessellated as one run.

    ``points`` is the concatenation of the sets (float32 CUDA tensor (N, 3)),
    ``set_off`` the n_sets + 1 offsets (host). Every set gets its own grid
    (``grid_res`` per set, else from ``params.grid_density``); cells see only
    the generators of their own set and neighbour ids index the concatenation.

    The plan, workspace and output buffers are made once. :meth:`run`
    enqueues the whole path with the fixed no-sync schedule (no host wait), so
    it can be recorded by :meth:`capture` into a CUDA graph and replayed with
    :meth:`replay` after new coordinates are copied into :attr:`points`.
    :meth:`result` then reads the status and returns the cells.
    """

    def __init__(self, points: torch.Tensor, set_off, params: Params | None = None, grid_res=None,
                 nbr_per_cell: int = 20, geom_guess: dict | None = None):
        base = params or Params()
        self.params = Params(**{**base.__dict__, "no_sync": True, "stage_times": False})
        self.points = _check_points(points).clone()
        n = self.points.shape[0]
        self.n = n
        dev = self.points.device
        self.set_off_host = [int(x) for x in set_off]
        if self.set_off_host[-1] != n:
            raise ValueError("set_off[-1] must equal the number of points")
        self.n_sets = len(self.set_off_host) - 1
        plan, self.total_cells = batch_plan(self.set_off_host, self.params, grid_res)
        raw = torch.frombuffer(bytearray(bytes(plan)), dtype=torch.uint8)
        self.plan = raw.to(dev)
        self.set_off = torch.tensor(self.set_off_host, dtype=torch.int64, device=dev)
        self.grid_res = [plan[i].G for i in range(self.n_sets)]
        b = ctypes.c_size_t()
        L.check(L.load().vt_batch_workspace_size(ctypes.byref(self.params.c()), n, self.total_cells, ctypes.byref(b)))
        self.ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
        guess = {"nbr": nbr_per_cell * n + 64, **(geom_guess or {})}
        self.cells = _alloc(self.params, n, dev, False, guess)
        self.graph = None
        self._pc = self.params.c()

    def run(self) -> None:
        """Enqueue one tessellation of :attr:`points` on the current stream."""
        o = _out_struct(self.cells)
        st = L.VtStats()
        L.check(L.load().vt_tessellate_batch(_ptr(self.points), self.n, _ptr(self.plan), _ptr(self.set_off),
                                             self.n_sets, self.total_cells, ctypes.byref(self._pc), ctypes.byref(o),
                                             ctypes.byref(st), _ptr(self.ws), self.ws.numel(),
                                             _stream(self.points.device)))
        self.launch_stats = st.as_dict()

    def capture(self) -> None:
        """Record :meth:`run` in a CUDA graph (after one eager warm-up run)."""
        self.run()
        torch.cuda.synchronize(self.points.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.points.device)
        s.wait_stream(torch.cuda.current_stream(self.points.device))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run()
        torch.cuda.current_stream(self.points.device).wait_stream(s)
        self.graph = g

    def replay(self) -> None:
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def result(self, strict: bool = True) -> Cells:
        """Status of the last run (blocking) and the cells as views of the
        batch's buffers. Raises VtError on bad input, unvalidated cells
        (``strict``) or outputs that did not fit (VT_ERR_CAPACITY: call
        :meth:`grow` and run again)."""
        o = _out_struct(self.cells)
        st = L.VtStats()
        code = L.load().vt_read_stats(_ptr(self.ws), self.ws.numel(), ctypes.byref(st), ctypes.byref(o),
                                      _stream(self.points.device))
        self.needed = {"nbr": o.needed_nbr, "vtx": o.needed_vtx, "face": o.needed_face,
                       "face_vtx": o.needed_face_vtx}
        if code not in (L.VT_OK, L.VT_ERR_UNVALIDATED) or (strict and code != L.VT_OK):
            L.check(code)
        out = Cells(**{k: getattr(self.cells, k) for k in ("vol", "cen", "m2", "nbr_off", "nbr", "vtx_off", "vtx",
                                                         "face_off", "face_nbr", "face_vtx_off", "face_vtx")})
        stats = dict(self.launch_stats)
        for k in ("fp64_rechecks", "capacity_retries", "precision_retries", "unvalidated"):
            stats[k] = getattr(st, k)
        stats["clip_events"] = list(st.clip_events)
        stats["status"] = L.STATUS_NAMES.get(code, code)
        out.stats = stats
        _unvalidated_ids(self.params, self.n, self.ws, self.points.device, _stream(self.points.device), code, out)
        _trim(out, o)
        return out

    def grow(self) -> None:
        """Reallocate the variable-length outputs to the sizes the last run
        needed (drops a captured graph, whose pointers would be stale)."""
        self.cells = _alloc(self.params, self.n, self.points.device, False, self.needed)
        self.graph = None


def tessellate_batch(points: torch.Tensor, set_off, params: Params | None = None, grid_res=None,
                     strict: bool = True) -> Cells:
    """One-shot batch. With the default synchronising schedule this is
    vt_tessellate_batch with the per-pass re-queue and the stage times of
    ``params.stage_times``; with ``params.no_sync`` it runs a :class:`Batch`.
    Variable-length outputs that do not fit are reallocated from the exact
    counts and written again by vt_emit."""
    params = params or Params()
    if params.no_sync:
        b = Batch(points, set_off, params, grid_res)
        b.run()
        try:
            return b.result(strict)
        except L.VtError as e:
            if e.code != L.VT_ERR_CAPACITY:
                raise
        b.grow()
        b.run()
        return b.result(strict)
    pts = _check_points(points)
    n = pts.shape[0]
    dev = pts.device
    lib = L.load()
    off = [int(x) for x in set_off]
    if off[-1] != n:
        raise ValueError("set_off[-1] must equal the number of points")
    plan, total = batch_plan(off, params, grid_res)
    plan_d = torch.frombuffer(bytearray(bytes(plan)), dtype=torch.uint8).to(dev)
    off_d = torch.tensor(off, dtype=torch.int64, device=dev)
    b = ctypes.c_size_t()
    pc = params.c()
    L.check(lib.vt_batch_workspace_size(ctypes.byref(pc), n, total, ctypes.byref(b)))
    ws = torch.empty(max(b.value, 256), dtype=torch.uint8, device=dev)
    cells = _alloc(params, n, dev, False)
    o = _out_struct(cells)
    st = L.VtStats()
    s = _stream(dev)
    code = lib.vt_tessellate_batch(_ptr(pts), n, _ptr(plan_d), _ptr(off_d), len(off) - 1, total, ctypes.byref(pc),
                                   ctypes.byref(o), ctypes.byref(st), _ptr(ws), ws.numel(), s)
    if code == L.VT_ERR_CAPACITY:
        guess = {"nbr": o.needed_nbr, "vtx": o.needed_vtx, "face": o.needed_face, "face_vtx": o.needed_face_vtx}
        fresh = _alloc(Params(**{**params.__dict__, "emit": tuple(x for x in params.emit if x in ("nbr", "geom"))}),
                       n, dev, False, guess, host_csr=host_csr)
        for name in ("nbr_off", "nbr", "vtx_off", "vtx", "face_off", "face_nbr", "face_vtx_off", "face_vtx"):
            setattr(cells, name, getattr(fresh, name))
        o = _out_struct(cells)
        code = lib.vt_emit(n, ctypes.byref(pc), ctypes.byref(o), _ptr(ws), ws.numel(), s)
    cells.stats = st.as_dict()
    if code in (L.VT_OK, L.VT_ERR_UNVALIDATED):
        code = _unvalidated_ids(params, n, ws, dev, s, code, cells)
        cells.stats["unvalidated"] = cells.unvalidated.numel()
    cells.stats["status"] = L.STATUS_NAMES.get(code, code)
    if code not in (L.VT_OK, L.VT_ERR_UNVALIDATED) or (strict and code != L.VT_OK):
        L.check(code)
    _trim(cells, o)
    return cells


# ---------------------------------------------------------------------------
# stage calls (vt_grid_build, vt_knn, vt_clip_cells, vt_emit)
# ---------------------------------------------------------------------------

def grid_build(points: torch.Tensor, params: Params | None = None, workspace: Workspace | None = None):
    """Stable grid counting sort. Returns (sorted float32[n,4], perm int32[n],
    cell_off int32[G^3+1], G, workspace)."""
    params = params or Params()
    pts = _check_points(points)
    n = pts.shape[0]
    dev = pts.device
    lib = L.load()
    G = grid_resolution(params, n)
    ws = workspace if workspace is not None and workspace.fits(params, n) else Workspace(params, n, dev)
    sorted_ = torch.empty((max(n, 1), 4), dtype=torch.float32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cell_off = torch.empty(G**3 + 1, dtype=torch.int32, device=dev)
    L.check(lib.vt_grid_build(_ptr(pts), n, ctypes.byref(params.c()), G, _ptr(sorted_), _ptr(perm), _ptr(cell_off),
                              _ptr(ws.buf), ws.buf.numel(), _stream(dev)))
    L.check(lib.vt_read_status(_ptr(ws.buf), ws.buf.numel(), _stream(dev)))
    return sorted_[:n], perm[:n], cell_off, G, ws


def knn(sorted_: torch.Tensor, cell_off: torch.Tensor, G: int, k: int, params: Params | None = None,
        queries: torch.Tensor | None = None, workspace: Workspace | None = None):
    """k nearest neighbours (sorted indices, nearest first) and squared
    distances (float64 for fp64, float32 for fp32)."""
    params = params or Params()
    n = sorted_.shape[0]
    dev = sorted_.device
    lib = L.load()
    ws = workspace if workspace is not None and workspace.fits(params, n) else Workspace(params, n, dev)
    nq = n if queries is None else queries.numel()
    nbr = torch.empty((max(nq, 1), k), dtype=torch.int32, device=dev)
    d2 = torch.empty((max(nq, 1), k), dtype=torch.float64 if params.precision == "fp64" else torch.float32, device=dev)
    q = None if queries is None else queries.to(torch.int32).contiguous()
    L.check(lib.vt_knn(_ptr(sorted_), _ptr(cell_off), G, n, _ptr(q), nq, k, ctypes.byref(params.c()), _ptr(nbr),
                       _ptr(d2), _ptr(ws.buf), ws.buf.numel(), _stream(dev)))
    return nbr[:nq], d2[:nq]


def clip_cells(sorted_: torch.Tensor, cell_off: torch.Tensor, G: int, nbr: torch.Tensor | None,
               d2: torch.Tensor | None, params: Params | None = None, queries: torch.Tensor | None = None,
               workspace: Workspace | None = None):
    """Clips the cells of ``queries`` (default all) with their lists (k =
    nbr.shape[1]; nbr=None runs the exhaustive mode). Returns (Cells with
    vol/cen/m2 written for validated cells, failed sorted indices, workspace)."""
    params = params or Params()
    n = sorted_.shape[0]
    dev = sorted_.device
    lib = L.load()
    ws = workspace if workspace is not None and workspace.fits(params, n) else Workspace(params, n, dev)
    nq = n if queries is None else queries.numel()
    k = 0 if nbr is None else nbr.shape[1]
    cells = Cells()
    e = set(params.emit)
    if "vol" in e:
        cells.vol = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    if "cen" in e:
        cells.cen = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
    if "m2" in e:
        cells.m2 = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    o = _out_struct(cells)
    failed = torch.empty(max(nq, 1), dtype=torch.int32, device=dev)
    n_failed = torch.zeros(1, dtype=torch.int32, device=dev)
    q = None if queries is None else queries.to(torch.int32).contiguous()
    L.check(lib.vt_clip_cells(_ptr(sorted_), _ptr(cell_off), G, n, _ptr(q), nq,
                              None if nbr is None else _ptr(nbr.contiguous()),
                              None if d2 is None else _ptr(d2.contiguous()), k, ctypes.byref(params.c()),
                              ctypes.byref(o), _ptr(failed), _ptr(n_failed), _ptr(ws.buf), ws.buf.numel(),
                              _stream(dev)))
    nf = int(n_failed.item())
    return cells, failed[:nf], ws


def emit(n: int, params: Params, workspace: Workspace, guess: dict | None = None) -> Cells:
    """Writes the neighbour CSR / geometry of the last clipping on
    ``workspace`` (vt_emit)."""
    lib = L.load()
    dev = workspace.buf.device
    p2 = Params(**{**params.__dict__, "emit": tuple(x for x in params.emit if x in ("nbr", "geom"))})
    cells = _alloc(p2, n, dev, False, guess)
    o = _out_struct(cells)
    code = lib.vt_emit(n, ctypes.byref(params.c()), ctypes.byref(o), _ptr(workspace.buf), workspace.buf.numel(),
                       _stream(dev))
    if code == L.VT_ERR_CAPACITY:
        return emit(n, params, workspace, {"nbr": o.needed_nbr, "vtx": o.needed_vtx, "face": o.needed_face,
                                           "face_vtx": o.needed_face_vtx})
    L.check(code)
    _trim(cells, o)
    return cells


def probe_fma(precision: str = "fp32") -> float:
    """Measured FMA throughput of the current device in TFLOP/s (vt_probe_fma)."""
    out = ctypes.c_double()
    dev = torch.device("cuda", torch.cuda.current_device())
    L.check(L.load().vt_probe_fma(_PREC[precision], ctypes.byref(out), _stream(dev)))
    return float(out.value)


def launch_count() -> int:
    return int(L.load().vt_launch_count())


def version() -> str:
    return L.load().vt_version().decode()


# ---------------------------------------------------------------------------
# adjoint of the cell moments, autograd and Lloyd relaxation
# ---------------------------------------------------------------------------

def moments_adjoint(points: torch.Tensor, cells: Cells, gV: torch.Tensor | None = None,
                    gC: torch.Tensor | None = None, gM: torch.Tensor | None = None,
                    precision: str = "fp64", params: Params | None = None) -> torch.Tensor:
    """d(sum gV.V + gC.c + gM.M2)/d(points) as float64 [n, 3] (vt_moments_adjoint).

    ``cells`` must come from :func:`tessellate` on ``points`` with emit
    including vol, cen and geom in the original index space. ``precision``
    ("fp64" or "fp32") is that of the face integrals: "fp32" for cells of the
    FP32 form. ``params`` gives the box and whether it is periodic (the
    tessellation's parameters; default the unit box)."""
    pts = _check_points(points)
    n = pts.shape[0]
    dev = pts.device
    grad = torch.empty((max(n, 1), 3), dtype=torch.float64, device=dev)
    o = _out_struct(cells)

    def f64(t):
        return None if t is None else t.to(device=dev, dtype=torch.float64).contiguous()

    gV, gC, gM = f64(gV), f64(gC), f64(gM)
    pc = Params(**{**(params or Params()).__dict__, "precision": precision}).c()
    L.check(L.load().vt_moments_adjoint(_ptr(pts), n, ctypes.byref(o), _ptr(gV), _ptr(gC), _ptr(gM),
                                        ctypes.byref(pc), _ptr(grad), _stream(dev)))
    return grad[:n]


class VoronoiMoments(torch.autograd.Function):
    """(V, c, M2) of every Voronoi cell of ``points``, differentiable in the points.

    forward: one tessellation (emit vol, cen, m2 and the geometry the adjoint
    needs). backward: the hand-written adjoint kernel (vt_moments_adjoint)."""

    @staticmethod
    def forward(ctx, points: torch.Tensor, params: Params | None = None):
        p = params or Params()
        p = Params(**{**p.__dict__, "emit": ("vol", "cen", "m2", "geom"), "index_space": "original"})
        cells = tessellate(points.detach(), p)
        ctx.cells = cells
        ctx.precision = p.precision
        ctx.params = p
        ctx.save_for_backward(points)
        return cells.vol, cells.cen, cells.m2

    @staticmethod
    def backward(ctx, gV, gC, gM):
        (points,) = ctx.saved_tensors
        g = moments_adjoint(points.detach(), ctx.cells, gV, gC, gM, precision=ctx.precision, params=ctx.params)
        return g.to(points.dtype), None


def voronoi_moments(points: torch.Tensor, params: Params | None = None):
    return VoronoiMoments.apply(points, params)


def lloyd_step(points: torch.Tensor, grad: torch.Tensor, vol: torch.Tensor, params: Params | None = None
               ) -> torch.Tensor:
    """One Lloyd update p <- p - grad / (2 vol) (vt_lloyd_step): the cell
    centroids when ``grad`` is the gradient of sum_i M2_i. Float32 points,
    FP64 gradient and volumes, all on the device; in a periodic box
    (``params.periodic``) the new points are wrapped into [box_lo, box_hi)."""
    pts = _check_points(points)
    n = pts.shape[0]
    dev = pts.device
    g = grad.to(device=dev, dtype=torch.float64).contiguous()
    v = vol.to(device=dev, dtype=torch.float64).contiguous()
    out = torch.empty_like(pts)
    pc = (params or Params()).c()
    L.check(L.load().vt_lloyd_step(_ptr(pts), n, _ptr(g), _ptr(v), ctypes.byref(pc), _ptr(out), _stream(dev)))
    return out


def lloyd(points: torch.Tensor, iterations: int, params: Params | None = None, checkpoint: str | None = None,
          checkpoint_every: int = 10, resume: bool = False, callback=None) -> torch.Tensor:
    """Lloyd relaxation: minimises sum_i M2_i by p <- p - g / (2 V), g the
    adjoint gradient of the loss (the step lands on the cell centroids).

    With ``checkpoint`` the points and the iteration are saved every
    ``checkpoint_every`` iterations (written to a temporary file and renamed,
    so an interrupted write leaves the previous checkpoint intact);
    ``resume=True`` continues from the file, or starts from ``points`` when
    no checkpoint has been written yet. The pipeline is deterministic, so a
    resumed run reproduces the points of an uninterrupted one bit for bit. In
    a periodic box (``params.periodic``) the new points are wrapped back into
    [box_lo, box_hi)."""
    import os

    p = points.detach().clone()
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        state = torch.load(checkpoint, map_location=p.device, weights_only=True)
        p = state["points"].to(p.device)
        start = int(state["iteration"])
    for it in range(start, iterations):
        q = p.clone().requires_grad_(True)
        vol, cen, m2 = voronoi_moments(q, params)
        loss = m2.sum()
        loss.backward()
        with torch.no_grad():
            p = lloyd_step(p, q.grad, vol.detach(), params)
        if callback is not None:
            callback(it, float(loss.detach()))
        if checkpoint and ((it + 1) % checkpoint_every == 0 or it + 1 == iterations):
            tmp = f"{checkpoint}.{os.getpid()}.tmp"
            torch.save({"points": p.cpu(), "iteration": it + 1}, tmp)
            os.replace(tmp, checkpoint)
    return p
