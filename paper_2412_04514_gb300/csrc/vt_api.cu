// vt_api.cu -- the C ABI (include/vt.h): argument checks, workspace layout
// and the host-side orchestration of the pass loop. Every step of the
// computation runs in the kernels of grid.cu, knn.cu, clip.cu, emit.cu and
// scan.cu; the host only launches them and reads a status block once per
// pass.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vt_internal.cuh"

namespace vt {

namespace {
thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_params(const vt_params* p)
{
    if (!p) return fail(VT_ERR_INVALID_ARG, "params is NULL");
    if (p->k0 < 1 || p->k0 > 256) return fail(VT_ERR_INVALID_ARG, "k0 must be in [1, 256], got %d", p->k0);
    if (p->k_max < p->k0 || p->k_max > 256)
        return fail(VT_ERR_INVALID_ARG, "k_max must be in [k0, 256], got %d", p->k_max);
    if (p->grid_res < 0 || p->grid_res > 1024) return fail(VT_ERR_INVALID_ARG, "grid_res must be in [0, 1024]");
    if (p->grid_res == 0 && !(p->grid_density > 0.0f))
        return fail(VT_ERR_INVALID_ARG, "grid_density must be > 0 when grid_res is 0");
    const int t = p->threads_per_cell;
    if (!(t == 0 || t == 8 || t == 16 || t == 32))
        return fail(VT_ERR_INVALID_ARG, "threads_per_cell must be 0, 8, 16 or 32, got %d", t);
    if (p->precision != VT_FP64 && p->precision != VT_FP32_RECHECK)
        return fail(VT_ERR_INVALID_ARG, "precision must be VT_FP64 or VT_FP32_RECHECK");
    if (p->index_space != VT_INDEX_ORIGINAL && p->index_space != VT_INDEX_SORTED)
        return fail(VT_ERR_INVALID_ARG, "index_space must be VT_INDEX_ORIGINAL or VT_INDEX_SORTED");
    if (p->flags & ~(VT_FLAG_STAGE_TIMES | VT_FLAG_NO_SYNC | VT_FLAG_PERIODIC | VT_FLAG_FUSED))
        return fail(VT_ERR_INVALID_ARG, "unknown flag bits 0x%x", p->flags);
    if (p->emit & ~(VT_EMIT_NBR | VT_EMIT_VOL | VT_EMIT_CEN | VT_EMIT_M2 | VT_EMIT_GEOM))
        return fail(VT_ERR_INVALID_ARG, "unknown emit bits 0x%x", p->emit);
    for (int a = 0; a < 3; ++a)
        if (!(std::isfinite(p->box_lo[a]) && std::isfinite(p->box_hi[a]) && p->box_hi[a] > p->box_lo[a]))
            return fail(VT_ERR_INVALID_ARG, "box must satisfy lo < hi (finite) on every axis");
    if (p->flags & VT_FLAG_PERIODIC) {
        // images shifted by more than two periods must be unable to cut: |L| <= 2 min L_a
        double l2 = 0, lmin = 0;
        for (int a = 0; a < 3; ++a) {
            const double L = (double)p->box_hi[a] - (double)p->box_lo[a];
            l2 += L * L;
            lmin = a == 0 || L < lmin ? L : lmin;
        }
        if (l2 > 4.0 * lmin * lmin)
            return fail(VT_ERR_INVALID_ARG, "a periodic box needs |L|^2 <= 4 min L_a^2 (got %g > %g)", l2,
                        4.0 * lmin * lmin);
    }
    return VT_OK;
}

// periodic lists pack a sorted index in 24 bits
int check_periodic_n(const vt_params* p, int64_t n)
{
    if ((p->flags & VT_FLAG_PERIODIC) && n >= ((int64_t)1 << 24))
        return fail(VT_ERR_INVALID_ARG, "a periodic box holds fewer than 2^24 points per call, got %lld", (long long)n);
    return VT_OK;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(VT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// true when device code can use p as it is: device or managed memory, or
// pinned host memory (mapped at the same address under unified addressing);
// NULL passes (optional buffers). A kernel is never launched on a pointer
// that fails, so a pageable host buffer is an argument error, not a fault.
bool device_accessible(const void* p)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.devicePointer == p;
}

// the caller's buffers of a call (skipped while the stream is being captured:
// the same buffers were checked by the uncaptured calls before)
int check_buffers(void* stream, const void* pts, const void* ws, const vt_cells_out* out,
                  const void* extra0 = nullptr, const void* extra1 = nullptr)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) (void)cudaGetLastError();
    if (cs != cudaStreamCaptureStatusNone) return VT_OK;
    if (!device_accessible(pts)) return fail(VT_ERR_INVALID_ARG, "pts is not device-accessible memory");
    if (!device_accessible(ws)) return fail(VT_ERR_INVALID_ARG, "the workspace is not device-accessible memory");
    if (!device_accessible(extra0) || !device_accessible(extra1))
        return fail(VT_ERR_INVALID_ARG, "the batch plan and set offsets must be device-accessible memory");
    if (out) {
        const void* ps[] = {out->vol, out->cen, out->m2, out->nbr_off, out->nbr, out->vtx_off, out->vtx,
                            out->face_off, out->face_nbr, out->face_vtx_off, out->face_vtx, out->perm};
        for (const void* q : ps)
            if (!device_accessible(q))
                return fail(VT_ERR_INVALID_ARG,
                            "an output buffer is not device-accessible memory (device, managed or pinned host)");
    }
    return VT_OK;
}

}  // namespace

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

int check_device_buffers(void* stream, const void* const* ptrs, const char* const* names, int count)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) (void)cudaGetLastError();
    if (cs != cudaStreamCaptureStatusNone) return VT_OK;
    for (int i = 0; i < count; ++i)
        if (!device_accessible(ptrs[i]))
            return fail(VT_ERR_INVALID_ARG, "%s is not device-accessible memory (device, managed or pinned host)",
                        names[i]);
    return VT_OK;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

static int grid_res_for(const vt_params* p, int64_t n)
{
    if (p->grid_res > 0) return p->grid_res;
    if (n <= 0) return 1;
    double g = std::ceil(std::cbrt((double)n / (double)p->grid_density) - 1e-9);
    double cap = std::ceil(std::cbrt(8.0 * (double)n)) + 1.0;
    if (g > cap) g = cap;
    if (g > 1024) g = 1024;
    if (g < 1) g = 1;
    return (int)g;
}

GridDesc make_grid(const vt_params* p, int G)
{
    GridDesc g;
    g.G = G;
    double ext_max = 0;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = p->box_lo[a];
        g.hi[a] = p->box_hi[a];
        const float ext = p->box_hi[a] - p->box_lo[a];
        g.scale[a] = (float)G / ext;
        g.cw[a] = ((double)p->box_hi[a] - (double)p->box_lo[a]) / (double)G;
        ext_max = std::fmax(ext_max, (double)p->box_hi[a] - (double)p->box_lo[a]);
    }
    // cell assignment in float32 may differ from exact arithmetic by a few
    // ulps of the scaled coordinate; the shell-walk stop rule stays clear of it
    g.margin = 16.0 * ext_max * std::ldexp(1.0, -24);
    g.cell_base = 0;
    g.pt_begin = 0;
    g.npts = 0;
    g.periodic = (p->flags & VT_FLAG_PERIODIC) ? 1 : 0;
    g.reserved = 0;
    return g;
}

Layout make_layout(const vt_params* p, int64_t n, int64_t cells, bool batch)
{
    Layout L{};
    L.G = grid_res_for(p, n);
    L.n = n;
    L.g3 = cells >= 0 ? cells : (int64_t)L.G * L.G * L.G;
    const int64_t nn = n > 0 ? n : 1;
    // list-mode passes run in chunks of knn_cap / k cells; the no-sync schedule
    // runs each pass in one launch, so its buffer holds n * max(k_max, the
    // range-list capacity) entries
    const bool nosync = (p->flags & VT_FLAG_NO_SYNC) != 0;
    // the first pass computes the second pass's list too when k doubles
    // within k_max (2 k0 entries per cell, all cells at once)
    const int kmx = p->k_max > RANGE_CAP ? p->k_max : RANGE_CAP;
    const int kpre = 2 * p->k0 <= p->k_max ? 2 * p->k0 : p->k0;
    // the fused schedule clips from the grid walk: no list buffer (one small
    // block keeps the layout uniform) and no saved polyhedra
    const bool fused = (p->flags & VT_FLAG_FUSED) != 0;
    int64_t cap = fused ? 64 : nn * (int64_t)(nosync ? (kmx > kpre ? kmx : kpre) : kpre);
    if (!fused && cap < (int64_t)p->k_max * 64) cap = (int64_t)p->k_max * 64;
    L.knn_cap = cap;
    // the robust variant's lists have their own buffer (the regular lists of
    // the first pass stay in place for the second): n / 8 cells of 128
    int64_t rc = nn / 8 > 65536 ? nn / 8 : 65536;
    L.rob_cap = rc * 128;
    const bool recs = (p->emit & (VT_EMIT_NBR | VT_EMIT_GEOM)) != 0;
    L.rec_stride = !recs ? 0
                         : ((p->emit & VT_EMIT_GEOM) ? (p->precision == VT_FP64 ? REC_STRIDE_GEOM : REC_STRIDE_GEOM_F32)
                                                     : REC_STRIDE_NBR);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    // the regions vt_emit reads come first: their offsets depend only on n
    // and the emit bits, so vt_emit works after single-set and batch runs alike
    L.status = take(sizeof(DevStatus));
    L.rec = take(L.rec_stride * (size_t)nn);
    L.cnt = take(sizeof(int32_t) * 4 * nn);
    L.off64 = take(sizeof(int64_t) * 4 * (nn + 1));
    L.scan_emit = take(scan_tmp_bytes(nn));
    L.cid = take(sizeof(int32_t) * nn);
    L.ticket = take(sizeof(int32_t) * nn);
    L.sorted = take(sizeof(float4) * nn);
    L.perm = take(sizeof(int32_t) * nn);
    L.list_a = take(sizeof(int32_t) * nn * 7);  // seven cell lists of n entries
    L.state_stride = fused ? 0 : clip_state_bytes(p->precision);
    L.state = take(L.state_stride * (size_t)nn);
    L.counts = take(sizeof(int32_t) * (L.g3 + 1));
    L.cell_off = take(sizeof(int32_t) * (L.g3 + 1));
    L.big = take(sizeof(int32_t) * (L.g3 + 1));
    size_t st1 = scan_tmp_bytes(L.g3), st2 = scan_tmp_bytes(nn);
    L.scan_tmp = take(st1 > st2 ? st1 : st2);
    L.knn_nbr = take(sizeof(int32_t) * L.knn_cap);
    // list keys: float in the FP32 form (its lists, range lists included, carry float keys)
    L.knn_d2 = take((p->precision == VT_FP64 ? sizeof(double) : sizeof(float)) * L.knn_cap);
    L.rob_nbr = take(sizeof(int32_t) * L.rob_cap);
    L.rob_d2 = take(sizeof(double) * L.rob_cap);
    L.set_of = batch ? take(sizeof(int32_t) * nn) : 0;
    L.ctr = take(sizeof(int32_t) * (4 * VT_MAX_PASSES + 8));
    L.rlen = take(sizeof(int32_t) * nn);
    L.total = off;
    return L;
}

}  // namespace vt

using namespace vt;

namespace vt_host {

// list length of the robust variant's exhaustive pass (nearest first, then the walk)
constexpr int ROBUST_EXH_K = 128;


// CUDA-event timing of kernel groups on the call's stream (VT_FLAG_STAGE_TIMES)
// CUDA-event stage timer (VT_FLAG_STAGE_TIMES); every stage is also an NVTX
// range, visible to any profiler that records NVTX (free when none does)
struct StageTimer {
    enum { GRID = 0, KNN = 1, CLIP = 2, EMIT = 3, KNNL = 4 };  // KNNL: the k-nearest-neighbour lists (within KNN)
    bool on = false;
    int nvtx_depth = 0;
    cudaStream_t s = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[5];
    std::vector<int> clip_pass;  // pass index of each CLIP event pair
    int pass = 0;
    int open_stage = -1;
    void begin(int stage)
    {
        static const char* const names[5] = {"vt grid sort", "vt range lists", "vt clip", "vt emit", "vt kNN"};
        nvtxRangePushA(names[stage]);
        ++nvtx_depth;
        if (!on) return;
        // without events the call runs untimed (stage times stay 0); the
        // failed creation is cleared so later launch checks do not see it
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess) {
            (void)cudaGetLastError();
            on = false;
            return;
        }
        if (cudaEventCreate(&b) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaEventDestroy(a);
            on = false;
            return;
        }
        cudaEventRecord(a, s);
        ev[stage].push_back({a, b});
        if (stage == CLIP) clip_pass.push_back(pass);
        open_stage = stage;
    }
    void per_pass(double* out, int n)
    {
        for (size_t i = 0; i < ev[CLIP].size(); ++i) {
            float ms = 0;
            if (clip_pass[i] < n && cudaEventElapsedTime(&ms, ev[CLIP][i].first, ev[CLIP][i].second) == cudaSuccess)
                out[clip_pass[i]] += ms;
        }
    }
    void end()
    {
        if (nvtx_depth > 0) {
            nvtxRangePop();
            --nvtx_depth;
        }
        if (!on || open_stage < 0) return;
        cudaEventRecord(ev[open_stage].back().second, s);
        open_stage = -1;
    }
    // call after the stream is synchronised
    double total(int stage)
    {
        double t = 0;
        for (auto& e : ev[stage]) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) t += ms;
        }
        return t;
    }
    ~StageTimer()
    {
        for (auto& v : ev)
            for (auto& e : v) {
                cudaEventDestroy(e.first);
                cudaEventDestroy(e.second);
            }
    }
};

struct Ctx {
    Layout L;
    uint8_t* base;
    cudaStream_t s;
    DevStatus* st;
    GridDesc g;
    // batches (null for a single point set)
    const GridDesc* sets = nullptr;
    const int64_t* set_off = nullptr;
    int nsets = 1;
    StageTimer* timer = nullptr;
    int* clip_launches = nullptr;
    int* knn_launches = nullptr;
    template <typename X>
    X* at(size_t off) const { return reinterpret_cast<X*>(base + off); }
    int32_t* set_of() const { return sets ? at<int32_t>(L.set_of) : nullptr; }
};

int make_ctx(const vt_params* p, int64_t n, void* ws, size_t ws_bytes, void* stream, Ctx& c, int64_t cells = -1,
             bool batch = false)
{
    int e = check_params(p);
    if (e) return e;
    if (n < 0 || n > (int64_t)INT32_MAX / 2) return fail(VT_ERR_INVALID_ARG, "n out of range: %lld", (long long)n);
    e = check_periodic_n(p, n);
    if (e) return e;
    c.L = make_layout(p, n, cells, batch);
    if (!ws) return fail(VT_ERR_WORKSPACE, "workspace is NULL");
    if (ws_bytes < c.L.total)
        return fail(VT_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes needed", ws_bytes, c.L.total);
    c.base = (uint8_t*)ws;
    c.s = (cudaStream_t)stream;
    c.st = c.at<DevStatus>(c.L.status);
    c.g = make_grid(p, c.L.G);
    c.g.npts = n;
    return VT_OK;
}

int read_status(const Ctx& c, DevStatus& h)
{
    cudaError_t e = cudaMemcpyAsync(&h, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    return VT_OK;
}

int zero_counters(const Ctx& c)
{
    cudaError_t e = cudaMemsetAsync(&c.st->n_fail_next, 0, 2 * sizeof(int32_t), c.s);
    return e == cudaSuccess ? VT_OK : cuda_fail(e, "counter reset");
}

__global__ void k_iota(int32_t* a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// one clip pass over `list` (m cells, or *m_dev cells when m_dev is set):
// kNN with k in chunks that fit the list buffer, then the clipper. With
// `exhaustive` the clipper then walks every generator within 2R (k = 0: no
// list, the regular variant resumes its saved state instead). Failures go to
// the given lists and counters.
int clip_pass(const Ctx& c, const vt_params* p, const int32_t* list, int64_t m, const int32_t* m_dev, int k,
              bool exhaustive, int k_prev, int variant, int knn_prec, vt_cells_out* out, int32_t* fail_next,
              int32_t* ctr_next, int32_t* fail_robust, int32_t* ctr_robust, int k_list = 0, bool reuse = false,
              int k_next = 0)
{
    const Layout& L = c.L;
    ClipArgs a{};
    a.sorted = c.at<float4>(L.sorted);
    a.cell_off = c.at<int32_t>(L.cell_off);
    a.g = c.g;
    a.sets = c.sets;
    a.set_of = c.set_of();
    a.nq_dev = m_dev;
    a.n = L.n;
    a.k = k;
    a.exhaustive = exhaustive ? 1 : 0;
    a.emit = p->emit;
    a.index_space = p->index_space;
    a.vol = (p->emit & VT_EMIT_VOL) ? out->vol : nullptr;
    a.cen = (p->emit & VT_EMIT_CEN) ? out->cen : nullptr;
    a.m2 = (p->emit & VT_EMIT_M2) ? out->m2 : nullptr;
    a.rec = L.rec_stride ? c.at<uint8_t>(L.rec) : nullptr;
    a.rec_stride = L.rec_stride;
    a.fail_next = fail_next;
    a.fail_robust = fail_robust;
    a.ctr_next = ctr_next;
    a.ctr_robust = ctr_robust;
    a.k_prev = k_prev;
    a.state = L.state_stride ? c.at<uint8_t>(L.state) : nullptr;  // none in the fused schedule
    a.state_stride = L.state_stride;
    a.st = c.st;
    a.rec_f32 = p->precision != VT_FP64 ? 1 : 0;
    a.queue = c.at<int32_t>(c.L.ctr) + CTR_QUEUE;
    const int tpc = p->threads_per_cell;
    StageTimer dummy;
    StageTimer& T = c.timer ? *c.timer : dummy;
    if (k == 0) {
        a.queries = list;
        a.nq = m;
        a.nq_cap = m;
        T.begin(StageTimer::CLIP);
        cudaError_t e = launch_clip(a, variant, tpc, c.s);
        T.end();
        if (c.clip_launches) ++*c.clip_launches;
        return e == cudaSuccess ? VT_OK : cuda_fail(e, "clip launch");
    }
    // k_list > k: the kNN computes k_list entries per cell (the next pass's
    // list too) and the clipper uses the first k; reuse: the lists of all
    // cells are already in the buffer, indexed by sorted cell index
    const int kl = k_list > k ? k_list : k;
    a.kstride = kl;
    a.k_next = k_next > k && k_next <= kl ? k_next : 0;
    a.by_cell = reuse ? 1 : 0;
    const bool rob = variant >= 2;  // the robust variants' lists have their own buffer
    int32_t* lnbr = c.at<int32_t>(rob ? L.rob_nbr : L.knn_nbr);
    void* ld2 = c.at<void>(rob ? L.rob_d2 : L.knn_d2);
    // chunks of the list buffer; a device-counted pass runs the same chunks
    // as launches that each clamp to the count they find (empty ones exit)
    const int64_t chunk = reuse ? (m > 0 ? m : 1) : (rob ? L.rob_cap : L.knn_cap) / kl;
    for (int64_t o = 0; o < m; o += chunk) {
        const int64_t cnt = (m - o) < chunk ? (m - o) : chunk;
        const int32_t* q = list ? list + o : nullptr;
        if (!list && o > 0) return fail(VT_ERR_INVALID_ARG, "internal: implicit list needs one chunk");
        if (!reuse) {
            T.begin(StageTimer::KNNL);
            cudaError_t e = launch_knn(a.sorted, a.cell_off, c.g, L.n, q, cnt, kl, knn_prec, lnbr, ld2, c.st, c.s,
                                       c.sets, c.set_of(), m_dev, o, c.at<int32_t>(L.ctr) + CTR_QUEUE);
            T.end();
            if (c.knn_launches) ++*c.knn_launches;
            if (e != cudaSuccess) return cuda_fail(e, "knn launch");
        }
        a.queries = q;
        a.nq = cnt;
        a.nq_cap = cnt;
        a.nq_off = o;
        a.nbr = lnbr;
        a.d2 = ld2;
        T.begin(StageTimer::CLIP);
        cudaError_t e = launch_clip(a, variant, tpc, c.s);
        T.end();
        if (c.clip_launches) ++*c.clip_launches;
        if (e != cudaSuccess) return cuda_fail(e, "clip launch");
    }
    return VT_OK;
}

// the last pass for resumed regular cells (`list`, m cells or *m_dev): range
// lists of every generator that can still cut, sorted nearest first, clipped
// as complete lists; cells with more candidates than a list holds go to
// over_list / over_ctr and the exhaustive walk. Failures go to fail_robust.
int range_pass(const Ctx& c, const vt_params* p, const int32_t* list, int64_t m, const int32_t* m_dev, int k_prev,
               int variant, vt_cells_out* out, int32_t* over_list, int32_t* over_ctr, int32_t* fail_robust,
               int32_t* ctr_robust, int32_t* unval, int32_t* ctr_unval)
{
    const Layout& L = c.L;
    StageTimer dummy;
    StageTimer& T = c.timer ? *c.timer : dummy;
    cudaError_t e = cudaMemsetAsync(over_ctr, 0, sizeof(int32_t), c.s);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    const int64_t chunk = L.knn_cap / RANGE_CAP;
    for (int64_t o = 0; o < m; o += chunk) {
        const int64_t cnt = (m - o) < chunk ? (m - o) : chunk;
        RangeArgs r{};
        r.sorted = c.at<float4>(L.sorted);
        r.cell_off = c.at<int32_t>(L.cell_off);
        r.g = c.g;
        r.sets = c.sets;
        r.set_of = c.set_of();
        r.queries = list + o;
        r.nq = cnt;
        r.nq_dev = m_dev;
        r.nq_off = o;
        r.state = c.at<uint8_t>(L.state);
        r.state_stride = L.state_stride;
        r.pos_off = clip_state_pos_offset(p->precision);
        r.precision = p->precision;
        r.rnbr = c.at<int32_t>(L.knn_nbr);
        r.rd2 = c.at<void>(L.knn_d2);
        r.rlen = c.at<int32_t>(L.rlen);
        r.over_list = over_list;
        r.over_ctr = over_ctr;
        r.st = c.st;
        r.queue = c.at<int32_t>(L.ctr) + CTR_QUEUE;
        T.begin(StageTimer::KNN);
        e = launch_range(r, c.s);
        T.end();
        if (c.knn_launches) ++*c.knn_launches;
        if (e != cudaSuccess) return cuda_fail(e, "range launch");
        ClipArgs a{};
        a.sorted = r.sorted;
        a.cell_off = r.cell_off;
        a.g = c.g;
        a.sets = c.sets;
        a.set_of = c.set_of();
        a.nq_dev = m_dev;
        a.n = L.n;
        a.queries = r.queries;
        a.nq = cnt;
        a.nq_cap = cnt;
        a.nq_off = o;
        a.nbr = r.rnbr;
        a.d2 = r.rd2;
        a.k = RANGE_CAP;
        a.klen = r.rlen;
        a.complete = 1;
        a.restore = 1;
        a.emit = p->emit;
        a.index_space = p->index_space;
        a.vol = (p->emit & VT_EMIT_VOL) ? out->vol : nullptr;
        a.cen = (p->emit & VT_EMIT_CEN) ? out->cen : nullptr;
        a.m2 = (p->emit & VT_EMIT_M2) ? out->m2 : nullptr;
        a.rec = L.rec_stride ? c.at<uint8_t>(L.rec) : nullptr;
        a.rec_stride = L.rec_stride;
        a.fail_next = unval;  // a complete list never asks for more
        a.ctr_next = ctr_unval;
        a.fail_robust = fail_robust;
        a.ctr_robust = ctr_robust;
        a.state = c.at<uint8_t>(L.state);
        a.state_stride = L.state_stride;
        a.st = c.st;
        a.rec_f32 = p->precision != VT_FP64 ? 1 : 0;
        a.queue = c.at<int32_t>(c.L.ctr) + CTR_QUEUE;
        T.begin(StageTimer::CLIP);
        e = launch_clip(a, variant, p->threads_per_cell, c.s);
        T.end();
        if (c.clip_launches) ++*c.clip_launches;
        if (e != cudaSuccess) return cuda_fail(e, "clip launch");
    }
    // the overflowed cells: the clipper's own walk, resuming the saved state
    return clip_pass(c, p, over_list, m, over_ctr, 0, true, k_prev, variant, p->precision, out, unval, ctr_unval,
                     fail_robust, ctr_robust);
}

int status_errors(const DevStatus& h)
{
    if (h.check_fail) return fail(VT_ERR_INTERNAL, "a debug bounds check failed (code %d)", h.check_fail);
    if (h.bad_point)
        return fail(VT_ERR_INVALID_ARG, "point %d is not finite or not inside [box_lo, box_hi)", h.bad_point - 1);
    if (h.duplicate) return fail(VT_ERR_DUPLICATE_POINTS, "two generators coincide");
    return VT_OK;
}

int emit_outputs(const Ctx& c, const vt_params* p, vt_cells_out* out)
{
    const Layout& L = c.L;
    const int64_t n = L.n;
    if (!(p->emit & (VT_EMIT_NBR | VT_EMIT_GEOM))) return VT_OK;
    const bool nosync = (p->flags & VT_FLAG_NO_SYNC) != 0;
    if (n == 0 && nosync) return VT_OK;
    if (n == 0) {
        int64_t z = 0;
        if ((p->emit & VT_EMIT_NBR) && out->nbr_off)
            cudaMemcpyAsync(out->nbr_off, &z, sizeof(z), cudaMemcpyHostToDevice, c.s);
        if (p->emit & VT_EMIT_GEOM) {
            if (out->vtx_off) cudaMemcpyAsync(out->vtx_off, &z, sizeof(z), cudaMemcpyHostToDevice, c.s);
            if (out->face_off) cudaMemcpyAsync(out->face_off, &z, sizeof(z), cudaMemcpyHostToDevice, c.s);
            if (out->face_vtx_off) cudaMemcpyAsync(out->face_vtx_off, &z, sizeof(z), cudaMemcpyHostToDevice, c.s);
        }
        cudaStreamSynchronize(c.s);
        out->needed_nbr = out->needed_vtx = out->needed_face = out->needed_face_vtx = 0;
        return VT_OK;
    }
    EmitArgs e{};
    e.n = n;
    e.emit = p->emit;
    e.vtx_f32 = p->precision != VT_FP64 ? 1 : 0;
    e.rec = c.at<uint8_t>(L.rec);
    e.rec_stride = L.rec_stride;
    e.cnt = c.at<int32_t>(L.cnt);
    e.off64 = c.at<int64_t>(L.off64);
    e.scan_tmp = c.at<void>(L.scan_emit);
    e.st = c.st;
    // a buffer may be NULL only when its capacity is 0
    if ((p->emit & VT_EMIT_NBR) && (!out->nbr_off || (!out->nbr && out->nbr_cap > 0)))
        return fail(VT_ERR_INVALID_ARG, "VT_EMIT_NBR needs nbr_off and nbr");
    if ((p->emit & VT_EMIT_GEOM) &&
        (!out->vtx_off || !out->face_off || !out->face_vtx_off || (!out->vtx && out->vtx_cap > 0) ||
         (!out->face_nbr && out->face_cap > 0) || (!out->face_vtx && out->face_vtx_cap > 0)))
        return fail(VT_ERR_INVALID_ARG, "VT_EMIT_GEOM needs every geometry pointer");
    StageTimer dummy;
    StageTimer& T = c.timer ? *c.timer : dummy;
    T.begin(StageTimer::EMIT);
    cudaError_t ce = launch_emit_count(e, c.s);
    T.end();
    if (ce != cudaSuccess) return cuda_fail(ce, "emit count");
    if (nosync) {  // capacities are checked on the device; vt_read_stats reports them
        ce = launch_emit_write(e, *out, c.s);
        return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "emit write");
    }
    DevStatus h;
    int r = read_status(c, h);
    if (r) return r;
    out->needed_nbr = h.totals[0];
    out->needed_vtx = h.totals[1];
    out->needed_face = h.totals[2];
    out->needed_face_vtx = h.totals[3];
    if (h.record_overflow) return fail(VT_ERR_CAPACITY, "%d cells exceed the per-cell record size", h.record_overflow);
    if (p->emit & VT_EMIT_NBR) {
        if (out->nbr_cap < h.totals[0])
            return fail(VT_ERR_CAPACITY, "nbr_cap %lld < needed %lld", (long long)out->nbr_cap, (long long)h.totals[0]);
    }
    if (p->emit & VT_EMIT_GEOM) {
        if (out->vtx_cap < h.totals[1] || out->face_cap < h.totals[2] || out->face_vtx_cap < h.totals[3])
            return fail(VT_ERR_CAPACITY, "geometry buffers too small (need vtx %lld, faces %lld, face_vtx %lld)",
                        (long long)h.totals[1], (long long)h.totals[2], (long long)h.totals[3]);
    }
    T.begin(StageTimer::EMIT);
    ce = launch_emit_write(e, *out, c.s);
    T.end();
    if (ce != cudaSuccess) return cuda_fail(ce, "emit write");
    return VT_OK;
}


// the whole path on an initialised context (single set or batch)
int tessellate_run(Ctx& c, const float* pts, int64_t n, const vt_params* p, vt_cells_out* out, vt_stats* stats)
{
    if (!out) return fail(VT_ERR_INVALID_ARG, "out is NULL");
    if (n > 0 && !pts) return fail(VT_ERR_INVALID_ARG, "pts is NULL");
    if ((p->emit & VT_EMIT_VOL) && n > 0 && !out->vol) return fail(VT_ERR_INVALID_ARG, "VT_EMIT_VOL needs vol");
    if ((p->emit & VT_EMIT_CEN) && n > 0 && !out->cen) return fail(VT_ERR_INVALID_ARG, "VT_EMIT_CEN needs cen");
    if ((p->emit & VT_EMIT_M2) && n > 0 && !out->m2) return fail(VT_ERR_INVALID_ARG, "VT_EMIT_M2 needs m2");
    const bool nosync = (p->flags & VT_FLAG_NO_SYNC) != 0;
    const bool fused = (p->flags & VT_FLAG_FUSED) != 0;  // one walk pass from the box, no lists
    if (nosync && (p->flags & VT_FLAG_STAGE_TIMES))
        return fail(VT_ERR_INVALID_ARG, "VT_FLAG_STAGE_TIMES needs the synchronising schedule");
    const int64_t l0 = launches();
    vt_stats S{};
    S.grid_res = c.sets ? 0 : c.L.G;
    const Layout& L = c.L;
    StageTimer timer;
    timer.on = (p->flags & VT_FLAG_STAGE_TIMES) != 0;
    timer.s = c.s;
    c.timer = &timer;
    c.clip_launches = &S.clip_launches;
    c.knn_launches = &S.knn_launches;
    cudaError_t ce = cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c.at<int32_t>(L.ctr), 0, sizeof(int32_t) * (4 * VT_MAX_PASSES + 8), c.s);
    if (ce != cudaSuccess) return cuda_fail(ce, "status reset");
    if (n > 0) {
        timer.begin(StageTimer::GRID);
        BatchArgs b{c.sets, c.set_off, c.nsets, c.set_of()};
        ce = launch_grid_build(pts, n, c.g, c.at<float4>(L.sorted), c.at<int32_t>(L.perm), c.at<int32_t>(L.cell_off),
                               c.at<int32_t>(L.cid), c.at<int32_t>(L.ticket), c.at<int32_t>(L.counts),
                               c.at<int32_t>(L.big), c.at<void>(L.scan_tmp), c.st, c.s, c.sets ? &b : nullptr, L.g3);
        timer.end();
        if (ce != cudaSuccess) return cuda_fail(ce, "grid build");
        if (out->perm) {
            ce = cudaMemcpyAsync(out->perm, c.at<int32_t>(L.perm), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c.s);
            if (ce != cudaSuccess) return cuda_fail(ce, "perm copy");
        }
    }
    // six lists of n cells: regular current/next, robust current/next, robust new, unvalidated
    int32_t* lists = c.at<int32_t>(L.list_a);
    int32_t* reg_cur = lists;
    int32_t* reg_nxt = lists + n;
    int32_t* rob_cur = lists + 2 * n;
    int32_t* rob_nxt = lists + 3 * n;
    int32_t* rob_new = lists + 4 * n;
    int32_t* unval = lists + 5 * n;
    // the FP32 form's robust cells run first in FP32 with the robust capacity
    // (variant 3); what that cannot finish goes to the FP64 robust variant
    // through this list
    int32_t* rob64 = lists + 6 * n;
    const bool fp32 = p->precision != VT_FP64;
    const int variant_rob = fp32 ? 3 : 2;
    const int prec_rob = fp32 ? p->precision : VT_FP64;
    const int variant_reg = p->precision == VT_FP64 ? 1 : 0;
    int r = VT_OK;
    DevStatus h{};

    if (nosync && n > 0) {
        // fixed schedule, counts stay on the device: capturable in a CUDA graph.
        // Pass i reads its regular cells from the list pass i-1 appended to
        // (count ctr_reg[i-1]); robust cells of pass i are the new ones
        // (ctr_new[i]) and the ones carried from pass i-1 (ctr_rob[i-1]).
        int32_t* ctr_reg = c.at<int32_t>(L.ctr);
        int32_t* ctr_new = ctr_reg + VT_MAX_PASSES;
        int32_t* ctr_rob = ctr_new + VT_MAX_PASSES;
        int32_t* regl[2] = {reg_cur, reg_nxt};
        int32_t* robl[2] = {rob_cur, rob_nxt};
        // the first two list passes (k0 and 2 k0) run as one launch over the
        // 2 k0 list when 2 k0 <= k_max (same cells as a re-queue: validation
        // is tested before every entry)
        int ks[VT_MAX_PASSES];
        int np_ = 0;
        const bool merge = !fused && 2 * p->k0 <= p->k_max;
        if (!fused)
            for (int k = merge ? 2 * p->k0 : p->k0; k <= p->k_max && np_ < VT_MAX_PASSES - 1; k *= 2) ks[np_++] = k;
        ks[np_++] = 0;
        int k_prev = 0;
        int lp = 0;  // logical pass (stats)
        if (merge) S.k_of_pass[lp++] = p->k0;
        for (int pi = 0; pi < np_; ++pi) {
            const int kk = ks[pi];
            if (lp < VT_MAX_PASSES) S.k_of_pass[lp] = kk;
            ++lp;
            const int32_t* q = pi == 0 ? nullptr : regl[pi % 2];
            const int32_t* qn = pi == 0 ? nullptr : &ctr_reg[pi - 1];
            // the exhaustive pass always concludes; anything it still hands on
            // is counted as unvalidated rather than dropped
            const bool last = kk == 0;
            int32_t* rn = last ? unval : regl[(pi + 1) % 2];
            int32_t* rc = last ? &c.st->n_unval : &ctr_reg[pi];
            int32_t* bn = last ? unval : robl[(pi + 1) % 2];
            int32_t* bc = last ? &c.st->n_unval : &ctr_rob[pi];
            const int kr = last ? ROBUST_EXH_K : kk;  // the robust variant's list
            const bool merged = merge && pi == 0;
            if (last && pi > 0)
                r = range_pass(c, p, q, n, qn, k_prev, variant_reg, out, regl[(pi + 1) % 2], &ctr_reg[pi], rob_new,
                               &ctr_new[pi], unval, &c.st->n_unval);
            else
                r = clip_pass(c, p, q, n, qn, merged ? p->k0 : kk, last, k_prev, variant_reg, p->precision, out, rn,
                              rc, rob_new, &ctr_new[pi], merged ? kk : 0, false, merged ? kk : 0);
            if (r) return r;
            int32_t* ctr64 = ctr_rob + VT_MAX_PASSES;
            int32_t* fl = fp32 ? rob64 : unval;
            int32_t* fc = fp32 ? &ctr64[pi] : &c.st->n_unval;
            r = clip_pass(c, p, rob_new, n, &ctr_new[pi], kr, last, 0, variant_rob, prec_rob, out, bn, bc, fl, fc);
            if (r) return r;
            if (pi > 0) {
                r = clip_pass(c, p, robl[pi % 2], n, &ctr_rob[pi - 1], kr, last, 0, variant_rob, prec_rob, out, bn, bc,
                              fl, fc);
                if (r) return r;
            }
            if (fp32) {
                r = clip_pass(c, p, rob64, n, &ctr64[pi], kr, last, 0, 2, VT_FP64, out, bn, bc, unval,
                              &c.st->n_unval);
                if (r) return r;
            }
            if (kk) k_prev = kk;
        }
        S.passes = lp;
        ce = launch_mark_unvalidated(unval, &c.st->n_unval, 0, n, c.at<float4>(L.sorted), p->index_space,
                                     (p->emit & VT_EMIT_VOL) ? out->vol : nullptr,
                                     (p->emit & VT_EMIT_CEN) ? out->cen : nullptr,
                                     (p->emit & VT_EMIT_M2) ? out->m2 : nullptr, c.st, c.s);
        if (ce != cudaSuccess) return cuda_fail(ce, "unvalidated marks");
        r = emit_outputs(c, p, out);
        S.launches = (int)(launches() - l0);
        if (stats) *stats = S;
        return r;
    }

    int64_t m_reg = n, m_rob = 0, n_unval = 0;
    bool implicit = true;  // the first pass runs over all cells without a list
    int k = fused ? p->k_max + 1 : p->k0;  // fused: the exhaustive walk is the first pass
    int k_prev = 0;  // regular cells resume from their saved state after list entry k_prev

    while (m_reg + m_rob > 0) {
        const bool exhaustive = k > p->k_max;
        const int kk = exhaustive ? 0 : k;
        const bool merged = implicit && !exhaustive && 2 * k <= p->k_max && (int64_t)2 * k * m_reg <= L.knn_cap;
        if (S.passes < VT_MAX_PASSES) {
            S.k_of_pass[S.passes] = kk;
            S.cells_of_pass[S.passes] = m_reg + m_rob;
        }
        timer.pass = S.passes;
        ++S.passes;
        if (exhaustive) S.exhaustive_cells = m_reg + m_rob;
        int64_t got_next = 0, got_rob = 0;
        if (m_reg > 0) {
            if ((r = zero_counters(c))) return r;
            if (implicit && (int64_t)kk * m_reg > L.knn_cap) {
                k_iota<<<(unsigned)((m_reg + 255) / 256 < 152 * 64 ? (m_reg + 255) / 256 : 152 * 64), 256, 0, c.s>>>(
                    reg_cur, m_reg);
                count_launch();
                implicit = false;
            }
            const bool by_range = exhaustive && k_prev > 0 && !implicit;
            if (by_range)
                r = range_pass(c, p, reg_cur, m_reg, nullptr, k_prev, variant_reg, out, reg_nxt, &c.st->n_range_over,
                               rob_new, &c.st->n_fail_robust, unval + n_unval, &c.st->n_fail_next);
            else
                // the first two list passes (k and 2 k) run as one launch over
                // the 2 k list when 2 k <= k_max: a cell the first k entries
                // leave open continues at entry k (validation is tested before
                // every entry, so the cells are those of a re-queue)
                r = clip_pass(c, p, implicit ? nullptr : reg_cur, m_reg, nullptr, kk, exhaustive, k_prev, variant_reg,
                              p->precision, out, reg_nxt, &c.st->n_fail_next, rob_new, &c.st->n_fail_robust,
                              merged ? 2 * kk : 0, false, merged ? 2 * kk : 0);
            if (r) return r;
            if ((r = read_status(c, h))) return r;
            if ((r = status_errors(h))) return r;
            got_next = h.n_fail_next;
            got_rob = h.n_fail_robust;
            if (exhaustive && got_next > 0) {
                // the exhaustive pass concludes every cell; what it hands on
                // is unvalidated (range lists write it to unval + n_unval)
                if (!by_range) {
                    ce = cudaMemcpyAsync(unval + n_unval, reg_nxt, sizeof(int32_t) * got_next,
                                         cudaMemcpyDeviceToDevice, c.s);
                    if (ce != cudaSuccess) return cuda_fail(ce, "list copy");
                }
                n_unval += got_next;
                got_next = 0;
            }
        }
        implicit = false;
        if (got_rob > 0) {
            ce = cudaMemcpyAsync(rob_cur + m_rob, rob_new, sizeof(int32_t) * got_rob, cudaMemcpyDeviceToDevice, c.s);
            if (ce != cudaSuccess) return cuda_fail(ce, "list copy");
            m_rob += got_rob;
        }
        int64_t rob_next = 0;
        const int kr = exhaustive ? ROBUST_EXH_K : (merged ? 2 * kk : kk);
        if (m_rob > 0) {
            if ((r = zero_counters(c))) return r;
            r = clip_pass(c, p, rob_cur, m_rob, nullptr, kr, exhaustive, 0, variant_rob, prec_rob, out, rob_nxt,
                          &c.st->n_fail_next, fp32 ? rob64 : unval + n_unval, &c.st->n_fail_robust);
            if (r) return r;
            if ((r = read_status(c, h))) return r;
            if ((r = status_errors(h))) return r;
            rob_next = h.n_fail_next;
            const int64_t failed = h.n_fail_robust;
            if (fp32 && failed > 0) {  // the FP64 robust variant for what FP32 could not finish
                if ((r = zero_counters(c))) return r;
                r = clip_pass(c, p, rob64, failed, nullptr, kr, exhaustive, 0, 2, VT_FP64, out, rob_nxt + rob_next,
                              &c.st->n_fail_next, unval + n_unval, &c.st->n_fail_robust);
                if (r) return r;
                if ((r = read_status(c, h))) return r;
                if ((r = status_errors(h))) return r;
                rob_next += h.n_fail_next;
                n_unval += h.n_fail_robust;
            } else if (!fp32) {
                n_unval += failed;
            }
        }
        std::swap(reg_cur, reg_nxt);
        std::swap(rob_cur, rob_nxt);
        m_reg = got_next;
        m_rob = rob_next;
        if (exhaustive) {
            if (m_rob > 0) {  // cannot happen: the exhaustive pass always concludes
                ce = cudaMemcpyAsync(unval + n_unval, rob_cur, sizeof(int32_t) * m_rob, cudaMemcpyDeviceToDevice, c.s);
                if (ce != cudaSuccess) return cuda_fail(ce, "list copy");
                n_unval += m_rob;
            }
            break;
        }
        if (merged) {  // the second list pass ran inside this one
            if (S.passes < VT_MAX_PASSES) {
                S.k_of_pass[S.passes] = 2 * k;
                S.cells_of_pass[S.passes] = h.n_second;
            }
            ++S.passes;
            k *= 2;
        }
        k_prev = k;
        k *= 2;
    }
    S.unvalidated = n_unval;
    if (n_unval > 0) {
        ce = launch_mark_unvalidated(unval, nullptr, n_unval, n_unval, c.at<float4>(L.sorted), p->index_space,
                                     (p->emit & VT_EMIT_VOL) ? out->vol : nullptr,
                                     (p->emit & VT_EMIT_CEN) ? out->cen : nullptr,
                                     (p->emit & VT_EMIT_M2) ? out->m2 : nullptr, c.st, c.s);
        if (ce != cudaSuccess) return cuda_fail(ce, "unvalidated marks");
    }
    r = emit_outputs(c, p, out);
    if ((r = r ? r : read_status(c, h)) || (r = h.check_fail ? status_errors(h) : VT_OK)) {
        if (stats) *stats = S;
        return r;
    }
    S.fp64_rechecks = (int64_t)h.fp64_rechecks;
    S.capacity_retries = (int64_t)h.capacity_events;
    S.precision_retries = (int64_t)h.precision_events;
    for (int a = 0; a < 5; ++a) S.clip_events[a] = (int64_t)h.detail[a];
    S.knn_candidates = (int64_t)h.knn_evals;
    S.knn_queries = (int64_t)h.knn_queries;
    S.walk_cells = (int64_t)h.walk_cells;
    S.walk_candidates = (int64_t)h.walk_cands;
    S.launches = (int)(launches() - l0);
    if (timer.on) {
        S.ms_grid = timer.total(StageTimer::GRID);
        S.ms_knn_lists = timer.total(StageTimer::KNNL);
        S.ms_knn = timer.total(StageTimer::KNN) + S.ms_knn_lists;
        S.ms_clip = timer.total(StageTimer::CLIP);
        S.ms_emit = timer.total(StageTimer::EMIT);
        timer.per_pass(S.ms_clip_pass, VT_MAX_PASSES);
    }
    if (stats) *stats = S;
    if (n_unval > 0) return fail(VT_ERR_UNVALIDATED, "%lld cells could not be validated", (long long)n_unval);
    return VT_OK;
}

}  // namespace vt_host

using namespace vt_host;

extern "C" {

void vt_params_default(vt_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k0 = 16;
    p->k_max = 32;
    p->grid_density = 2.0f;
    p->grid_res = 0;
    p->threads_per_cell = 0;
    p->precision = VT_FP32_RECHECK;
    p->emit = VT_EMIT_NBR | VT_EMIT_VOL | VT_EMIT_CEN;
    p->index_space = VT_INDEX_ORIGINAL;
    for (int a = 0; a < 3; ++a) { p->box_lo[a] = 0.0f; p->box_hi[a] = 1.0f; }
}

int vt_grid_resolution(const vt_params* p, int64_t n)
{
    if (check_params(p)) return -1;
    return grid_res_for(p, n);
}

int vt_workspace_size(const vt_params* p, int64_t n, size_t* bytes)
{
    int e = check_params(p);
    if (e) return e;
    if (n < 0 || !bytes) return fail(VT_ERR_INVALID_ARG, "n < 0 or bytes is NULL");
    e = check_periodic_n(p, n);
    if (e) return e;
    *bytes = make_layout(p, n).total;
    return VT_OK;
}

int vt_grid_build(const float* pts, int64_t n, const vt_params* p, int G, float* sorted, int32_t* perm,
                  int32_t* cell_off, void* ws, size_t ws_bytes, void* stream)
{
    Ctx c;
    int e = make_ctx(p, n, ws, ws_bytes, stream, c);
    if (e) return e;
    if (G != c.L.G) return fail(VT_ERR_INVALID_ARG, "G = %d differs from vt_grid_resolution = %d", G, c.L.G);
    if ((n > 0 && (!pts || !sorted || !perm)) || !cell_off) return fail(VT_ERR_INVALID_ARG, "NULL buffer");
    {
        const void* ptrs[] = {pts, sorted, perm, cell_off, ws};
        const char* names[] = {"pts", "sorted", "perm", "cell_off", "the workspace"};
        if ((e = check_device_buffers(stream, ptrs, names, 5))) return e;
    }
    cudaError_t ce = cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s);
    if (ce != cudaSuccess) return cuda_fail(ce, "status reset");
    ce = launch_grid_build(pts, n, c.g, (float4*)sorted, perm, cell_off, c.at<int32_t>(c.L.cid),
                           c.at<int32_t>(c.L.ticket), c.at<int32_t>(c.L.counts), c.at<int32_t>(c.L.big),
                           c.at<void>(c.L.scan_tmp), c.st, c.s);
    return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "grid build");
}

int vt_knn(const float* sorted, const int32_t* cell_off, int G, int64_t n, const int32_t* queries, int64_t nq, int k,
           const vt_params* p, int32_t* nbr, void* d2, void* ws, size_t ws_bytes, void* stream)
{
    Ctx c;
    int e = make_ctx(p, n, ws, ws_bytes, stream, c);
    if (e) return e;
    if (G != c.L.G) return fail(VT_ERR_INVALID_ARG, "G = %d differs from vt_grid_resolution = %d", G, c.L.G);
    if (k < 1 || k > 256) return fail(VT_ERR_INVALID_ARG, "k must be in [1, 256], got %d", k);
    if (nq < 0 || (nq > 0 && (!sorted || !cell_off || !nbr))) return fail(VT_ERR_INVALID_ARG, "bad buffers");
    if (!queries && nq > n) return fail(VT_ERR_INVALID_ARG, "nq > n without a query list");
    {
        const void* ptrs[] = {sorted, cell_off, queries, nbr, d2, ws};
        const char* names[] = {"sorted", "cell_off", "queries", "nbr", "d2", "the workspace"};
        if ((e = check_device_buffers(stream, ptrs, names, 6))) return e;
    }
    cudaError_t ce = launch_knn((const float4*)sorted, cell_off, c.g, n, queries, nq, k, p->precision, nbr, d2, c.st, c.s,
                                nullptr, nullptr, nullptr, 0, c.at<int32_t>(c.L.ctr) + CTR_QUEUE);
    return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "knn");
}

int vt_clip_cells(const float* sorted, const int32_t* cell_off, int G, int64_t n, const int32_t* queries, int64_t nq,
                  const int32_t* nbr, const void* d2, int k, const vt_params* p, vt_cells_out* out, int32_t* failed,
                  int32_t* n_failed, void* ws, size_t ws_bytes, void* stream)
{
    Ctx c;
    int e = make_ctx(p, n, ws, ws_bytes, stream, c);
    if (e) return e;
    if (G != c.L.G) return fail(VT_ERR_INVALID_ARG, "G = %d differs from vt_grid_resolution = %d", G, c.L.G);
    if (k < 0 || k > 256) return fail(VT_ERR_INVALID_ARG, "k must be in [0, 256]");
    if (!out || !failed || !n_failed || !sorted || !cell_off) return fail(VT_ERR_INVALID_ARG, "NULL buffer");
    if (k > 0 && (!nbr || !d2)) return fail(VT_ERR_INVALID_ARG, "list mode needs nbr and d2");
    if (!queries && nq > n) return fail(VT_ERR_INVALID_ARG, "nq > n without a query list");
    {
        const void* ptrs[] = {sorted, cell_off, queries, nbr, d2, failed, n_failed};
        const char* names[] = {"sorted", "cell_off", "queries", "nbr", "d2", "failed", "n_failed"};
        if ((e = check_device_buffers(stream, ptrs, names, 7))) return e;
        if ((e = check_buffers(stream, nullptr, ws, out))) return e;
    }
    ClipArgs a{};
    a.sorted = (const float4*)sorted;
    a.cell_off = cell_off;
    a.g = c.g;
    a.n = n;
    a.queries = queries;
    a.nq = nq;
    a.nbr = nbr;
    a.d2 = d2;
    a.k = k;
    a.exhaustive = k == 0 ? 1 : 0;
    a.nq_cap = nq;
    a.emit = p->emit;
    a.index_space = p->index_space;
    a.vol = (p->emit & VT_EMIT_VOL) ? out->vol : nullptr;
    a.cen = (p->emit & VT_EMIT_CEN) ? out->cen : nullptr;
    a.m2 = (p->emit & VT_EMIT_M2) ? out->m2 : nullptr;
    a.rec = c.L.rec_stride ? c.at<uint8_t>(c.L.rec) : nullptr;
    a.rec_stride = c.L.rec_stride;
    a.fail_next = failed;
    a.fail_robust = failed;
    a.ctr_next = n_failed;
    a.ctr_robust = n_failed;
    a.st = c.st;
    a.rec_f32 = p->precision != VT_FP64 ? 1 : 0;
    a.queue = c.at<int32_t>(c.L.ctr) + CTR_QUEUE;
    cudaError_t ce = launch_clip(a, p->precision == VT_FP64 ? 1 : 0, p->threads_per_cell, c.s);
    return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "clip");
}

int vt_emit(int64_t n, const vt_params* p, vt_cells_out* out, void* ws, size_t ws_bytes, void* stream)
{
    Ctx c;
    int e = make_ctx(p, n, ws, ws_bytes, stream, c);
    if (e) return e;
    if (!out) return fail(VT_ERR_INVALID_ARG, "out is NULL");
    e = check_buffers(stream, nullptr, ws, out);
    if (e) return e;
    return emit_outputs(c, p, out);
}

int vt_tessellate(const float* pts, int64_t n, const vt_params* p, vt_cells_out* out, vt_stats* stats, void* ws,
                  size_t ws_bytes, void* stream)
{
    Ctx c;
    int e = make_ctx(p, n, ws, ws_bytes, stream, c);
    if (e) return e;
    e = check_buffers(stream, pts, ws, out);
    if (e) return e;
    return tessellate_run(c, pts, n, p, out, stats);
}

int vt_batch_plan(const int64_t* set_off, int n_sets, const vt_params* p, const int* grid_res, vt_set_desc* plan,
                  int64_t* total_cells)
{
    int e = check_params(p);
    if (e) return e;
    if (n_sets < 1 || !set_off || !plan || !total_cells) return fail(VT_ERR_INVALID_ARG, "bad batch plan arguments");
    if (set_off[0] != 0) return fail(VT_ERR_INVALID_ARG, "set_off[0] must be 0");
    int64_t cells = 0;
    for (int sidx = 0; sidx < n_sets; ++sidx) {
        const int64_t ns = set_off[sidx + 1] - set_off[sidx];
        if (ns < 0) return fail(VT_ERR_INVALID_ARG, "set_off must be non-decreasing");
        int G = grid_res && grid_res[sidx] > 0 ? grid_res[sidx] : grid_res_for(p, ns);
        if (G > 1024) return fail(VT_ERR_INVALID_ARG, "grid resolution of set %d above 1024", sidx);
        GridDesc g = make_grid(p, G);
        g.cell_base = cells;
        g.pt_begin = set_off[sidx];
        g.npts = ns;
        std::memcpy(&plan[sidx], &g, sizeof(g));
        cells += (int64_t)G * G * G;
    }
    if (cells > (int64_t)INT32_MAX / 2) return fail(VT_ERR_INVALID_ARG, "too many grid cells in the batch");
    *total_cells = cells;
    return VT_OK;
}

int vt_batch_workspace_size(const vt_params* p, int64_t n_total, int64_t total_cells, size_t* bytes)
{
    int e = check_params(p);
    if (e) return e;
    if (n_total < 0 || total_cells < 1 || !bytes) return fail(VT_ERR_INVALID_ARG, "bad batch sizes");
    e = check_periodic_n(p, n_total);
    if (e) return e;
    *bytes = make_layout(p, n_total, total_cells, true).total;
    return VT_OK;
}

int vt_tessellate_batch(const float* pts, int64_t n_total, const vt_set_desc* plan, const int64_t* set_off,
                        int n_sets, int64_t total_cells, const vt_params* p, vt_cells_out* out, vt_stats* stats,
                        void* ws, size_t ws_bytes, void* stream)
{
    if (n_sets < 1 || !plan || !set_off || total_cells < 1)
        return fail(VT_ERR_INVALID_ARG, "a batch needs its device plan, set offsets and cell count");
    Ctx c;
    int e = make_ctx(p, n_total, ws, ws_bytes, stream, c, total_cells, true);
    if (e) return e;
    e = check_buffers(stream, pts, ws, out, plan, set_off);
    if (e) return e;
    c.sets = reinterpret_cast<const GridDesc*>(plan);
    c.set_off = set_off;
    c.nsets = n_sets;
    return tessellate_run(c, pts, n_total, p, out, stats);
}

int vt_moments_adjoint(const float* pts, int64_t n, const vt_cells_out* cells, const double* gV, const double* gC,
                       const double* gM, const vt_params* p, double* grad, void* stream)
{
    if (n < 0) return fail(VT_ERR_INVALID_ARG, "n must be >= 0");
    vt_params dflt;
    if (!p) {
        vt_params_default(&dflt);
        dflt.precision = VT_FP64;
        p = &dflt;
    }
    int ce0 = check_params(p);
    if (ce0) return ce0;
    const int precision = p->precision;
    if (n == 0) return VT_OK;
    if (!pts || !cells || !grad) return fail(VT_ERR_INVALID_ARG, "NULL argument");
    if (!cells->vol || !cells->cen || !cells->vtx_off || !cells->vtx || !cells->face_off || !cells->face_nbr ||
        !cells->face_vtx_off || !cells->face_vtx)
        return fail(VT_ERR_INVALID_ARG, "the adjoint needs vol, cen and the geometry of the tessellation");
    {
        const void* ptrs[] = {pts, gV, gC, gM, grad};
        const char* names[] = {"pts", "gV", "gC", "gM", "grad"};
        int r = check_device_buffers(stream, ptrs, names, 5);
        if (!r) r = check_buffers(stream, nullptr, nullptr, cells);
        if (r) return r;
    }
    cudaError_t e = launch_adjoint(pts, n, *cells, gV, gC, gM, grad, precision, make_grid(p, 1), (cudaStream_t)stream);
    return e == cudaSuccess ? VT_OK : cuda_fail(e, "adjoint");
}

int vt_lloyd_step(const float* pts, int64_t n, const double* grad, const double* vol, const vt_params* p,
                  float* out, void* stream)
{
    if (n < 0) return fail(VT_ERR_INVALID_ARG, "n must be >= 0");
    int e = check_params(p);
    if (e) return e;
    if (n == 0) return VT_OK;
    if (!pts || !grad || !vol || !out) return fail(VT_ERR_INVALID_ARG, "NULL argument");
    const void* ptrs[] = {pts, grad, vol, out};
    const char* names[] = {"pts", "grad", "vol", "out"};
    if ((e = check_device_buffers(stream, ptrs, names, 4))) return e;
    cudaError_t ce = launch_lloyd_step(pts, n, grad, vol, make_grid(p, 1), out, (cudaStream_t)stream);
    return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "lloyd step");
}

int vt_read_status(void* ws, size_t ws_bytes, void* stream)
{
    if (!ws || ws_bytes < sizeof(DevStatus)) return fail(VT_ERR_WORKSPACE, "workspace too small");
    Ctx c;
    c.base = (uint8_t*)ws;
    c.s = (cudaStream_t)stream;
    c.st = (DevStatus*)ws;  // the status block is the first region of every layout
    DevStatus h;
    int r = read_status(c, h);
    if (r) return r;
    return status_errors(h);
}

int vt_cluster_index(const float* pts, int64_t n_total, const vt_set_desc* plan, const int64_t* set_off, int n_sets,
                     int64_t total_cells, const vt_params* p, double* index, void* ws, size_t ws_bytes, void* stream)
{
    if (!index || n_sets < 1) return fail(VT_ERR_INVALID_ARG, "index is NULL or n_sets < 1");
    if (!plan && n_sets != 1) return fail(VT_ERR_INVALID_ARG, "several sets need a plan");
    Ctx c;
    int e = plan ? make_ctx(p, n_total, ws, ws_bytes, stream, c, total_cells, true)
                 : make_ctx(p, n_total, ws, ws_bytes, stream, c);
    if (e) return e;
    if (n_total > 0 && !pts) return fail(VT_ERR_INVALID_ARG, "pts is NULL");
    if ((e = check_buffers(stream, pts, ws, nullptr, plan, set_off))) return e;
    if (plan) {
        if (!set_off) return fail(VT_ERR_INVALID_ARG, "a plan needs set_off");
        c.sets = reinterpret_cast<const GridDesc*>(plan);
        c.set_off = set_off;
        c.nsets = n_sets;
    }
    const Layout& L = c.L;
    // the per-set counts use the list-key buffer (4 bytes per list entry at least)
    if ((int64_t)n_sets > L.knn_cap / 2) return fail(VT_ERR_INVALID_ARG, "more sets than the workspace can count");
    std::vector<GridDesc> h_sets(n_sets);
    cudaError_t ce = cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s);
    if (ce != cudaSuccess) return cuda_fail(ce, "status reset");
    if (plan) {
        ce = cudaMemcpyAsync(h_sets.data(), plan, sizeof(GridDesc) * n_sets, cudaMemcpyDeviceToHost, c.s);
        if (ce != cudaSuccess) return cuda_fail(ce, "plan read");
    } else {
        h_sets[0] = c.g;
        h_sets[0].npts = n_total;
    }
    unsigned long long* acc = c.at<unsigned long long>(L.knn_d2);
    if (n_total > 0) {
        BatchArgs b{c.sets, c.set_off, c.nsets, c.set_of()};
        ce = launch_grid_build(pts, n_total, c.g, c.at<float4>(L.sorted), c.at<int32_t>(L.perm),
                               c.at<int32_t>(L.cell_off), c.at<int32_t>(L.cid), c.at<int32_t>(L.ticket),
                               c.at<int32_t>(L.counts), c.at<int32_t>(L.big), c.at<void>(L.scan_tmp), c.st, c.s,
                               c.sets ? &b : nullptr, L.g3);
        if (ce == cudaSuccess)
            ce = launch_pair_counts(c.at<int32_t>(L.cell_off), L.g3, c.sets, c.sets ? n_sets : 1, acc, c.s);
        if (ce != cudaSuccess) return cuda_fail(ce, "grid build");
    } else {
        ce = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * n_sets, c.s);
        if (ce != cudaSuccess) return cuda_fail(ce, "clear");
    }
    std::vector<unsigned long long> h_acc(n_sets);
    ce = cudaMemcpyAsync(h_acc.data(), acc, sizeof(unsigned long long) * n_sets, cudaMemcpyDeviceToHost, c.s);
    if (ce != cudaSuccess) return cuda_fail(ce, "count read");
    DevStatus h;
    int r = read_status(c, h);
    if (r) return r;
    if ((r = status_errors(h))) return r;
    for (int sidx = 0; sidx < n_sets; ++sidx) {
        const double ns = (double)h_sets[sidx].npts;
        const double g3 = (double)h_sets[sidx].G * h_sets[sidx].G * h_sets[sidx].G;
        index[sidx] = ns < 2 ? 0.0 : g3 * (double)h_acc[sidx] / (ns * (ns - 1.0));
    }
    return VT_OK;
}

int vt_read_stats(void* ws, size_t ws_bytes, vt_stats* stats, vt_cells_out* out, void* stream)
{
    if (!ws || ws_bytes < sizeof(DevStatus)) return fail(VT_ERR_WORKSPACE, "workspace too small");
    Ctx c;
    c.base = (uint8_t*)ws;
    c.s = (cudaStream_t)stream;
    c.st = (DevStatus*)ws;
    DevStatus h;
    int r = read_status(c, h);
    if (r) return r;
    if (stats) {
        stats->fp64_rechecks = (int64_t)h.fp64_rechecks;
        stats->capacity_retries = (int64_t)h.capacity_events;
        stats->precision_retries = (int64_t)h.precision_events;
        stats->unvalidated = h.n_unval;
        for (int a = 0; a < 5; ++a) stats->clip_events[a] = (int64_t)h.detail[a];
        stats->knn_candidates = (int64_t)h.knn_evals;
        stats->knn_queries = (int64_t)h.knn_queries;
        stats->walk_cells = (int64_t)h.walk_cells;
        stats->walk_candidates = (int64_t)h.walk_cands;
    }
    if (out) {
        out->needed_nbr = h.totals[0];
        out->needed_vtx = h.totals[1];
        out->needed_face = h.totals[2];
        out->needed_face_vtx = h.totals[3];
    }
    if ((r = status_errors(h))) return r;
    if (h.record_overflow) return fail(VT_ERR_CAPACITY, "%d cells exceed the per-cell record size", h.record_overflow);
    if (h.cap_overflow) return fail(VT_ERR_CAPACITY, "an output buffer was too small (needed_* hold the sizes)");
    if (h.n_unval) return fail(VT_ERR_UNVALIDATED, "%d cells could not be validated", h.n_unval);
    return VT_OK;
}

int vt_unvalidated_cells(const vt_params* p, int64_t n, int32_t* ids, int64_t cap, int64_t* count, void* ws,
                         size_t ws_bytes, void* stream)
{
    int e = check_params(p);
    if (e) return e;
    if (!count) return fail(VT_ERR_INVALID_ARG, "count is NULL");
    if (n < 0 || n > (int64_t)INT32_MAX / 2) return fail(VT_ERR_INVALID_ARG, "n out of range: %lld", (long long)n);
    if (cap < 0 || (cap > 0 && !ids)) return fail(VT_ERR_INVALID_ARG, "ids is NULL with cap > 0");
    // the sorted points and the cell lists precede every region whose size
    // depends on the grid, so their offsets are the same for one set and for
    // a batch of n points in total
    const Layout L = make_layout(p, n);
    const int64_t nn = n > 0 ? n : 1;
    if (!ws || ws_bytes < L.list_a + sizeof(int32_t) * 7 * (size_t)nn)
        return fail(VT_ERR_WORKSPACE, "workspace too small for %lld points", (long long)n);
    if (cap > 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) (void)cudaGetLastError();
        if (cs != cudaStreamCaptureStatusNone)
            return fail(VT_ERR_INVALID_ARG, "vt_unvalidated_cells reads a count and cannot be captured");
        if (!device_accessible(ids)) return fail(VT_ERR_INVALID_ARG, "ids is not device-accessible memory");
    }
    Ctx c;
    c.base = (uint8_t*)ws;
    c.s = (cudaStream_t)stream;
    c.st = reinterpret_cast<DevStatus*>(c.base + L.status);
    DevStatus h;
    int r = read_status(c, h);
    if (r) return r;
    const int64_t cnt = h.n_unval;
    *count = cnt;
    if (!ids) return VT_OK;  // the count only
    if (cnt > cap)
        return fail(VT_ERR_CAPACITY, "%lld unvalidated cells, cap %lld", (long long)cnt, (long long)cap);
    // the unvalidated list is the sixth of the cell lists
    const int32_t* list = reinterpret_cast<const int32_t*>(c.base + L.list_a) + 5 * nn;
    cudaError_t ce = launch_unvalidated_ids(list, cnt, reinterpret_cast<const float4*>(c.base + L.sorted),
                                            p->index_space, ids, c.s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c.s);
    return ce == cudaSuccess ? VT_OK : cuda_fail(ce, "unvalidated ids");
}

const char* vt_last_error(void) { return g_err.c_str(); }

int64_t vt_launch_count(void) { return launches(); }

const char* vt_version(void) { return "vt 0.1.0 (sm_103a)"; }

}  // extern "C"
