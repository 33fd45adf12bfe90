// tune.cu -- autotuner of the launch parameters (threads per cell, initial k,
// k_max, grid density). The paper fixes these by hand for its hardware; here
// they are picked by timing the whole path on the caller's own points (or a
// seeded sample of them) with CUDA events, one parameter at a time: grid
// density first (per clustering class for a batch), then k0, then the k_max
// multiple, then threads per cell. Every candidate runs once untimed and
// `reps` times timed; the minimum counts. Host code only: it calls the public
// entry points of this library, so every tuned run is an ordinary run.
#include <cmath>
#include <cstring>
#include <vector>

#include "vt_internal.cuh"

namespace {

constexpr double kInf = 1e300;

struct Cand {
    int tpc, k0, mult;
    float rho[VT_TUNE_CLASSES];
};

bool same(const Cand& a, const Cand& b)
{
    if (a.tpc != b.tpc || a.k0 != b.k0 || a.mult != b.mult) return false;
    for (int c = 0; c < VT_TUNE_CLASSES; ++c)
        if (a.rho[c] != b.rho[c]) return false;
    return true;
}

int kmax_of(int k0, int mult)
{
    const int k = k0 * mult;
    return k > 256 ? 256 : k;
}

vt_params params_of(const vt_params* base, const Cand& c, int cls)
{
    vt_params p = *base;
    p.threads_per_cell = c.tpc;
    p.k0 = c.k0;
    p.k_max = kmax_of(c.k0, c.mult);
    p.grid_density = c.rho[cls];
    p.grid_res = 0;
    return p;
}

int check_space(const vt_tune_space* s)
{
    if (!s) return vt::set_error(VT_ERR_INVALID_ARG, "tune space is NULL");
    if (s->n_tpc < 1 || s->n_tpc > 4 || s->n_k0 < 1 || s->n_k0 > 8 || s->n_kmax < 1 || s->n_kmax > 4 ||
        s->n_rho < 1 || s->n_rho > 8 || s->reps < 1 || s->reps > 50)
        return vt::set_error(VT_ERR_INVALID_ARG, "tune space sizes out of range");
    for (int i = 0; i < s->n_tpc; ++i)
        if (!(s->tpc[i] == 8 || s->tpc[i] == 16 || s->tpc[i] == 32))
            return vt::set_error(VT_ERR_INVALID_ARG, "threads_per_cell candidates must be 8, 16 or 32");
    for (int i = 0; i < s->n_k0; ++i)
        if (s->k0[i] < 1 || s->k0[i] > 256) return vt::set_error(VT_ERR_INVALID_ARG, "k0 candidates must be in [1, 256]");
    for (int i = 0; i < s->n_kmax; ++i)
        if (s->kmax_mult[i] < 1 || s->kmax_mult[i] > 256)
            return vt::set_error(VT_ERR_INVALID_ARG, "k_max multiples must be in [1, 256]");
    for (int i = 0; i < s->n_rho; ++i)
        if (!(s->rho[i] > 0.0f) || !std::isfinite(s->rho[i]))
            return vt::set_error(VT_ERR_INVALID_ARG, "grid densities must be positive");
    return VT_OK;
}

// the parameters whose workspace is largest: smallest density, largest k
vt_params widest(const vt_params* base, const vt_tune_space* s)
{
    vt_params p = *base;
    float rmin = s->rho[0];
    int kmax0 = 1, mmax = 1;
    for (int i = 0; i < s->n_rho; ++i) rmin = std::fmin(rmin, s->rho[i]);
    for (int i = 0; i < s->n_k0; ++i) kmax0 = s->k0[i] > kmax0 ? s->k0[i] : kmax0;
    for (int i = 0; i < s->n_kmax; ++i) mmax = s->kmax_mult[i] > mmax ? s->kmax_mult[i] : mmax;
    if (base->k0 > kmax0) kmax0 = base->k0;
    const int bmult = base->k_max / base->k0 > mmax ? base->k_max / base->k0 : mmax;
    p.grid_density = std::fmin(rmin, base->grid_density);
    p.grid_res = 0;
    p.k0 = kmax0;
    p.k_max = kmax_of(kmax0, bmult);
    return p;
}

// one timed candidate: run() enqueues (and may synchronise) one tessellation
// and returns its status; the time is the minimum over reps of the event
// interval around it
template <typename Run>
double time_runs(Run run, int reps, cudaStream_t s, int& status)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return kInf;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return kInf;
    }
    double best = kInf;
    status = run();  // untimed warm-up
    for (int r = 0; r < reps && status == VT_OK; ++r) {
        cudaEventRecord(a, s);
        status = run();
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            status = VT_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (status == VT_OK && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return status == VT_OK ? best : kInf;
}

// coordinate descent over the space; eval(c) returns the candidate's time
template <typename Eval>
int descend(const vt_params* base, const vt_tune_space* s, const bool* classes_used, Eval eval, vt_tune_result* res)
{
    std::vector<Cand> seen;
    std::vector<double> seen_ms;
    auto try_ = [&](const Cand& c, int cls) {
        for (size_t i = 0; i < seen.size(); ++i)
            if (same(seen[i], c)) return seen_ms[i];
        int status = VT_OK;
        const double ms = eval(c, status);
        seen.push_back(c);
        seen_ms.push_back(ms);
        if (res->n_tried < VT_TUNE_MAX_TRIED) {
            vt_tune_trial& t = res->tried[res->n_tried];
            t.threads_per_cell = c.tpc;
            t.k0 = c.k0;
            t.k_max = kmax_of(c.k0, c.mult);
            t.cls = cls;
            t.grid_density = c.rho[cls < 0 ? 0 : cls];
            t.ms = ms >= kInf ? -1.0 : ms;
            t.status = status;
        }
        ++res->n_tried;
        return ms;
    };
    Cand cur{};
    cur.tpc = base->threads_per_cell ? base->threads_per_cell : 32;
    cur.k0 = base->k0;
    cur.mult = base->k_max / base->k0 > 0 ? base->k_max / base->k0 : 1;
    for (int c = 0; c < VT_TUNE_CLASSES; ++c) cur.rho[c] = base->grid_density;
    double best = try_(cur, 0);
    for (int c = 0; c < VT_TUNE_CLASSES; ++c) {
        if (!classes_used[c]) continue;
        for (int i = 0; i < s->n_rho; ++i) {
            Cand t = cur;
            t.rho[c] = s->rho[i];
            const double ms = try_(t, c);
            if (ms < best) { best = ms; cur = t; }
        }
    }
    for (int i = 0; i < s->n_k0; ++i) {
        Cand t = cur;
        t.k0 = s->k0[i];
        const double ms = try_(t, 0);
        if (ms < best) { best = ms; cur = t; }
    }
    for (int i = 0; i < s->n_kmax; ++i) {
        Cand t = cur;
        t.mult = s->kmax_mult[i];
        const double ms = try_(t, 0);
        if (ms < best) { best = ms; cur = t; }
    }
    for (int i = 0; i < s->n_tpc; ++i) {
        Cand t = cur;
        t.tpc = s->tpc[i];
        const double ms = try_(t, 0);
        if (ms < best) { best = ms; cur = t; }
    }
    if (best >= kInf) return vt::set_error(VT_ERR_UNVALIDATED, "no candidate of the tune space completed");
    int first = 0;
    while (first < VT_TUNE_CLASSES - 1 && !classes_used[first]) ++first;
    res->best = params_of(base, cur, first);
    for (int c = 0; c < VT_TUNE_CLASSES; ++c) res->density_of_class[c] = cur.rho[c];
    res->best_ms = best;
    return VT_OK;
}

}  // namespace

extern "C" {

void vt_tune_space_default(vt_tune_space* s)
{
    std::memset(s, 0, sizeof(*s));
    const int tpc[3] = {8, 16, 32};
    const int k0[5] = {8, 12, 16, 24, 32};
    const int mult[3] = {1, 2, 4};
    const float rho[5] = {1.f, 2.f, 3.f, 4.f, 6.f};
    s->n_tpc = 3;
    std::memcpy(s->tpc, tpc, sizeof(tpc));
    s->n_k0 = 5;
    std::memcpy(s->k0, k0, sizeof(k0));
    s->n_kmax = 3;
    std::memcpy(s->kmax_mult, mult, sizeof(mult));
    s->n_rho = 5;
    std::memcpy(s->rho, rho, sizeof(rho));
    s->reps = 3;
}

int vt_cluster_class(double index)
{
    if (!(index < 2.0)) {
        if (index < 8.0) return 1;
        if (index < 32.0) return 2;
        return 3;
    }
    return 0;
}

int vt_autotune_workspace_size(const vt_params* base, const vt_tune_space* s, int64_t n, size_t* bytes)
{
    int e = check_space(s);
    if (e) return e;
    if (!base || !bytes) return vt::set_error(VT_ERR_INVALID_ARG, "NULL argument");
    const vt_params w = widest(base, s);
    return vt_workspace_size(&w, n, bytes);
}

int vt_autotune(const float* pts, int64_t n, const vt_params* base, const vt_tune_space* s, vt_cells_out* out,
                vt_tune_result* res, void* ws, size_t ws_bytes, void* stream)
{
    int e = check_space(s);
    if (e) return e;
    if (!base || !out || !res) return vt::set_error(VT_ERR_INVALID_ARG, "NULL argument");
    if (base->flags & VT_FLAG_STAGE_TIMES) return vt::set_error(VT_ERR_INVALID_ARG, "tune without stage times");
    std::memset(res, 0, sizeof(*res));
    const bool used[VT_TUNE_CLASSES] = {true, false, false, false};
    cudaStream_t st = (cudaStream_t)stream;
    auto eval = [&](const Cand& c, int& status) {
        const vt_params p = params_of(base, c, 0);
        auto run = [&]() {
            vt_cells_out o = *out;
            int r = vt_tessellate(pts, n, &p, &o, nullptr, ws, ws_bytes, stream);
            if (r == VT_OK && (p.flags & VT_FLAG_NO_SYNC)) r = vt_read_stats(ws, ws_bytes, nullptr, &o, stream);
            return r;
        };
        return time_runs(run, s->reps, st, status);
    };
    return descend(base, s, used, eval, res);
}

int vt_autotune_batch_workspace_size(const int64_t* set_off, int n_sets, const vt_params* base,
                                     const vt_tune_space* s, size_t* bytes)
{
    int e = check_space(s);
    if (e) return e;
    if (!base || !bytes || !set_off || n_sets < 1) return vt::set_error(VT_ERR_INVALID_ARG, "NULL argument");
    const vt_params w = widest(base, s);
    std::vector<vt_set_desc> plan(n_sets);
    int64_t cells = 0;
    if ((e = vt_batch_plan(set_off, n_sets, &w, nullptr, plan.data(), &cells))) return e;
    return vt_batch_workspace_size(&w, set_off[n_sets], cells, bytes);
}

int vt_autotune_batch(const float* pts, const int64_t* set_off_host, const int64_t* set_off_dev, int n_sets,
                      const int* set_class, const vt_params* base, const vt_tune_space* s, vt_set_desc* plan_dev,
                      vt_cells_out* out, vt_tune_result* res, void* ws, size_t ws_bytes, void* stream)
{
    int e = check_space(s);
    if (e) return e;
    if (!base || !out || !res || !set_off_host || !set_off_dev || !set_class || !plan_dev || n_sets < 1)
        return vt::set_error(VT_ERR_INVALID_ARG, "NULL argument");
    if (base->flags & VT_FLAG_STAGE_TIMES) return vt::set_error(VT_ERR_INVALID_ARG, "tune without stage times");
    std::memset(res, 0, sizeof(*res));
    bool used[VT_TUNE_CLASSES] = {false, false, false, false};
    for (int i = 0; i < n_sets; ++i) {
        if (set_class[i] < 0 || set_class[i] >= VT_TUNE_CLASSES)
            return vt::set_error(VT_ERR_INVALID_ARG, "set class out of range");
        used[set_class[i]] = true;
    }
    const int64_t n_total = set_off_host[n_sets];
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<vt_set_desc> plan(n_sets);
    std::vector<int> gres(n_sets);
    auto eval = [&](const Cand& c, int& status) {
        // grid resolution of every set from the density of its class
        for (int i = 0; i < n_sets; ++i) {
            const vt_params pc = params_of(base, c, set_class[i]);
            gres[i] = vt_grid_resolution(&pc, set_off_host[i + 1] - set_off_host[i]);
        }
        const vt_params p = params_of(base, c, 0);
        int64_t cells = 0;
        status = vt_batch_plan(set_off_host, n_sets, &p, gres.data(), plan.data(), &cells);
        if (status) return kInf;
        if (cudaMemcpyAsync(plan_dev, plan.data(), sizeof(vt_set_desc) * n_sets, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            status = VT_ERR_CUDA;
            return kInf;
        }
        auto run = [&]() {
            vt_cells_out o = *out;
            int r = vt_tessellate_batch(pts, n_total, plan_dev, set_off_dev, n_sets, cells, &p, &o, nullptr, ws,
                                        ws_bytes, stream);
            if (r == VT_OK && (p.flags & VT_FLAG_NO_SYNC)) r = vt_read_stats(ws, ws_bytes, nullptr, &o, stream);
            return r;
        };
        return time_runs(run, s->reps, st, status);
    };
    return descend(base, s, used, eval, res);
}

}  // extern "C"
