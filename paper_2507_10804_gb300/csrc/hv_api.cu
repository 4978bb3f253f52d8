// hv_api.cu -- the C ABI of libhv: validation, workspace layout and the
// executor that drives the forward sweep, the checkpointed adjoint sweep and
// the final reductions (paper section 3: H_d v by two wave solves per source
// plus the forward field; section 2.1, eq. (grad): misfit gradient).
#include "hv_internal.h"

#include <atomic>

#include <functional>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <memory>
#include <set>
#include <utility>

namespace hvi {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace hvi

#define HV_CK(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)
#define HV_RT(call)                                                                                   \
    do {                                                                                              \
        int r_ = (call);                                                                              \
        if (r_ != HV_OK) return r_;                                                                   \
    } while (0)

extern "C" const char *hv_last_error(void) { return hvi::g_err.c_str(); }
extern "C" int hv_version(void) { return 100; }

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int build_rectiles(hv_handle *h, const hvi::Tiling &t)
{
    long long key = (long long)t.TX * 65536 + t.TZ;
    if (h->rectiles.count(key)) return HV_OK;
    std::vector<int> off((size_t)h->ns * (t.ntiles + 1)), rec((size_t)h->ns * h->nr), pos((size_t)h->ns * h->nr);
    for (int s = 0; s < h->ns; ++s) {
        std::vector<std::pair<int, int>> tr;   // (tile, receiver)
        for (int r = 0; r < h->nr; ++r) {
            int z = h->h_rec_zx[2 * ((size_t)s * h->nr + r)], x = h->h_rec_zx[2 * ((size_t)s * h->nr + r) + 1];
            tr.push_back({(z / t.TZ) * t.ntx + (x / t.TX), r});
        }
        std::stable_sort(tr.begin(), tr.end(), [](auto &a, auto &b) { return a.first < b.first; });
        int *o = off.data() + (size_t)s * (t.ntiles + 1);
        size_t i = 0;
        for (int tile = 0; tile <= t.ntiles; ++tile) {
            while (i < tr.size() && tr[i].first < tile) ++i;
            o[tile] = (int)i;
        }
        for (size_t q = 0; q < tr.size(); ++q) {
            int r = tr[q].second;
            int z = h->h_rec_zx[2 * ((size_t)s * h->nr + r)], x = h->h_rec_zx[2 * ((size_t)s * h->nr + r) + 1];
            rec[(size_t)s * h->nr + q] = r;
            pos[(size_t)s * h->nr + q] = (z + hvi::GH) * h->P + (x + hvi::GH);
        }
    }
    hvi::RecTiles rt;
    rt.TX = t.TX;
    rt.TZ = t.TZ;
    rt.ntiles = t.ntiles;
    HV_CK(cudaMalloc(&rt.off, off.size() * sizeof(int)));
    HV_CK(cudaMalloc(&rt.rec, rec.size() * sizeof(int)));
    HV_CK(cudaMalloc(&rt.pos, pos.size() * sizeof(int)));
    HV_CK(cudaMemcpy(rt.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    HV_CK(cudaMemcpy(rt.rec, rec.data(), rec.size() * sizeof(int), cudaMemcpyHostToDevice));
    HV_CK(cudaMemcpy(rt.pos, pos.data(), pos.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->rectiles[key] = rt;
    return HV_OK;
}

const hvi::RecTiles &rectiles_for(const hv_handle *h, const hvi::Tiling &t)
{
    return h->rectiles.at((long long)t.TX * 65536 + t.TZ);
}

// ---------------------------------------------------------------- workspace layout
struct Layout {
    bool history = false;     // keep every time level instead of snapshots
    bool resident = false;    // H v on the shared-memory-resident kernels (history of Q^n, per-pair images)
    int slots = 0;            // snapshot pairs per shot (binomial mode)
    int G = 1;                // adjoint shot groups (partial images)
    size_t fb = 0;            // bytes of one field batch (all shots)
    size_t C = 0, b = 0, zero = 0, work = 0, store = 0, D = 0, dd = 0, img = 0, part = 0, total = 0;
    size_t cnt = 0, cnt_bytes = 0;   // per (shot group, tile) step counters (dataflow launch mode)
    size_t fields_end = 0;    // the field regions (all first) end here: the tensor maps cover [0, fields_end)
};

constexpr int kResidualBlocks = 1024;
// Forward levels in flight besides the snapshots: the current state (2), and
// the two outputs of a fused double step.
constexpr int kWorkBatches = 4;

int make_layout(const hv_handle *h, int op, int k, int ckpt, Layout &L)
{
    if (op < HV_OP_FWD || op > HV_OP_MISFITS) return hvi::fail(HV_EINVAL, "unknown operation %d", op);
    const bool adjoint = (op == HV_OP_MIGRATE || op == HV_OP_GRAD || op == HV_OP_HV);
    const bool born = (op == HV_OP_BORN || op == HV_OP_HV);
    const bool models = op == HV_OP_MISFITS;
    if (born && (k < 1 || k > 65535)) return hvi::fail(HV_EINVAL, "k = %d vectors; need 1 <= k <= 65535", k);
    if (models && (k < 1 || k > 65535)) return hvi::fail(HV_EINVAL, "k = %d models; need 1 <= k <= 65535", k);
    if (!born && !models) k = 1;
    if (adjoint) {
        if (ckpt != HV_CKPT_ALL && ckpt < 1)
            return hvi::fail(HV_EINVAL, "checkpoint budget %d; use HV_CKPT_ALL or a value >= 1", ckpt);
        L.history = (ckpt == HV_CKPT_ALL) || (ckpt >= h->nt - 1);
        L.slots = L.history ? 0 : ckpt;
        L.G = hvk::adj_groups(h);
    }
    L.fb = align256((size_t)h->ns * h->fsize * sizeof(float));
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    const size_t fbytes = h->fsize * sizeof(float);
    if (models) {             // k coefficient fields, a ring of three field batches per model, data, partial sums
        L.C = take((size_t)k * fbytes);
        L.work = take((size_t)3 * k * L.fb);
        L.fields_end = o;
        L.dd = take((size_t)k * h->ns * h->nt * h->nr * sizeof(float));
        L.part = take((size_t)k * kResidualBlocks * sizeof(double));
        L.total = o;
        return HV_OK;
    }
    L.C = take(fbytes);
    if (born) L.b = take((size_t)k * fbytes);
    L.zero = take(L.fb);
    if (!adjoint || !L.history) L.work = take(kWorkBatches * L.fb);
    if (adjoint) L.store = take(L.history ? (size_t)h->nt * L.fb : (size_t)2 * L.slots * L.fb);
    if (born || adjoint) L.D = take((size_t)2 * k * L.fb);
    L.fields_end = o;         // every region above is a whole number of fields (fsize is 64-float aligned)
    const size_t ndata = (size_t)h->ns * h->nt * h->nr;
    if (op == HV_OP_HV) L.dd = take((size_t)k * ndata * sizeof(float));
    if (op == HV_OP_GRAD || op == HV_OP_MISFIT) L.dd = take(ndata * sizeof(float));
    L.resident = op == HV_OP_HV && L.history && h->resident && !h->img_f64 && hvk::resident_fits(h);
    if (adjoint) L.img = take((size_t)(L.resident ? h->ns : L.G) * k * h->fsize * sizeof(double));
    if (op == HV_OP_GRAD || op == HV_OP_MISFIT) L.part = take(kResidualBlocks * sizeof(double));
    L.cnt_bytes = (size_t)hvk::adj_groups(h) * hvk::max_tiles(h) * sizeof(int);
    L.cnt = take(L.cnt_bytes);
    L.total = o;
    return HV_OK;
}

// ---------------------------------------------------------------- profiling
cudaEvent_t take_event(hv_handle *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets the launches of its scope with events when profiling is on.
struct ProfScope {
    hv_handle *h;
    cudaStream_t st;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(hv_handle *hh, cudaStream_t s, int k) : h(hh), st(s), kind(k)
    {
        if (h->prof_on) {
            a = take_event(h);
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope()
    {
        if (a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, st);
            h->prof_rec.push_back({kind, {a, b}});
        }
    }
};

// ---------------------------------------------------------------- executor
struct Exec {
    hv_handle *h;
    cudaStream_t st;
    Layout L;
    char *ws;
    int k;
    float *C, *b, *zero;
    float *D;            // 2 k field batches: Born fields (first sweep), adjoint fields (reversal)
    double *img;
    hvk::TmaMaps maps;   // tensor maps of this call's workspace
    // Forward levels live in a pool of field batches (3 working + 2 per snapshot
    // slot, contiguous).  A snapshot pins the two batches of the current state
    // (reference counts) instead of copying them; a forward step writes into
    // any batch that is neither pinned nor part of the current state.
    std::vector<float *> pool;
    std::vector<int> refs;
    std::vector<std::pair<int, int>> slot_b;   // slot -> (batch of u^j, batch of u^{j-1}), -1 = zero
    int cur_i = -1, prev_i = -1;               // pool indices of the current state (-1: zero batch)
    const float *cur, *prev;
    int j;               // current state index: cur = u^j, prev = u^{j-1}
    // Dataflow ordering of the stencil steps (HV_LAUNCH_DATAFLOW): the step
    // counters, the items of all steps launched so far in this call, and the
    // calling thread's launch count right after the last step.
    int *cnt = nullptr;
    int need = 0;
    long long last_tl = -1;

    // Ordering of the next stencil step, which completes `items` items per
    // (shot group, tile): tile waits if the previous kernel this thread
    // launched was the previous step, else a wait for every earlier kernel.
    hvk::StepDeps deps(int items)
    {
        hvk::StepDeps d;
        d.cnt = cnt;
        d.need = need;
        d.flow = cnt != nullptr && last_tl == hvk::thread_launches();
        need += items;
        if (d.flow && h->inject_wait) {   // testing the timeout path: a count no step reaches
            d.need += 1 << 24;
            h->inject_wait = false;
        }
        return d;
    }
    void launched_step() { last_tl = hvk::thread_launches(); }
    // The adjoint's tile configuration: the FP64-image check has one of its own.
    int adj_cfg() const { return h->img_f64 ? hvk::adj_f64_cfg() : h->cfg[2]; }

    float *batch(char *base, size_t i) const { return reinterpret_cast<float *>(base + i * L.fb); }
    float *Dbuf(int parity) const { return reinterpret_cast<float *>(reinterpret_cast<char *>(D) + (size_t)parity * k * L.fb); }
    float *hist(int n) const { return n == 0 ? zero : batch(ws + L.store, (size_t)(n - 1)); }
    const float *ptr(int i) const { return i < 0 ? zero : pool[i]; }

    int pick_free() const
    {
        for (size_t i = 0; i < pool.size(); ++i)
            if (refs[i] == 0 && (int)i != cur_i && (int)i != prev_i) return (int)i;
        return -1;
    }

    int init(hv_handle *hh, cudaStream_t s, const Layout &l, void *w, int kk)
    {
        h = hh; st = s; L = l; ws = (char *)w; k = kk;
        C = reinterpret_cast<float *>(ws + L.C);
        b = L.b ? reinterpret_cast<float *>(ws + L.b) : nullptr;
        zero = reinterpret_cast<float *>(ws + L.zero);
        D = reinterpret_cast<float *>(ws + L.D);
        img = reinterpret_cast<double *>(ws + L.img);
        if (L.work) {
            const int n = kWorkBatches + (L.history ? 0 : 2 * L.slots);   // work and snapshot batches are contiguous
            for (int i = 0; i < n; ++i) pool.push_back(batch(ws + L.work, i));
            refs.assign(n, 0);
            slot_b.assign(L.slots, {-1, -1});
        }
        cur = prev = zero;
        cur_i = prev_i = -1;
        j = 0;
        const hvi::Tiling t0 = hvk::tiling(h, h->cfg[0]), t1 = hvk::tiling(h, h->cfg[1]), t2 = hvk::tiling(h, adj_cfg());
        const bool one_tiling = t0.TX == t1.TX && t0.TX == t2.TX && t0.TZ == t1.TZ && t0.TZ == t2.TZ;
        if (h->launch_mode == HV_LAUNCH_DATAFLOW && one_tiling) {
            cnt = reinterpret_cast<int *>(ws + L.cnt);
            HV_CK(cudaMemsetAsync(cnt, 0, L.cnt_bytes, st));
        }
        return hvk::make_maps(h, ws, (long long)(L.fields_end / (h->fsize * sizeof(float))), &maps);
    }

    // One forward step from the current state.  born: advance the Born fields
    // too (first sweep of H v / Born map).  target: write u^{n+1} there
    // (stored-history mode) instead of into a pool batch.
    int forward(int n, bool born, float *d_u, float *d_du, float *target, int kind = HV_K_FWD)
    {
        ProfScope ps(h, st, kind);
        if (n != j) return hvi::fail(HV_EINVAL, "internal: forward step %d from state %d", n, j);
        int ni = -1;
        float *next = target;
        if (!next) {
            ni = pick_free();
            if (ni < 0) return hvi::fail(HV_EINVAL, "internal: no free forward buffer");
            next = pool[ni];
        }
        hvk::FwdLaunch a{};
        a.u_cur = cur; a.u_prev = prev; a.u_next = next; a.C = C;
        a.n = n;
        if (born) {
            a.b = b; a.k = k;
            a.du_cur = Dbuf(n & 1);
            a.du_io = Dbuf((n + 1) & 1);
            a.d_du = d_du;
        }
        a.d_u = d_u;
        const int cfg = born ? h->cfg[0] : h->cfg[1];
        a.deps = deps(born ? k : 1);
        HV_RT(hvk::launch_fwd(h, cfg, rectiles_for(h, hvk::tiling(h, cfg)), maps, a, st));
        launched_step();
        prev = cur;
        prev_i = cur_i;
        cur = next;
        cur_i = ni;
        j = n + 1;
        return HV_OK;
    }

    // Two recomputation steps in one launch (k_fwd2): u^{j+1}, u^{j+2} into two
    // free batches.  Falls back to two single steps where it does not apply.
    int forward2(int n)
    {
        if (n != j) return hvi::fail(HV_EINVAL, "internal: forward step %d from state %d", n, j);
        const int i1 = pick_free();
        int i2 = -1;
        for (size_t i = 0; i < pool.size(); ++i)
            if (refs[i] == 0 && (int)i != cur_i && (int)i != prev_i && (int)i != i1) {
                i2 = (int)i;
                break;
            }
        if (!h->fuse_steps || cnt != nullptr || i1 < 0 || i2 < 0) {
            HV_RT(forward(n, false, nullptr, nullptr, nullptr, HV_K_ADVANCE));
            return forward(n + 1, false, nullptr, nullptr, nullptr, HV_K_ADVANCE);
        }
        ProfScope ps(h, st, HV_K_ADVANCE);
        hvk::Fwd2Launch a{};
        a.u_cur = cur; a.u_prev = prev; a.u_next1 = pool[i1]; a.u_next2 = pool[i2]; a.C = C; a.n = n;
        HV_RT(hvk::launch_fwd2(h, h->cfg[1], rectiles_for(h, hvk::tiling(h, h->cfg[1])), maps, a, st));
        launched_step();
        prev = pool[i1];
        prev_i = i1;
        cur = pool[i2];
        cur_i = i2;
        j = n + 2;
        return HV_OK;
    }

    // Pin the current state in `slot` (no copy).
    int save(int slot)
    {
        if (slot < 0 || slot >= (int)slot_b.size()) return hvi::fail(HV_EINVAL, "internal: snapshot slot %d", slot);
        auto &sb = slot_b[slot];
        if (sb.first >= 0) --refs[sb.first];
        if (sb.second >= 0) --refs[sb.second];
        sb = {cur_i, prev_i};
        if (cur_i >= 0) ++refs[cur_i];
        if (prev_i >= 0) ++refs[prev_i];
        return HV_OK;
    }

    void restore(int slot, int state)
    {
        if (slot < 0) {
            cur_i = prev_i = -1;
            j = 0;
        } else {
            cur_i = slot_b[slot].first;
            prev_i = slot_b[slot].second;
            j = state;
        }
        cur = ptr(cur_i);
        prev = ptr(prev_i);
    }

    int adjoint(int n, const float *u, const float *r, int r_per_vector, float rscale, int kk)
    {
        ProfScope ps(h, st, HV_K_ADJ);
        hvk::AdjLaunch a{};
        a.u = u;
        a.lam1 = Dbuf((n + 1) & 1);
        a.lam_io = Dbuf(n & 1);
        a.C = C;
        a.r = r;
        a.r_per_vector = r_per_vector;
        a.rscale = rscale;
        a.img = img;
        a.img_f64 = h->img_f64;
        a.n = n;
        a.k = kk;
        a.G = L.G;
        a.deps = deps(kk);
        HV_RT(hvk::launch_adj(h, adj_cfg(), rectiles_for(h, hvk::tiling(h, adj_cfg())), maps, a, st));
        launched_step();
        return HV_OK;
    }

    // Zero the ghost bands of every field batch this call's kernels write:
    // the zero state, the forward-level pool, the stored levels and the
    // Born/adjoint fields.
    int zero_ghosts(bool with_store)
    {
        const long long per_batch = (long long)h->ns;
        HV_RT(hvk::launch_zero_ghosts(h, zero, per_batch, st));
        if (!pool.empty()) HV_RT(hvk::launch_zero_ghosts(h, pool[0], (long long)pool.size() * per_batch, st));
        if (with_store && L.history) HV_RT(hvk::launch_zero_ghosts(h, hist(1), (long long)h->nt * per_batch, st));
        if (L.D) HV_RT(hvk::launch_zero_ghosts(h, D, 2LL * k * per_batch, st));
        return HV_OK;
    }

    const float *u_for(int n)
    {
        if (j == n) return cur;
        if (j == n + 1) return prev;
        return nullptr;
    }
};

int check_common(hv_handle *h, const void *ws, size_t ws_bytes, int op, int k, int ckpt, Layout &L)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != h->device) return hvi::fail(HV_EINVAL, "current device %d is not the handle's device %d", dev, h->device);
    HV_RT(make_layout(h, op, k, ckpt, L));
    if (!ws) return hvi::fail(HV_EINVAL, "null workspace");
    if (((uintptr_t)ws & 255u) != 0) return hvi::fail(HV_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return hvi::fail(HV_ENOMEM, "workspace of %zu bytes; this call needs %zu", ws_bytes, L.total);
    return HV_OK;
}

const std::vector<hvi::Action> *schedule_for(hv_handle *h, int slots)
{
    std::lock_guard<std::mutex> g(h->mu);
    auto it = h->schedules.find(slots);
    if (it != h->schedules.end()) return &it->second;
    std::vector<hvi::Action> acts;
    long long adv = 0;
    hvi::build_schedule(h->nt, slots, acts, &adv);
    auto r = h->schedules.emplace(slots, std::move(acts));
    return &r.first->second;
}

// Extra work of a merged call (hv_apply_batch): the forward data are sampled
// into fwd_data during the first sweep and after_sweep runs (the residuals
// of the gradient slots, which overwrite those slots' Born data, and the misfits).
struct BatchExtra {
    float *fwd_data = nullptr;
    std::function<int(cudaStream_t)> after_sweep;
};
int run_adjoint_body(hv_handle *h, int kind, const float *in, int kk, double *phi, int ckpt, void *ws,
                     const Layout &L, cudaStream_t st, const BatchExtra *bx = nullptr);
int run_resident_hv(hv_handle *h, int kk, void *ws, const Layout &L, cudaStream_t st);

std::string graph_key(const void *ws, size_t bytes, int k, int ckpt, const int *cfg, int mode, bool fuse, bool res,
                      unsigned long long wait_ns)
{
    char buf[208];
    snprintf(buf, sizeof(buf), "%p/%zu/%d/%d/%d.%d.%d/%d/%d/%d/%llu", ws, bytes, k, ckpt, cfg[0], cfg[1], cfg[2], mode,
             (int)fuse, (int)res, wait_ns);
    return buf;
}

// Keeps an instantiated graph under `key`; the cache holds the kMaxGraphs most
// recent (a server's arena offsets and batch sizes make many keys).  An
// evicted graph still in flight is freed when it completes.
constexpr size_t kMaxGraphs = 32;
cudaGraphExec_t cache_graph(hv_handle *h, const std::string &key, cudaGraphExec_t ex)
{
    while (h->graphs.size() >= kMaxGraphs && !h->graph_order.empty()) {
        auto old = h->graphs.find(h->graph_order.front());
        if (old != h->graphs.end()) {
            cudaGraphExecDestroy(old->second);
            h->graphs.erase(old);
        }
        h->graph_order.pop_front();
    }
    h->graphs.emplace(key, ex);
    h->graph_order.push_back(key);
    return ex;
}

// The shared driver of migrate / misfit_grad / hessian_apply.
//   kind 0: migrate   r = user data,                         scale h^2
//   kind 1: gradient  r = f(m) - d_obs (computed),           scale h^2 / sigma^2
//   kind 2: H v       r = F v (Born data, computed),         scale h^2 / sigma^2
int run_adjoint(hv_handle *h, int kind, const float *m, const float *in, int k, float *out32, double *out64,
                double *phi, int ckpt, void *ws, size_t ws_bytes, cudaStream_t st, double *ext = nullptr)
{
    const int op = kind == 0 ? HV_OP_MIGRATE : (kind == 1 ? HV_OP_GRAD : HV_OP_HV);
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, op, kind == 2 ? k : 1, ckpt, L));
    const int kk = (kind == 2) ? k : 1;
    const bool born = (kind == 2);
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_RT(hvk::launch_prep(h, m, born ? in : nullptr, born ? kk : 0, reinterpret_cast<float *>((char *)ws + L.C),
                               born ? reinterpret_cast<float *>((char *)ws + L.b) : nullptr, st));
    }
    // Everything between the model preparation and the final fold touches only
    // the workspace and the handle, so for H v it can be captured once as a
    // CUDA graph and replayed (hv_set_graphs).
    // (A pending wait-timeout injection runs eagerly: a graph would keep it.)
    const bool graph = born && h->graphs_on && !h->prof_on && !h->inject_wait;
    if (graph) {
        const std::string key =
            graph_key(ws, L.total, kk, ckpt, h->cfg, h->launch_mode + 16 * (int)h->img_f64, h->fuse_steps, L.resident,
                      h->wait_ns);
        auto it = h->graphs.find(key);
        cudaGraphExec_t ge = it == h->graphs.end() ? nullptr : it->second;
        if (!ge) {
            cudaStream_t cs = h->capture_stream;
            HV_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int rc = run_adjoint_body(h, kind, in, kk, phi, ckpt, ws, L, cs);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (rc != HV_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            ge = cache_graph(h, key, ex);
        }
        HV_CK(cudaGraphLaunch(ge, st));
    } else {
        HV_RT(run_adjoint_body(h, kind, in, kk, phi, ckpt, ws, L, st));
    }
    {
        ProfScope ps(h, st, HV_K_OTHER);
        const int fmt = h->img_f64 && !L.resident ? hvk::kImgF64 : hvk::kImgPairs;
        if (ext)   // the extended image of this handle's shots, not folded (hv_hessian_apply_partial)
            return hvk::launch_partial_image(h, m, reinterpret_cast<double *>((char *)ws + L.img), fmt,
                                             L.resident ? h->ns : L.G, kk, ext, st);
        HV_RT(hvk::launch_finalize(h, m, reinterpret_cast<double *>((char *)ws + L.img), fmt, L.resident ? h->ns : L.G, kk,
                                   out32, out64, reinterpret_cast<double *>((char *)ws + L.D), st));
    }
    return HV_OK;
}

// H v with every level stored on the shared-memory-resident kernels: the
// forward fields write Q^n into the history region, the Born fields of every
// (shot, vector) pair write the Born data, and the adjoint fields of every pair
// write the pair's image; the fold sums the pairs' images over shots.
int run_resident_hv(hv_handle *h, int kk, void *ws, const Layout &L, cudaStream_t st)
{
    const hvi::RecTiles &rt = rectiles_for(h, hvk::tiling(h, h->cfg[2]));
    hvk::ResLaunch a{};
    a.base = ws;
    a.C = reinterpret_cast<const float *>((char *)ws + L.C);
    a.b = reinterpret_cast<const float *>((char *)ws + L.b);
    a.q = reinterpret_cast<float *>((char *)ws + L.store);
    a.dd = reinterpret_cast<float *>((char *)ws + L.dd);
    a.rscale = (float)(h->h * h->h / (h->sigma * h->sigma));
    a.img = (char *)ws + L.img;
    a.rec = rt.rec;
    a.pos = rt.pos;
    a.k = kk;
    {
        ProfScope ps(h, st, HV_K_FWD);
        HV_RT(hvk::launch_resident(h, 0, a, st));
        HV_RT(hvk::launch_resident(h, 1, a, st));
    }
    ProfScope ps(h, st, HV_K_ADJ);
    return hvk::launch_resident(h, 2, a, st);
}

// The part of run_adjoint between preparation and fold (all on `st`).
int run_adjoint_body(hv_handle *h, int kind, const float *in, int kk, double *phi, int ckpt, void *ws,
                     const Layout &L, cudaStream_t st, const BatchExtra *bx)
{
    (void)ckpt;
    if (L.resident && !bx) return run_resident_hv(h, kk, ws, L, st);
    Exec E;
    HV_RT(E.init(h, st, L, ws, kk));
    const bool born = (kind == 2);
    HV_CK(cudaMemsetAsync(E.zero, 0, L.fb, st));
    HV_RT(E.zero_ghosts(true));
    HV_CK(cudaMemsetAsync((char *)ws + L.D, 0, (size_t)2 * kk * L.fb, st));
    float *dd = (kind != 0) ? reinterpret_cast<float *>((char *)ws + L.dd) : nullptr;

    const std::vector<hvi::Action> *sched = L.history ? nullptr : schedule_for(h, L.slots);
    size_t ai = 0;
    // ---- first sweep
    for (int n = 0; n < h->nt; ++n) {
        float *target = L.history ? E.hist(n + 1) : nullptr;
        if (sched) {
            const hvi::Action &a = (*sched)[ai++];
            if (a.op != hvi::ACT_FORWARD || a.a0 != n) return hvi::fail(HV_EINVAL, "internal: schedule order");
        }
        float *d_u = bx ? bx->fwd_data : (kind == 1 ? dd : nullptr);
        HV_RT(E.forward(n, born, d_u, kind == 2 ? dd : nullptr, target));
        if (sched && ai < sched->size() && (*sched)[ai].op == hvi::ACT_SAVE) HV_RT(E.save((*sched)[ai++].a0));
    }
    // ---- adjoint sources
    const float *r = in;
    int r_per_vector = 0;
    float rscale = (float)(h->h * h->h);
    if (kind == 1) {
        ProfScope ps(h, st, HV_K_OTHER);
        double *part = reinterpret_cast<double *>((char *)ws + L.part);
        HV_RT(hvk::launch_residual(h, dd, in, dd, part, kResidualBlocks, st));
        HV_RT(hvk::launch_reduce_phi(part, kResidualBlocks, 0.5 / (h->sigma * h->sigma), phi, st));
        r = dd;
        rscale = (float)(h->h * h->h / (h->sigma * h->sigma));
    } else if (kind == 2) {
        if (bx && bx->after_sweep) {
            ProfScope ps(h, st, HV_K_OTHER);
            HV_RT(bx->after_sweep(st));
        }
        r = dd;
        r_per_vector = 1;
        rscale = (float)(h->h * h->h / (h->sigma * h->sigma));
    }
    // ---- reversal
    HV_CK(cudaMemsetAsync((char *)ws + L.D, 0, (size_t)2 * kk * L.fb, st));
    HV_CK(cudaMemsetAsync((char *)ws + L.img, 0, (size_t)L.G * kk * h->fsize * sizeof(double), st));
    if (L.history) {
        for (int n = h->nt - 1; n >= 0; --n) HV_RT(E.adjoint(n, E.hist(n), r, r_per_vector, rscale, kk));
    } else {
        for (; ai < sched->size(); ++ai) {
            const hvi::Action &a = (*sched)[ai];
            switch (a.op) {
            case hvi::ACT_SAVE: HV_RT(E.save(a.a0)); break;
            case hvi::ACT_RESTORE: E.restore(a.a0, a.a1); break;
            case hvi::ACT_ADVANCE:
                if (ai + 1 < sched->size() && (*sched)[ai + 1].op == hvi::ACT_ADVANCE) {
                    HV_RT(E.forward2(E.j));             // two consecutive recomputation steps
                    ++ai;
                } else {
                    HV_RT(E.forward(E.j, false, nullptr, nullptr, nullptr, HV_K_ADVANCE));
                }
                break;
            case hvi::ACT_ADJOINT: {
                const float *u = E.u_for(a.a0);
                if (!u) return hvi::fail(HV_EINVAL, "internal: adjoint step %d from state %d", a.a0, E.j);
                HV_RT(E.adjoint(a.a0, u, r, r_per_vector, rscale, kk));
                break;
            }
            default: return hvi::fail(HV_EINVAL, "internal: forward step inside the reversal");
            }
        }
    }
    return HV_OK;
}

int validate_create(const hv_grid *g, const hv_acq *a)
{
    if (!g || !a) return hvi::fail(HV_EINVAL, "null grid or acquisition");
    if (g->nz < 1 || g->nx < 1) return hvi::fail(HV_EINVAL, "grid %d x %d; need nz, nx >= 1", g->nz, g->nx);
    if (g->nb < 0) return hvi::fail(HV_EINVAL, "sponge width %d < 0", g->nb);
    if (!(g->h > 0)) return hvi::fail(HV_EINVAL, "grid spacing must be > 0");
    long long NZ = g->nz + 2LL * g->nb, NX = g->nx + 2LL * g->nb;
    if (NZ > 65535 || NX > (1 << 20)) return hvi::fail(HV_EINVAL, "padded grid %lld x %lld too large", NZ, NX);
    if (a->ns < 1 || a->nr < 1 || a->nt < 1)
        return hvi::fail(HV_EINVAL, "ns = %d, nr = %d, nt = %d; all must be >= 1", a->ns, a->nr, a->nt);
    if (a->ns > 65535) return hvi::fail(HV_EINVAL, "ns = %d > 65535", a->ns);
    if (!a->src_iz || !a->src_ix || !a->rec_iz || !a->rec_ix) return hvi::fail(HV_EINVAL, "null acquisition array");
    if (!(a->dt > 0) || !(a->vmax > 0) || !(a->sigma > 0) || !(a->f0 > 0))
        return hvi::fail(HV_EINVAL, "dt, f0, vmax and sigma must be > 0");
    if (!(a->R > 0 && a->R < 1)) return hvi::fail(HV_EINVAL, "sponge reflection coefficient must lie in (0, 1)");
    for (int s = 0; s < a->ns; ++s) {
        if (a->src_iz[s] < 0 || a->src_iz[s] >= g->nz || a->src_ix[s] < 0 || a->src_ix[s] >= g->nx)
            return hvi::fail(HV_EINVAL, "shot %d source node (%d, %d) outside the %d x %d interior", s, a->src_iz[s],
                             a->src_ix[s], g->nz, g->nx);
        std::set<long long> seen;
        for (int r = 0; r < a->nr; ++r) {
            size_t i = (size_t)s * a->nr + r;
            if (a->rec_iz[i] < 0 || a->rec_iz[i] >= g->nz || a->rec_ix[i] < 0 || a->rec_ix[i] >= g->nx)
                return hvi::fail(HV_EINVAL, "shot %d receiver %d node (%d, %d) outside the interior", s, r,
                                 a->rec_iz[i], a->rec_ix[i]);
            if (!seen.insert((long long)a->rec_iz[i] * g->nx + a->rec_ix[i]).second)
                return hvi::fail(HV_EINVAL, "shot %d receiver %d duplicates another receiver's node", s, r);
        }
    }
    return HV_OK;
}

}  // namespace

extern "C" int hv_create(const hv_grid *g, const hv_acq *a, hv_handle **out)
{
    if (!out) return hvi::fail(HV_EINVAL, "null output handle pointer");
    *out = nullptr;
    HV_RT(validate_create(g, a));
    static std::atomic<unsigned long long> next_serial{1};
    hv_handle *h = new hv_handle();
    h->serial = next_serial++;
    h->nz = g->nz; h->nx = g->nx; h->nb = g->nb; h->h = g->h;
    h->NZ = g->nz + 2 * g->nb;
    h->NX = g->nx + 2 * g->nb;
    h->P = ((h->NX + 2 * hvi::GH) + 31) / 32 * 32;
    h->rows = h->NZ + 2 * hvi::GH;
    h->fsize = ((size_t)h->rows * h->P + 63) / 64 * 64;
    h->ns = a->ns; h->nr = a->nr; h->nt = a->nt;
    h->dt = a->dt; h->f0 = a->f0; h->t0 = a->t0; h->vmax = a->vmax; h->R = a->R; h->sigma = a->sigma;
    h->h_src_zx.resize(2 * (size_t)h->ns);
    h->h_rec_zx.resize(2 * (size_t)h->ns * h->nr);
    for (int s = 0; s < h->ns; ++s) {
        h->h_src_zx[2 * s] = a->src_iz[s] + h->nb;
        h->h_src_zx[2 * s + 1] = a->src_ix[s] + h->nb;
    }
    for (size_t i = 0; i < (size_t)h->ns * h->nr; ++i) {
        h->h_rec_zx[2 * i] = a->rec_iz[i] + h->nb;
        h->h_rec_zx[2 * i + 1] = a->rec_ix[i] + h->nb;
    }
    auto cleanup_fail = [&](int rc) {
        hv_destroy(h);
        return rc;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return cleanup_fail(hvi::fail(HV_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    if ((e = cudaMalloc(&h->wavelet, sizeof(float) * h->nt)) != cudaSuccess ||
        (e = cudaMalloc(&h->az, sizeof(float) * h->NZ)) != cudaSuccess ||
        (e = cudaMalloc(&h->ax, sizeof(float) * h->NX)) != cudaSuccess ||
        (e = cudaMalloc(&h->src_zx, sizeof(int) * h->h_src_zx.size())) != cudaSuccess ||
        (e = cudaMalloc(&h->rec_zx, sizeof(int) * h->h_rec_zx.size())) != cudaSuccess ||
        (e = cudaMalloc(&h->status, sizeof(int))) != cudaSuccess || (e = cudaMemset(h->status, 0, sizeof(int))) != cudaSuccess)
        return cleanup_fail(hvi::fail(HV_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e)));
    if ((e = cudaMemcpy(h->src_zx, h->h_src_zx.data(), sizeof(int) * h->h_src_zx.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(h->rec_zx, h->h_rec_zx.data(), sizeof(int) * h->h_rec_zx.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return cleanup_fail(hvi::fail(HV_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e)));
    int rc = hvk::launch_setup(h, 0);
    if (rc != HV_OK) return cleanup_fail(rc);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess)
        return cleanup_fail(hvi::fail(HV_ECUDA, "set-up kernels: %s", cudaGetErrorString(e)));
    for (int c = 0; c < hvk::tile_menu_size(); ++c)
        if ((rc = build_rectiles(h, hvk::tiling(h, c))) != HV_OK) return cleanup_fail(rc);
    if ((rc = hvk::prepare_kernels(h)) != HV_OK) return cleanup_fail(rc);
    if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup_fail(hvi::fail(HV_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    *out = h;
    return HV_OK;
}

extern "C" int hv_destroy(hv_handle *h)
{
    if (!h) return HV_OK;
    cudaDeviceSynchronize();
    cudaFree(h->wavelet);
    cudaFree(h->az);
    cudaFree(h->ax);
    cudaFree(h->src_zx);
    cudaFree(h->rec_zx);
    cudaFree(h->status);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (auto &r : h->prof_rec) {
        cudaEventDestroy(r.second.first);
        cudaEventDestroy(r.second.second);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (auto &kv : h->rectiles) {
        cudaFree(kv.second.off);
        cudaFree(kv.second.rec);
        cudaFree(kv.second.pos);
    }
    delete h;
    return HV_OK;
}

extern "C" int hv_workspace_size(const hv_handle *h, int op, int k, int ckpt, size_t *bytes)
{
    if (!h || !bytes) return hvi::fail(HV_EINVAL, "null handle or output");
    Layout L;
    if (op == HV_OP_FWD || op == HV_OP_BORN || op == HV_OP_WAVEFIELD || op == HV_OP_MISFIT || op == HV_OP_MISFITS)
        ckpt = HV_CKPT_ALL;
    HV_RT(make_layout(h, op, k, ckpt, L));
    *bytes = L.total;
    return HV_OK;
}

extern "C" int hv_fwd_model(hv_handle *h, const float *m, float *d, void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_fwd_model");
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_FWD, 1, HV_CKPT_ALL, L));
    if (!m || !d) return hvi::fail(HV_EINVAL, "null model or data pointer");
    cudaStream_t st = (cudaStream_t)stream;
    Exec E;
    HV_RT(E.init(h, st, L, ws, 0));
    HV_CK(cudaMemsetAsync(E.zero, 0, L.fb, st));
    HV_RT(E.zero_ghosts(false));
    HV_RT(hvk::launch_prep(h, m, nullptr, 0, E.C, nullptr, st));
    for (int n = 0; n < h->nt; ++n) HV_RT(E.forward(n, false, d, nullptr, nullptr));
    return HV_OK;
}

extern "C" int hv_misfit(hv_handle *h, const float *m, const float *d_obs, double *phi, void *ws, size_t ws_bytes,
                         void *stream)
{
    hvi::Range nvtx_range("hv_misfit");
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_MISFIT, 1, HV_CKPT_ALL, L));
    if (!m || !d_obs || !phi) return hvi::fail(HV_EINVAL, "null model, data or phi pointer");
    cudaStream_t st = (cudaStream_t)stream;
    Exec E;
    HV_RT(E.init(h, st, L, ws, 0));
    HV_CK(cudaMemsetAsync(E.zero, 0, L.fb, st));
    HV_RT(E.zero_ghosts(false));
    HV_RT(hvk::launch_prep(h, m, nullptr, 0, E.C, nullptr, st));
    float *dd = reinterpret_cast<float *>((char *)ws + L.dd);
    for (int n = 0; n < h->nt; ++n) HV_RT(E.forward(n, false, dd, nullptr, nullptr));
    double *part = reinterpret_cast<double *>((char *)ws + L.part);
    HV_RT(hvk::launch_residual(h, dd, d_obs, dd, part, kResidualBlocks, st));
    HV_RT(hvk::launch_reduce_phi(part, kResidualBlocks, 0.5 / (h->sigma * h->sigma), phi, st));
    return HV_OK;
}

namespace {

// The forward sweep of hv_misfit_models: the k models' field batches side by
// side in a ring of three (u^{n-1}, u^n, u^{n+1}), one launch per step for all
// of them, receiver samples into the data region.  Touches only the workspace
// and the handle.
int misfit_models_sweep(hv_handle *h, int k, const Layout &L, char *w, cudaStream_t st)
{
    hvk::TmaMaps maps;
    HV_RT(hvk::make_maps(h, w, (long long)(L.fields_end / (h->fsize * sizeof(float))), &maps));
    const size_t rb = (size_t)k * L.fb;
    float *ring[3];
    for (int r = 0; r < 3; ++r) ring[r] = reinterpret_cast<float *>(w + L.work + r * rb);
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_CK(cudaMemsetAsync(w + L.work, 0, 3 * rb, st));   // u^{-1} = u^0 = 0 and every ghost band
    }
    const int cfg = h->cfg[1];
    const hvi::RecTiles &rt = rectiles_for(h, hvk::tiling(h, cfg));
    for (int n = 0; n < h->nt; ++n) {
        ProfScope ps(h, st, HV_K_FWD);
        hvk::FwdLaunch a{};
        a.u_cur = ring[n % 3];
        a.u_prev = ring[(n + 2) % 3];
        a.u_next = ring[(n + 1) % 3];
        a.C = reinterpret_cast<const float *>(w + L.C);
        a.d_u = reinterpret_cast<float *>(w + L.dd);
        a.n = n;
        a.models = k;
        HV_RT(hvk::launch_fwd(h, cfg, rt, maps, a, st));
    }
    return HV_OK;
}

}  // namespace

extern "C" int hv_misfit_models(hv_handle *h, int k, const float *const *m, const float *const *d_obs,
                                double *const *phi, void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_misfit_models");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "hv_misfit_models: k = %d models; need 1 <= k <= 65535", k);
    if (!m || !d_obs || !phi) return hvi::fail(HV_EINVAL, "hv_misfit_models: null pointer array");
    for (int i = 0; i < k; ++i)
        if (!m[i] || !d_obs[i] || !phi[i])
            return hvi::fail(HV_EINVAL, "hv_misfit_models: null model, data or phi pointer for model %d", i);
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_MISFITS, k, HV_CKPT_ALL, L));
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    {
        ProfScope ps(h, st, HV_K_OTHER);
        float *C = reinterpret_cast<float *>(w + L.C);
        for (int i = 0; i < k; ++i) HV_RT(hvk::launch_prep(h, m[i], nullptr, 0, C + (size_t)i * h->fsize, nullptr, st));
    }
    // The sweep touches only the workspace and the handle: captured once per
    // workspace and replayed, as for H v (hv_set_graphs).
    if (h->graphs_on && !h->prof_on && !h->inject_wait) {
        const std::string key = "models/" + graph_key(ws, L.total, k, 0, h->cfg, h->launch_mode, false, false, h->wait_ns);
        auto it = h->graphs.find(key);
        cudaGraphExec_t ge = it == h->graphs.end() ? nullptr : it->second;
        if (!ge) {
            cudaStream_t cs = h->capture_stream;
            HV_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int rc = misfit_models_sweep(h, k, L, w, cs);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (rc != HV_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            ge = cache_graph(h, key, ex);
        }
        HV_CK(cudaGraphLaunch(ge, st));
    } else {
        HV_RT(misfit_models_sweep(h, k, L, w, st));
    }
    ProfScope ps(h, st, HV_K_OTHER);
    const size_t ndata = (size_t)h->ns * h->nt * h->nr;
    float *dd = reinterpret_cast<float *>(w + L.dd);
    double *part = reinterpret_cast<double *>(w + L.part);
    for (int i = 0; i < k; ++i) {
        float *di = dd + (size_t)i * ndata;
        double *pi = part + (size_t)i * kResidualBlocks;
        HV_RT(hvk::launch_residual(h, di, d_obs[i], di, pi, kResidualBlocks, st));
        HV_RT(hvk::launch_reduce_phi(pi, kResidualBlocks, 0.5 / (h->sigma * h->sigma), phi[i], st));
    }
    return HV_OK;
}

// ---------------------------------------------------------------- misfit engine
// Misfit requests that join a running sweep at the next time step
// (hv_engine_*): a fixed set of slots, each a model with its own coefficient
// field, ring of three field batches, data and step counter; one launch per
// tick advances every occupied slot by one step.
struct hv_engine {
    hv_handle *h = nullptr;
    int slots = 0;
    char *ws = nullptr;
    Layout L;
    int *join_dev = nullptr;           // [slots] tick of each slot's step 0 (kFreeSlot: free)
    hvk::TmaMaps maps;
    std::vector<int> join;
    std::vector<const float *> dobs;
    std::vector<double *> phi;
    int tick = 0;                      // launches since the last rebase
    int active = 0;
    bool dirty = true;                 // join differs from join_dev
    // The device-resident loop (hv_engine_post / serve / poll): its tables in
    // the workspace after join_dev, host-mapped mailboxes, its graph.
    bool loop = false;                 // a request was posted: join and tick are refused from then on
    int *post = nullptr, *seen = nullptr, *step = nullptr, *fin = nullptr, *ctl = nullptr;
    const float **dobs_tbl = nullptr;
    double **phi_tbl = nullptr;
    int *hmap = nullptr;               // pinned, mapped: ack[slots], done[slots], stop
    int *hmap_dev = nullptr;
    cudaEvent_t init_done = nullptr;   // the tables' initialisation (first post)
    cudaEvent_t ran = nullptr;         // recorded after the last launch of the loop
    bool launched = false;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int seq = 0;
    std::vector<int> slot_seq;         // sequence number posted into each slot (0: free)
};

namespace {

constexpr int kFreeSlot = 1 << 30;     // later than any tick: a free slot takes no step
constexpr int kRebaseTick = 1 << 28;

constexpr int kLoopBlocks = 1024;       // residual blocks of one misfit: kResidualBlocks, as hv_misfit
constexpr int kLoopMaxIter = 1 << 20;   // iterations of one launch of the loop, at most
constexpr int kLoopIdle = 200;          // iterations with no occupied slot before the loop ends

size_t loop_bytes(int slots)
{
    const size_t i = align256((size_t)slots * sizeof(int));
    return 3 * i + align256((size_t)(slots + 1) * sizeof(int)) + 256 + 2 * align256((size_t)slots * sizeof(void *));
}

size_t engine_bytes(const Layout &L, int slots)
{
    return L.total + align256((size_t)slots * sizeof(int)) + loop_bytes(slots);
}

}  // namespace

extern "C" int hv_engine_workspace_size(const hv_handle *h, int slots, size_t *bytes)
{
    if (!h || !bytes) return hvi::fail(HV_EINVAL, "hv_engine_workspace_size: null handle or output");
    Layout L;
    HV_RT(make_layout(h, HV_OP_MISFITS, slots, HV_CKPT_ALL, L));
    *bytes = engine_bytes(L, slots);
    return HV_OK;
}

extern "C" int hv_engine_create(hv_handle *h, int slots, void *ws, size_t ws_bytes, hv_engine **out)
{
    if (!out) return hvi::fail(HV_EINVAL, "hv_engine_create: null output pointer");
    *out = nullptr;
    if (slots < 1 || slots > 65535) return hvi::fail(HV_EINVAL, "hv_engine_create: %d slots; need 1..65535", slots);
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_MISFITS, slots, HV_CKPT_ALL, L));
    if (ws_bytes < engine_bytes(L, slots))
        return hvi::fail(HV_ENOMEM, "hv_engine_create: workspace of %zu bytes; %zu needed", ws_bytes, engine_bytes(L, slots));
    hv_engine *e = new hv_engine();
    e->h = h;
    e->slots = slots;
    e->ws = (char *)ws;
    e->L = L;
    e->join_dev = reinterpret_cast<int *>(e->ws + L.total);
    {
        char *q = e->ws + L.total + align256((size_t)slots * sizeof(int));
        const size_t i = align256((size_t)slots * sizeof(int));
        e->post = reinterpret_cast<int *>(q);
        e->seen = reinterpret_cast<int *>(q + i);
        e->step = reinterpret_cast<int *>(q + 2 * i);
        e->fin = reinterpret_cast<int *>(q + 3 * i);
        e->ctl = reinterpret_cast<int *>(q + 3 * i + align256((size_t)(slots + 1) * sizeof(int)));
        e->dobs_tbl = reinterpret_cast<const float **>(q + 3 * i + align256((size_t)(slots + 1) * sizeof(int)) + 256);
        e->phi_tbl = reinterpret_cast<double **>(reinterpret_cast<char *>(e->dobs_tbl) +
                                                 align256((size_t)slots * sizeof(void *)));
    }
    e->slot_seq.assign(slots, 0);
    e->join.assign(slots, kFreeSlot);
    e->dobs.assign(slots, nullptr);
    e->phi.assign(slots, nullptr);
    int rc = hvk::make_maps(h, ws, (long long)(L.fields_end / (h->fsize * sizeof(float))), &e->maps);
    if (rc != HV_OK) {
        delete e;
        return rc;
    }
    *out = e;
    return HV_OK;
}

extern "C" int hv_engine_destroy(hv_engine *e)
{
    if (!e) return HV_OK;
    if (e->launched && cudaEventQuery(e->ran) == cudaErrorNotReady) {   // end the loop after its iteration
        reinterpret_cast<volatile int *>(e->hmap)[2 * e->slots] = 1;
        cudaEventSynchronize(e->ran);
    }
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->ran) cudaEventDestroy(e->ran);
    if (e->init_done) cudaEventDestroy(e->init_done);
    if (e->hmap) cudaFreeHost(e->hmap);
    delete e;
    return HV_OK;
}

extern "C" int hv_engine_join(hv_engine *e, const float *m, const float *d_obs, double *phi, void *stream, int *slot)
{
    if (!e || !m || !d_obs || !phi || !slot) return hvi::fail(HV_EINVAL, "hv_engine_join: null argument");
    *slot = -1;
    if (e->loop) return hvi::fail(HV_EINVAL, "hv_engine_join: the engine serves posted requests (hv_engine_post)");
    int j = 0;
    while (j < e->slots && e->join[j] != kFreeSlot) ++j;
    if (j == e->slots) return hvi::fail(HV_EBUSY, "hv_engine_join: all %d slots are taken", e->slots);
    hv_handle *h = e->h;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fbytes = h->fsize * sizeof(float);
    if (e->active == 0) e->tick = 0;   // nothing in flight depends on the old count once every slot is free
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_RT(hvk::launch_prep(h, m, nullptr, 0, reinterpret_cast<float *>(e->ws + e->L.C) + (size_t)j * h->fsize,
                               nullptr, st));
        HV_CK(cudaMemsetAsync(e->ws + e->L.work + (size_t)3 * j * h->ns * fbytes, 0, (size_t)3 * h->ns * fbytes, st));
    }
    e->join[j] = e->tick;
    e->dobs[j] = d_obs;
    e->phi[j] = phi;
    e->dirty = true;
    ++e->active;
    *slot = j;
    return HV_OK;
}

extern "C" int hv_engine_tick(hv_engine *e, void *stream, int *done, int *n_done)
{
    hvi::Range nvtx_range("hv_engine_tick");
    if (!e || !done || !n_done) return hvi::fail(HV_EINVAL, "hv_engine_tick: null argument");
    *n_done = 0;
    if (e->loop) return hvi::fail(HV_EINVAL, "hv_engine_tick: the engine serves posted requests (hv_engine_post)");
    if (e->active == 0) return HV_OK;
    hv_handle *h = e->h;
    cudaStream_t st = (cudaStream_t)stream;
    if (e->tick >= kRebaseTick) {      // keep the counters far below kFreeSlot
        int base = kFreeSlot;
        for (int v : e->join) base = std::min(base, v);
        for (int &v : e->join)
            if (v != kFreeSlot) v -= base;
        e->tick -= base;
        e->dirty = true;
    }
    if (e->dirty) {                    // pageable source: staged before the call returns
        HV_CK(cudaMemcpyAsync(e->join_dev, e->join.data(), (size_t)e->slots * sizeof(int), cudaMemcpyHostToDevice, st));
        e->dirty = false;
    }
    int ymax = 0;
    for (int j = 0; j < e->slots; ++j)
        if (e->join[j] != kFreeSlot) ymax = j + 1;
    {
        ProfScope ps(h, st, HV_K_FWD);
        hvk::FwdLaunch a{};
        a.u_cur = a.u_prev = reinterpret_cast<const float *>(e->ws + e->L.work);
        a.u_next = reinterpret_cast<float *>(e->ws + e->L.work);
        a.C = reinterpret_cast<const float *>(e->ws + e->L.C);
        a.d_u = reinterpret_cast<float *>(e->ws + e->L.dd);
        a.n = e->tick;
        a.models = ymax;
        a.slot_join = e->join_dev;
        const int cfg = h->cfg[1];
        HV_RT(hvk::launch_fwd(h, cfg, rectiles_for(h, hvk::tiling(h, cfg)), e->maps, a, st));
    }
    const size_t ndata = (size_t)h->ns * h->nt * h->nr;
    for (int j = 0; j < e->slots; ++j) {
        if (e->join[j] == kFreeSlot || e->tick - e->join[j] != h->nt - 1) continue;
        ProfScope ps(h, st, HV_K_OTHER);
        float *dj = reinterpret_cast<float *>(e->ws + e->L.dd) + (size_t)j * ndata;
        double *pj = reinterpret_cast<double *>(e->ws + e->L.part) + (size_t)j * kResidualBlocks;
        HV_RT(hvk::launch_residual(h, dj, e->dobs[j], dj, pj, kResidualBlocks, st));
        HV_RT(hvk::launch_reduce_phi(pj, kResidualBlocks, 0.5 / (h->sigma * h->sigma), e->phi[j], st));
        e->join[j] = kFreeSlot;
        e->dirty = true;
        --e->active;
        done[(*n_done)++] = j;
    }
    ++e->tick;
    return HV_OK;
}

namespace {

// The loop's graph: a conditional while node whose body is a switch over
// the iterations: the forward step launched over the first 1, 2, 4, ...
// slots, followed by k_loop_control and an if node holding the finishing
// slots' misfits; or k_loop_control alone.  Each node's body is captured into
// the graph the node owns.
int capture_into(cudaStream_t cs, cudaGraph_t g, const std::function<int()> &launch)
{
    HV_CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int rc = launch();
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &out);
    if (rc != HV_OK) return rc;
    if (ce != cudaSuccess) return hvi::fail(HV_ECUDA, "misfit loop capture: %s", cudaGetErrorString(ce));
    return HV_OK;
}

int add_conditional(cudaGraph_t g, cudaGraphConditionalHandle hc, cudaGraphConditionalNodeType type, unsigned size,
                    const cudaGraphNode_t *dep, cudaGraphNode_t *node, cudaGraph_t *bodies)
{
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = type;
    np.conditional.size = size;
    HV_CK(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &np));
    for (unsigned i = 0; i < size; ++i) bodies[i] = np.conditional.phGraph_out[i];
    return HV_OK;
}

int build_loop_graph(hv_engine *e)
{
    hv_handle *h = e->h;
    if (!e->cap) HV_CK(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking));
    HV_CK(cudaGraphCreate(&e->graph, 0));
    hvk::LoopParams lp{};
    HV_CK(cudaGraphConditionalHandleCreate(&lp.cond, e->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t wnode, snode;
    cudaGraph_t body;
    HV_RT(add_conditional(e->graph, lp.cond, cudaGraphCondTypeWhile, 1, nullptr, &wnode, &body));
    int nsizes = 1;                    // step launches over the first 1, 2, 4, ... slots, the last all of them
    while ((1 << (nsizes - 1)) < e->slots) ++nsizes;
    // Every launch starts with the body without a step (the default is applied per launch), so
    // a relaunch never advances a slot twice.
    HV_CK(cudaGraphConditionalHandleCreate(&lp.cond_step, body, (unsigned)nsizes, cudaGraphCondAssignDefault));
    lp.slots = e->slots;
    lp.nt = h->nt;
    lp.nblk = kLoopBlocks;
    lp.ndata = (size_t)h->ns * h->nt * h->nr;
    lp.scale = 0.5 / (h->sigma * h->sigma);
    lp.max_iter = kLoopMaxIter;
    lp.idle_max = kLoopIdle;
    lp.post = e->post;
    lp.seen = e->seen;
    lp.step = e->step;
    lp.join = e->join_dev;
    lp.fin = e->fin;
    lp.ctl = e->ctl;
    lp.dobs = e->dobs_tbl;
    lp.phi = e->phi_tbl;
    lp.data = reinterpret_cast<float *>(e->ws + e->L.dd);
    lp.part = reinterpret_cast<double *>(e->ws + e->L.part);
    lp.ack = e->hmap_dev;
    lp.done = e->hmap_dev + e->slots;
    lp.stop = e->hmap_dev + 2 * e->slots;
    lp.nsizes = nsizes;
    std::vector<cudaGraph_t> sb(nsizes + 1);
    HV_RT(add_conditional(body, lp.cond_step, cudaGraphCondTypeSwitch, (unsigned)nsizes + 1, nullptr, &snode,
                          sb.data()));
    for (int i = 0; i <= nsizes; ++i) {
        const bool step = i < nsizes;
        hvk::LoopParams li = lp;
        li.after_tick = step ? 1 : 0;
        if (step) HV_CK(cudaGraphConditionalHandleCreate(&li.cond_fin, sb[i], 0, 0));
        HV_RT(capture_into(e->cap, sb[i], [&] {
            int rc = HV_OK;
            if (step) {
                hvk::FwdLaunch a{};
                a.u_cur = a.u_prev = reinterpret_cast<const float *>(e->ws + e->L.work);
                a.u_next = reinterpret_cast<float *>(e->ws + e->L.work);
                a.C = reinterpret_cast<const float *>(e->ws + e->L.C);
                a.d_u = lp.data;
                a.n = 0;               // k_fwd's step of slot j: 0 - join[j] = step[j]
                a.models = std::min(e->slots, 1 << i);
                a.slot_join = e->join_dev;
                a.plain = true;        // first in its body
                const int cfg = h->cfg[1];
                rc = hvk::launch_fwd(h, cfg, rectiles_for(h, hvk::tiling(h, cfg)), e->maps, a, e->cap);
            }
            // behind the step by programmatic dependent launch: resident while the step drains
            if (rc == HV_OK) rc = hvk::launch_loop_control(li, e->cap, step);
            return rc;
        }));
        if (!step) continue;
        cudaGraphNode_t root[2];
        size_t nroot = 2, nall = 0;
        HV_CK(cudaGraphGetRootNodes(sb[i], root, &nroot));
        HV_CK(cudaGraphGetNodes(sb[i], nullptr, &nall));
        std::vector<cudaGraphNode_t> all(nall);
        HV_CK(cudaGraphGetNodes(sb[i], all.data(), &nall));
        if (nroot != 1 || nall != 2) return hvi::fail(HV_ECUDA, "misfit loop: step body of %zu nodes", nall);
        const cudaGraphNode_t ctrl = all[0] == root[0] ? all[1] : all[0];
        cudaGraphNode_t fnode;
        cudaGraph_t fb;
        HV_RT(add_conditional(sb[i], li.cond_fin, cudaGraphCondTypeIf, 1, &ctrl, &fnode, &fb));
        HV_RT(capture_into(e->cap, fb, [&] { return hvk::launch_loop_finish(li, e->cap); }));
    }
    HV_CK(cudaGraphInstantiate(&e->exec, e->graph, 0));
    return HV_OK;
}

}  // namespace

extern "C" int hv_engine_post(hv_engine *e, const float *m, const float *d_obs, double *phi, void *stream, int *slot)
{
    hvi::Range nvtx_range("hv_engine_post");
    if (!e || !m || !d_obs || !phi || !slot) return hvi::fail(HV_EINVAL, "hv_engine_post: null argument");
    *slot = -1;
    if (!e->loop && e->active > 0)
        return hvi::fail(HV_EINVAL, "hv_engine_post: slots joined with hv_engine_join are still running");
    hv_handle *h = e->h;
    cudaStream_t st = (cudaStream_t)stream;
    const int S = e->slots;
    if (!e->loop) {                                // first post: mailboxes, tables, events
        HV_CK(cudaHostAlloc(reinterpret_cast<void **>(&e->hmap), (2 * (size_t)S + 1) * sizeof(int), cudaHostAllocMapped));
        memset(e->hmap, 0, (2 * (size_t)S + 1) * sizeof(int));
        HV_CK(cudaHostGetDevicePointer(reinterpret_cast<void **>(&e->hmap_dev), e->hmap, 0));
        HV_CK(cudaEventCreateWithFlags(&e->init_done, cudaEventDisableTiming));
        HV_CK(cudaEventCreateWithFlags(&e->ran, cudaEventDisableTiming));
        HV_CK(cudaMemsetAsync(e->post, 0, (size_t)S * sizeof(int), st));
        HV_CK(cudaMemsetAsync(e->seen, 0, (size_t)S * sizeof(int), st));
        HV_CK(cudaMemsetAsync(e->step, 0xff, (size_t)S * sizeof(int), st));   // -1: free
        HV_CK(cudaMemsetAsync(e->fin, 0, (size_t)(S + 1) * sizeof(int), st));
        HV_CK(cudaMemsetAsync(e->ctl, 0, 4 * sizeof(int), st));
        HV_CK(cudaEventRecord(e->init_done, st));
        e->loop = true;
    }
    int j = 0;
    while (j < S && e->slot_seq[j] != 0) ++j;
    if (j == S) return hvi::fail(HV_EBUSY, "hv_engine_post: all %d slots are taken", S);
    const size_t fbytes = h->fsize * sizeof(float);
    e->seq = e->seq == INT_MAX ? 1 : e->seq + 1;   // never 0, the value of a slot that was never posted
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_RT(hvk::launch_prep(h, m, nullptr, 0, reinterpret_cast<float *>(e->ws + e->L.C) + (size_t)j * h->fsize,
                               nullptr, st));
        HV_CK(cudaMemsetAsync(e->ws + e->L.work + (size_t)3 * j * h->ns * fbytes, 0, (size_t)3 * h->ns * fbytes, st));
        HV_RT(hvk::launch_loop_post(e->post, e->dobs_tbl, e->phi_tbl, j, e->seq, d_obs, phi, st));
    }
    e->slot_seq[j] = e->seq;
    *slot = j;
    return HV_OK;
}

extern "C" int hv_engine_serve(hv_engine *e, void *stream)
{
    hvi::Range nvtx_range("hv_engine_serve");
    if (!e) return hvi::fail(HV_EINVAL, "hv_engine_serve: null engine");
    if (!e->loop) return hvi::fail(HV_EINVAL, "hv_engine_serve: nothing was posted to this engine");
    if (e->launched && cudaEventQuery(e->ran) == cudaErrorNotReady) return HV_OK;   // running
    cudaStream_t st = (cudaStream_t)stream;
    if (!e->exec) {
        const int rc = build_loop_graph(e);
        if (rc != HV_OK) {                         // a later call builds it again from scratch
            if (e->graph) cudaGraphDestroy(e->graph);
            e->graph = nullptr;
            return rc;
        }
    }
    reinterpret_cast<volatile int *>(e->hmap)[2 * e->slots] = 0;                   // no stop request
    HV_CK(cudaStreamWaitEvent(st, e->init_done, 0));
    HV_CK(cudaGraphLaunch(e->exec, st));
    HV_CK(cudaEventRecord(e->ran, st));
    e->launched = true;
    return HV_OK;
}

extern "C" int hv_engine_poll(hv_engine *e, int *done, int *n_done, int *running)
{
    if (!e || !done || !n_done) return hvi::fail(HV_EINVAL, "hv_engine_poll: null argument");
    *n_done = 0;
    if (e->loop) {
        const volatile int *dn = e->hmap + e->slots;
        for (int j = 0; j < e->slots; ++j)
            if (e->slot_seq[j] != 0 && dn[j] == e->slot_seq[j]) {
                done[(*n_done)++] = j;
                e->slot_seq[j] = 0;
            }
    }
    if (running) *running = e->launched && cudaEventQuery(e->ran) == cudaErrorNotReady;
    return HV_OK;
}

extern "C" int hv_engine_stop(hv_engine *e)
{
    if (!e) return hvi::fail(HV_EINVAL, "hv_engine_stop: null engine");
    if (e->hmap) reinterpret_cast<volatile int *>(e->hmap)[2 * e->slots] = 1;
    return HV_OK;
}

extern "C" int hv_engine_active(const hv_engine *e, int *active)
{
    if (!e || !active) return hvi::fail(HV_EINVAL, "hv_engine_active: null argument");
    *active = e->active;
    return HV_OK;
}

extern "C" int hv_wavefield(hv_handle *h, const float *m, int n_out, const int *steps, float *out, void *ws,
                            size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_wavefield");
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_WAVEFIELD, 1, HV_CKPT_ALL, L));
    if (!m || !out || !steps || n_out < 1) return hvi::fail(HV_EINVAL, "null pointer or n_out < 1");
    for (int i = 0; i < n_out; ++i)
        if (steps[i] < 0 || steps[i] >= h->nt || (i > 0 && steps[i] <= steps[i - 1]))
            return hvi::fail(HV_EINVAL, "steps must be ascending and in [0, nt)");
    cudaStream_t st = (cudaStream_t)stream;
    Exec E;
    HV_RT(E.init(h, st, L, ws, 0));
    HV_CK(cudaMemsetAsync(E.zero, 0, L.fb, st));
    HV_RT(E.zero_ghosts(false));
    HV_RT(hvk::launch_prep(h, m, nullptr, 0, E.C, nullptr, st));
    int i = 0;
    for (int n = 0; n <= steps[n_out - 1]; ++n) {
        HV_RT(E.forward(n, false, nullptr, nullptr, nullptr));
        if (n == steps[i]) {
            HV_RT(hvk::launch_copy_wavefield(h, E.cur, out + (size_t)i * h->ns * h->NZ * h->NX, st));
            ++i;
        }
    }
    return HV_OK;
}

extern "C" int hv_born(hv_handle *h, const float *m, const float *dm, int k, float *dd, void *ws, size_t ws_bytes,
                       void *stream)
{
    hvi::Range nvtx_range("hv_born");
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_BORN, k, HV_CKPT_ALL, L));
    if (!m || !dm || !dd) return hvi::fail(HV_EINVAL, "null model, perturbation or output");
    cudaStream_t st = (cudaStream_t)stream;
    Exec E;
    HV_RT(E.init(h, st, L, ws, k));
    HV_CK(cudaMemsetAsync(E.zero, 0, L.fb, st));
    HV_RT(E.zero_ghosts(false));
    HV_CK(cudaMemsetAsync((char *)ws + L.D, 0, (size_t)2 * k * L.fb, st));
    HV_RT(hvk::launch_prep(h, m, dm, k, E.C, E.b, st));
    for (int n = 0; n < h->nt; ++n) HV_RT(E.forward(n, true, nullptr, dd, nullptr));
    return HV_OK;
}

extern "C" int hv_migrate(hv_handle *h, const float *m, const float *r, float *g, int ckpt, void *ws, size_t ws_bytes,
                          void *stream)
{
    hvi::Range nvtx_range("hv_migrate");
    if (!m || !r || !g) return hvi::fail(HV_EINVAL, "null model, data or output");
    return run_adjoint(h, 0, m, r, 1, g, nullptr, nullptr, ckpt, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int hv_misfit_grad(hv_handle *h, const float *m, const float *d_obs, double *phi, float *grad, int ckpt,
                              void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_misfit_grad");
    if (!m || !d_obs || !phi || !grad) return hvi::fail(HV_EINVAL, "null model, data, phi or gradient");
    return run_adjoint(h, 1, m, d_obs, 1, grad, nullptr, phi, ckpt, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int hv_hessian_apply(hv_handle *h, const float *m, const float *v, int k, float *Hv, int ckpt, void *ws,
                                size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_hessian_apply");
    if (!m || !v || !Hv) return hvi::fail(HV_EINVAL, "null model, vector or output");
    return run_adjoint(h, 2, m, v, k, Hv, nullptr, nullptr, ckpt, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int hv_hessian_apply_f64out(hv_handle *h, const float *m, const float *v, int k, double *Hv, int ckpt,
                                       void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_hessian_apply_f64out");
    if (!m || !v || !Hv) return hvi::fail(HV_EINVAL, "null model, vector or output");
    return run_adjoint(h, 2, m, v, k, nullptr, Hv, nullptr, ckpt, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int hv_hessian_apply_partial(hv_handle *h, const float *m, const float *v, int k, double *ext, int ckpt,
                                        void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_hessian_apply_partial");
    if (!m || !v || !ext) return hvi::fail(HV_EINVAL, "null model, vector or output");
    return run_adjoint(h, 2, m, v, k, nullptr, nullptr, nullptr, ckpt, ws, ws_bytes, (cudaStream_t)stream, ext);
}

extern "C" int hv_image_fold(hv_handle *h, const double *ext, int k, float *out, double *out64, void *stream)
{
    hvi::Range nvtx_range("hv_image_fold");
    if (!h || !ext || (!out && !out64)) return hvi::fail(HV_EINVAL, "null handle, image or output");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "k = %d; need 1 <= k <= 65535", k);
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != h->device) return hvi::fail(HV_EINVAL, "current device %d is not the handle's device %d", dev, h->device);
    return hvk::launch_fold_ext(h, ext, k, out, out64, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- merged calls
namespace {

struct BatchLayout {
    int K = 0;                 // Born vectors: the Hessian vectors, then one per gradient
    Layout L;                  // HV_OP_HV with K vectors, or HV_OP_MISFIT when K = 0
    size_t vstage = 0, ostage = 0, fwd = 0, rscr = 0, part = 0, total = 0;
};

int batch_check(const hv_handle *h, const hv_batch *b)
{
    if (!h || !b) return hvi::fail(HV_EINVAL, "null handle or batch");
    if (b->n_hv < 0 || b->n_grad < 0 || b->n_misfit < 0 || b->n_hv + b->n_grad + b->n_misfit == 0)
        return hvi::fail(HV_EINVAL, "empty batch or negative counts");
    if ((b->n_hv && (!b->v || !b->k || !b->Hv)) || (b->n_grad && (!b->grad_dobs || !b->grad_phi || !b->grad)) ||
        (b->n_misfit && (!b->misfit_dobs || !b->misfit_phi)))
        return hvi::fail(HV_EINVAL, "batch: null array");
    long long K = b->n_grad;
    for (int i = 0; i < b->n_hv; ++i) {
        if (b->k[i] < 1 || !b->v[i] || !b->Hv[i]) return hvi::fail(HV_EINVAL, "batch: H v entry %d is empty", i);
        K += b->k[i];
    }
    for (int g = 0; g < b->n_grad; ++g)
        if (!b->grad_dobs[g] || !b->grad_phi[g] || !b->grad[g]) return hvi::fail(HV_EINVAL, "batch: gradient %d", g);
    for (int q = 0; q < b->n_misfit; ++q)
        if (!b->misfit_dobs[q] || !b->misfit_phi[q]) return hvi::fail(HV_EINVAL, "batch: misfit %d", q);
    if (K > 65535) return hvi::fail(HV_EINVAL, "batch: %lld vectors; at most 65535", K);
    return HV_OK;
}

int batch_layout(const hv_handle *h, const hv_batch *b, int ckpt, BatchLayout &B)
{
    HV_RT(batch_check(h, b));
    B.K = b->n_grad;
    for (int i = 0; i < b->n_hv; ++i) B.K += b->k[i];
    if (B.K > 0) HV_RT(make_layout(h, HV_OP_HV, B.K, ckpt, B.L));
    else HV_RT(make_layout(h, HV_OP_MISFIT, 1, HV_CKPT_ALL, B.L));
    const size_t N = (size_t)h->nz * h->nx, ndata = (size_t)h->ns * h->nt * h->nr;
    size_t o = B.L.total;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    if (B.K > 0) {
        B.vstage = take((size_t)B.K * N * sizeof(float));
        B.ostage = take((size_t)B.K * N * sizeof(float));
        B.fwd = take(ndata * sizeof(float));
    }
    B.rscr = take(ndata * sizeof(float));
    B.part = take((size_t)(b->n_grad + b->n_misfit) * kResidualBlocks * sizeof(double));
    B.total = o;
    return HV_OK;
}

}  // namespace

extern "C" int hv_batch_workspace_size(const hv_handle *h, const hv_batch *b, int ckpt, size_t *bytes)
{
    if (!bytes) return hvi::fail(HV_EINVAL, "null output");
    BatchLayout B;
    HV_RT(batch_layout(h, b, ckpt, B));
    *bytes = B.total;
    return HV_OK;
}

extern "C" int hv_apply_batch(hv_handle *h, const float *m, const hv_batch *b, int ckpt, void *ws, size_t ws_bytes,
                              void *stream)
{
    hvi::Range nvtx_range("hv_apply_batch");
    if (!m) return hvi::fail(HV_EINVAL, "null model");
    BatchLayout B;
    HV_RT(batch_layout(h, b, ckpt, B));
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != h->device) return hvi::fail(HV_EINVAL, "current device %d is not the handle's device %d", dev, h->device);
    if (!ws || ((uintptr_t)ws & 255u) != 0) return hvi::fail(HV_EINVAL, "workspace must be non-null and 256-byte aligned");
    if (ws_bytes < B.total) return hvi::fail(HV_ENOMEM, "workspace of %zu bytes; this batch needs %zu", ws_bytes, B.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    const size_t N = (size_t)h->nz * h->nx, ndata = (size_t)h->ns * h->nt * h->nr;
    const double phi_scale = 0.5 / (h->sigma * h->sigma);
    double *part = reinterpret_cast<double *>(w + B.part);
    float *rscr = reinterpret_cast<float *>(w + B.rscr);
    // The misfits of the batch from the forward data: r = d - d_obs (discarded), phi in FP64.
    auto misfits = [&](const float *fwd, cudaStream_t s) -> int {
        for (int q = 0; q < b->n_misfit; ++q) {
            double *pq = part + (size_t)(b->n_grad + q) * kResidualBlocks;
            HV_RT(hvk::launch_residual(h, fwd, b->misfit_dobs[q], rscr, pq, kResidualBlocks, s));
            HV_RT(hvk::launch_reduce_phi(pq, kResidualBlocks, phi_scale, b->misfit_phi[q], s));
        }
        return HV_OK;
    };
    if (B.K == 0) {                               // misfits only: one forward sweep
        Exec E;
        HV_RT(E.init(h, st, B.L, ws, 0));
        HV_CK(cudaMemsetAsync(E.zero, 0, B.L.fb, st));
        HV_RT(E.zero_ghosts(false));
        HV_RT(hvk::launch_prep(h, m, nullptr, 0, E.C, nullptr, st));
        float *fwd = reinterpret_cast<float *>(w + B.L.dd);
        for (int n = 0; n < h->nt; ++n) HV_RT(E.forward(n, false, fwd, nullptr, nullptr));
        return misfits(fwd, st);
    }
    // Gather the vectors: the H v vectors in entry order, then a zero vector per gradient
    // (its Born field stays zero; its adjoint source becomes the residual).
    float *V = reinterpret_cast<float *>(w + B.vstage), *O = reinterpret_cast<float *>(w + B.ostage);
    float *fwd = reinterpret_cast<float *>(w + B.fwd);
    size_t at = 0;
    for (int i = 0; i < b->n_hv; ++i) {
        HV_CK(cudaMemcpyAsync(V + at * N, b->v[i], (size_t)b->k[i] * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        at += b->k[i];
    }
    const size_t g0 = at;
    if (b->n_grad) HV_CK(cudaMemsetAsync(V + g0 * N, 0, (size_t)b->n_grad * N * sizeof(float), st));
    const Layout &L = B.L;
    float *dd = reinterpret_cast<float *>(w + L.dd);
    BatchExtra bx;
    bx.fwd_data = fwd;
    bx.after_sweep = [&](cudaStream_t s) -> int {
        for (int g = 0; g < b->n_grad; ++g) {       // gradient slot: r = f(m) - d_obs replaces its Born data
            double *pg = part + (size_t)g * kResidualBlocks;
            HV_RT(hvk::launch_residual(h, fwd, b->grad_dobs[g], dd + (g0 + g) * ndata, pg, kResidualBlocks, s));
            HV_RT(hvk::launch_reduce_phi(pg, kResidualBlocks, phi_scale, b->grad_phi[g], s));
        }
        return misfits(fwd, s);
    };
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_RT(hvk::launch_prep(h, m, V, B.K, reinterpret_cast<float *>(w + L.C), reinterpret_cast<float *>(w + L.b), st));
    }
    HV_RT(run_adjoint_body(h, 2, V, B.K, nullptr, ckpt, ws, L, st, &bx));
    {
        ProfScope ps(h, st, HV_K_OTHER);
        HV_RT(hvk::launch_finalize(h, m, reinterpret_cast<double *>(w + L.img), h->img_f64 ? hvk::kImgF64 : hvk::kImgPairs,
                                   L.G, B.K, O, nullptr, reinterpret_cast<double *>(w + L.D), st));
    }
    at = 0;
    for (int i = 0; i < b->n_hv; ++i) {
        HV_CK(cudaMemcpyAsync(b->Hv[i], O + at * N, (size_t)b->k[i] * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        at += b->k[i];
    }
    for (int g = 0; g < b->n_grad; ++g)
        HV_CK(cudaMemcpyAsync(b->grad[g], O + (g0 + g) * N, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HV_OK;
}

extern "C" int hv_count_nonfinite(const float *x, size_t n, unsigned long long *count, void *stream)
{
    if (!count || (n > 0 && !x)) return hvi::fail(HV_EINVAL, "hv_count_nonfinite: null pointer");
    return hvk::launch_count_nonfinite(x, n, count, (cudaStream_t)stream);
}

extern "C" int hv_profile(hv_handle *h, int enable)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    h->prof_on = enable != 0;
    return HV_OK;
}

extern "C" int hv_profile_read(hv_handle *h, long long *launches, double *ms)
{
    if (!h || !launches || !ms) return hvi::fail(HV_EINVAL, "null handle or output");
    for (int k = 0; k < HV_K_COUNT; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
    }
    for (auto &r : h->prof_rec) {
        HV_CK(cudaEventSynchronize(r.second.second));
        float t = 0.f;
        HV_CK(cudaEventElapsedTime(&t, r.second.first, r.second.second));
        launches[r.first] += 1;
        ms[r.first] += t;
        h->ev_pool.push_back(r.second.first);
        h->ev_pool.push_back(r.second.second);
    }
    h->prof_rec.clear();
    return HV_OK;
}

extern "C" long long hv_kernel_launches(void) { return hvk::launches_so_far(); }

// ---------------------------------------------------------------- allocation-free Hessian apply
//
// hv_hessian_apply_static serves callers that cannot allocate device memory
// at the point of the call: code that runs under a device-memory budget owned
// by someone else (a host application that hands out every byte from its own
// pool), a real-time loop where an allocation could stall, or a caller that
// has no way to size and pass a workspace.  It needs no handle and no
// workspace: the problem tables and the scratch fields live in the array
// below, which every GPU that loads the library holds until the process
// exits.  It runs exactly the kernels of hv_hessian_apply.
namespace {

__device__ __align__(256) unsigned char g_hv_static_scratch[HV_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
std::map<int, void *> g_static_base;   // device ordinal -> device address of the array

// Device address of the scratch array on `dev` (the current device).  Looked
// up once per device; in host code the symbol itself is only a stand-in.
int static_scratch_base(int dev, void **base)
{
    std::lock_guard<std::mutex> g(g_static_mu);
    auto it = g_static_base.find(dev);
    if (it != g_static_base.end()) {
        *base = it->second;
        return HV_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_hv_static_scratch);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    g_static_base[dev] = p;
    *base = p;
    return HV_OK;
}

// Receiver tables of one tiling, on the host.
void static_rectile_tables(const hv_handle *h, const hvi::Tiling &t, std::vector<int> &off, std::vector<int> &rec,
                           std::vector<int> &pos)
{
    off.assign((size_t)h->ns * (t.ntiles + 1), 0);
    rec.assign((size_t)h->ns * h->nr, 0);
    pos.assign((size_t)h->ns * h->nr, 0);
    for (int s = 0; s < h->ns; ++s) {
        std::vector<std::pair<int, int>> tr;
        for (int r = 0; r < h->nr; ++r) {
            int z = h->h_rec_zx[2 * ((size_t)s * h->nr + r)], x = h->h_rec_zx[2 * ((size_t)s * h->nr + r) + 1];
            tr.push_back({(z / t.TZ) * t.ntx + (x / t.TX), r});
        }
        std::stable_sort(tr.begin(), tr.end(), [](auto &a, auto &b) { return a.first < b.first; });
        size_t i = 0;
        for (int tile = 0; tile <= t.ntiles; ++tile) {
            while (i < tr.size() && tr[i].first < tile) ++i;
            off[(size_t)s * (t.ntiles + 1) + tile] = (int)i;
        }
        for (size_t q = 0; q < tr.size(); ++q) {
            int r = tr[q].second;
            int z = h->h_rec_zx[2 * ((size_t)s * h->nr + r)], x = h->h_rec_zx[2 * ((size_t)s * h->nr + r) + 1];
            rec[(size_t)s * h->nr + q] = r;
            pos[(size_t)s * h->nr + q] = (z + hvi::GH) * h->P + (x + hvi::GH);
        }
    }
}

}  // namespace

extern "C" int hv_hessian_apply_static(const hv_grid *g, const hv_acq *a, const float *m, const float *v, int k,
                                       float *Hv, int ckpt, void *stream)
{
    HV_RT(validate_create(g, a));
    if (!m || !v || !Hv) return hvi::fail(HV_EINVAL, "null model, vector or output");
    cudaStream_t st = (cudaStream_t)stream;
    // The tables below are copied from host vectors that die with this call;
    // a capture would record copies from freed host memory.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HV_CK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return hvi::fail(HV_EINVAL, "hv_hessian_apply_static: the stream is being captured; call it outside capture");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    void *base = nullptr;
    HV_RT(static_scratch_base(dev, &base));

    // A host-only handle whose device arrays point into the scratch array.
    std::unique_ptr<hv_handle> hp(new hv_handle());
    hv_handle *h = hp.get();
    h->device = dev;
    h->nz = g->nz; h->nx = g->nx; h->nb = g->nb; h->h = g->h;
    h->NZ = g->nz + 2 * g->nb;
    h->NX = g->nx + 2 * g->nb;
    h->P = ((h->NX + 2 * hvi::GH) + 31) / 32 * 32;
    h->rows = h->NZ + 2 * hvi::GH;
    h->fsize = ((size_t)h->rows * h->P + 63) / 64 * 64;
    h->ns = a->ns; h->nr = a->nr; h->nt = a->nt;
    h->dt = a->dt; h->f0 = a->f0; h->t0 = a->t0; h->vmax = a->vmax; h->R = a->R; h->sigma = a->sigma;
    h->h_src_zx.resize(2 * (size_t)h->ns);
    h->h_rec_zx.resize(2 * (size_t)h->ns * h->nr);
    for (int s = 0; s < h->ns; ++s) {
        h->h_src_zx[2 * s] = a->src_iz[s] + h->nb;
        h->h_src_zx[2 * s + 1] = a->src_ix[s] + h->nb;
    }
    for (size_t i = 0; i < (size_t)h->ns * h->nr; ++i) {
        h->h_rec_zx[2 * i] = a->rec_iz[i] + h->nb;
        h->h_rec_zx[2 * i + 1] = a->rec_ix[i] + h->nb;
    }
    // This path always runs tile configuration 0 for all three kernel kinds
    // (the temporary handle's default), so one set of receiver tables serves.
    const hvi::Tiling tf = hvk::tiling(h, 0);
    std::vector<int> off_f, rec_f, pos_f;
    static_rectile_tables(h, tf, off_f, rec_f, pos_f);

    // Carve the array: the status word (always at offset 0, read by
    // hv_static_status), the tables, then the workspace of hv_hessian_apply.
    size_t o = 0;
    auto carve = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return (char *)base + at;
    };
    h->status = (int *)carve(sizeof(int));
    h->wavelet = (float *)carve(sizeof(float) * h->nt);
    h->az = (float *)carve(sizeof(float) * h->NZ);
    h->ax = (float *)carve(sizeof(float) * h->NX);
    h->src_zx = (int *)carve(sizeof(int) * h->h_src_zx.size());
    h->rec_zx = (int *)carve(sizeof(int) * h->h_rec_zx.size());
    hvi::RecTiles rf;
    rf.TX = tf.TX; rf.TZ = tf.TZ; rf.ntiles = tf.ntiles;
    rf.off = (int *)carve(sizeof(int) * off_f.size());
    rf.rec = (int *)carve(sizeof(int) * rec_f.size());
    rf.pos = (int *)carve(sizeof(int) * pos_f.size());
    const size_t tables = o;
    Layout L;
    HV_RT(make_layout(h, HV_OP_HV, k, ckpt, L));
    if (o > HV_STATIC_SCRATCH_BYTES || L.total > HV_STATIC_SCRATCH_BYTES - o)
        return hvi::fail(HV_ENOMEM,
                         "hv_hessian_apply_static: this problem needs %zu bytes of scratch (%zu of tables, %zu of "
                         "fields); the static array holds %zu; use hv_hessian_apply with a workspace",
                         tables + L.total, tables, L.total, (size_t)HV_STATIC_SCRATCH_BYTES);
    void *ws = (char *)base + tables;

    // Tables (rewritten on every call: the array keeps the previous call's contents).
    HV_CK(cudaMemcpyAsync(h->src_zx, h->h_src_zx.data(), sizeof(int) * h->h_src_zx.size(), cudaMemcpyHostToDevice, st));
    HV_CK(cudaMemcpyAsync(h->rec_zx, h->h_rec_zx.data(), sizeof(int) * h->h_rec_zx.size(), cudaMemcpyHostToDevice, st));
    HV_CK(cudaMemcpyAsync(rf.off, off_f.data(), sizeof(int) * off_f.size(), cudaMemcpyHostToDevice, st));
    HV_CK(cudaMemcpyAsync(rf.rec, rec_f.data(), sizeof(int) * rec_f.size(), cudaMemcpyHostToDevice, st));
    HV_CK(cudaMemcpyAsync(rf.pos, pos_f.data(), sizeof(int) * pos_f.size(), cudaMemcpyHostToDevice, st));
    // The status word is not cleared here: it collects timeouts of every call
    // until hv_static_status reads and clears it (the array starts zeroed).
    h->rectiles[(long long)rf.TX * 65536 + rf.TZ] = rf;
    HV_RT(hvk::launch_setup(h, st));
    HV_RT(hvk::prepare_kernels(h));
    int rc = run_adjoint(h, 2, m, v, k, Hv, nullptr, nullptr, ckpt, ws, HV_STATIC_SCRATCH_BYTES - tables, st);
    // The pageable-host copies above are staged before cudaMemcpyAsync returns, so the
    // host tables may go out of scope now; the device pointers are not freed (they
    // belong to the static array).
    h->rectiles.clear();
    return rc;
}

extern "C" int hv_static_status(int *device_status)
{
    if (!device_status) return hvi::fail(HV_EINVAL, "null output");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    void *base = nullptr;
    HV_RT(static_scratch_base(dev, &base));
    HV_CK(cudaDeviceSynchronize());
    HV_CK(cudaMemcpy(device_status, base, sizeof(int), cudaMemcpyDeviceToHost));
    HV_CK(cudaMemset(base, 0, sizeof(int)));
    return HV_OK;
}

extern "C" int hv_status(hv_handle *h, int *device_status)
{
    if (!h || !device_status) return hvi::fail(HV_EINVAL, "null handle or output");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != h->device) return hvi::fail(HV_EINVAL, "current device %d is not the handle's device %d", dev, h->device);
    HV_CK(cudaDeviceSynchronize());
    HV_CK(cudaMemcpy(device_status, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    HV_CK(cudaMemset(h->status, 0, sizeof(int)));
    return HV_OK;
}

extern "C" int hv_set_image_precision(hv_handle *h, int mode)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    if (mode != HV_IMAGE_PAIRS && mode != HV_IMAGE_FP64) return hvi::fail(HV_EINVAL, "image precision mode %d", mode);
    h->img_f64 = mode == HV_IMAGE_FP64;
    return HV_OK;
}

extern "C" int hv_set_wait_limit(hv_handle *h, double seconds)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    if (!(seconds >= 1e-4 && seconds <= 60.0))
        return hvi::fail(HV_EINVAL, "wait limit %g s; need 1e-4 <= limit <= 60", seconds);
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return HV_OK;
}

extern "C" int hv_inject_wait_timeout(hv_handle *h)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    h->inject_wait = true;
    return HV_OK;
}

extern "C" int hv_tile_menu(int index, int *TX, int *TZ)
{
    if (index < 0 || index >= hvk::tile_menu_size()) return hvi::fail(HV_EINVAL, "tile configuration %d not in the menu", index);
    hv_handle dummy;
    dummy.NX = dummy.NZ = 1;
    hvi::Tiling t = hvk::tiling(&dummy, index);
    if (TX) *TX = t.TX;
    if (TZ) *TZ = t.TZ;
    return HV_OK;
}

extern "C" int hv_tile_menu_size(void) { return hvk::tile_menu_size(); }

extern "C" int hv_tile_menu_info(int index, int *info)
{
    if (index < 0 || index >= hvk::tile_menu_size()) return hvi::fail(HV_EINVAL, "tile configuration %d not in the menu", index);
    if (!info) return hvi::fail(HV_EINVAL, "null output");
    hvk::menu_info(index, info);
    return HV_OK;
}

extern "C" int hv_set_tiles(hv_handle *h, const int *cfg)
{
    if (!h || !cfg) return hvi::fail(HV_EINVAL, "null handle or configuration");
    for (int i = 0; i < 3; ++i)
        if (cfg[i] < 0 || cfg[i] >= hvk::tile_menu_size())
            return hvi::fail(HV_EINVAL, "tile configuration %d not in the menu", cfg[i]);
    for (int i = 0; i < 3; ++i) h->cfg[i] = cfg[i];
    return HV_OK;
}

extern "C" int hv_get_tiles(const hv_handle *h, int *cfg)
{
    if (!h || !cfg) return hvi::fail(HV_EINVAL, "null handle or output");
    for (int i = 0; i < 3; ++i) cfg[i] = h->cfg[i];
    return HV_OK;
}

extern "C" int hv_set_graphs(hv_handle *h, int enable)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    h->graphs_on = enable != 0;
    return HV_OK;
}

extern "C" int hv_set_resident(hv_handle *h, int enable)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    h->resident = enable != 0;
    return HV_OK;
}

extern "C" int hv_resident_fits(const hv_handle *h)
{
    return h && hvk::resident_fits(h) ? 1 : 0;
}

extern "C" int hv_set_step_fusion(hv_handle *h, int enable)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    h->fuse_steps = enable != 0;
    return HV_OK;
}

extern "C" int hv_set_launch_mode(hv_handle *h, int mode)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    if (mode < HV_LAUNCH_PLAIN || mode > HV_LAUNCH_DATAFLOW) return hvi::fail(HV_EINVAL, "launch mode %d", mode);
    h->launch_mode = mode;
    return HV_OK;
}

// Times every tile configuration of the three stencil kernels on this
// handle's grid with k vectors (on zeroed fields: the kernels have no
// data-dependent work) and keeps the fastest per kernel kind.
extern "C" int hv_autotune(hv_handle *h, int k, void *ws, size_t ws_bytes, void *stream, int *chosen, float *ms)
{
    hvi::Range nvtx_range("hv_autotune");
    Layout L;
    HV_RT(check_common(h, ws, ws_bytes, HV_OP_HV, k, 1, L));
    cudaStream_t st = (cudaStream_t)stream;
    HV_CK(cudaMemsetAsync(ws, 0, L.total, st));
    Exec E;
    HV_RT(E.init(h, st, L, ws, k));
    if (E.pool.size() < 4) return hvi::fail(HV_EINVAL, "internal: autotune needs four forward batches");
    const float *dd = reinterpret_cast<const float *>((char *)ws + L.dd);
    const int nmenu = hvk::tile_menu_size();
    cudaEvent_t e0, e1;
    HV_CK(cudaEventCreate(&e0));
    HV_CK(cudaEventCreate(&e1));
    constexpr int kReps = 6;
    const bool fused = h->fuse_steps && h->launch_mode != HV_LAUNCH_DATAFLOW && h->nt >= 2;
    std::vector<float> tm((size_t)nmenu * 3, 1e30f);
    float best[3] = {1e30f, 1e30f, 1e30f};
    int arg[3] = {0, 0, 0};
    int rc = HV_OK;
    for (int c = 0; c < nmenu && rc == HV_OK; ++c) {
        const hvi::RecTiles &rt = rectiles_for(h, hvk::tiling(h, c));
        for (int kind = 0; kind < 3 && rc == HV_OK; ++kind) {
            // The fields rotate through three pool batches (and the two vector
            // batches) as in a sweep, so each launch reads what the one before it
            // wrote, with the cache behaviour of the real sequence.
            for (int rep = 0; rep <= kReps && rc == HV_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, st);
                float *f0 = E.pool[rep % 3], *f1 = E.pool[(rep + 1) % 3], *f2 = E.pool[(rep + 2) % 3];
                float *d0 = E.Dbuf(rep % 2), *d1 = E.Dbuf((rep + 1) % 2);
                if (kind == 2) {
                    hvk::AdjLaunch a{};
                    a.u = f1; a.lam1 = d1; a.lam_io = d0; a.C = E.C; a.r = dd;
                    a.r_per_vector = 1; a.rscale = 1.0f; a.img = E.img; a.n = 0; a.k = k; a.G = L.G;
                    rc = hvk::launch_adj(h, c, rt, E.maps, a, st);
                } else if (kind == 1 && fused) {
                    hvk::Fwd2Launch a{};      // recomputation runs fused double steps: time one, halve it
                    const int q = 2 * rep;   // two levels per launch, over four batches
                    a.u_prev = E.pool[q % 4]; a.u_cur = E.pool[(q + 1) % 4];
                    a.u_next1 = E.pool[(q + 2) % 4]; a.u_next2 = E.pool[(q + 3) % 4]; a.C = E.C;
                    a.n = 0;
                    rc = hvk::launch_fwd2(h, c, rt, E.maps, a, st);
                } else {
                    hvk::FwdLaunch a{};
                    a.u_cur = f1; a.u_prev = f0; a.u_next = f2; a.C = E.C; a.n = 0;
                    if (kind == 0) {
                        a.b = E.b; a.k = k; a.du_cur = d1; a.du_io = d0;
                    }
                    rc = hvk::launch_fwd(h, c, rt, E.maps, a, st);
                }
            }
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess && rc == HV_OK) rc = hvi::fail(HV_ECUDA, "autotune: %s", cudaGetErrorString(e));
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            t /= kReps;
            if (kind == 1 && fused) t *= 0.5f;   // per step
            if (ms) ms[c * 3 + kind] = t;
            tm[c * 3 + kind] = t;
            if (t < best[kind]) {
                best[kind] = t;
                arg[kind] = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != HV_OK) return rc;
    if (h->launch_mode == HV_LAUNCH_DATAFLOW) {
        // Dataflow ordering needs one tile shape for the three kinds: take the
        // shape with the least weighted time (a binomially checkpointed H v
        // runs about 1.8 recompute steps per forward+Born and adjoint step),
        // then the fastest entry of that shape per kind.
        const float wgt[3] = {1.0f, 1.8f, 1.0f};
        float best_sum = 1e30f;
        for (int s = 0; s < nmenu; ++s) {
            const hvi::Tiling ts = hvk::tiling(h, s);
            int pick[3] = {s, s, s};
            float sum = 0.f;
            for (int kind = 0; kind < 3; ++kind) {
                float bt = 1e30f;
                for (int c = 0; c < nmenu; ++c) {
                    const hvi::Tiling tc = hvk::tiling(h, c);
                    if (tc.TX == ts.TX && tc.TZ == ts.TZ && tm[c * 3 + kind] < bt) {
                        bt = tm[c * 3 + kind];
                        pick[kind] = c;
                    }
                }
                sum += wgt[kind] * bt;
            }
            if (sum < best_sum) {
                best_sum = sum;
                for (int i = 0; i < 3; ++i) arg[i] = pick[i];
            }
        }
    }
    for (int i = 0; i < 3; ++i) h->cfg[i] = arg[i];
    if (chosen)
        for (int i = 0; i < 3; ++i) chosen[i] = arg[i];
    return HV_OK;
}

// ---------------------------------------------------------------- approximations
// Point-spread-function approximation (section 3.2; PsiDO row form, section 3.5).

namespace {

constexpr int kMaxPsfBatchesPerAxis = 8;
constexpr int kMaxPsfRadius = 40;

int psf_batches_per_axis(int n_batches)
{
    for (int B = 1; B <= kMaxPsfBatchesPerAxis; ++B)
        if (B * B == n_batches) return B;
    return 0;
}

int psf_geometry(int nz, int nx, int S, int n_batches, hvk::PsfGeo &g)
{
    if (S < 1) return hvi::fail(HV_EINVAL, "PSF lattice spacing %d; need >= 1", S);
    const int B = psf_batches_per_axis(n_batches);
    if (B == 0) return hvi::fail(HV_EINVAL, "n_batches = %d; need B * B with 1 <= B <= %d", n_batches, kMaxPsfBatchesPerAxis);
    g.nz = nz;
    g.nx = nx;
    g.S = S;
    g.B = B;
    g.R = (B * S - 1) / 2;
    g.cz0 = S / 2;
    g.cx0 = S / 2;
    if (g.cz0 >= nz || g.cx0 >= nx)
        return hvi::fail(HV_EINVAL, "first PSF sample point (%d, %d) is off the %d x %d grid", g.cz0, g.cx0, nz, nx);
    if (g.R > kMaxPsfRadius) return hvi::fail(HV_EINVAL, "PSF window radius %d exceeds %d", g.R, kMaxPsfRadius);
    g.na = (nz - 1 - g.cz0) / S + 1;
    g.nb = (nx - 1 - g.cx0) / S + 1;
    return HV_OK;
}

// Workspace of the build: impulse batches, their H v, then the H v workspace.
struct PsfLayout {
    size_t vec = 0, hv = 0, inner = 0, inner_bytes = 0, total = 0;
};

int psf_layout(hv_handle *h, int n_batches, int ckpt, PsfLayout &P)
{
    Layout L;
    HV_RT(make_layout(h, HV_OP_HV, n_batches, ckpt, L));
    const size_t vb = align256((size_t)n_batches * h->nz * h->nx * sizeof(float));
    P.vec = 0;
    P.hv = vb;
    P.inner = 2 * vb;
    P.inner_bytes = L.total;
    P.total = P.inner + L.total;
    return HV_OK;
}

}  // namespace

extern "C" int hv_approx_psf_workspace_size(hv_handle *h, int n_batches, int ckpt, size_t *bytes)
{
    if (!h || !bytes) return hvi::fail(HV_EINVAL, "null handle or output");
    if (psf_batches_per_axis(n_batches) == 0)
        return hvi::fail(HV_EINVAL, "n_batches = %d; need B * B with 1 <= B <= %d", n_batches, kMaxPsfBatchesPerAxis);
    PsfLayout P;
    HV_RT(psf_layout(h, n_batches, ckpt, P));
    *bytes = P.total;
    return HV_OK;
}

using HessFn = std::function<int(const float *, int, float *)>;
static int psf_finish(const hvk::PsfGeo &g, int device, float *vec, float *hv, const HessFn &hess, cudaStream_t st,
                      hv_approx **out);
static int pdo_finish(const hvk::LrGeo &g, int device, float *vp, float *hvp, const HessFn &hess, cudaStream_t st,
                      hv_approx **out);
static int lr_finish(int nz, int nx, double hh, int device, double delta, double gamma, int rank, const float *omega,
                     int k, float *Y, const HessFn &hess, cudaStream_t st, hv_approx **out);

// The high-pass filter around an operator during a build (sections 3.2, 3.7):
// X -> F_hp Op(F_hp X), the filter's transforms and a scratch of kmax fields
// allocated here and freed (after the stream drains) when the build returns.
namespace {
struct Filter {
    hvk::Highpass F;
    float *T = nullptr;
    cudaStream_t st = nullptr;
    bool made = false;
    int init(int nz, int nx, double hh, double rho_c, int kmax, cudaStream_t s)
    {
        st = s;
        made = true;
        HV_RT(hvk::highpass_create(F, nz, nx, hh, rho_c, kmax));
        HV_CK(cudaMalloc(&T, (size_t)kmax * nz * nx * sizeof(float)));
        return HV_OK;
    }
    HessFn wrap(const HessFn &inner)
    {
        return [this, inner](const float *X, int k, float *Z) {
            const size_t N = (size_t)F.nz * F.nx;
            for (int q0 = 0; q0 < k; q0 += F.kmax) {
                const int kb = std::min(F.kmax, k - q0);
                HV_RT(hvk::highpass_apply(F, X + q0 * N, kb, T, st));
                HV_RT(inner(T, kb, Z + q0 * N));
                HV_RT(hvk::highpass_apply(F, Z + q0 * N, kb, Z + q0 * N, st));
            }
            return HV_OK;
        };
    }
    ~Filter()
    {
        if (!made) return;
        if (st) cudaStreamSynchronize(st);
        cudaFree(T);
        hvk::highpass_destroy(F);
    }
};
}  // namespace

extern "C" int hv_set_highpass(hv_handle *h, double rho_c)
{
    if (!h) return hvi::fail(HV_EINVAL, "null handle");
    if (!(rho_c >= 0)) return hvi::fail(HV_EINVAL, "high-pass cutoff %g; need >= 0 (0: off)", rho_c);
    h->highpass = rho_c;
    return HV_OK;
}

extern "C" int hv_highpass_apply(int nz, int nx, double h, double rho_c, const float *v, int k, float *out,
                                 void *stream)
{
    hvi::Range nvtx_range("hv_highpass_apply");
    if (!v || !out || k < 1) return hvi::fail(HV_EINVAL, "null field or k < 1");
    cudaStream_t st = (cudaStream_t)stream;
    hvk::Highpass F;
    int rc = hvk::highpass_create(F, nz, nx, h, rho_c, std::min(k, 64));
    if (rc == HV_OK) rc = hvk::highpass_apply(F, v, k, out, st);
    cudaStreamSynchronize(st);
    hvk::highpass_destroy(F);
    return rc;
}

// An operator wrapped in the high-pass filter: F_hp Op F_hp.
struct hv_filtered {
    hv_operator inner{};
    hvk::Highpass F;
    float *T = nullptr;
    int max_k = 0;
    std::mutex mu;
    cudaEvent_t done = nullptr;   // the last apply's use of T and the transforms
};

namespace {
int filtered_apply(void *ctx, const float *v, int k, float *out, void *stream)
{
    hv_filtered *f = static_cast<hv_filtered *>(ctx);
    std::lock_guard<std::mutex> g(f->mu);
    cudaStream_t st = (cudaStream_t)stream;
    // applies from different streams share the scratch: order this one after the last
    HV_CK(cudaStreamWaitEvent(st, f->done, 0));
    const size_t N = (size_t)f->inner.nz * f->inner.nx;
    int rc = HV_OK;
    for (int q0 = 0; q0 < k && rc == HV_OK; q0 += f->max_k) {
        const int kb = std::min(f->max_k, k - q0);
        rc = hvk::highpass_apply(f->F, v + q0 * N, kb, f->T, st);
        if (rc == HV_OK) {
            const int r = f->inner.apply(f->inner.ctx, f->T, kb, out + q0 * N, stream);
            if (r != HV_OK) rc = hvi::fail(r, "the inner operator's apply returned %d", r);
        }
        if (rc == HV_OK) rc = hvk::highpass_apply(f->F, out + q0 * N, kb, out + q0 * N, st);
    }
    const cudaError_t e = cudaEventRecord(f->done, st);
    if (rc == HV_OK && e != cudaSuccess) rc = hvi::fail(HV_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    return rc;
}
}  // namespace

extern "C" int hv_filtered_create(const hv_operator *inner, double rho_c, int max_k, hv_filtered **out)
{
    if (out) *out = nullptr;
    if (!out || !inner || !inner->apply) return hvi::fail(HV_EINVAL, "null operator or output");
    if (max_k < 1 || max_k > 4096) return hvi::fail(HV_EINVAL, "max_k = %d; need 1..4096", max_k);
    hv_filtered *f = new hv_filtered;
    f->inner = *inner;
    f->max_k = max_k;
    int rc = hvk::highpass_create(f->F, inner->nz, inner->nx, inner->h, rho_c, max_k);
    if (rc == HV_OK && cudaMalloc(&f->T, (size_t)max_k * inner->nz * inner->nx * sizeof(float)) != cudaSuccess)
        rc = hvi::fail(HV_ECUDA, "high-pass scratch: out of device memory");
    if (rc == HV_OK && cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming) != cudaSuccess)
        rc = hvi::fail(HV_ECUDA, "cudaEventCreate failed");
    if (rc != HV_OK) {
        hv_filtered_destroy(f);
        return rc;
    }
    *out = f;
    return HV_OK;
}

extern "C" int hv_filtered_operator(hv_filtered *f, hv_operator *op)
{
    if (!f || !op) return hvi::fail(HV_EINVAL, "null filtered operator or output");
    op->nz = f->inner.nz;
    op->nx = f->inner.nx;
    op->h = f->inner.h;
    op->apply = filtered_apply;
    op->ctx = f;
    return HV_OK;
}

extern "C" int hv_filtered_destroy(hv_filtered *f)
{
    if (!f) return HV_OK;
    cudaDeviceSynchronize();
    cudaFree(f->T);
    hvk::highpass_destroy(f->F);
    if (f->done) cudaEventDestroy(f->done);
    delete f;
    return HV_OK;
}

extern "C" int hv_approx_build_psf(hv_handle *h, const float *m, int spacing_cells, int n_batches, int ckpt,
                                   hv_approx **out, void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_psf");
    if (out) *out = nullptr;
    if (!h || !out || !m) return hvi::fail(HV_EINVAL, "null handle, model or output");
    hvk::PsfGeo g;
    HV_RT(psf_geometry(h->nz, h->nx, spacing_cells, n_batches, g));
    PsfLayout P;
    HV_RT(psf_layout(h, n_batches, ckpt, P));
    if (!ws) return hvi::fail(HV_EINVAL, "null workspace");
    if (((uintptr_t)ws & 255u) != 0) return hvi::fail(HV_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < P.total) return hvi::fail(HV_ENOMEM, "workspace of %zu bytes; the PSF build needs %zu", ws_bytes, P.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    float *vec = reinterpret_cast<float *>(w + P.vec);
    float *hv = reinterpret_cast<float *>(w + P.hv);
    HessFn hess = [&](const float *X, int k, float *Z) {
        return run_adjoint(h, 2, m, X, k, Z, nullptr, nullptr, ckpt, w + P.inner, P.inner_bytes, st);
    };
    if (h->highpass > 0) {
        Filter F;
        HV_RT(F.init(h->nz, h->nx, h->h, h->highpass, n_batches, st));
        return psf_finish(g, h->device, vec, hv, F.wrap(hess), st, out);
    }
    return psf_finish(g, h->device, vec, hv, hess, st, out);
}

// The PSF build after the geometry: impulse batches, one batched operator
// application, window extraction.
static int psf_finish(const hvk::PsfGeo &g, int device, float *vec, float *hv, const HessFn &hess, cudaStream_t st,
                      hv_approx **out)
{
    const int n_batches = g.B * g.B;
    HV_CK(cudaMemsetAsync(vec, 0, (size_t)n_batches * g.nz * g.nx * sizeof(float), st));
    HV_RT(hvk::launch_psf_impulses(g, vec, st));
    HV_RT(hess(vec, n_batches, hv));
    hv_approx *a = new hv_approx;
    a->kind = 0;
    a->device = device;
    a->g = g;
    const size_t W = 2 * (size_t)g.R + 1;
    cudaError_t e = cudaMalloc(&a->psf, (size_t)g.na * g.nb * W * W * sizeof(float));
    if (e != cudaSuccess) {
        delete a;
        return hvi::fail(HV_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    int rc = hvk::launch_psf_extract(g, hv, a->psf, st);
    if (rc != HV_OK) {
        cudaFree(a->psf);
        delete a;
        return rc;
    }
    *out = a;
    return HV_OK;
}

// Pseudo-differential operator probing (section 3.4, appendix A).
namespace {
struct PdoLayout {
    size_t vp = 0, hvp = 0, inner = 0, inner_bytes = 0, total = 0;
};
int pdo_layout(hv_handle *h, int ckpt, PdoLayout &P)
{
    Layout L;
    HV_RT(make_layout(h, HV_OP_HV, 1, ckpt, L));
    const size_t fb = align256((size_t)h->nz * h->nx * sizeof(float));
    P.vp = 0;
    P.hvp = fb;
    P.inner = 2 * fb;
    P.inner_bytes = L.total;
    P.total = P.inner + L.total;
    return HV_OK;
}
}  // namespace

extern "C" int hv_approx_pdo_workspace_size(hv_handle *h, int ckpt, size_t *bytes)
{
    if (!h || !bytes) return hvi::fail(HV_EINVAL, "null handle or output");
    PdoLayout P;
    HV_RT(pdo_layout(h, ckpt, P));
    *bytes = P.total;
    return HV_OK;
}

extern "C" int hv_approx_build_pdo(hv_handle *h, const float *m, double rho0, int r, int ckpt, hv_approx **out,
                                   void *ws, size_t ws_bytes, void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_pdo");
    if (out) *out = nullptr;
    if (!h || !out || !m) return hvi::fail(HV_EINVAL, "null handle, model or output");
    hvk::LrGeo g;
    HV_RT(hvk::lr_samples(h->nz, h->nx, h->h, rho0, r, g));
    PdoLayout P;
    HV_RT(pdo_layout(h, ckpt, P));
    if (!ws) return hvi::fail(HV_EINVAL, "null workspace");
    if (((uintptr_t)ws & 255u) != 0) return hvi::fail(HV_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < P.total) return hvi::fail(HV_ENOMEM, "workspace of %zu bytes; the PDO build needs %zu", ws_bytes, P.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    float *vp = reinterpret_cast<float *>(w + P.vp);
    float *hvp = reinterpret_cast<float *>(w + P.hvp);
    HessFn hess = [&](const float *X, int k, float *Z) {
        return run_adjoint(h, 2, m, X, k, Z, nullptr, nullptr, ckpt, w + P.inner, P.inner_bytes, st);
    };
    if (h->highpass > 0) {
        Filter F;
        HV_RT(F.init(h->nz, h->nx, h->h, h->highpass, 1, st));
        return pdo_finish(g, h->device, vp, hvp, F.wrap(hess), st, out);
    }
    return pdo_finish(g, h->device, vp, hvp, hess, st, out);
}

// The PDO build after the sample geometry: probe, one operator application,
// spectral separation and weights.
static int pdo_finish(const hvk::LrGeo &g, int device, float *vp, float *hvp, const HessFn &hess, cudaStream_t st,
                      hv_approx **out)
{
    HV_RT(hvk::launch_pdo_probe(g, vp, st));
    HV_RT(hess(vp, 1, hvp));
    hv_approx *a = new hv_approx;
    a->kind = 1;
    a->device = device;
    int rc = hvk::lr_create(a->lr, g);
    if (rc == HV_OK) rc = hvk::pdo_columns(a->lr, hvp, st);
    if (rc != HV_OK) {
        hvk::lr_destroy(a->lr);
        delete a;
        return rc;
    }
    *out = a;
    return HV_OK;
}

// Low-rank approximation (section 3.1) with the Matern prior (section 2.1).
extern "C" int hv_approx_lr_workspace_size(hv_handle *h, int k, int ckpt, size_t *bytes)
{
    if (!h || !bytes) return hvi::fail(HV_EINVAL, "null handle or output");
    Layout L;
    HV_RT(make_layout(h, HV_OP_HV, k, ckpt, L));
    *bytes = align256((size_t)k * h->nz * h->nx * sizeof(float)) + L.total;
    return HV_OK;
}

extern "C" int hv_approx_build_lr(hv_handle *h, const float *m, double delta, double gamma, int rank,
                                  const float *omega, int k, int ckpt, hv_approx **out, void *ws, size_t ws_bytes,
                                  void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_lr");
    if (out) *out = nullptr;
    if (!h || !m || !omega || !out) return hvi::fail(HV_EINVAL, "null handle, model, test vectors or output");
    if (rank < 1 || k < rank || k > 256) return hvi::fail(HV_EINVAL, "rank %d with %d test vectors; need 1 <= rank <= k <= 256", rank, k);
    Layout L;
    HV_RT(make_layout(h, HV_OP_HV, k, ckpt, L));
    const size_t N = (size_t)h->nz * h->nx, yb = align256((size_t)k * N * sizeof(float));
    if (!ws) return hvi::fail(HV_EINVAL, "null workspace");
    if (((uintptr_t)ws & 255u) != 0) return hvi::fail(HV_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < yb + L.total) return hvi::fail(HV_ENOMEM, "workspace of %zu bytes; the LR build needs %zu", ws_bytes, yb + L.total);
    cudaStream_t st = (cudaStream_t)stream;
    float *Y = reinterpret_cast<float *>(ws);
    char *inner = (char *)ws + yb;
    return lr_finish(h->nz, h->nx, h->h, h->device, delta, gamma, rank, omega, k, Y,
                     [&](const float *X, int kk, float *Z) {
                         return run_adjoint(h, 2, m, X, kk, Z, nullptr, nullptr, ckpt, inner, L.total, st);
                     },
                     st, out);
}

// The LR build after the argument checks: Y = H_d omega, then the double pass.
static int lr_finish(int nz, int nx, double hh, int device, double delta, double gamma, int rank, const float *omega,
                     int k, float *Y, const HessFn &hess, cudaStream_t st, hv_approx **out)
{
    hv_approx *a = new hv_approx;
    a->kind = 3;
    a->device = device;
    a->nz = nz;
    a->nx = nx;
    int rc = hvk::prior_create(a->low.prior, nz, nx, hh, delta, gamma);
    if (rc == HV_OK) rc = hess(omega, k, Y);
    if (rc == HV_OK) rc = hvk::build_lowrank(a->low, Y, k, rank, (size_t)nz * nx, hess, st);
    if (rc != HV_OK) {
        hvk::lowrank_destroy(a->low);
        delete a;
        return rc;
    }
    *out = a;
    return HV_OK;
}

namespace {

// Device scratch of the *_op builds, freed after the stream has drained.
struct OpScratch {
    std::vector<void *> p;
    cudaStream_t st = nullptr;
    int get(float **out, size_t n)
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(out), n * sizeof(float));
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "build scratch: %s", cudaGetErrorString(e));
        p.push_back(*out);
        return HV_OK;
    }
    ~OpScratch()
    {
        if (st) cudaStreamSynchronize(st);
        for (void *q : p) cudaFree(q);
    }
};

int check_operator(const hv_operator *op)
{
    if (!op || !op->apply) return hvi::fail(HV_EINVAL, "null operator or apply function");
    if (op->nz < 1 || op->nx < 1 || !(op->h > 0)) return hvi::fail(HV_EINVAL, "operator grid %d x %d, h = %g", op->nz, op->nx, op->h);
    return HV_OK;
}

HessFn op_fn(const hv_operator *op, cudaStream_t st)
{
    return [op, st](const float *X, int k, float *Z) {
        const int rc = op->apply(op->ctx, X, k, Z, (void *)st);
        return rc == HV_OK ? HV_OK : hvi::fail(rc, "the operator's apply returned %d", rc);
    };
}

}  // namespace

extern "C" int hv_approx_build_psf_op(const hv_operator *op, int spacing_cells, int n_batches, hv_approx **out,
                                      void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_psf_op");
    if (out) *out = nullptr;
    if (!out) return hvi::fail(HV_EINVAL, "null output");
    HV_RT(check_operator(op));
    hvk::PsfGeo g;
    HV_RT(psf_geometry(op->nz, op->nx, spacing_cells, n_batches, g));
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    OpScratch sc;
    sc.st = st;
    float *vec = nullptr, *hv = nullptr;
    const size_t n = (size_t)n_batches * op->nz * op->nx;
    HV_RT(sc.get(&vec, n));
    HV_RT(sc.get(&hv, n));
    return psf_finish(g, dev, vec, hv, op_fn(op, st), st, out);
}

extern "C" int hv_approx_build_pdo_op(const hv_operator *op, double rho0, int r, hv_approx **out, void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_pdo_op");
    if (out) *out = nullptr;
    if (!out) return hvi::fail(HV_EINVAL, "null output");
    HV_RT(check_operator(op));
    hvk::LrGeo g;
    HV_RT(hvk::lr_samples(op->nz, op->nx, op->h, rho0, r, g));
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    OpScratch sc;
    sc.st = st;
    float *vp = nullptr, *hvp = nullptr;
    HV_RT(sc.get(&vp, (size_t)op->nz * op->nx));
    HV_RT(sc.get(&hvp, (size_t)op->nz * op->nx));
    return pdo_finish(g, dev, vp, hvp, op_fn(op, st), st, out);
}

extern "C" int hv_approx_build_lr_op(const hv_operator *op, double delta, double gamma, int rank, const float *omega,
                                     int k, hv_approx **out, void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_lr_op");
    if (out) *out = nullptr;
    if (!out || !omega) return hvi::fail(HV_EINVAL, "null test vectors or output");
    HV_RT(check_operator(op));
    if (rank < 1 || k < rank || k > 256) return hvi::fail(HV_EINVAL, "rank %d with %d test vectors; need 1 <= rank <= k <= 256", rank, k);
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    OpScratch sc;
    sc.st = st;
    float *Y = nullptr;
    HV_RT(sc.get(&Y, (size_t)k * op->nz * op->nx));
    return lr_finish(op->nz, op->nx, op->h, dev, delta, gamma, rank, omega, k, Y, op_fn(op, st), st, out);
}

extern "C" int hv_approx_lr_eigs(const hv_approx *a, double *lambda, float *V, void *stream)
{
    if (!a || a->kind != 3) return hvi::fail(HV_EINVAL, "not a low-rank approximation");
    if (lambda)
        for (int i = 0; i < a->low.r; ++i) lambda[i] = a->low.lam[i];
    if (V)
        HV_CK(cudaMemcpyAsync(V, a->low.V, (size_t)a->low.r * a->low.N * sizeof(float), cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
    return HV_OK;
}

extern "C" int hv_prior_apply(int nz, int nx, double h, double delta, double gamma, const float *v, int k, float *out,
                              int op, void *stream)
{
    hvi::Range nvtx_range("hv_prior_apply");
    if (!v || !out || k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "null field or k outside [1, 65535]");
    if (op < 0 || op > 3) return hvi::fail(HV_EINVAL, "prior operation %d", op);
    hvk::Prior P;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = hvk::prior_create(P, nz, nx, h, delta, gamma);
    if (rc == HV_OK) {
        if (op == 0) rc = hvk::prior_A(P, v, out, k, st);
        else if (op == 1) rc = hvk::prior_Ainv(P, v, out, k, st);
        else if (op == 2) rc = hvk::prior_R(P, v, out, k, st);
        else rc = hvk::prior_Rinv(P, v, out, k, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);   // the tables are freed below
    if (rc == HV_OK && e != cudaSuccess) rc = hvi::fail(HV_ECUDA, "prior apply: %s", cudaGetErrorString(e));
    hvk::prior_destroy(P);
    return rc;
}

static int build_psfplus_common(const hv_approx *psf, const hv_approx *pdo, double tol, bool spd, hv_approx **out,
                                void *stream)
{
    if (out) *out = nullptr;
    if (!psf || !pdo || !out) return hvi::fail(HV_EINVAL, "null approximation or output");
    if (psf->kind != 0 || pdo->kind != 1) return hvi::fail(HV_EINVAL, "PSF+ needs a PSF and a PDO approximation");
    if (psf->device != pdo->device) return hvi::fail(HV_EINVAL, "the PSF and PDO approximations are on different devices");
    if (psf->g.nz != pdo->lr.g.nz || psf->g.nx != pdo->lr.g.nx)
        return hvi::fail(HV_EINVAL, "the PSF and PDO approximations are on different grids");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != psf->device) return hvi::fail(HV_EINVAL, "current device %d is not the approximations' device", dev);
    hv_approx *a = new hv_approx;
    a->kind = 2;
    a->device = psf->device;
    a->g = psf->g;
    int rc = hvk::build_psfplus(psf->g, psf->psf, pdo->lr, tol, spd, a->lr, (cudaStream_t)stream);
    if (rc != HV_OK) {
        hvk::lr_destroy(a->lr);
        delete a;
        return rc;
    }
    *out = a;
    return HV_OK;
}

extern "C" int hv_approx_build_psfplus(const hv_approx *psf, const hv_approx *pdo, double tol, hv_approx **out,
                                       void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_psfplus");
    return build_psfplus_common(psf, pdo, tol, false, out, stream);
}

extern "C" int hv_approx_build_psfplus_sqrt(const hv_approx *psf, const hv_approx *pdo, double tol, hv_approx **out,
                                            void *stream)
{
    hvi::Range nvtx_range("hv_approx_build_psfplus_sqrt");
    return build_psfplus_common(psf, pdo, tol, true, out, stream);
}

extern "C" int hv_approx_sqrt_pdo(const hv_approx *pdo, hv_approx **out, void *stream)
{
    hvi::Range nvtx_range("hv_approx_sqrt_pdo");
    if (out) *out = nullptr;
    if (!pdo || !out) return hvi::fail(HV_EINVAL, "null approximation or output");
    if (pdo->kind != 1 || pdo->lr.spd) return hvi::fail(HV_EINVAL, "the square root is taken of a PDO approximation of H_d");
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != pdo->device) return hvi::fail(HV_EINVAL, "current device %d is not the approximation's device", dev);
    hv_approx *a = new hv_approx;
    a->kind = 1;
    a->device = pdo->device;
    int rc = hvk::pdo_sqrt(pdo->lr, a->lr, (cudaStream_t)stream);
    if (rc != HV_OK) {
        hvk::lr_destroy(a->lr);
        delete a;
        return rc;
    }
    *out = a;
    return HV_OK;
}

extern "C" int hv_approx_pdo_symbol(const hv_approx *a, float *cols, float *weights, void *stream)
{
    if (!a || (a->kind != 1 && a->kind != 2)) return hvi::fail(HV_EINVAL, "not a low-rank-symbol approximation");
    if (!cols && !weights) return hvi::fail(HV_EINVAL, "null outputs");
    const size_t n = (size_t)a->lr.g.r * a->lr.g.nz * a->lr.g.nx;
    cudaStream_t st = (cudaStream_t)stream;
    HV_CK(cudaStreamWaitEvent(st, a->lr.done, 0));
    if (cols) HV_CK(cudaMemcpyAsync(cols, a->lr.a, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (weights) HV_CK(cudaMemcpyAsync(weights, a->lr.b, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    return HV_OK;
}

extern "C" int hv_approx_apply(const hv_approx *a, const float *v, int k, float *out, int mode, void *stream)
{
    hvi::Range nvtx_range("hv_approx_apply");
    if (!a) return hvi::fail(HV_EINVAL, "null approximation");
    if (mode < HV_APPROX_H || mode > HV_APPROX_SQRT_T) return hvi::fail(HV_EINVAL, "unknown apply mode %d", mode);
    const bool spd = (a->kind == 1 || a->kind == 2) && a->lr.spd;
    const bool ok = mode == HV_APPROX_H || (a->kind == 3 && mode == HV_APPROX_INVSQRT) ||
                    (spd && (mode == HV_APPROX_SQRT || mode == HV_APPROX_SQRT_T));
    if (!ok) return hvi::fail(HV_ENOTSUP, "apply mode %d is not provided for this approximation", mode);
    if (!v || !out) return hvi::fail(HV_EINVAL, "null vector or output");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "k = %d vectors; need 1 <= k <= 65535", k);
    int dev = -1;
    HV_CK(cudaGetDevice(&dev));
    if (dev != a->device) return hvi::fail(HV_EINVAL, "current device %d is not the approximation's device %d", dev, a->device);
    if (a->kind == 3)
        return hvk::lowrank_apply(const_cast<hvk::LowRank &>(a->low), v, k, out, mode == HV_APPROX_H ? 0 : 2,
                                  (cudaStream_t)stream);
    if (a->kind != 0) {
        const int op = mode == HV_APPROX_SQRT ? hvk::kLrForward
                       : mode == HV_APPROX_SQRT_T ? hvk::kLrTranspose
                       : spd ? hvk::kLrGram : hvk::kLrForward;
        return hvk::lr_apply(const_cast<hvk::LrSym &>(a->lr), v, k, out, (cudaStream_t)stream, op);
    }
    return hvk::launch_psf_apply(a->g, a->psf, v, k, out, (cudaStream_t)stream);
}

int hvi::approx_device(const hv_approx *a) { return a ? a->device : -1; }

extern "C" int hv_approx_info(const hv_approx *a, int *info)
{
    if (!a || !info) return hvi::fail(HV_EINVAL, "null approximation or output");
    if (a->kind == 3) {
        const int vals[11] = {3, a->low.r, 0, 0, 0, 0, 0, 0, 0, a->nz, a->nx};
        for (int i = 0; i < 11; ++i) info[i] = vals[i];
        return HV_OK;
    }
    if (a->kind != 0) {
        const hvk::LrGeo &l = a->lr.g;
        const int vals[11] = {a->kind, l.r, a->lr.spd ? 1 : 0, 0, 0, 0, 0, 0, 0, l.nz, l.nx};
        for (int i = 0; i < 11; ++i) info[i] = vals[i];
        return HV_OK;
    }
    const hvk::PsfGeo &g = a->g;
    const int vals[11] = {a->kind, g.na * g.nb, g.R, g.na, g.nb, g.S, g.B, g.cz0, g.cx0, g.nz, g.nx};
    for (int i = 0; i < 11; ++i) info[i] = vals[i];
    return HV_OK;
}

extern "C" int hv_approx_psfs(const hv_approx *a, float *psf, void *stream)
{
    if (!a || !psf) return hvi::fail(HV_EINVAL, "null approximation or output");
    if (a->kind != 0) return hvi::fail(HV_EINVAL, "not a PSF approximation");
    const size_t W = 2 * (size_t)a->g.R + 1;
    HV_CK(cudaMemcpyAsync(psf, a->psf, (size_t)a->g.na * a->g.nb * W * W * sizeof(float), cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream));
    return HV_OK;
}

extern "C" int hv_approx_destroy(hv_approx *a)
{
    if (!a) return HV_OK;
    if (a->kind == 3) {
        cudaDeviceSynchronize();
        hvk::lowrank_destroy(a->low);
    } else if (a->kind != 0) {
        if (a->lr.done) cudaEventSynchronize(a->lr.done);
        hvk::lr_destroy(a->lr);
    }
    if (a->kind == 0) cudaFree(a->psf);
    delete a;
    return HV_OK;
}
