// hv_server.cpp -- request serving for many concurrent clients (MCMC chains
// asking for misfits, optimisers asking for gradients and Hessian actions;
// paper sections 2.2-2.3 use exactly these three quantities).
//
// One device arena holds every admitted request's workspace; a scheduler
// thread admits queued requests when a stream and enough arena memory are
// free and runs each on its own stream, so requests that arrive while others
// run overlap with them on the GPU.  Continuous batching: when it admits an
// H v, gradient or misfit request, the queued requests on the same problem
// and model join it (up to the server's vector limit, if the merged
// workspace fits) and run as one merged call (hv_apply_batch: one forward
// sweep, the H v vectors and the gradients as one batch of Born vectors),
// whose results are bitwise those of separate calls; queued applies of one
// Hessian approximation in one mode join into one apply of all their vectors.
// Misfit requests (MCMC chains' proposals) go to a misfit lane per problem,
// looked after by a second thread: a misfit engine (hv_engine_*) whose slots
// each hold one model with its own step counter, ticked by that thread or
// served by the engine's device-resident loop, so a misfit joins a running
// sweep at its next time step; where no lane fits in the arena, queued
// misfits at different models run as one sweep of all the models
// (hv_misfit_models).  Completion is detected
// with events; the scheduler never blocks on the device (event queries plus
// short sleeps), and every host wait is bounded.
#include "hv_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) in 256-byte units, with coalescing.
class Arena {
  public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes;
                size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_[*off] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off)
    {
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t bytes = u->second;
        used_.erase(u);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

  private:
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> used_;
};

struct Req {
    unsigned long long id;
    hv_request r;
    int status = HV_REQ_QUEUED;
    size_t ws = 0, off = 0;
    int slot = -1;
    int batch = 1;            // requests that ran in the same launch sequence
    bool no_lane = false;     // a misfit left to the scheduler (its lane did not fit)
    double t_submit = 0, t_start = 0, t_done = 0;
};

// A misfit lane: the misfit engine of one problem (hv_engine_*) in an arena
// block.  Host-ticked (default): requests join on the lane's stream and the
// lane thread enqueues the ticks, keeping up to kLookahead in flight.  Device
// loop (hv_server_set_engine_loop): the engine's device-resident loop runs on
// the lane's stream, requests are prepared and posted on a second stream and
// join the loop at its next time step, and the lane thread polls the
// engine's host-mapped completion words.
constexpr int kLookahead = 8;
struct Lane {
    hv_engine *e = nullptr;
    unsigned long long serial = 0;              // the problem's hv_create serial
    bool device_loop = false;
    int slots = 0;
    size_t off = 0;
    cudaStream_t st = nullptr;                  // joins and ticks, or the loop
    cudaStream_t post_st = nullptr;             // device loop: the requests' preparation and posts
    std::vector<unsigned long long> slot_req;   // request per engine slot (0: free)
    int active = 0;                             // occupied slots (joined or posted, not done)
    int busy = 0;                               // active + admitted, not yet joined or posted
    std::deque<cudaEvent_t> ticks;              // host-ticked: recorded after recent ticks, oldest first
    std::vector<std::pair<cudaEvent_t, std::vector<unsigned long long>>> finishing;   // done when the event is
    bool running = false;                       // device loop: the loop, at the last poll
    int failed = HV_OK;                         // a join, post, tick or launch failed: the lane takes no more
    double idle_since = -1;
};

}  // namespace

struct hv_server {
    int device = 0;
    size_t budget = 0;
    char *arena_base = nullptr;
    Arena *arena = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<std::vector<unsigned long long>> slot_reqs;   // request ids per slot (empty = free)
    std::vector<size_t> slot_off;                              // arena offset held by the slot
    int merge_max = 64;                                        // vectors per merged call (< 2: no merging)
    int engine_slots = 64;                                     // slots per misfit lane (0: misfits run as calls)
    bool engine_loop = false;                                  // lanes created from now on run the device loop
    std::unordered_map<hv_handle *, Lane> lanes;               // lane thread only
    int lane_reqs = 0;                                         // requests admitted to lanes and not done (under mu)
    std::vector<cudaEvent_t> ev_pool;                          // lane thread only
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<unsigned long long> queue;
    std::unordered_map<unsigned long long, Req> reqs;
    unsigned long long next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker, lane_worker;
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

int op_of(int kind)
{
    return kind == HV_REQ_HV ? HV_OP_HV : (kind == HV_REQ_GRAD ? HV_OP_GRAD : HV_OP_MISFIT);
}

int request_ws(const hv_request &r, size_t *bytes)
{
    if (r.kind == HV_REQ_APPROX) {
        *bytes = 0;
        return HV_OK;
    }
    return hv_workspace_size(r.problem, op_of(r.kind), r.kind == HV_REQ_HV ? r.k : 1, r.ckpt, bytes);
}

// Enqueue one request on its stream and record the slot's completion event
// (also after a failed enqueue, so that its memory is released only once
// whatever was enqueued has finished).
int launch(hv_server *S, const Req &q)
{
    void *ws = S->arena_base + q.off;
    void *st = (void *)S->streams[q.slot];
    const hv_request &r = q.r;
    int rc;
    if (r.kind == HV_REQ_HV) rc = hv_hessian_apply(r.problem, r.m, r.v, r.k, r.out, r.ckpt, ws, q.ws, st);
    else if (r.kind == HV_REQ_GRAD) rc = hv_misfit_grad(r.problem, r.m, r.d_obs, r.phi, r.out, r.ckpt, ws, q.ws, st);
    else if (r.kind == HV_REQ_APPROX) rc = hv_approx_apply(r.approx, r.v, r.k, r.out, r.approx_mode, st);
    else rc = hv_misfit(r.problem, r.m, r.d_obs, r.phi, ws, q.ws, st);
    cudaError_t e = cudaEventRecord(S->events[q.slot], S->streams[q.slot]);
    if (rc == HV_OK && e != cudaSuccess) rc = HV_ECUDA;
    return rc;
}

// The merged call of several requests on one problem and model.
struct Merged {
    std::vector<const float *> v, gd, md;
    std::vector<int> k;
    std::vector<float *> out, g;
    std::vector<double *> gp, mp;
    int ckpt = HV_CKPT_ALL;
    hv_batch b{};
    void add(const hv_request &r)
    {
        if (r.kind == HV_REQ_HV) {
            v.push_back(r.v);
            k.push_back(r.k);
            out.push_back(r.out);
        } else if (r.kind == HV_REQ_GRAD) {
            gd.push_back(r.d_obs);
            gp.push_back(r.phi);
            g.push_back(r.out);
        } else {
            md.push_back(r.d_obs);
            mp.push_back(r.phi);
        }
    }
    const hv_batch *make()
    {
        b.n_hv = (int)v.size();
        b.v = v.data();
        b.k = k.data();
        b.Hv = out.data();
        b.n_grad = (int)gd.size();
        b.grad_dobs = gd.data();
        b.grad_phi = gp.data();
        b.grad = g.data();
        b.n_misfit = (int)md.size();
        b.misfit_dobs = md.data();
        b.misfit_phi = mp.data();
        return &b;
    }
};

int launch_merged(hv_server *S, const std::vector<Req> &qs, size_t ws_bytes)
{
    const int slot = qs[0].slot;
    Merged M;
    for (const Req &q : qs) {
        M.add(q.r);
        if (q.r.kind != HV_REQ_MISFIT) M.ckpt = q.r.ckpt;
    }
    int rc = hv_apply_batch(qs[0].r.problem, qs[0].r.m, M.make(), M.ckpt, S->arena_base + qs[0].off, ws_bytes,
                            (void *)S->streams[slot]);
    cudaError_t e = cudaEventRecord(S->events[slot], S->streams[slot]);
    if (rc == HV_OK && e != cudaSuccess) rc = HV_ECUDA;
    return rc;
}

bool mergeable(const hv_request &r) { return r.kind == HV_REQ_HV || r.kind == HV_REQ_GRAD || r.kind == HV_REQ_MISFIT; }

// A merged group of misfits at more than one model runs as one sweep of all
// the models (hv_misfit_models); other merged groups share one model.
bool models_group(hv_server *S, const std::vector<unsigned long long> &ids)
{
    const hv_request &r0 = S->reqs[ids[0]].r;
    bool other = false;
    for (auto id : ids) {
        const hv_request &r = S->reqs[id].r;
        if (r.kind != HV_REQ_MISFIT) return false;
        other |= r.m != r0.m;
    }
    return ids.size() > 1 && other;
}

int launch_merged_models(hv_server *S, const std::vector<Req> &qs, size_t ws_bytes)
{
    const int slot = qs[0].slot;
    std::vector<const float *> m, d;
    std::vector<double *> phi;
    for (const Req &q : qs) {
        m.push_back(q.r.m);
        d.push_back(q.r.d_obs);
        phi.push_back(q.r.phi);
    }
    int rc = hv_misfit_models(qs[0].r.problem, (int)qs.size(), m.data(), d.data(), phi.data(),
                              S->arena_base + qs[0].off, ws_bytes, (void *)S->streams[slot]);
    cudaError_t e = cudaEventRecord(S->events[slot], S->streams[slot]);
    if (rc == HV_OK && e != cudaSuccess) rc = HV_ECUDA;
    return rc;
}

// Points per field of an approximation (its grid).
size_t approx_points(const hv_approx *a)
{
    int info[11] = {};
    if (hv_approx_info(a, info) != HV_OK) return 0;
    return (size_t)info[9] * info[10];
}

// Applies of one approximation in one mode, merged: the vectors gathered into
// the arena block (vectors, then outputs), one apply of all of them, the
// outputs scattered back.
int launch_merged_approx(hv_server *S, const std::vector<Req> &qs)
{
    const int slot = qs[0].slot;
    cudaStream_t st = S->streams[slot];
    const hv_approx *a = qs[0].r.approx;
    const size_t N = approx_points(a);
    int K = 0;
    for (const Req &q : qs) K += q.r.k;
    float *V = reinterpret_cast<float *>(S->arena_base + qs[0].off), *O = V + (size_t)K * N;
    int rc = HV_OK;
    size_t at = 0;
    for (const Req &q : qs) {
        if (rc == HV_OK && cudaMemcpyAsync(V + at * N, q.r.v, (size_t)q.r.k * N * sizeof(float), cudaMemcpyDeviceToDevice,
                                           st) != cudaSuccess)
            rc = hvi::fail(HV_ECUDA, "merged apply: gathering the vectors failed");
        at += q.r.k;
    }
    if (rc == HV_OK) rc = hv_approx_apply(a, V, K, O, qs[0].r.approx_mode, (void *)st);
    at = 0;
    for (const Req &q : qs) {
        if (rc == HV_OK && cudaMemcpyAsync(q.r.out, O + at * N, (size_t)q.r.k * N * sizeof(float),
                                           cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = hvi::fail(HV_ECUDA, "merged apply: scattering the outputs failed");
        at += q.r.k;
    }
    cudaError_t e = cudaEventRecord(S->events[slot], st);
    if (rc == HV_OK && e != cudaSuccess) rc = HV_ECUDA;
    return rc;
}

// The queued requests that can run merged with the one at `head`: same problem
// and model; H v and gradients with the same checkpoint budget; at most
// merge_max Born vectors in all.
std::vector<unsigned long long> merge_group(hv_server *S, std::deque<unsigned long long>::iterator head)
{
    std::vector<unsigned long long> ids{*head};
    const hv_request &r0 = S->reqs[*head].r;
    if (S->merge_max < 2) return ids;
    if (r0.kind == HV_REQ_APPROX) {              // applies of one approximation in one mode
        int vecs = r0.k;
        for (auto it = std::next(head); it != S->queue.end(); ++it) {
            const hv_request &r = S->reqs[*it].r;
            if (r.kind != HV_REQ_APPROX || r.approx != r0.approx || r.approx_mode != r0.approx_mode) continue;
            if (vecs + r.k > S->merge_max) continue;
            vecs += r.k;
            ids.push_back(*it);
        }
        return ids;
    }
    if (!mergeable(r0)) return ids;
    if (r0.kind == HV_REQ_MISFIT) {              // misfits on the problem at other models: one sweep of all models
        std::vector<unsigned long long> mids{*head};
        bool other = false;
        for (auto it = std::next(head); it != S->queue.end() && (int)mids.size() < S->merge_max; ++it) {
            const hv_request &r = S->reqs[*it].r;
            if (r.kind != HV_REQ_MISFIT || r.problem != r0.problem) continue;
            other |= r.m != r0.m;
            mids.push_back(*it);
        }
        if (other) return mids;
    }
    int ckpt = r0.kind == HV_REQ_MISFIT ? 0 : r0.ckpt;
    bool have_ckpt = r0.kind != HV_REQ_MISFIT;
    int vecs = r0.kind == HV_REQ_HV ? r0.k : (r0.kind == HV_REQ_GRAD ? 1 : 0);
    for (auto it = std::next(head); it != S->queue.end(); ++it) {
        const hv_request &r = S->reqs[*it].r;
        if (!mergeable(r) || r.problem != r0.problem || r.m != r0.m) continue;
        if (r.kind != HV_REQ_MISFIT) {
            if (have_ckpt && r.ckpt != ckpt) continue;
            const int add = r.kind == HV_REQ_HV ? r.k : 1;
            if (vecs + add > S->merge_max) continue;
            vecs += add;
            ckpt = r.ckpt;
            have_ckpt = true;
        }
        ids.push_back(*it);
    }
    return ids;
}

int merged_ws(hv_server *S, const std::vector<unsigned long long> &ids, size_t *bytes)
{
    if (S->reqs[ids[0]].r.kind == HV_REQ_APPROX) {   // staging for the vectors and the outputs
        size_t K = 0;
        for (auto id : ids) K += S->reqs[id].r.k;
        *bytes = 2 * K * approx_points(S->reqs[ids[0]].r.approx) * sizeof(float);
        return HV_OK;
    }
    if (models_group(S, ids))
        return hv_workspace_size(S->reqs[ids[0]].r.problem, HV_OP_MISFITS, (int)ids.size(), 0, bytes);
    Merged M;
    for (auto id : ids) {
        const hv_request &r = S->reqs[id].r;
        M.add(r);
        if (r.kind != HV_REQ_MISFIT) M.ckpt = r.ckpt;
    }
    return hv_batch_workspace_size(S->reqs[ids[0]].r.problem, M.make(), M.ckpt, bytes);
}

// ---------------------------------------------------------------- misfit lanes
// A queued misfit that its problem's lane takes (lanes on, and one fits).
bool lane_bound(const hv_server *S, const Req &q)
{
    return q.r.kind == HV_REQ_MISFIT && S->engine_slots > 0 && !q.no_lane;
}

cudaEvent_t take_event(hv_server *S)
{
    cudaEvent_t e = nullptr;
    if (!S->ev_pool.empty()) {
        e = S->ev_pool.back();
        S->ev_pool.pop_back();
    } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

void lane_release(hv_server *S, Lane &L)
{
    hv_engine_destroy(L.e);                     // ends a running loop first
    cudaStreamSynchronize(L.st);
    if (L.post_st) cudaStreamSynchronize(L.post_st);
    for (cudaEvent_t e : L.ticks) S->ev_pool.push_back(e);
    for (auto &f : L.finishing) S->ev_pool.push_back(f.first);
    cudaStreamDestroy(L.st);
    if (L.post_st) cudaStreamDestroy(L.post_st);
    S->arena->release(L.off);
}

// The lane of problem p, created on first use with as many slots (up to
// engine_slots) as fit in an eighth of the budget and in kLaneCtas CTAs per
// step (the loop's step kernel launches the CTAs of every slot; those of free
// slots exit at once, but on a large grid they would still cost more than the
// step); nullptr if none fits now.
constexpr int kLaneCtas = 16384;
Lane *lane_for(hv_server *S, hv_handle *p)
{
    auto it = S->lanes.find(p);
    if (it != S->lanes.end() && it->second.serial != p->serial) {
        // The lane of a destroyed problem whose address a new problem reuses: it never
        // runs for the new one; released here once idle (requests of a destroyed problem
        // cannot be pending unless the caller broke the contract).
        Lane &L = it->second;
        if (L.busy != 0) return nullptr;
        lane_release(S, L);
        S->lanes.erase(it);
        it = S->lanes.end();
    }
    if (it != S->lanes.end()) return it->second.failed == HV_OK ? &it->second : nullptr;
    int slots = std::min(S->engine_slots, std::max(1, kLaneCtas / std::max(1, hvk::fwd_ctas_per_model(p, p->cfg[1]))));
    size_t bytes = 0;
    while (slots > 1 && (hv_engine_workspace_size(p, slots, &bytes) != HV_OK || bytes > S->budget / 8)) slots /= 2;
    if (hv_engine_workspace_size(p, slots, &bytes) != HV_OK) return nullptr;
    Lane L;
    if (!S->arena->alloc(bytes, &L.off)) return nullptr;
    if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess) {
        S->arena->release(L.off);
        return nullptr;
    }
    L.device_loop = S->engine_loop;
    if (L.device_loop && cudaStreamCreateWithFlags(&L.post_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(L.st);
        S->arena->release(L.off);
        return nullptr;
    }
    if (hv_engine_create(p, slots, S->arena_base + L.off, bytes, &L.e) != HV_OK) {
        cudaStreamDestroy(L.st);
        if (L.post_st) cudaStreamDestroy(L.post_st);
        S->arena->release(L.off);
        return nullptr;
    }
    L.slots = slots;
    L.serial = p->serial;
    L.slot_req.assign(slots, 0);
    return &(S->lanes[p] = std::move(L));
}

struct Join {
    hv_handle *p;
    unsigned long long id;
    const float *m, *d_obs;
    double *phi;
};

// A lane's occupied slots all fail with rc; the lane takes no more requests.
void lane_fail(Lane &L, int rc, std::vector<std::pair<unsigned long long, int>> &finished)
{
    L.failed = rc;
    for (int q = 0; q < L.slots; ++q)
        if (L.slot_req[q]) {
            finished.push_back({L.slot_req[q], rc});
            L.slot_req[q] = 0;
        }
    L.busy -= L.active;
    L.active = 0;
}

// Host-ticked lane: ticks until kLookahead are in flight; the requests of a
// tick that finishes slots are done once the event after it has completed.
bool lane_ticks(hv_server *S, Lane &L, std::vector<std::pair<unsigned long long, int>> &finished)
{
    bool any = false;
    std::vector<int> done(L.slots);
    while (L.active > 0 && L.failed == HV_OK) {
        while (!L.ticks.empty() && cudaEventQuery(L.ticks.front()) != cudaErrorNotReady) {
            S->ev_pool.push_back(L.ticks.front());
            L.ticks.pop_front();
        }
        if ((int)L.ticks.size() >= kLookahead) break;
        int nd = 0;
        int rc = hv_engine_tick(L.e, (void *)L.st, done.data(), &nd);
        cudaEvent_t ev = take_event(S);
        if (rc == HV_OK && (!ev || cudaEventRecord(ev, L.st) != cudaSuccess)) rc = HV_ECUDA;
        if (ev) L.ticks.push_back(ev);
        any = true;
        if (rc != HV_OK) {
            lane_fail(L, rc, finished);
            break;
        }
        if (nd > 0) {
            std::vector<unsigned long long> ids;
            for (int q = 0; q < nd; ++q) {
                ids.push_back(L.slot_req[done[q]]);
                L.slot_req[done[q]] = 0;
            }
            L.active -= nd;
            L.busy -= nd;
            cudaEvent_t f = take_event(S);
            if (f && cudaEventRecord(f, L.st) == cudaSuccess) {
                L.finishing.push_back({f, ids});
            } else {
                if (f) S->ev_pool.push_back(f);
                for (auto id : ids) finished.push_back({id, HV_ECUDA});
            }
        }
    }
    return any;
}

// Device-loop lane: the finished slots reported by the engine; the loop
// relaunched if it has ended while requests are out.
bool lane_poll(Lane &L, std::vector<std::pair<unsigned long long, int>> &finished)
{
    if (L.active == 0 && !L.running) return false;
    std::vector<int> done(L.slots);
    int nd = 0, run = 0;
    if (hv_engine_poll(L.e, done.data(), &nd, &run) != HV_OK) run = 0;
    for (int q = 0; q < nd; ++q) {
        finished.push_back({L.slot_req[done[q]], HV_OK});
        L.slot_req[done[q]] = 0;
    }
    L.active -= nd;
    L.busy -= nd;
    if (L.active > 0 && !run && L.failed == HV_OK) {
        const int rc = hv_engine_serve(L.e, (void *)L.st);
        if (rc == HV_OK) run = 1;
        else lane_fail(L, rc, finished);
    }
    L.running = run != 0;
    return nd > 0;
}

// Outside the lock: the admitted requests joined to (or posted to) their
// lanes, then every lane ticked or polled.  Returns whether anything was
// enqueued or finished; `finished` collects requests done (HV_OK) or failed.
bool lane_work(hv_server *S, const std::vector<Join> &joins, std::vector<std::pair<unsigned long long, int>> &finished)
{
    bool any = !joins.empty();
    for (const Join &j : joins) {
        Lane &L = S->lanes[j.p];
        int slot = -1;
        int rc = L.failed;
        if (rc == HV_OK)
            rc = L.device_loop ? hv_engine_post(L.e, j.m, j.d_obs, j.phi, (void *)L.post_st, &slot)
                               : hv_engine_join(L.e, j.m, j.d_obs, j.phi, (void *)L.st, &slot);
        if (rc != HV_OK) {
            if (L.failed == HV_OK) L.failed = rc;
            --L.busy;
            finished.push_back({j.id, rc});
            continue;
        }
        L.slot_req[slot] = j.id;
        ++L.active;
    }
    for (auto &kv : S->lanes) any |= kv.second.device_loop ? lane_poll(kv.second, finished)
                                                          : lane_ticks(S, kv.second, finished);
    return any;
}

// Under the lock: the statuses of finished (or failed) lane requests, the
// host-ticked lanes' requests whose last tick has completed, and lanes idle
// for a while released.  Returns whether a request finished.
bool lane_completions(hv_server *S, std::vector<std::pair<unsigned long long, int>> &finished)
{
    bool any = false;
    const double t = S->now();
    for (auto &f : finished) {
        Req &q = S->reqs[f.first];
        q.status = f.second;
        q.t_done = t;
        --S->lane_reqs;
        any = true;
    }
    finished.clear();
    for (auto it = S->lanes.begin(); it != S->lanes.end();) {
        Lane &L = it->second;
        for (size_t i = 0; i < L.finishing.size();) {
            const cudaError_t e = cudaEventQuery(L.finishing[i].first);
            if (e == cudaErrorNotReady) {
                ++i;
                continue;
            }
            for (auto id : L.finishing[i].second) {
                Req &q = S->reqs[id];
                q.status = e == cudaSuccess ? HV_OK : HV_ECUDA;
                q.t_done = t;
                --S->lane_reqs;
            }
            S->ev_pool.push_back(L.finishing[i].first);
            L.finishing.erase(L.finishing.begin() + i);
            any = true;
        }
        if (L.busy != 0 || !L.finishing.empty()) {
            L.idle_since = -1;
            ++it;
            continue;
        }
        if (L.idle_since < 0) L.idle_since = t;
        if (t - L.idle_since < 0.2 || cudaStreamQuery(L.st) == cudaErrorNotReady) {
            ++it;
            continue;
        }
        lane_release(S, L);
        it = S->lanes.erase(it);
    }
    return any;
}

// The lane thread: admits queued misfits into their problems' lanes (a
// misfit whose lane does not fit in the arena is left to the scheduler), then
// joins or posts them and ticks or polls the lanes outside the lock, so that
// the lanes advance whatever the scheduler thread is enqueueing.
void lane_loop(hv_server *S)
{
    cudaSetDevice(S->device);
    std::vector<std::pair<unsigned long long, int>> lane_failed;
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop.load()) {
        bool progress = lane_completions(S, lane_failed);
        if (progress) S->cv_done.notify_all();
        std::vector<Join> joins;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            Req &q = S->reqs[*it];
            if (!lane_bound(S, q)) {
                ++it;
                continue;
            }
            Lane *L = lane_for(S, q.r.problem);
            if (!L) {                              // no room for a lane: the scheduler runs it as a call
                q.no_lane = true;
                S->cv_work.notify_all();
                ++it;
                continue;
            }
            if (L->busy >= L->slots) {
                ++it;
                continue;
            }
            ++L->busy;
            ++S->lane_reqs;
            q.status = HV_REQ_RUNNING;
            q.t_start = S->now();
            q.batch = L->busy;
            joins.push_back({q.r.problem, q.id, q.r.m, q.r.d_obs, q.r.phi});
            it = S->queue.erase(it);
        }
        bool active = !joins.empty();
        for (auto &kv : S->lanes) active |= kv.second.active > 0 || kv.second.running;
        if (active) {
            lk.unlock();
            progress |= lane_work(S, joins, lane_failed);
            lk.lock();
        }
        if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(active ? 10 : 50));
    }
}

void worker_loop(hv_server *S)
{
    cudaSetDevice(S->device);
    std::vector<int> failed(S->slot_reqs.size(), HV_OK);   // enqueue status per running slot
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop.load()) {
        bool progress = false;
        // completions
        for (size_t sl = 0; sl < S->slot_reqs.size(); ++sl) {
            if (S->slot_reqs[sl].empty()) continue;
            cudaError_t e = cudaEventQuery(S->events[sl]);
            if (e == cudaErrorNotReady) continue;
            const double t = S->now();
            for (auto id : S->slot_reqs[sl]) {
                Req &q = S->reqs[id];
                q.status = failed[sl] != HV_OK ? failed[sl] : (e == cudaSuccess ? HV_OK : HV_ECUDA);
                q.t_done = t;
            }
            S->arena->release(S->slot_off[sl]);
            S->slot_reqs[sl].clear();
            failed[sl] = HV_OK;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // admissions, in arrival order; a request that does not fit yet is passed
        std::vector<std::vector<Req>> admitted;
        std::vector<size_t> admitted_ws;
        std::vector<bool> admitted_models;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            if (lane_bound(S, S->reqs[*it])) {   // the lane thread admits it
                ++it;
                continue;
            }
            int slot = -1;
            for (size_t sl = 0; sl < S->slot_reqs.size(); ++sl)
                if (S->slot_reqs[sl].empty()) {
                    slot = (int)sl;
                    break;
                }
            if (slot < 0) {
                ++it;
                continue;
            }
            std::vector<unsigned long long> ids = merge_group(S, it);
            size_t ws = S->reqs[*it].ws, off = 0;
            if (ids.size() > 1 && merged_ws(S, ids, &ws) != HV_OK) {
                ids.resize(1);
                ws = S->reqs[*it].ws;
            }
            bool fits = S->arena->alloc(ws, &off);
            if (!fits && ids.size() > 1) {        // the merged call does not fit: try the request alone
                ids.resize(1);
                ws = S->reqs[*it].ws;
                fits = S->arena->alloc(ws, &off);
            }
            if (!fits) {
                ++it;
                continue;
            }
            std::vector<Req> group;
            const double t = S->now();
            for (auto id : ids) {
                Req &q = S->reqs[id];
                q.off = off;
                q.slot = slot;
                q.t_start = t;
                q.status = HV_REQ_RUNNING;
                q.batch = (int)ids.size();
                group.push_back(q);
            }
            S->slot_reqs[slot] = ids;
            S->slot_off[slot] = off;
            admitted_models.push_back(models_group(S, ids));
            admitted.push_back(group);
            admitted_ws.push_back(ws);
            // Erasing from a deque invalidates its iterators: work by index.  The merged
            // requests all sit behind the head, so removing them leaves the head's index.
            const size_t head = (size_t)(it - S->queue.begin());
            for (size_t i = 1; i < ids.size(); ++i)
                S->queue.erase(std::find(S->queue.begin() + head + 1, S->queue.end(), ids[i]));
            it = S->queue.erase(S->queue.begin() + head);
        }
        if (!admitted.empty()) {
            lk.unlock();                          // enqueueing thousands of launches takes a while
            std::vector<int> rcs;
            for (size_t i = 0; i < admitted.size(); ++i) {
                const std::vector<Req> &g = admitted[i];
                rcs.push_back(g.size() == 1                  ? launch(S, g[0])
                              : g[0].r.kind == HV_REQ_APPROX ? launch_merged_approx(S, g)
                              : admitted_models[i]           ? launch_merged_models(S, g, admitted_ws[i])
                                                             : launch_merged(S, g, admitted_ws[i]));
            }
            lk.lock();
            for (size_t i = 0; i < admitted.size(); ++i) failed[admitted[i][0].slot] = rcs[i];
            progress = true;
        }
        if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" int hv_server_create(size_t hbm_budget, int max_concurrent, hv_server **out)
{
    if (!out || hbm_budget < 4096 || max_concurrent < 1 || max_concurrent > 256)
        return hvi::fail(HV_EINVAL, "hv_server_create: need a budget >= 4 KiB and 1..256 concurrent requests");
    *out = nullptr;
    hv_server *S = new hv_server();
    S->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_base, hbm_budget);
    if (e != cudaSuccess) {
        delete S;
        return hvi::fail(e == cudaErrorMemoryAllocation ? HV_ENOMEM : HV_ECUDA, "hv_server_create: %s",
                         cudaGetErrorString(e));
    }
    S->budget = hbm_budget;
    S->arena = new Arena(hbm_budget);
    S->streams.resize(max_concurrent);
    S->events.resize(max_concurrent);
    S->slot_reqs.assign(max_concurrent, {});
    S->slot_off.assign(max_concurrent, 0);
    for (int i = 0; i < max_concurrent; ++i) {
        cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming);
    }
    S->worker = std::thread(worker_loop, S);
    S->lane_worker = std::thread(lane_loop, S);
    *out = S;
    return HV_OK;
}

extern "C" int hv_server_destroy(hv_server *S, double timeout_s)
{
    if (!S) return HV_OK;
    int rc = HV_OK;
    {
        // wait (bounded) for running requests
        auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
        std::unique_lock<std::mutex> lk(S->mu);
        S->queue.clear();
        auto busy = [&] {
            for (auto &ids : S->slot_reqs)
                if (!ids.empty()) return true;
            return S->lane_reqs > 0;
        };
        while (busy()) {
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && busy()) {
                rc = hvi::fail(HV_ETIMEOUT, "hv_server_destroy: requests still running after %.1f s", timeout_s);
                break;
            }
        }
    }
    S->stop.store(true);
    S->cv_work.notify_all();
    S->worker.join();
    S->lane_worker.join();
    if (rc == HV_OK) {
        for (auto &kv : S->lanes) lane_release(S, kv.second);
        for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
        for (auto st : S->streams) cudaStreamDestroy(st);
        for (auto ev : S->events) cudaEventDestroy(ev);
        cudaFree(S->arena_base);
        delete S->arena;
        delete S;
    }
    // on timeout the server's device memory is left in place (work may still use it)
    return rc;
}

extern "C" int hv_submit(hv_server *S, const hv_request *r, unsigned long long *id)
{
    if (!S || !r || !id) return hvi::fail(HV_EINVAL, "hv_submit: null argument");
    const bool approx = r->kind == HV_REQ_APPROX;
    if ((!approx && (!r->problem || !r->m)) || (r->kind == HV_REQ_HV && (!r->v || !r->out || r->k < 1)) ||
        (r->kind == HV_REQ_GRAD && (!r->d_obs || !r->out || !r->phi)) || (r->kind == HV_REQ_MISFIT && (!r->d_obs || !r->phi)) ||
        (approx && (!r->approx || !r->v || !r->out || r->k < 1 || r->approx_mode < HV_APPROX_H ||
                    r->approx_mode > HV_APPROX_SQRT_T)) || r->kind < HV_REQ_HV || r->kind > HV_REQ_APPROX)
        return hvi::fail(HV_EINVAL, "hv_submit: incomplete request of kind %d", r->kind);
    const int dev = approx ? hvi::approx_device(r->approx) : r->problem->device;
    if (dev != S->device) return hvi::fail(HV_EINVAL, "hv_submit: %s on another device", approx ? "approximation" : "problem");
    size_t ws = 0;
    HV_RT_INTERNAL(request_ws(*r, &ws));
    if (((ws + 255) & ~(size_t)255) > S->budget)
        return hvi::fail(HV_ENOMEM, "hv_submit: request needs %zu bytes, the server budget is %zu", ws, S->budget);
    std::lock_guard<std::mutex> g(S->mu);
    Req q;
    q.id = S->next_id++;
    q.r = *r;
    q.ws = ws;
    q.t_submit = S->now();
    S->reqs[q.id] = q;
    S->queue.push_back(q.id);
    *id = q.id;
    S->cv_work.notify_all();
    return HV_OK;
}

extern "C" int hv_poll(hv_server *S, unsigned long long id, int *status)
{
    if (!S || !status) return hvi::fail(HV_EINVAL, "hv_poll: null argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return hvi::fail(HV_EINVAL, "hv_poll: unknown request %llu", id);
    *status = it->second.status;
    return HV_OK;
}

extern "C" int hv_wait(hv_server *S, unsigned long long id, double timeout_s, int *status)
{
    if (!S || !status) return hvi::fail(HV_EINVAL, "hv_wait: null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
    for (;;) {
        auto it = S->reqs.find(id);
        if (it == S->reqs.end()) return hvi::fail(HV_EINVAL, "hv_wait: unknown request %llu", id);
        int st = it->second.status;
        if (st != HV_REQ_QUEUED && st != HV_REQ_RUNNING) {
            *status = st;
            return HV_OK;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            *status = S->reqs[id].status;
            if (*status == HV_REQ_QUEUED || *status == HV_REQ_RUNNING)
                return hvi::fail(HV_ETIMEOUT, "hv_wait: request %llu not done after %.3f s", id, timeout_s);
            return HV_OK;
        }
    }
}

extern "C" int hv_request_get_info(hv_server *S, unsigned long long id, hv_request_info *info)
{
    if (!S || !info) return hvi::fail(HV_EINVAL, "hv_request_get_info: null argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return hvi::fail(HV_EINVAL, "hv_request_get_info: unknown request %llu", id);
    const Req &q = it->second;
    info->kind = q.r.kind;
    info->status = q.status;
    info->t_submit = q.t_submit;
    info->t_start = q.t_start;
    info->t_done = q.t_done;
    info->ws_bytes = q.ws;
    info->batch = q.batch;
    return HV_OK;
}

extern "C" int hv_server_set_engine(hv_server *S, int slots)
{
    if (!S || slots < 0 || slots > 65535)
        return hvi::fail(HV_EINVAL, "hv_server_set_engine: null server or slots outside 0..65535");
    std::lock_guard<std::mutex> g(S->mu);
    S->engine_slots = slots;
    return HV_OK;
}

extern "C" int hv_server_set_engine_loop(hv_server *S, int enable)
{
    if (!S) return hvi::fail(HV_EINVAL, "hv_server_set_engine_loop: null server");
    std::lock_guard<std::mutex> g(S->mu);
    S->engine_loop = enable != 0;
    return HV_OK;
}

extern "C" int hv_server_set_batching(hv_server *S, int max_vectors)
{
    if (!S || max_vectors < 0 || max_vectors > 65535)
        return hvi::fail(HV_EINVAL, "hv_server_set_batching: null server or max_vectors outside 0..65535");
    std::lock_guard<std::mutex> g(S->mu);
    S->merge_max = max_vectors;
    return HV_OK;
}
