// Continuous-batching forecast server.
//
// A request is a Parareal (§3.1, Eq. 9) or two-level MGRIT (§3.2) solve of one initial
// state.  Requests wait in a FIFO queue and are admitted at the start of a tick while the
// slot limit and the device-memory budget allow; the budget counts each request's own state,
// its share of the staging buffers and the plan workspace its slices need.
//
// Lanes.  Calls on one plan must not overlap (a plan's workspace is shared), so the active
// requests are partitioned into lanes: requests that share a plan (fine or coarse) are in
// the same lane.  Every lane runs on its own CUDA stream with its own staging buffers, so
// the work of different lanes (different truncations with their own plans) overlaps on the
// device; within a lane the work is ordered on its stream.
//
// Every tick advances every active request by one iteration, with ONE host
// synchronisation per tick for all lanes:
//  * Parareal requests of one lane that share plans and steppers form a group: the fine
//    propagation of all their slices is one batched propagate call, and their serial
//    coarse chains advance together (one batched coarse step per chain position, then each
//    request's FP64 correction).  Newly admitted requests of a group get their initial
//    coarse chains batched the same way, without a host synchronisation.
//  * MGRIT requests run one cycle each, enqueued on their lane without synchronising.
// Norms and status words go to pinned host memory and are read after the tick's
// synchronisation.  A request's spectral state stays in device memory from admission to
// completion.  With FP64 plans a request's result equals its result alone up to the
// rounding order of the small-batch implicit solve; with split-precision plans the batch
// width selects the Legendre kernel (narrow FP32 contraction or tcgen05 GEMM) and the
// implicit-solve kernel, so results agree within the split-precision tolerance.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "swe_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long id = 0;
    swe_request_desc d{};
    int64_t per = 0;              // complex values per state (fine plan)
    size_t bytes = 0;             // device memory charged to the budget while held
    std::vector<double2> U0;      // host copy until admission
    // Parareal state
    double2* U = nullptr;         // [S+1]
    double2* Fo = nullptr;        // [S]
    double2* Gold = nullptr;      // [S]
    unsigned long long* red = nullptr;
    // MGRIT state
    swe_mgrit_t mg = nullptr;
    double2* u0 = nullptr;        // device copy of the initial state (MGRIT)
    // pinned host words filled by the tick: 6 reduction words and the status words of the
    // request's two plans (fine / coarse level)
    unsigned long long* red_host = nullptr;
    int* bits_host = nullptr;
    bool fresh = false;           // admitted in this tick: initial guess not yet computed
    int iters_done = 0;
    int status = 0;               // 0 queued, 1 active, 2 done, 3 failed
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<double> norms;
};

bool same_group(const swe_request_desc& a, const swe_request_desc& b) {
    return a.method == SWE_METHOD_PARAREAL && b.method == SWE_METHOD_PARAREAL && a.fine_plan == b.fine_plan &&
           a.coarse_plan == b.coarse_plan && memcmp(&a.fine, &b.fine, sizeof(a.fine)) == 0 &&
           memcmp(&a.coarse, &b.coarse, sizeof(a.coarse)) == 0;
}

struct Lane {
    cudaStream_t st = nullptr;
    double2* stage_in = nullptr;
    double2* stage_out = nullptr;
    size_t stage_bytes = 0;
};

double norm_of(const unsigned long long* red) {
    double nrm = 0.0;
    for (int q = 0; q < 3; ++q) {
        double dd, vv;
        memcpy(&dd, &red[q], sizeof(double));
        memcpy(&vv, &red[3 + q], sizeof(double));
        if (vv > 0) nrm = fmax(nrm, dd / vv);
    }
    return nrm;
}

}  // namespace

struct swe_server {
    swe_server_desc d{};
    long long next_id = 1;
    std::deque<long long> queue;
    std::map<long long, std::unique_ptr<Request>> reqs;
    size_t bytes_active = 0;
    int n_active = 0;
    std::vector<Lane> lanes;      // stream pool, reused tick to tick
};

static swe_status lane_get(swe_server* s, int n) {
    while ((int)s->lanes.size() < n) {
        Lane L;
        SWE_CHECK_CUDA(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
        s->lanes.push_back(L);
    }
    return SWE_OK;
}

static swe_status ensure_stage(Lane& L, size_t bytes) {
    if (bytes <= L.stage_bytes) return SWE_OK;
    SWE_CHECK_CUDA(cudaStreamSynchronize(L.st));
    cudaFree(L.stage_in);
    cudaFree(L.stage_out);
    L.stage_in = L.stage_out = nullptr;
    L.stage_bytes = 0;
    SWE_CHECK_CUDA(cudaMalloc((void**)&L.stage_in, bytes));
    SWE_CHECK_CUDA(cudaMalloc((void**)&L.stage_out, bytes));
    L.stage_bytes = bytes;
    return SWE_OK;
}

// device memory charged to a request: its own state, staging for its slices (two buffers)
// and the plan workspace its propagations claim (batches are chunked, so at most one chunk's
// worth per plan; the workspace is shared by the plan's requests, so this is an upper bound)
static size_t request_bytes(const swe_request_desc& d, int64_t per) {
    const size_t st = sizeof(double2) * per;
    const size_t stage = 2 * st * (size_t)d.S;
    if (d.method == SWE_METHOD_PARAREAL)
        return st * (3 * (size_t)d.S + 1) + 64 + stage + stepper_bytes_chunked(d.fine_plan, d.S) +
               stepper_bytes_chunked(d.coarse_plan, 1);
    // MGRIT with levels (fine, coarse): all time points of both levels plus transfer arrays,
    // and the relaxation workspaces of both levels (S intervals per batched step)
    const size_t n0 = (size_t)d.S * d.cf;
    const size_t per_c = 3 * (size_t)d.coarse_plan->nc * sizeof(double2);
    return st * (n0 + 1 + (size_t)d.S + 2) + per_c * (4 * ((size_t)d.S + 1)) +
           stepper_bytes_chunked(d.fine_plan, d.S) + stepper_bytes_chunked(d.coarse_plan, d.S);
}

static void free_request(Request& r) {
    cudaFree(r.U);
    cudaFree(r.Fo);
    cudaFree(r.Gold);
    cudaFree(r.red);
    cudaFree(r.u0);
    r.U = r.Fo = r.Gold = r.u0 = nullptr;
    r.red = nullptr;
    if (r.mg) swe_mgrit_destroy(r.mg);
    r.mg = nullptr;
    if (r.red_host) cudaFreeHost(r.red_host);
    if (r.bits_host) cudaFreeHost(r.bits_host);
    r.red_host = nullptr;
    r.bits_host = nullptr;
}

// device buffers; the initial guess is computed later in the tick (batched per group for
// Parareal, swe_mgrit_init for MGRIT), on the request's lane
static swe_status admit_alloc(Request& r) {
    const size_t st = sizeof(double2) * r.per;
    SWE_CHECK_CUDA(cudaHostAlloc((void**)&r.red_host, sizeof(unsigned long long) * 6, cudaHostAllocDefault));
    SWE_CHECK_CUDA(cudaHostAlloc((void**)&r.bits_host, sizeof(int) * 2, cudaHostAllocDefault));
    memset(r.red_host, 0, sizeof(unsigned long long) * 6);
    memset(r.bits_host, 0, sizeof(int) * 2);
    if (r.d.method == SWE_METHOD_PARAREAL) {
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.U, st * (r.d.S + 1)));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.Fo, st * r.d.S));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.Gold, st * r.d.S));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.red, sizeof(unsigned long long) * 6));
    } else {
        swe_mgrit_desc md{};
        md.L = 2;
        md.cf = r.d.cf;
        md.nu = r.d.nu_relax;
        md.N0 = r.d.S * r.d.cf;
        md.cycle = 1;
        md.plan[0] = r.d.fine_plan;
        md.plan[1] = r.d.coarse_plan;
        md.step[0] = r.d.fine;
        md.step[1] = r.d.coarse;
        SWE_CHECK(swe_mgrit_create(&md, &r.mg));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.u0, st));
    }
    return SWE_OK;
}

// a finished request leaves its slot; its device memory stays charged to the budget until the
// result is fetched (swe_server_result)
static void finish(swe_server* s, Request& r, double t) {
    r.status = 2;
    r.t_done = t;
    s->n_active -= 1;
}

// initial guess of newly admitted Parareal requests of one group, batched: U_{n+1} = G(U_n)
static swe_status parareal_group_init(Lane& L, std::vector<Request*>& g) {
    const swe_request_desc& d = g[0]->d;
    const int64_t per = g[0]->per;
    const size_t st = sizeof(double2) * per;
    int maxS = 0;
    for (Request* r : g) maxS = std::max(maxS, r->d.S);
    SWE_CHECK(ensure_stage(L, st * g.size()));
    for (Request* r : g) SWE_CHECK_CUDA(cudaMemcpyAsync(r->U, r->U0.data(), st, cudaMemcpyHostToDevice, L.st));
    std::vector<Request*> at;
    for (int n = 0; n < maxS; ++n) {
        at.clear();
        for (Request* r : g)
            if (r->d.S > n) at.push_back(r);
        for (size_t i = 0; i < at.size(); ++i)
            SWE_CHECK_CUDA(cudaMemcpyAsync(L.stage_in + per * i, at[i]->U + per * n, st, cudaMemcpyDeviceToDevice,
                                           L.st));
        SWE_CHECK(propagate_G(d.coarse_plan, d.fine_plan, &d.coarse, (const double*)L.stage_in,
                              (double*)L.stage_out, (int)at.size(), L.st));
        for (size_t i = 0; i < at.size(); ++i) {
            SWE_CHECK_CUDA(cudaMemcpyAsync(at[i]->Gold + per * n, L.stage_out + per * i, st, cudaMemcpyDeviceToDevice,
                                           L.st));
            SWE_CHECK_CUDA(cudaMemcpyAsync(at[i]->U + per * (n + 1), L.stage_out + per * i, st,
                                           cudaMemcpyDeviceToDevice, L.st));
        }
    }
    return SWE_OK;
}

// one Parareal iteration for every request of one group, batched
static swe_status parareal_group_tick(Lane& L, std::vector<Request*>& g) {
    const swe_request_desc& d = g[0]->d;
    const int64_t per = g[0]->per;
    const size_t st = sizeof(double2) * per;
    int total = 0, maxS = 0;
    for (Request* r : g) {
        total += r->d.S;
        maxS = std::max(maxS, r->d.S);
    }
    SWE_CHECK(ensure_stage(L, st * total));
    // fine propagation of all slices of all requests in one call
    int off = 0;
    for (Request* r : g) {
        SWE_CHECK_CUDA(cudaMemcpyAsync(L.stage_in + per * off, r->U, st * r->d.S, cudaMemcpyDeviceToDevice, L.st));
        off += r->d.S;
    }
    SWE_CHECK(propagate_F(d.fine_plan, &d.fine, (const double*)L.stage_in, (double*)L.stage_out, total, L.st));
    off = 0;
    for (Request* r : g) {
        SWE_CHECK_CUDA(cudaMemcpyAsync(r->Fo, L.stage_out + per * off, st * r->d.S, cudaMemcpyDeviceToDevice, L.st));
        SWE_CHECK_CUDA(cudaMemsetAsync(r->red, 0, sizeof(unsigned long long) * 6, L.st));
        off += r->d.S;
    }
    // coarse chains, advanced together: one batched coarse step per chain position
    std::vector<Request*> at;
    for (int n = 0; n < maxS; ++n) {
        at.clear();
        for (Request* r : g)
            if (r->d.S > n) at.push_back(r);
        for (size_t i = 0; i < at.size(); ++i)
            SWE_CHECK_CUDA(cudaMemcpyAsync(L.stage_in + per * i, at[i]->U + per * n, st, cudaMemcpyDeviceToDevice,
                                           L.st));
        SWE_CHECK(propagate_G(d.coarse_plan, d.fine_plan, &d.coarse, (const double*)L.stage_in,
                              (double*)L.stage_out, (int)at.size(), L.st));
        for (size_t i = 0; i < at.size(); ++i) {
            Request* r = at[i];
            SWE_CHECK(parareal_correct_launch(L.stage_out + per * i, r->Fo + per * n, r->Gold + per * n,
                                              r->U + per * (n + 1), d.fine_plan->nc, r->red, d.fine_plan->flags,
                                              L.st));
        }
    }
    for (Request* r : g)
        SWE_CHECK_CUDA(cudaMemcpyAsync(r->red_host, r->red, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToHost,
                                       L.st));
    return SWE_OK;
}

// lanes: connected components of the "shares a plan" relation among the given requests
static std::vector<std::vector<Request*>> make_lanes(const std::vector<Request*>& act) {
    const int n = (int)act.size();
    std::vector<int> parent(n);
    for (int i = 0; i < n; ++i) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const swe_request_desc &a = act[i]->d, &b = act[j]->d;
            if (a.fine_plan == b.fine_plan || a.fine_plan == b.coarse_plan || a.coarse_plan == b.fine_plan ||
                a.coarse_plan == b.coarse_plan)
                parent[find(i)] = find(j);
        }
    std::map<int, std::vector<Request*>> comp;
    for (int i = 0; i < n; ++i) comp[find(i)].push_back(act[i]);
    std::vector<std::vector<Request*>> out;
    for (auto& kv : comp) out.push_back(kv.second);
    return out;
}

// enqueue one tick of one lane on its stream (no host synchronisation)
static swe_status lane_tick(Lane& L, std::vector<Request*>& lane) {
    // status words of this lane's plans: cleared first, read back after its work
    std::vector<swe_plan*> plans;
    for (Request* r : lane)
        for (swe_plan* q : {r->d.fine_plan, r->d.coarse_plan})
            if (std::find(plans.begin(), plans.end(), q) == plans.end()) plans.push_back(q);
    for (swe_plan* q : plans) SWE_CHECK(plan_flags_clear(q, L.st));
    // Parareal groups; fresh members first get their batched initial coarse chains
    std::vector<std::vector<Request*>> groups;
    for (Request* r : lane) {
        if (r->d.method != SWE_METHOD_PARAREAL) continue;
        bool placed = false;
        for (auto& g : groups)
            if (same_group(g[0]->d, r->d)) {
                g.push_back(r);
                placed = true;
                break;
            }
        if (!placed) groups.push_back({r});
    }
    for (auto& g : groups) {
        std::vector<Request*> fresh;
        for (Request* r : g)
            if (r->fresh) fresh.push_back(r);
        if (!fresh.empty()) SWE_CHECK(parareal_group_init(L, fresh));
        SWE_CHECK(parareal_group_tick(L, g));
    }
    // MGRIT requests: initial guess for fresh ones, then one cycle each
    for (Request* r : lane) {
        if (r->d.method != SWE_METHOD_MGRIT2) continue;
        if (r->fresh) {
            SWE_CHECK_CUDA(
                cudaMemcpyAsync(r->u0, r->U0.data(), sizeof(double2) * r->per, cudaMemcpyHostToDevice, L.st));
            SWE_CHECK(swe_mgrit_init(r->mg, (const double*)r->u0, L.st));
        }
        SWE_CHECK(mgrit_cycle_enqueue(r->mg, L.st, r->red_host, r->bits_host));
    }
    for (Request* r : lane)
        if (r->d.method == SWE_METHOD_PARAREAL) {
            SWE_CHECK(plan_flags_fetch(r->d.fine_plan, &r->bits_host[0], L.st));
            SWE_CHECK(plan_flags_fetch(r->d.coarse_plan, &r->bits_host[1], L.st));
        }
    return SWE_OK;
}

extern "C" swe_status swe_request_bytes(const swe_request_desc* d, size_t* bytes) {
    if (!d || !bytes || !d->fine_plan || !d->coarse_plan || d->S < 1 ||
        (d->method == SWE_METHOD_MGRIT2 && d->cf < 2)) {
        swe_set_error("swe_request_bytes: invalid request");
        return SWE_EINVAL;
    }
    *bytes = request_bytes(*d, 3 * d->fine_plan->nc);
    return SWE_OK;
}

extern "C" swe_status swe_server_create(const swe_server_desc* d, swe_server_t* out) {
    if (!d || !out || d->max_active < 1) {
        swe_set_error("swe_server_create: invalid descriptor");
        return SWE_EINVAL;
    }
    swe_server* s = new swe_server();
    s->d = *d;
    const swe_status st = lane_get(s, 1);
    if (st != SWE_OK) {
        delete s;
        return st;
    }
    *out = s;
    return SWE_OK;
}

extern "C" swe_status swe_server_destroy(swe_server_t s) {
    if (!s) return SWE_OK;
    for (auto& L : s->lanes) cudaStreamSynchronize(L.st);
    for (auto& kv : s->reqs) free_request(*kv.second);
    for (auto& L : s->lanes) {
        cudaFree(L.stage_in);
        cudaFree(L.stage_out);
        cudaStreamDestroy(L.st);
    }
    delete s;
    return SWE_OK;
}

extern "C" swe_status swe_server_submit(swe_server_t s, const swe_request_desc* d, long long* id) {
    if (!s || !d || !id || !d->fine_plan || !d->coarse_plan || !d->U0_host || d->S < 1 || d->iters < 1) {
        swe_set_error("swe_server_submit: invalid request");
        return SWE_EINVAL;
    }
    if (d->method != SWE_METHOD_PARAREAL && d->method != SWE_METHOD_MGRIT2) {
        swe_set_error("swe_server_submit: unknown method %d", d->method);
        return SWE_EINVAL;
    }
    if (d->method == SWE_METHOD_MGRIT2 && d->cf < 2) {
        swe_set_error("swe_server_submit: MGRIT requests need cf >= 2");
        return SWE_EINVAL;
    }
    if (d->coarse_plan->M > d->fine_plan->M) {
        swe_set_error("swe_server_submit: coarse truncation must not exceed the fine one");
        return SWE_EINVAL;
    }
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->d = *d;
    r->per = 3 * d->fine_plan->nc;
    r->bytes = request_bytes(*d, r->per);
    if (r->bytes > s->d.hbm_budget_bytes) {
        swe_set_error("swe_server_submit: request needs %zu bytes, more than the %zu-byte budget", r->bytes,
                      s->d.hbm_budget_bytes);
        return SWE_EINVAL;
    }
    r->U0.assign((const double2*)d->U0_host, (const double2*)d->U0_host + r->per);
    r->t_submit = now_s();
    *id = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    return SWE_OK;
}

extern "C" swe_status swe_server_step(swe_server_t s, int* n_active, int* n_queued, int* n_done_now) {
    if (!s) {
        swe_set_error("swe_server_step: NULL server");
        return SWE_EINVAL;
    }
    // admission (FIFO) by slot limit and device-memory budget
    while (!s->queue.empty() && s->n_active < s->d.max_active) {
        Request& r = *s->reqs[s->queue.front()];
        if (s->bytes_active + r.bytes > s->d.hbm_budget_bytes) break;
        s->queue.pop_front();
        const swe_status e = admit_alloc(r);
        if (e != SWE_OK) {
            r.status = 3;
            free_request(r);
            return e;
        }
        s->bytes_active += r.bytes;
        s->n_active += 1;
        r.status = 1;
        r.fresh = true;
        r.t_admit = now_s();
    }
    std::vector<Request*> act;
    for (auto& kv : s->reqs)
        if (kv.second->status == 1) act.push_back(kv.second.get());
    auto lanes = make_lanes(act);
    SWE_CHECK(lane_get(s, (int)lanes.size()));
    for (size_t li = 0; li < lanes.size(); ++li) SWE_CHECK(lane_tick(s->lanes[li], lanes[li]));
    // one synchronisation for every lane
    for (size_t li = 0; li < lanes.size(); ++li) SWE_CHECK_CUDA(cudaStreamSynchronize(s->lanes[li].st));
    const double t = now_s();
    int done = 0;
    int bits = 0;
    for (Request* r : act) {
        std::vector<double2>().swap(r->U0);
        r->fresh = false;
        bits |= r->bits_host[0] | r->bits_host[1];
        r->norms.push_back(norm_of(r->red_host));
        if (++r->iters_done >= r->d.iters) {
            finish(s, *r, t);
            ++done;
        }
    }
    if (n_active) *n_active = s->n_active;
    if (n_queued) *n_queued = (int)s->queue.size();
    if (n_done_now) *n_done_now = done;
    if (bits) return plan_flags_status(bits, "swe_server_step", 0);
    return SWE_OK;
}

extern "C" swe_status swe_server_result(swe_server_t s, long long id, double* U_host, double* timing_host) {
    if (!s || s->reqs.find(id) == s->reqs.end()) {
        swe_set_error("swe_server_result: unknown request %lld", id);
        return SWE_EINVAL;
    }
    Request& r = *s->reqs[id];
    if (r.status != 2) {
        swe_set_error("swe_server_result: request %lld is not finished", id);
        return SWE_EINVAL;
    }
    if (U_host) {
        if (r.d.method == SWE_METHOD_PARAREAL) {
            SWE_CHECK_CUDA(cudaMemcpy(U_host, r.U, sizeof(double2) * r.per * (r.d.S + 1), cudaMemcpyDeviceToHost));
        } else {
            cudaStream_t st = s->lanes[0].st;
            SWE_CHECK(swe_mgrit_cpoints(r.mg, U_host, st));
            SWE_CHECK_CUDA(cudaStreamSynchronize(st));
        }
    }
    if (timing_host) {
        timing_host[0] = r.t_done - r.t_submit;     // latency
        timing_host[1] = r.t_admit - r.t_submit;    // queueing
        timing_host[2] = (double)r.iters_done;
    }
    free_request(r);
    s->bytes_active -= r.bytes;
    s->reqs.erase(id);
    return SWE_OK;
}

extern "C" swe_status swe_server_norms(swe_server_t s, long long id, double* norms_host, int max_norms, int* n) {
    if (!s || s->reqs.find(id) == s->reqs.end()) {
        swe_set_error("swe_server_norms: unknown request %lld", id);
        return SWE_EINVAL;
    }
    Request& r = *s->reqs[id];
    const int k = std::min<int>(max_norms, (int)r.norms.size());
    for (int i = 0; i < k && norms_host; ++i) norms_host[i] = r.norms[i];
    if (n) *n = (int)r.norms.size();
    return SWE_OK;
}
