// Continuous-batching forecast server.
//
// A request is a Parareal (§3.1, Eq. 9) or MGRIT (§3.2) solve of one initial
// state.  Requests wait in a FIFO queue and are admitted at the start of a
// tick while the device-memory budget and the slot limit allow.  Every tick
// advances every active request by one iteration:
//  * Parareal requests that share plans and steppers are batched into the same
//    launches: the fine propagation of all their slices is ONE propagate call,
//    and their serial coarse chains advance together, one batched coarse step
//    per chain position, followed by each request's FP64 correction.  Requests
//    admitted later join the batch at the next tick (continuous batching).
//  * MGRIT requests run one cycle each.
// A request's spectral state stays in device memory from admission to
// completion; results are copied out on request.  Every kernel acts on each
// state column independently, so a request's result does not depend on which
// other requests share its launches.
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
    size_t bytes = 0;             // device memory held while active
    std::vector<double2> U0;      // host copy until admission
    // Parareal state
    double2* U = nullptr;         // [S+1]
    double2* Fo = nullptr;        // [S]
    double2* Gold = nullptr;      // [S]
    unsigned long long* red = nullptr;
    // MGRIT state
    swe_mgrit_t mg = nullptr;
    int iters_done = 0;
    int status = 0;               // 0 queued, 1 active, 2 done, 3 failed
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<double> norms;
};

bool same_group(const swe_request_desc& a, const swe_request_desc& b) {
    return a.fine_plan == b.fine_plan && a.coarse_plan == b.coarse_plan &&
           memcmp(&a.fine, &b.fine, sizeof(a.fine)) == 0 && memcmp(&a.coarse, &b.coarse, sizeof(a.coarse)) == 0;
}

}  // namespace

struct swe_server {
    swe_server_desc d{};
    long long next_id = 1;
    std::deque<long long> queue;
    std::map<long long, std::unique_ptr<Request>> reqs;
    size_t bytes_active = 0;
    int n_active = 0;
    cudaStream_t st = nullptr;
    double2* stage_in = nullptr;
    double2* stage_out = nullptr;
    size_t stage_bytes = 0;
};

static swe_status ensure_stage(swe_server* s, size_t bytes) {
    if (bytes <= s->stage_bytes) return SWE_OK;
    SWE_CHECK_CUDA(cudaStreamSynchronize(s->st));
    cudaFree(s->stage_in);
    cudaFree(s->stage_out);
    s->stage_in = s->stage_out = nullptr;
    s->stage_bytes = 0;
    SWE_CHECK_CUDA(cudaMalloc((void**)&s->stage_in, bytes));
    SWE_CHECK_CUDA(cudaMalloc((void**)&s->stage_out, bytes));
    s->stage_bytes = bytes;
    return SWE_OK;
}

static size_t request_bytes(const swe_request_desc& d, int64_t per) {
    const size_t st = sizeof(double2) * per;
    if (d.method == SWE_METHOD_PARAREAL) return st * (3 * (size_t)d.S + 1) + 64;
    // MGRIT with levels (fine, coarse): all time points of both levels plus transfer arrays
    const size_t n0 = (size_t)d.S * d.cf;
    return st * (n0 + 1 + 4 * ((size_t)d.S + 1) + (size_t)d.S);
}

static swe_status admit(swe_server* s, Request& r) {
    const int64_t per = r.per;
    const size_t st = sizeof(double2) * per;
    if (r.d.method == SWE_METHOD_PARAREAL) {
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.U, st * (r.d.S + 1)));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.Fo, st * r.d.S));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.Gold, st * r.d.S));
        SWE_CHECK_CUDA(cudaMalloc((void**)&r.red, sizeof(unsigned long long) * 6));
        SWE_CHECK_CUDA(cudaMemcpyAsync(r.U, r.U0.data(), st, cudaMemcpyHostToDevice, s->st));
        // initial guess: serial coarse chain U_{n+1} = G(U_n), Gold_n = U_{n+1}
        for (int n = 0; n < r.d.S; ++n) {
            SWE_CHECK(propagate_G(r.d.coarse_plan, r.d.fine_plan, &r.d.coarse, (const double*)(r.U + per * n),
                                  (double*)(r.Gold + per * n), 1, s->st));
            SWE_CHECK_CUDA(
                cudaMemcpyAsync(r.U + per * (n + 1), r.Gold + per * n, st, cudaMemcpyDeviceToDevice, s->st));
        }
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
        double2* u0;
        SWE_CHECK_CUDA(cudaMalloc((void**)&u0, st));
        SWE_CHECK_CUDA(cudaMemcpyAsync(u0, r.U0.data(), st, cudaMemcpyHostToDevice, s->st));
        swe_status e = swe_mgrit_init(r.mg, (const double*)u0, s->st);
        SWE_CHECK_CUDA(cudaStreamSynchronize(s->st));
        cudaFree(u0);
        SWE_CHECK(e);
    }
    std::vector<double2>().swap(r.U0);
    r.status = 1;
    r.t_admit = now_s();
    return SWE_OK;
}

// a finished request leaves its slot; its device memory stays counted against the
// budget until the result is fetched (swe_server_result)
static void finish(swe_server* s, Request& r, double t) {
    r.status = 2;
    r.t_done = t;
    s->n_active -= 1;
}

// one Parareal iteration for every active Parareal request of one group, batched
static swe_status parareal_group_tick(swe_server* s, std::vector<Request*>& g) {
    const swe_request_desc& d = g[0]->d;
    const int64_t per = g[0]->per;
    const size_t st = sizeof(double2) * per;
    int total = 0, maxS = 0;
    for (Request* r : g) {
        total += r->d.S;
        maxS = std::max(maxS, r->d.S);
    }
    SWE_CHECK(ensure_stage(s, st * total));
    // fine propagation of all slices of all requests in one call
    int off = 0;
    for (Request* r : g) {
        SWE_CHECK_CUDA(cudaMemcpyAsync(s->stage_in + per * off, r->U, st * r->d.S, cudaMemcpyDeviceToDevice, s->st));
        off += r->d.S;
    }
    SWE_CHECK(propagate_F(d.fine_plan, &d.fine, (const double*)s->stage_in, (double*)s->stage_out, total, s->st));
    off = 0;
    for (Request* r : g) {
        SWE_CHECK_CUDA(cudaMemcpyAsync(r->Fo, s->stage_out + per * off, st * r->d.S, cudaMemcpyDeviceToDevice, s->st));
        SWE_CHECK_CUDA(cudaMemsetAsync(r->red, 0, sizeof(unsigned long long) * 6, s->st));
        off += r->d.S;
    }
    // coarse chains, advanced together: one batched coarse step per chain position
    std::vector<Request*> at;
    for (int n = 0; n < maxS; ++n) {
        at.clear();
        for (Request* r : g)
            if (r->d.S > n) at.push_back(r);
        for (size_t i = 0; i < at.size(); ++i)
            SWE_CHECK_CUDA(cudaMemcpyAsync(s->stage_in + per * i, at[i]->U + per * n, st, cudaMemcpyDeviceToDevice,
                                           s->st));
        SWE_CHECK(propagate_G(d.coarse_plan, d.fine_plan, &d.coarse, (const double*)s->stage_in,
                              (double*)s->stage_out, (int)at.size(), s->st));
        for (size_t i = 0; i < at.size(); ++i) {
            Request* r = at[i];
            SWE_CHECK(parareal_correct_launch(s->stage_out + per * i, r->Fo + per * n, r->Gold + per * n,
                                              r->U + per * (n + 1), d.fine_plan->nc, r->red, d.fine_plan->flags,
                                              s->st));
        }
    }
    return SWE_OK;
}

extern "C" swe_status swe_server_create(const swe_server_desc* d, swe_server_t* out) {
    if (!d || !out || d->max_active < 1) {
        swe_set_error("swe_server_create: invalid descriptor");
        return SWE_EINVAL;
    }
    swe_server* s = new swe_server();
    s->d = *d;
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return swe_cuda_status(e, "swe_server_create");
    }
    *out = s;
    return SWE_OK;
}

extern "C" swe_status swe_server_destroy(swe_server_t s) {
    if (!s) return SWE_OK;
    cudaStreamSynchronize(s->st);
    for (auto& kv : s->reqs) {
        Request& r = *kv.second;
        cudaFree(r.U);
        cudaFree(r.Fo);
        cudaFree(r.Gold);
        cudaFree(r.red);
        if (r.mg) swe_mgrit_destroy(r.mg);
    }
    cudaFree(s->stage_in);
    cudaFree(s->stage_out);
    cudaStreamDestroy(s->st);
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
        s->bytes_active += r.bytes;
        s->n_active += 1;
        swe_status e = admit(s, r);
        if (e != SWE_OK) {
            r.status = 3;
            s->n_active -= 1;
            return e;
        }
    }
    // group the active Parareal requests by plans and steppers
    std::vector<std::vector<Request*>> groups;
    std::vector<Request*> mg;
    for (auto& kv : s->reqs) {
        Request* r = kv.second.get();
        if (r->status != 1) continue;
        if (r->d.method == SWE_METHOD_MGRIT2) {
            mg.push_back(r);
            continue;
        }
        bool placed = false;
        for (auto& g : groups)
            if (same_group(g[0]->d, r->d)) {
                g.push_back(r);
                placed = true;
                break;
            }
        if (!placed) groups.push_back({r});
    }
    // status words of the Parareal groups' plans: cleared before their launches and read back
    // before any MGRIT cycle (which clears the words of its own plans) runs on the stream
    std::vector<swe_plan*> pplans;
    for (auto& g : groups)
        for (swe_plan* q : {g[0]->d.fine_plan, g[0]->d.coarse_plan})
            if (std::find(pplans.begin(), pplans.end(), q) == pplans.end()) pplans.push_back(q);
    std::vector<int> pbits(pplans.size(), 0);
    for (swe_plan* q : pplans) SWE_CHECK(plan_flags_clear(q, s->st));
    for (auto& g : groups) SWE_CHECK(parareal_group_tick(s, g));
    for (size_t i = 0; i < pplans.size(); ++i) SWE_CHECK(plan_flags_fetch(pplans[i], &pbits[i], s->st));
    std::vector<double> mg_norm(mg.size(), 0.0);
    for (size_t i = 0; i < mg.size(); ++i) {
        int k = 0;
        SWE_CHECK(mgrit_cycle(mg[i]->mg, 1, 0.0, &k, &mg_norm[i], s->st));
    }
    SWE_CHECK_CUDA(cudaStreamSynchronize(s->st));
    {
        int bits = 0;
        for (int b : pbits) bits |= b;
        if (bits) {
            for (swe_plan* q : pplans) SWE_CHECK(plan_flags_clear(q, s->st));
            SWE_CHECK_CUDA(cudaStreamSynchronize(s->st));
            return plan_flags_status(bits, "swe_server_step", 0);
        }
    }
    const double t = now_s();
    int done = 0;
    for (auto& g : groups)
        for (Request* r : g) {
            unsigned long long red[6];
            SWE_CHECK_CUDA(cudaMemcpy(red, r->red, sizeof(red), cudaMemcpyDeviceToHost));
            double nrm = 0.0;
            for (int q = 0; q < 3; ++q) {
                double dd, vv;
                memcpy(&dd, &red[q], sizeof(double));
                memcpy(&vv, &red[3 + q], sizeof(double));
                if (vv > 0) nrm = fmax(nrm, dd / vv);
            }
            r->norms.push_back(nrm);
            if (++r->iters_done >= r->d.iters) {
                finish(s, *r, t);
                ++done;
            }
        }
    for (size_t i = 0; i < mg.size(); ++i) {
        Request* r = mg[i];
        r->norms.push_back(mg_norm[i]);
        if (++r->iters_done >= r->d.iters) {
            finish(s, *r, t);
            ++done;
        }
    }
    if (n_active) *n_active = s->n_active;
    if (n_queued) *n_queued = (int)s->queue.size();
    if (n_done_now) *n_done_now = done;
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
            SWE_CHECK(swe_mgrit_cpoints(r.mg, U_host, s->st));
            SWE_CHECK_CUDA(cudaStreamSynchronize(s->st));
        }
    }
    if (timing_host) {
        timing_host[0] = r.t_done - r.t_submit;     // latency
        timing_host[1] = r.t_admit - r.t_submit;    // queueing
        timing_host[2] = (double)r.iters_done;
    }
    // free the request's device state
    cudaFree(r.U);
    cudaFree(r.Fo);
    cudaFree(r.Gold);
    cudaFree(r.red);
    r.U = r.Fo = r.Gold = nullptr;
    r.red = nullptr;
    if (r.mg) swe_mgrit_destroy(r.mg);
    r.mg = nullptr;
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
