// Parareal (§3.1, Eq. 9) on one GPU: the fine propagator runs on all S slices
// at once (one batched propagate_F), the coarse chain runs serially, the whole
// iteration is captured once into a CUDA graph and replayed, and the FP64 correction
// U^{k+1}_{n+1} = G(U^{k+1}_n) + F(U^k_n) - G(U^k_n) is fused with the
// per-field convergence norm.
#include <cstring>

#include "swe_internal.cuh"

struct swe_pint {
    swe_pint_desc d;
    int64_t nc = 0;
    double2* U = nullptr;      // [S+1][3][NC] current iterate
    double2* Fo = nullptr;     // [S][3][NC]   phi_f(U^k_n)
    double2* Gold = nullptr;   // [S][3][NC]   phi_c(U^k_n)
    double2* Gnew = nullptr;   // [3][NC]      phi_c(U^{k+1}_n)
    unsigned long long* red = nullptr;   // [6] max |dU_f|, max |U_f| (double bits)
    cudaStream_t cs = nullptr;
    // the whole iteration (fine sweep over all slices, serial coarse chain, corrections),
    // captured into one CUDA graph after one uncaptured iteration has sized every buffer
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_launches = 0;   // kernels per replay of the captured iteration
    bool ready = false;
    int passes = 0;                 // uncaptured iterations so far
    bool off = false;               // capture failed: stay uncaptured
    unsigned long long gen_f = 0, gen_c = 0;   // plan generations the graph was captured at
};

namespace {

__device__ __forceinline__ double cabs_inf(double2 v) { return fmax(fabs(v.x), fabs(v.y)); }

// Unext <- G + F - Gold ; Gold <- G ; reduce max |Unext_new - Unext_old| and max |Unext_new| per field
__global__ void k_parareal_correct(const double2* __restrict__ G, const double2* __restrict__ F,
                                   double2* __restrict__ Gold, double2* __restrict__ Unext, int64_t nc,
                                   unsigned long long* red, int* flags) {
    __shared__ double sd[3][8], sv[3][8];
    double md[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
    const int64_t n = 3 * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 g = G[i], f = F[i], go = Gold[i], uo = Unext[i];
        double2 u = make_double2(g.x + f.x - go.x, g.y + f.y - go.y);
        if (!isfinite(u.x) || !isfinite(u.y)) atomicOr(flags, 1);
        Unext[i] = u;
        Gold[i] = g;
        int fld = (int)(i / nc);
        double dd = cabs_inf(make_double2(u.x - uo.x, u.y - uo.y));
        double vv = cabs_inf(u);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (q == fld) {
                md[q] = fmax(md[q], dd);
                mv[q] = fmax(mv[q], vv);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) {
            md[q] = fmax(md[q], __shfl_xor_sync(0xffffffffu, md[q], o));
            mv[q] = fmax(mv[q], __shfl_xor_sync(0xffffffffu, mv[q], o));
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < 3; ++q) {
            sd[q][warp] = md[q];
            sv[q][warp] = mv[q];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        int q = threadIdx.x;
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmax(a, sd[q][w]);
            b = fmax(b, sv[q][w]);
        }
        // non-negative doubles order like their bit patterns
        atomicMax(&red[q], (unsigned long long)__double_as_longlong(a));
        atomicMax(&red[3 + q], (unsigned long long)__double_as_longlong(b));
    }
}

}  // namespace

// Parareal correction of one slice boundary (used by the serving loop as well):
// Unext <- G + F - Gold, Gold <- G, per-field max-norm reduction into red[6].
swe_status parareal_correct_launch(const double2* G, const double2* F, double2* Gold, double2* Unext, int64_t nc,
                                   unsigned long long* red, int* flags, cudaStream_t st) {
    const int64_t per = 3 * nc;
    k_parareal_correct<<<(unsigned)((per + 255) / 256 < 1184 ? (per + 255) / 256 : 1184), 256, 0, st>>>(
        G, F, Gold, Unext, nc, red, flags);
    SWE_CHECK_LAUNCH("k_parareal_correct");
    return SWE_OK;
}

extern "C" swe_status swe_pint_create(const swe_pint_desc* d, swe_pint_t* out) {
    if (!d || !out || !d->fine_plan || !d->coarse_plan || d->S < 1) {
        swe_set_error("swe_pint_create: invalid descriptor");
        return SWE_EINVAL;
    }
    if (d->coarse_plan->M > d->fine_plan->M) {
        swe_set_error("swe_pint_create: coarse truncation must not exceed the fine one");
        return SWE_EINVAL;
    }
    swe_pint* p = new swe_pint();
    p->d = *d;
    p->nc = d->fine_plan->nc;
    const size_t st = sizeof(double2) * 3 * p->nc;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->U, st * (d->S + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->Fo, st * d->S);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->Gold, st * d->S);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->Gnew, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->red, sizeof(unsigned long long) * 6);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        swe_pint_destroy(p);
        return swe_cuda_status(e, "swe_pint_create");
    }
    *out = p;
    return SWE_OK;
}

extern "C" swe_status swe_pint_destroy(swe_pint_t p) {
    if (!p) return SWE_OK;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cs) cudaStreamDestroy(p->cs);
    cudaFree(p->U);
    cudaFree(p->Fo);
    cudaFree(p->Gold);
    cudaFree(p->Gnew);
    cudaFree(p->red);
    delete p;
    return SWE_OK;
}

static swe_status coarse(swe_pint* p, const double2* in, double2* out) {
    return propagate_G(p->d.coarse_plan, p->d.fine_plan, &p->d.coarse, (const double*)in, (double*)out, 1, p->cs);
}

static swe_status join_user_stream(swe_pint* p, cudaStream_t user) {
    cudaEvent_t ev;
    SWE_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SWE_CHECK_CUDA(cudaEventRecord(ev, p->cs));
    SWE_CHECK_CUDA(cudaStreamWaitEvent(user, ev, 0));
    cudaEventDestroy(ev);
    return SWE_OK;
}

static swe_status wait_user_stream(swe_pint* p, cudaStream_t user) {
    cudaEvent_t ev;
    SWE_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SWE_CHECK_CUDA(cudaEventRecord(ev, user));
    SWE_CHECK_CUDA(cudaStreamWaitEvent(p->cs, ev, 0));
    cudaEventDestroy(ev);
    return SWE_OK;
}

extern "C" swe_status swe_pint_init(swe_pint_t p, const double* U0, void* stream) {
    if (!p || !U0) {
        swe_set_error("swe_pint_init: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(wait_user_stream(p, user));
    const int64_t per = 3 * p->nc;
    SWE_CHECK_CUDA(cudaMemcpyAsync(p->U, U0, sizeof(double2) * per, cudaMemcpyDeviceToDevice, p->cs));
    for (int n = 0; n < p->d.S; ++n) {
        SWE_CHECK(coarse(p, p->U + per * n, p->Gold + per * n));
        SWE_CHECK_CUDA(cudaMemcpyAsync(p->U + per * (n + 1), p->Gold + per * n, sizeof(double2) * per,
                                       cudaMemcpyDeviceToDevice, p->cs));
    }
    SWE_CHECK(join_user_stream(p, user));
    return SWE_OK;
}

// the serial part of one iteration: G chain + corrections (+ norm reduction)
static swe_status chain(swe_pint* p) {
    const int64_t per = 3 * p->nc;
    SWE_CHECK_CUDA(cudaMemsetAsync(p->red, 0, sizeof(unsigned long long) * 6, p->cs));
    for (int n = 0; n < p->d.S; ++n) {
        SWE_CHECK(coarse(p, p->U + per * n, p->Gnew));
        k_parareal_correct<<<(unsigned)((per + 255) / 256 < 1184 ? (per + 255) / 256 : 1184), 256, 0, p->cs>>>(
            p->Gnew, p->Fo + per * n, p->Gold + per * n, p->U + per * (n + 1), p->nc, p->red,
            p->d.fine_plan->flags);
        SWE_CHECK_LAUNCH("k_parareal_correct");
    }
    return SWE_OK;
}

// one iteration: the fine propagator on every slice at once, then the serial chain
static swe_status iteration_body(swe_pint* p) {
    SWE_CHECK(propagate_F(p->d.fine_plan, &p->d.fine, (const double*)p->U, (double*)p->Fo, p->d.S, p->cs));
    return chain(p);
}

extern "C" swe_status parareal_iterate(swe_pint_t p, int kmax, double tol, int* k_done, double* norm_hist,
                                       void* stream) {
    if (!p || kmax < 0) {
        swe_set_error("parareal_iterate: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(wait_user_stream(p, user));
    SWE_CHECK(plan_flags_clear(p->d.fine_plan, p->cs));
    if (p->d.coarse_plan != p->d.fine_plan) SWE_CHECK(plan_flags_clear(p->d.coarse_plan, p->cs));
    const int S = p->d.S;
    int k = 0;
    swe_status status = SWE_OK;
    for (; k < kmax; ++k) {
        if (p->d.use_graphs && !prof_enabled()) {
            if (p->ready && (p->gen_f != p->d.fine_plan->gen || p->gen_c != p->d.coarse_plan->gen)) {
                // a plan buffer the graph points into was reallocated: capture again
                SWE_CHECK_CUDA(cudaStreamSynchronize(p->cs));
                cudaGraphExecDestroy(p->gexec);
                cudaGraphDestroy(p->graph);
                p->gexec = nullptr;
                p->graph = nullptr;
                p->ready = false;
                p->passes = 0;
            }
            if (!p->ready && (p->off || p->passes < 1)) {
                p->passes += 1;
                SWE_CHECK(iteration_body(p));
            } else {
                if (!p->ready) {
                    const long long before = swe_launch_count();
                    const unsigned long long gf = p->d.fine_plan->gen, gc = p->d.coarse_plan->gen;
                    SWE_CHECK_CUDA(cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeThreadLocal));
                    const swe_status s = iteration_body(p);
                    cudaGraph_t g = nullptr;
                    const cudaError_t e = cudaStreamEndCapture(p->cs, &g);
                    // captured launches did not execute: count them at each replay instead
                    p->graph_launches = swe_launch_count() - before;
                    prof_launch(-p->graph_launches);
                    if (s != SWE_OK || e != cudaSuccess || gf != p->d.fine_plan->gen ||
                        gc != p->d.coarse_plan->gen) {
                        // not capturable as it stands: run uncaptured from now on
                        if (g) cudaGraphDestroy(g);
                        cudaGetLastError();
                        p->off = true;
                        SWE_CHECK(iteration_body(p));
                    } else {
                        p->graph = g;
                        SWE_CHECK_CUDA(cudaGraphInstantiate(&p->gexec, g, 0));
                        p->ready = true;
                        p->gen_f = gf;
                        p->gen_c = gc;
                    }
                }
                if (p->ready) {
                    SWE_CHECK_CUDA(cudaGraphLaunch(p->gexec, p->cs));
                    prof_launch(p->graph_launches);
                }
            }
        } else {
            SWE_CHECK(iteration_body(p));
        }
        unsigned long long red[6];
        SWE_CHECK_CUDA(cudaMemcpyAsync(red, p->red, sizeof(red), cudaMemcpyDeviceToHost, p->cs));
        int flag = 0, flag_c = 0;
        SWE_CHECK(plan_flags_fetch(p->d.fine_plan, &flag, p->cs));
        if (p->d.coarse_plan != p->d.fine_plan) SWE_CHECK(plan_flags_fetch(p->d.coarse_plan, &flag_c, p->cs));
        SWE_CHECK_CUDA(cudaStreamSynchronize(p->cs));
        flag |= flag_c;
        double nrm = 0.0;
        for (int q = 0; q < 3; ++q) {
            double dd, vv;
            memcpy(&dd, &red[q], sizeof(double));
            memcpy(&vv, &red[3 + q], sizeof(double));
            if (vv > 0) nrm = fmax(nrm, dd / vv);
        }
        if (norm_hist) norm_hist[k] = nrm;
        if (flag) {
            status = plan_flags_status(flag, "parareal_iterate", k + 1);
            // the condition is reported: leave the status words clear for the next call
            SWE_CHECK(plan_flags_clear(p->d.fine_plan, p->cs));
            if (p->d.coarse_plan != p->d.fine_plan) SWE_CHECK(plan_flags_clear(p->d.coarse_plan, p->cs));
            ++k;
            break;
        }
        if (tol > 0.0 && nrm < tol) {
            ++k;
            break;
        }
    }
    if (k_done) *k_done = k;
    SWE_CHECK(join_user_stream(p, user));
    return status;
}

extern "C" swe_status swe_pint_solution(swe_pint_t p, double* U_out, void* stream) {
    if (!p || !U_out) {
        swe_set_error("swe_pint_solution: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(wait_user_stream(p, user));
    SWE_CHECK_CUDA(cudaMemcpyAsync(U_out, p->U, sizeof(double2) * 3 * p->nc * (p->d.S + 1), cudaMemcpyDeviceToDevice,
                                   p->cs));
    SWE_CHECK(join_user_stream(p, user));
    return SWE_OK;
}

// Checkpoint / resume of the Parareal state (U^k_n, n = 0..S, and phi_c(U^k_n)).
// Pointers may be host (pageable or pinned) or device memory.
extern "C" swe_status swe_pint_load(swe_pint_t p, const double* U, const double* Gold, void* stream) {
    if (!p || !U) {
        swe_set_error("swe_pint_load: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(wait_user_stream(p, user));
    const int64_t per = 3 * p->nc;
    SWE_CHECK_CUDA(cudaMemcpyAsync(p->U, U, sizeof(double2) * per * (p->d.S + 1), cudaMemcpyDefault, p->cs));
    if (Gold) {
        SWE_CHECK_CUDA(cudaMemcpyAsync(p->Gold, Gold, sizeof(double2) * per * p->d.S, cudaMemcpyDefault, p->cs));
    } else {
        for (int n = 0; n < p->d.S; ++n) SWE_CHECK(coarse(p, p->U + per * n, p->Gold + per * n));
    }
    SWE_CHECK(join_user_stream(p, user));
    return SWE_OK;
}

extern "C" swe_status swe_pint_save(swe_pint_t p, double* U, double* Gold, void* stream) {
    if (!p || !U) {
        swe_set_error("swe_pint_save: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(wait_user_stream(p, user));
    const int64_t per = 3 * p->nc;
    SWE_CHECK_CUDA(cudaMemcpyAsync(U, p->U, sizeof(double2) * per * (p->d.S + 1), cudaMemcpyDefault, p->cs));
    if (Gold)
        SWE_CHECK_CUDA(cudaMemcpyAsync(Gold, p->Gold, sizeof(double2) * per * p->d.S, cudaMemcpyDefault, p->cs));
    SWE_CHECK(join_user_stream(p, user));
    return SWE_OK;
}
