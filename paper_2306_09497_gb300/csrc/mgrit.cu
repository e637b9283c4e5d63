// MGRIT (§3.2) on one GPU: full approximation scheme with F(CF)^nu relaxation,
// F-cycle followed by one V-cycle per level (§3.2.3), injection at C-points
// (§3.2.2) and spectral truncation / zero padding between spatial resolutions.
//
// Level l holds all N_l + 1 time points in HBM ([N_l+1][3][NC_l] complex128).
// Every relaxation is ONE batched, strided propagation over all C-intervals of the
// level (F-relaxation: cf - 1 launches of the stepper, each advancing every interval
// by one step); the FAS right-hand side, restriction and correction are fused
// element-wise kernels; only the coarsest level is a serial chain (two-step
// SL-SI-SETTLS there when selected, §3.2.4).
//
// Level system: u_0 = g_0, u_j = Phi_l(u_{j-1}) + g_j (g = 0 on level 0).
// Restriction to level l+1: v_i = R u_{cf i};  g_{l+1,i} = R(g_{cf i} + Phi_l(u_{cf i - 1}) - u_{cf i})
//   + v_i - Phi_{l+1}(v_{i-1});  correction: u_{cf i} += P(u_{l+1,i} - v_i), then F-relaxation.
// Initial guess: serial propagation on the coarsest level, injected upwards with F-relaxation.
#include <cstring>
#include <vector>

#include <algorithm>

#include "swe_internal.cuh"

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

inline unsigned nb(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

// index in a T_Mf state of coarse coefficient r (m, n from the coarse row table)
__device__ __forceinline__ int64_t fine_index(int64_t r, const int* srow_c, int Mc, int Mf) {
    const int m = srow_c[r];
    const int n = m + (int)(r - st_off(m, Mc));
    return st_off(m, Mf) + (n - m);
}

// v_i = R u_f[cf i], i = 0..Nc
__global__ void k_restrict(double2* __restrict__ v, const double2* __restrict__ uf, int cf, int Nc,
                           const int* __restrict__ srow_c, int Mc, int Mf) {
    const int64_t ncc = nc_state(Mc), ncf = nc_state(Mf);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)(Nc + 1) * 3 * ncc) return;
    const int64_t r = t % ncc;
    const int64_t fi = (t / ncc) % 3;
    const int64_t i = t / (3 * ncc);
    v[t] = uf[((int64_t)cf * i * 3 + fi) * ncf + fine_index(r, srow_c, Mc, Mf)];
}

// g_c[i] = R(g_f[cf i] + A[i-1] - u_f[cf i]) + v[i] - B[i-1]  (i >= 1),  g_c[0] = v[0]
__global__ void k_fas_rhs(double2* __restrict__ gc, const double2* __restrict__ v, const double2* __restrict__ B,
                          const double2* __restrict__ uf, const double2* __restrict__ gf,
                          const double2* __restrict__ A, int cf, int Nc, const int* __restrict__ srow_c, int Mc,
                          int Mf) {
    const int64_t ncc = nc_state(Mc), ncf = nc_state(Mf);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)(Nc + 1) * 3 * ncc) return;
    const int64_t r = t % ncc;
    const int64_t fi = (t / ncc) % 3;
    const int64_t i = t / (3 * ncc);
    if (i == 0) {
        gc[t] = v[t];
        return;
    }
    const int64_t fidx = fi * ncf + fine_index(r, srow_c, Mc, Mf);
    const int64_t fpos = (int64_t)cf * i * 3 * ncf + fidx;
    double2 x = csub(A[(i - 1) * 3 * ncf + fidx], uf[fpos]);
    if (gf) x = cadd(x, gf[fpos]);
    gc[t] = csub(cadd(x, v[t]), B[(i - 1) * 3 * ncc + fi * ncc + r]);
}

// u_f[cf i] += P(u_c[i] - v[i]), i = 1..Nc  (zero padding: only coefficients present at T_Mc)
__global__ void k_correct(double2* __restrict__ uf, const double2* __restrict__ uc, const double2* __restrict__ v,
                          int cf, int Nc, const int* __restrict__ srow_c, int Mc, int Mf) {
    const int64_t ncc = nc_state(Mc), ncf = nc_state(Mf);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)Nc * 3 * ncc) return;
    const int64_t r = t % ncc;
    const int64_t fi = (t / ncc) % 3;
    const int64_t i = 1 + t / (3 * ncc);
    const int64_t c = (i * 3 + fi) * ncc + r;
    const int64_t f = ((int64_t)cf * i * 3 + fi) * ncf + fine_index(r, srow_c, Mc, Mf);
    uf[f] = cadd(uf[f], csub(uc[c], v[c]));
}

// u_f[cf i] = P(u_c[i]), i = 1..Nc (initial-guess injection)
__global__ void k_inject(double2* __restrict__ uf, const double2* __restrict__ uc, int cf, int Nc,
                         const int* __restrict__ srow_f, int Mc, int Mf) {
    const int64_t ncc = nc_state(Mc), ncf = nc_state(Mf);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)Nc * 3 * ncf) return;
    const int64_t r = t % ncf;
    const int64_t fi = (t / ncf) % 3;
    const int64_t i = 1 + t / (3 * ncf);
    const int m = srow_f[r];
    const int n = m + (int)(r - st_off(m, Mf));
    double2 val = make_double2(0.0, 0.0);
    if (m <= Mc && n <= Mc) val = uc[(i * 3 + fi) * ncc + st_off(m, Mc) + (n - m)];
    uf[((int64_t)cf * i * 3 + fi) * ncf + r] = val;
}

// spatial truncation / padding of one state (any direction)
__global__ void k_retrunc(const double2* __restrict__ in, int Min, double2* __restrict__ out, int Mout,
                          const int* __restrict__ srow_out) {
    const int64_t nco = nc_state(Mout), nci = nc_state(Min);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * nco) return;
    const int64_t r = t % nco, fi = t / nco;
    const int m = srow_out[r];
    const int n = m + (int)(r - st_off(m, Mout));
    double2 val = make_double2(0.0, 0.0);
    if (m <= Min && n <= Min) val = in[fi * nci + st_off(m, Min) + (n - m)];
    out[t] = val;
}

// per-field max |new - old| and max |new| over the C-points; old <- new
__global__ void k_cnorm(const double2* __restrict__ u, double2* __restrict__ old, int cf, int Nc, int64_t nc,
                        unsigned long long* red, int* flags) {
    const int64_t total = (int64_t)(Nc + 1) * 3 * nc;
    double md[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t % nc;
        const int fld = (int)((t / nc) % 3);
        const int64_t i = t / (3 * nc);
        const double2 a = u[((int64_t)cf * i * 3 + fld) * nc + r];
        const double2 b = old[t];
        if (!isfinite(a.x) || !isfinite(a.y)) atomicOr(flags, 1);
        old[t] = a;
        const double d = fmax(fabs(a.x - b.x), fabs(a.y - b.y));
        const double w = fmax(fabs(a.x), fabs(a.y));
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q == fld) {
                md[q] = fmax(md[q], d);
                mv[q] = fmax(mv[q], w);
            }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) {
            md[q] = fmax(md[q], __shfl_xor_sync(0xffffffffu, md[q], o));
            mv[q] = fmax(mv[q], __shfl_xor_sync(0xffffffffu, mv[q], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&red[q], (unsigned long long)__double_as_longlong(md[q]));
            atomicMax(&red[3 + q], (unsigned long long)__double_as_longlong(mv[q]));
        }
    }
}

}  // namespace

struct MGLevel {
    swe_plan* plan = nullptr;
    swe_stepper_desc sd{};
    int N = 0;
    int64_t per = 0;            // complex values per state
    double2* u = nullptr;       // [N+1]
    double2* g = nullptr;       // [N+1] (levels >= 1)
    double2* v = nullptr;       // [N+1] restricted values (levels >= 1)
    double2* A = nullptr;       // [N_{l+1}] Phi_l(u_{cf i - 1})   (levels < L-1)
    double2* B = nullptr;       // [N] Phi_l(v_{i-1})              (levels >= 1)
    double2* x0 = nullptr;      // initial condition at this resolution
    bool g_on = false;
    bool two_step = false;
    // serial coarsest-level solve, captured into a CUDA graph after one uncaptured pass
    // (which sizes the plan's buffers); one graph per FAS right-hand-side state (g_on)
    struct Graph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long gen = 0;   // plan generation at capture
        long long launches = 0;       // kernels per replay
        int passes = 0;               // uncaptured passes so far
        bool off = false;             // capture failed: stay uncaptured
    } cg[2];
};

struct swe_mgrit {
    swe_mgrit_desc d{};
    std::vector<MGLevel> lv;
    double2* cold = nullptr;    // previous level-0 C-points
    unsigned long long* red = nullptr;
    cudaStream_t cs = nullptr;
    // the whole cycle (every level's relaxations, restrictions, coarse solve and corrections),
    // captured into one CUDA graph after one uncaptured cycle has sized every buffer
    struct CycleGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<unsigned long long> gens;   // generations of the level plans at capture
        long long launches = 0;
        int passes = 0;
        bool off = false;
    } cyc;
    bool capturing = false;     // inside the cycle capture: no nested graphs
};

static swe_status mg_step_batch(swe_mgrit* g, int l, const double2* in, int64_t in_stride, double2* out,
                                int64_t out_stride, const double2* add, int64_t add_stride, int S) {
    MGLevel& L = g->lv[l];
    swe_stepper_desc sd = L.sd;
    sd.nsteps = 1;
    if (sd.scheme == SWE_SLSI_SETTLS) sd.scheme = SWE_SLSI_SETTLS_1STEP;   // relaxations start at C-points
    return propagate_strided(L.plan, &sd, in, in_stride, out, out_stride, add, add_stride, S, g->cs);
}

static swe_status f_relax(swe_mgrit* g, int l) {
    MGLevel& L = g->lv[l];
    const int cf = g->d.cf, Nc = L.N / cf;
    for (int j = 1; j < cf; ++j)
        SWE_CHECK(mg_step_batch(g, l, L.u + (j - 1) * L.per, cf, L.u + j * L.per, cf, L.g_on ? L.g + j * L.per : nullptr,
                                cf, Nc));
    return SWE_OK;
}

static swe_status c_relax(swe_mgrit* g, int l) {
    MGLevel& L = g->lv[l];
    const int cf = g->d.cf, Nc = L.N / cf;
    return mg_step_batch(g, l, L.u + (cf - 1) * L.per, cf, L.u + cf * L.per, cf, L.g_on ? L.g + cf * L.per : nullptr,
                         cf, Nc);
}

static swe_status relax(swe_mgrit* g, int l) {
    SWE_CHECK(f_relax(g, l));
    for (int k = 0; k < g->d.nu; ++k) {
        SWE_CHECK(c_relax(g, l));
        SWE_CHECK(f_relax(g, l));
    }
    return SWE_OK;
}

static swe_status restrict_level(swe_mgrit* g, int l) {
    MGLevel& F = g->lv[l];
    MGLevel& C = g->lv[l + 1];
    const int cf = g->d.cf, Nc = C.N;
    // A_i = Phi_l(u_{cf i - 1}), i = 1..Nc
    SWE_CHECK(mg_step_batch(g, l, F.u + (cf - 1) * F.per, cf, F.A, 1, nullptr, 0, Nc));
    // v_i = R u_{cf i}
    k_restrict<<<nb((int64_t)(Nc + 1) * C.per), 256, 0, g->cs>>>(C.v, F.u, cf, Nc, C.plan->srow_m, C.plan->M,
                                                                   F.plan->M);
    SWE_CHECK_LAUNCH("k_restrict");
    // B_i = Phi_{l+1}(v_{i-1})
    SWE_CHECK(mg_step_batch(g, l + 1, C.v, 1, C.B, 1, nullptr, 0, Nc));
    k_fas_rhs<<<nb((int64_t)(Nc + 1) * C.per), 256, 0, g->cs>>>(C.g, C.v, C.B, F.u, F.g_on ? F.g : nullptr, F.A, cf,
                                                                  Nc, C.plan->srow_m, C.plan->M, F.plan->M);
    SWE_CHECK_LAUNCH("k_fas_rhs");
    SWE_CHECK_CUDA(cudaMemcpyAsync(C.u, C.v, sizeof(double2) * C.per * (Nc + 1), cudaMemcpyDeviceToDevice, g->cs));
    C.g_on = true;
    return SWE_OK;
}

static swe_status correct_level(swe_mgrit* g, int l) {
    MGLevel& F = g->lv[l];
    MGLevel& C = g->lv[l + 1];
    const int cf = g->d.cf, Nc = C.N;
    k_correct<<<nb((int64_t)Nc * C.per), 256, 0, g->cs>>>(F.u, C.u, C.v, cf, Nc, C.plan->srow_m, C.plan->M, F.plan->M);
    SWE_CHECK_LAUNCH("k_correct");
    return f_relax(g, l);
}

static swe_status solve_coarsest_body(swe_mgrit* g, int l) {
    MGLevel& L = g->lv[l];
    if (L.g_on)
        SWE_CHECK_CUDA(cudaMemcpyAsync(L.u, L.g, sizeof(double2) * L.per, cudaMemcpyDeviceToDevice, g->cs));
    for (int i = 1; i <= L.N; ++i) {
        double2* out = L.u + i * L.per;
        const double2* add = L.g_on ? L.g + i * L.per : nullptr;
        if (L.two_step && i >= 2) {
            // two-step SL-SI-SETTLS: the state one step earlier is u_{i-2}.  Its grid velocity
            // and N_R are exactly the current fields of step i-1, which sl_step keeps in the
            // workspace (swap): only step 2 transforms u_0 explicitly.
            char* ws;
            SWE_CHECK(plan_workspace(L.plan, sl_bytes(L.plan, 1), &ws));
            SWE_CHECK(sl_step(L.plan, L.sd.dt, L.sd.visc_nu, L.sd.visc_q, i == 2 ? L.u + (i - 2) * L.per : nullptr,
                              i > 2, L.u + (i - 1) * L.per, out, 1, ws, true, g->cs));
            if (add) SWE_CHECK(k_axpy(out, add, 1.0, L.per, g->cs));
        } else {
            SWE_CHECK(mg_step_batch(g, l, L.u + (i - 1) * L.per, 1, out, 1, add, 1, 1));
        }
    }
    return SWE_OK;
}

static void drop_graph(MGLevel::Graph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
}

static swe_status solve_coarsest(swe_mgrit* g, int l) {
    MGLevel& L = g->lv[l];
    if (g->capturing) return solve_coarsest_body(g, l);     // part of the captured cycle
    MGLevel::Graph& G = L.cg[L.g_on ? 1 : 0];
    if (G.exec && G.gen != L.plan->gen) {
        // a plan buffer the graph points into was reallocated since the capture
        SWE_CHECK_CUDA(cudaStreamSynchronize(g->cs));
        drop_graph(G);
        G.passes = 0;
    }
    if (!G.exec && (G.off || G.passes < 1)) {
        G.passes += 1;
        return solve_coarsest_body(g, l);
    }
    if (!G.exec) {
        const long long before = swe_launch_count();
        const unsigned long long gen0 = L.plan->gen;
        SWE_CHECK_CUDA(cudaStreamBeginCapture(g->cs, cudaStreamCaptureModeThreadLocal));
        const swe_status st = solve_coarsest_body(g, l);
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g->cs, &gr);
        // captured launches did not execute: they are counted at each replay instead
        G.launches = swe_launch_count() - before;
        prof_launch(-G.launches);
        if (st != SWE_OK || e != cudaSuccess || L.plan->gen != gen0) {
            // not capturable as it stands (e.g. a buffer had to grow): run it uncaptured from now on
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            G.off = true;
            return solve_coarsest_body(g, l);
        }
        G.graph = gr;
        SWE_CHECK_CUDA(cudaGraphInstantiate(&G.exec, gr, 0));
        G.gen = L.plan->gen;
    }
    SWE_CHECK_CUDA(cudaGraphLaunch(G.exec, g->cs));
    prof_launch(G.launches);
    return SWE_OK;
}

static swe_status v_cycle(swe_mgrit* g, int l) {
    const int Lc = (int)g->lv.size() - 1;
    if (l == Lc) return solve_coarsest(g, l);
    SWE_CHECK(relax(g, l));
    SWE_CHECK(restrict_level(g, l));
    SWE_CHECK(v_cycle(g, l + 1));
    return correct_level(g, l);
}

static swe_status f_cycle(swe_mgrit* g, int l) {
    const int Lc = (int)g->lv.size() - 1;
    if (l == Lc) return solve_coarsest(g, l);
    SWE_CHECK(relax(g, l));
    SWE_CHECK(restrict_level(g, l));
    if (l + 1 == Lc) {
        SWE_CHECK(solve_coarsest(g, l + 1));
    } else {
        SWE_CHECK(f_cycle(g, l + 1));
        SWE_CHECK(v_cycle(g, l + 1));
    }
    return correct_level(g, l);
}

static std::vector<unsigned long long> plan_gens(const swe_mgrit* g) {
    std::vector<unsigned long long> v;
    for (const auto& L : g->lv) v.push_back(L.plan->gen);
    return v;
}

static swe_status cycle_body(swe_mgrit* g) {
    for (size_t l = 1; l < g->lv.size(); ++l) g->lv[l].g_on = false;
    return g->d.cycle == 1 ? f_cycle(g, 0) : v_cycle(g, 0);
}

// One MGRIT iteration: uncaptured the first time (buffers, implicit-solve factors and launch
// configurations settle), then captured once and replayed as a single graph launch.  A plan
// buffer reallocated since the capture (generation changed) drops the graph and re-captures.
static swe_status run_cycle(swe_mgrit* g) {
    auto& C = g->cyc;
    if (prof_enabled()) return cycle_body(g);     // per-kernel timing needs uncaptured launches
    if (C.exec && C.gens != plan_gens(g)) {
        SWE_CHECK_CUDA(cudaStreamSynchronize(g->cs));
        cudaGraphExecDestroy(C.exec);
        cudaGraphDestroy(C.graph);
        C.exec = nullptr;
        C.graph = nullptr;
        C.passes = 0;
    }
    if (!C.exec && (C.off || C.passes < 1)) {
        C.passes += 1;
        return cycle_body(g);
    }
    if (!C.exec) {
        const long long before = swe_launch_count();
        const std::vector<unsigned long long> gens = plan_gens(g);
        SWE_CHECK_CUDA(cudaStreamBeginCapture(g->cs, cudaStreamCaptureModeThreadLocal));
        g->capturing = true;
        const swe_status st = cycle_body(g);
        g->capturing = false;
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g->cs, &gr);
        C.launches = swe_launch_count() - before;
        prof_launch(-C.launches);
        if (st != SWE_OK || e != cudaSuccess || gens != plan_gens(g)) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            C.off = true;
            return cycle_body(g);
        }
        C.graph = gr;
        SWE_CHECK_CUDA(cudaGraphInstantiate(&C.exec, gr, 0));
        C.gens = gens;
    }
    SWE_CHECK_CUDA(cudaGraphLaunch(C.exec, g->cs));
    prof_launch(C.launches);
    return SWE_OK;
}

extern "C" swe_status swe_mgrit_create(const swe_mgrit_desc* d, swe_mgrit_t* out) {
    if (!d || !out || d->L < 2 || d->L > 8 || d->cf < 2 || d->nu < 0 || d->N0 < d->cf) {
        swe_set_error("swe_mgrit_create: need 2 <= L <= 8, cf >= 2, nu >= 0, N0 >= cf");
        return SWE_EINVAL;
    }
    long long div = 1;
    for (int l = 1; l < d->L; ++l) div *= d->cf;
    if (d->N0 % div) {
        swe_set_error("swe_mgrit_create: N0 = %d is not divisible by cf^(L-1) = %lld", d->N0, div);
        return SWE_EINVAL;
    }
    for (int l = 0; l < d->L; ++l) {
        if (!d->plan[l]) {
            swe_set_error("swe_mgrit_create: plan of level %d is NULL", l);
            return SWE_EINVAL;
        }
        if (l > 0 && d->plan[l]->M > d->plan[l - 1]->M) {
            swe_set_error("swe_mgrit_create: level %d truncation exceeds level %d", l, l - 1);
            return SWE_EINVAL;
        }
    }
    swe_mgrit* g = new swe_mgrit();
    g->d = *d;
    g->lv.resize(d->L);
    int N = d->N0;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < d->L; ++l) {
        MGLevel& L = g->lv[l];
        L.plan = d->plan[l];
        L.sd = d->step[l];
        L.N = N;
        L.per = 3 * L.plan->nc;
        L.two_step = (l == d->L - 1) && (L.sd.scheme == SWE_SLSI_SETTLS);
        const size_t st = sizeof(double2) * L.per;
        if (e == cudaSuccess) e = cudaMalloc((void**)&L.u, st * (N + 1));
        if (e == cudaSuccess) e = cudaMalloc((void**)&L.x0, st);
        if (l > 0) {
            if (e == cudaSuccess) e = cudaMalloc((void**)&L.g, st * (N + 1));
            if (e == cudaSuccess) e = cudaMalloc((void**)&L.v, st * (N + 1));
            if (e == cudaSuccess) e = cudaMalloc((void**)&L.B, st * N);
        }
        if (l + 1 < d->L && e == cudaSuccess) e = cudaMalloc((void**)&L.A, st * (N / d->cf));
        N /= d->cf;
    }
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&g->cold, sizeof(double2) * g->lv[0].per * (g->lv[0].N / d->cf + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->red, sizeof(unsigned long long) * 6);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        swe_mgrit_destroy(g);
        return swe_cuda_status(e, "swe_mgrit_create");
    }
    *out = g;
    return SWE_OK;
}

extern "C" swe_status swe_mgrit_destroy(swe_mgrit_t g) {
    if (!g) return SWE_OK;
    if (g->cs) cudaStreamSynchronize(g->cs);
    for (auto& L : g->lv) {
        drop_graph(L.cg[0]);
        drop_graph(L.cg[1]);
        cudaFree(L.u);
        cudaFree(L.g);
        cudaFree(L.v);
        cudaFree(L.A);
        cudaFree(L.B);
        cudaFree(L.x0);
    }
    if (g->cyc.exec) cudaGraphExecDestroy(g->cyc.exec);
    if (g->cyc.graph) cudaGraphDestroy(g->cyc.graph);
    cudaFree(g->cold);
    cudaFree(g->red);
    if (g->cs) cudaStreamDestroy(g->cs);
    delete g;
    return SWE_OK;
}

static swe_status sync_in(swe_mgrit* g, cudaStream_t user) {
    cudaEvent_t ev;
    SWE_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SWE_CHECK_CUDA(cudaEventRecord(ev, user));
    SWE_CHECK_CUDA(cudaStreamWaitEvent(g->cs, ev, 0));
    cudaEventDestroy(ev);
    return SWE_OK;
}

static swe_status sync_out(swe_mgrit* g, cudaStream_t user) {
    cudaEvent_t ev;
    SWE_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SWE_CHECK_CUDA(cudaEventRecord(ev, g->cs));
    SWE_CHECK_CUDA(cudaStreamWaitEvent(user, ev, 0));
    cudaEventDestroy(ev);
    return SWE_OK;
}

extern "C" swe_status swe_mgrit_init(swe_mgrit_t g, const double* U0, void* stream) {
    if (!g || !U0) {
        swe_set_error("swe_mgrit_init: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(sync_in(g, user));
    const int Lc = (int)g->lv.size() - 1;
    // initial condition at every resolution
    SWE_CHECK_CUDA(cudaMemcpyAsync(g->lv[0].x0, U0, sizeof(double2) * g->lv[0].per, cudaMemcpyDeviceToDevice, g->cs));
    for (int l = 1; l <= Lc; ++l) {
        k_retrunc<<<nb(g->lv[l].per), 256, 0, g->cs>>>(g->lv[l - 1].x0, g->lv[l - 1].plan->M, g->lv[l].x0,
                                                       g->lv[l].plan->M, g->lv[l].plan->srow_m);
        SWE_CHECK_LAUNCH("k_retrunc");
    }
    for (auto& L : g->lv) L.g_on = false;
    // serial propagation on the coarsest level
    MGLevel& C = g->lv[Lc];
    SWE_CHECK_CUDA(cudaMemcpyAsync(C.u, C.x0, sizeof(double2) * C.per, cudaMemcpyDeviceToDevice, g->cs));
    SWE_CHECK(solve_coarsest(g, Lc));
    // inject upwards with F-relaxation
    for (int l = Lc - 1; l >= 0; --l) {
        MGLevel& F = g->lv[l];
        MGLevel& Cn = g->lv[l + 1];
        SWE_CHECK_CUDA(cudaMemcpyAsync(F.u, F.x0, sizeof(double2) * F.per, cudaMemcpyDeviceToDevice, g->cs));
        k_inject<<<nb((int64_t)Cn.N * F.per), 256, 0, g->cs>>>(F.u, Cn.u, g->d.cf, Cn.N, F.plan->srow_m, Cn.plan->M,
                                                                F.plan->M);
        SWE_CHECK_LAUNCH("k_inject");
        SWE_CHECK(f_relax(g, l));
    }
    // reference C-points for the convergence norm
    MGLevel& F0 = g->lv[0];
    const int Nc = F0.N / g->d.cf;
    SWE_CHECK_CUDA(cudaMemsetAsync(g->red, 0, sizeof(unsigned long long) * 6, g->cs));
    k_cnorm<<<256, 256, 0, g->cs>>>(F0.u, g->cold, g->d.cf, Nc, F0.plan->nc, g->red, F0.plan->flags);
    SWE_CHECK_LAUNCH("k_cnorm");
    SWE_CHECK(sync_out(g, user));
    return SWE_OK;
}

extern "C" swe_status mgrit_cycle(swe_mgrit_t g, int ncycles, double tol, int* k_done, double* norm_hist,
                                  void* stream) {
    if (!g || ncycles < 0) {
        swe_set_error("mgrit_cycle: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(sync_in(g, user));
    MGLevel& F0 = g->lv[0];
    // the distinct plans of the levels: each has its own status word
    std::vector<swe_plan*> plans;
    for (auto& lv : g->lv)
        if (std::find(plans.begin(), plans.end(), lv.plan) == plans.end()) plans.push_back(lv.plan);
    for (swe_plan* q : plans) SWE_CHECK(plan_flags_clear(q, g->cs));
    std::vector<int> bits(plans.size(), 0);
    const int Nc = F0.N / g->d.cf;
    int k = 0;
    swe_status status = SWE_OK;
    for (; k < ncycles; ++k) {
        SWE_CHECK(run_cycle(g));
        SWE_CHECK_CUDA(cudaMemsetAsync(g->red, 0, sizeof(unsigned long long) * 6, g->cs));
        k_cnorm<<<256, 256, 0, g->cs>>>(F0.u, g->cold, g->d.cf, Nc, F0.plan->nc, g->red, F0.plan->flags);
        SWE_CHECK_LAUNCH("k_cnorm");
        unsigned long long red[6];
        int flag = 0;
        SWE_CHECK_CUDA(cudaMemcpyAsync(red, g->red, sizeof(red), cudaMemcpyDeviceToHost, g->cs));
        for (size_t i = 0; i < plans.size(); ++i) SWE_CHECK(plan_flags_fetch(plans[i], &bits[i], g->cs));
        SWE_CHECK_CUDA(cudaStreamSynchronize(g->cs));
        for (int b : bits) flag |= b;
        double nrm = 0.0;
        for (int q = 0; q < 3; ++q) {
            double dd, vv;
            memcpy(&dd, &red[q], sizeof(double));
            memcpy(&vv, &red[3 + q], sizeof(double));
            if (vv > 0) nrm = fmax(nrm, dd / vv);
        }
        if (norm_hist) norm_hist[k] = nrm;
        if (flag) {
            status = plan_flags_status(flag, "mgrit_cycle", k + 1);
            // the condition is reported: leave the status words clear for the next call
            for (swe_plan* q : plans) SWE_CHECK(plan_flags_clear(q, g->cs));
            ++k;
            break;
        }
        if (tol > 0.0 && nrm < tol) {
            ++k;
            break;
        }
    }
    if (k_done) *k_done = k;
    SWE_CHECK(sync_out(g, user));
    return status;
}

// One cycle enqueued behind `user` without synchronising the host: the cycle, the C-point norm
// reduction and the copies of its six reduction words (red_host, pinned host memory) and of the
// levels' status words (bits_host[0..L-1]) all follow `user`'s prior work, and `user` waits for
// them; the host values are valid once `user` is synchronised.  Used by the server, which
// synchronises once per tick for all its requests.
swe_status mgrit_cycle_enqueue(swe_mgrit* g, cudaStream_t user, unsigned long long* red_host, int* bits_host) {
    SWE_CHECK(sync_in(g, user));
    MGLevel& F0 = g->lv[0];
    for (auto& L : g->lv) SWE_CHECK(plan_flags_clear(L.plan, g->cs));
    const int Nc = F0.N / g->d.cf;
    SWE_CHECK(run_cycle(g));
    SWE_CHECK_CUDA(cudaMemsetAsync(g->red, 0, sizeof(unsigned long long) * 6, g->cs));
    k_cnorm<<<256, 256, 0, g->cs>>>(F0.u, g->cold, g->d.cf, Nc, F0.plan->nc, g->red, F0.plan->flags);
    SWE_CHECK_LAUNCH("k_cnorm");
    SWE_CHECK_CUDA(cudaMemcpyAsync(red_host, g->red, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToHost, g->cs));
    for (size_t l = 0; l < g->lv.size(); ++l) SWE_CHECK(plan_flags_fetch(g->lv[l].plan, &bits_host[l], g->cs));
    return sync_out(g, user);
}

extern "C" swe_status swe_mgrit_cpoints(swe_mgrit_t g, double* U_out, void* stream) {
    if (!g || !U_out) {
        swe_set_error("swe_mgrit_cpoints: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    SWE_CHECK(sync_in(g, user));
    MGLevel& F0 = g->lv[0];
    const int Nc = F0.N / g->d.cf;
    SWE_CHECK_CUDA(cudaMemcpy2DAsync(U_out, sizeof(double2) * F0.per, F0.u, sizeof(double2) * F0.per * g->d.cf,
                                     sizeof(double2) * F0.per, Nc + 1, cudaMemcpyDefault, g->cs));
    SWE_CHECK(sync_out(g, user));
    return SWE_OK;
}
