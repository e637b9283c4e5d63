// Plan creation: Gaussian grid, associated Legendre table and FFT twiddles built on
// the device in FP64 (§2.2); workspace arena; scalar SHT entry points.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "swe_internal.cuh"

static thread_local char g_err[1024] = "";

void swe_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

swe_status swe_cuda_status(cudaError_t e, const char* what) {
    swe_set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
}

extern "C" const char* swe_last_error(void) { return g_err; }
extern "C" const char* swe_version(void) { return "swe_gb300 0.1 (sm_103a)"; }
extern "C" int64_t swe_ncoef(int M) { return M < 0 ? 0 : nc_state(M); }

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes: Newton iteration on P_nlat in colatitude t (mu = cos t),
// started from t = pi (j + 3/4) / (nlat + 1/2) for the j-th node from the north.
// dP/dt = nlat (mu P_nlat - P_{nlat-1}) / sin t;  w = 2 sin^2 t / (nlat (mu P_nlat - P_{nlat-1}))^2.
__global__ void k_gauss(int nlat, double* mu, double* w) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int nh = nlat / 2;
    if (j >= nh) return;
    double t = M_PI * ((double)j + 0.75) / ((double)nlat + 0.5);
    double pn = 0.0, pn1 = 0.0, x = 0.0;
    for (int it = 0; it < 60; ++it) {
        x = cos(t);
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < nlat; ++k) {
            double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        pn = p1;
        pn1 = p0;
        double dpdt = nlat * (x * pn - pn1) / sin(t);
        double dt = pn / dpdt;
        t -= dt;
        if (fabs(dt) < 1e-17) break;
    }
    x = cos(t);
    {
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < nlat; ++k) {
            double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        pn = p1;
        pn1 = p0;
    }
    double s = sin(t);
    double d = nlat * (x * pn - pn1);
    double wj = 2.0 * s * s / (d * d);
    mu[j] = x;
    mu[nlat - 1 - j] = -x;
    w[j] = wj;
    w[nlat - 1 - j] = wj;
}

// Normalised associated Legendre functions P_n^m(mu_j), n = m..M+1, j in the
// northern half, one thread per (m, j).  The sectoral value
// P_m^m = sqrt(1/2) prod_{k<=m} sqrt((2k+1)/(2k)) sin(t)^m is carried as v * 2^e
// so that it never underflows; the n-recurrence
// P_n = (mu P_{n-1} - eps_{n-1} P_{n-2}) / eps_n  runs on the scaled values and
// the output is ldexp(v, e), which underflows to zero only where the true value
// is below the double range.
__global__ void k_legendre(int M, int nlat2, const double* mu, double* P) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (j >= nlat2) return;
    const double x = mu[j];
    const double s = sqrt((1.0 - x) * (1.0 + x));
    const double big = 0x1p200, small = 0x1p-200;
    double v = 0.70710678118654752440;   // sqrt(1/2)
    int e = 0;
    for (int k = 1; k <= m; ++k) {
        v *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
        if (v < small) {
            v *= big;
            e -= 200;
        }
    }
    const int64_t base = ex_off(m, M) * nlat2;
    double pm2 = v;                                  // P_m^m (scaled)
    P[base + j] = ldexp(pm2, e);
    if (m + 1 > M + 1) return;
    double pm1 = sqrt(2.0 * m + 3.0) * x * pm2;      // P_{m+1}^m
    P[base + (int64_t)1 * nlat2 + j] = ldexp(pm1, e);
    for (int n = m + 2; n <= M + 1; ++n) {
        double pn = (x * pm1 - eps_nm(m, n - 1) * pm2) / eps_nm(m, n);
        pm2 = pm1;
        pm1 = pn;
        if (fabs(pm1) > big) {
            pm1 *= small;
            pm2 *= small;
            e += 200;
        }
        P[base + (int64_t)(n - m) * nlat2 + j] = ldexp(pm1, e);
    }
}

__global__ void k_twiddle(int N, double2* tw, float2* twf) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)N, &s, &c);
    tw[k] = make_double2(c, -s);
    twf[k] = make_float2((float)c, (float)-s);
}

__global__ void k_row_m(int M, int* row_m, int* srow_m) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > M) return;
    int64_t o = ex_off(m, M);
    for (int n = m; n <= M + 1; ++n) row_m[o + (n - m)] = m;
    int64_t so = st_off(m, M);
    for (int n = m; n <= M; ++n) srow_m[so + (n - m)] = m;
}

__global__ void k_row_coef(int M, double a, double* rc, float* rcf) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > M) return;
    auto il = [&](int n) { return (n >= 1 && n <= M && n >= m) ? -a * a / ((double)n * (n + 1.0)) : 0.0; };
    for (int n = m; n <= M + 1; ++n) {
        double* c = rc + (ex_off(m, M) + (n - m)) * RC_NUM;
        const double en = eps_nm(m, n), en1 = eps_nm(m, n + 1);
        c[RC_UC0] = m * il(n) / a;
        c[RC_UCM] = (n - 1 >= m) ? (n - 1.0) * en * il(n - 1) / a : 0.0;
        c[RC_UCP] = (n + 2.0) * en1 * il(n + 1) / a;
        c[RC_DCP] = n * en1 / a;
        c[RC_DCM] = (n + 1.0) * en / a;
        c[RC_P] = n >= 1 ? (n + 1.0) / n * en : 0.0;
        c[RC_Q] = n >= 1 ? n / (n + 1.0) * en1 : 0.0;
        c[RC_R] = n >= 1 ? (double)m / ((double)n * (n + 1.0)) : 0.0;
        c[RC_GM] = (n - 1 >= m) ? -(n - 1.0) * en : 0.0;
        c[RC_GP] = (n + 2.0) * en1;
        for (int k = 0; k < RC_NUM; ++k) rcf[(ex_off(m, M) + (n - m)) * RC_NUM + k] = (float)c[k];
    }
}

static bool factor_radices(int N, int* rad, int* nrad) {
    int k = 0;
    while (N % 4 == 0) { rad[k++] = 4; N /= 4; }
    while (N % 3 == 0) { rad[k++] = 3; N /= 3; }
    while (N % 2 == 0) { rad[k++] = 2; N /= 2; }
    *nrad = k;
    return N == 1;
}

extern "C" swe_status swe_plan_create(const swe_plan_desc* d, swe_plan_t* out) {
    if (!d || !out) {
        swe_set_error("swe_plan_create: null argument");
        return SWE_EINVAL;
    }
    *out = nullptr;
    if (d->M < 1 || d->nlat < d->M + 2 || (d->nlat & 1) || d->nlon <= 2 * (d->M + 1) ||
        d->nlon > 8192 || d->M > 2047) {
        swe_set_error("swe_plan_create: need M >= 1, even nlat >= M+2, 2(M+1) < nlon <= 8192 (M=%d nlat=%d nlon=%d)",
                      d->M, d->nlat, d->nlon);
        return SWE_EINVAL;
    }
    if (d->prec != SWE_FP64 && d->prec != SWE_SPLIT_BF16X3) {
        swe_set_error("swe_plan_create: unknown precision %d", (int)d->prec);
        return SWE_EINVAL;
    }
    swe_plan* p = new swe_plan();
    p->M = d->M;
    p->nlat = d->nlat;
    p->nlon = d->nlon;
    p->nlat2 = d->nlat / 2;
    p->a = d->a;
    p->omega = d->omega;
    p->g = d->g;
    p->phibar = d->phibar;
    p->prec = d->prec;
    p->nc = nc_state(d->M);
    p->ncx = nc_ext(d->M);
    // the longitude FFT runs on nlon/2 complex points (two real samples each)
    if ((d->nlon & 1) || !factor_radices(d->nlon / 2, p->rad, &p->nrad)) {
        delete p;
        swe_set_error("swe_plan_create: nlon=%d is not of the form 2^a 3^b with a >= 1", d->nlon);
        return SWE_EINVAL;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return swe_cuda_status(e, "cudaGetDevice");
    }
#define ALLOC(ptr, bytes)                                                      \
    do {                                                                       \
        cudaError_t e2 = cudaMalloc((void**)&(ptr), (bytes));                  \
        if (e2 != cudaSuccess) {                                               \
            swe_plan_destroy(p);                                               \
            return swe_cuda_status(e2, "cudaMalloc(plan tables)");             \
        }                                                                      \
    } while (0)
    ALLOC(p->mu, sizeof(double) * p->nlat);
    ALLOC(p->w, sizeof(double) * p->nlat);
    ALLOC(p->P, sizeof(double) * p->ncx * p->nlat2);
    ALLOC(p->row_m, sizeof(int) * p->ncx);
    ALLOC(p->srow_m, sizeof(int) * p->nc);
    ALLOC(p->tw, sizeof(double2) * p->nlon);
    ALLOC(p->twf, sizeof(float2) * p->nlon);
    ALLOC(p->flags, sizeof(int) * 4);
    ALLOC(p->rc, sizeof(double) * RC_NUM * p->ncx);
    ALLOC(p->rcf, sizeof(float) * RC_NUM * p->ncx);
#undef ALLOC
    cudaMemset(p->flags, 0, sizeof(int) * 4);
    k_gauss<<<(p->nlat2 + 63) / 64, 64>>>(p->nlat, p->mu, p->w);
    {
        dim3 g((p->nlat2 + 127) / 128, p->M + 1);
        k_legendre<<<g, 128>>>(p->M, p->nlat2, p->mu, p->P);
    }
    k_twiddle<<<(p->nlon + 255) / 256, 256>>>(p->nlon, p->tw, p->twf);
    k_row_m<<<(p->M + 1 + 127) / 128, 128>>>(p->M, p->row_m, p->srow_m);
    k_row_coef<<<(p->M + 1 + 127) / 128, 128>>>(p->M, p->a, p->rc, p->rcf);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        swe_plan_destroy(p);
        return swe_cuda_status(e, "plan table kernels");
    }
    if (p->prec == SWE_SPLIT_BF16X3) {
        swe_status s2 = split_tables_build(p);
        if (s2 == SWE_OK) s2 = small_tables_build(p);
        if (s2 != SWE_OK) {
            swe_plan_destroy(p);
            return s2;
        }
    }
    *out = p;
    return SWE_OK;
}

extern "C" swe_status swe_plan_destroy(swe_plan_t p) {
    if (!p) return SWE_OK;
    cudaFree(p->mu);
    cudaFree(p->w);
    cudaFree(p->P);
    cudaFree(p->row_m);
    cudaFree(p->srow_m);
    cudaFree(p->tw);
    cudaFree(p->twf);
    cudaFree(p->flags);
    cudaFree(p->thx);
    cudaFree(p->rc);
    cudaFree(p->rcf);
    split_tables_free(p);
    small_tables_free(p);
    for (int i = 0; i < p->ncn; ++i) {
        cudaFree(p->cn[i].fac);
        cudaFree(p->cn[i].fac32);
    }
    if (p->ws.base) cudaFree(p->ws.base);
    delete p;
    return SWE_OK;
}

extern "C" swe_status swe_plan_gauss(swe_plan_t p, double* mu_host, double* w_host) {
    if (!p || !mu_host || !w_host) {
        swe_set_error("swe_plan_gauss: null argument");
        return SWE_EINVAL;
    }
    SWE_CHECK_CUDA(cudaMemcpy(mu_host, p->mu, sizeof(double) * p->nlat, cudaMemcpyDeviceToHost));
    SWE_CHECK_CUDA(cudaMemcpy(w_host, p->w, sizeof(double) * p->nlat, cudaMemcpyDeviceToHost));
    return SWE_OK;
}

// Grows the plan's workspace arena (never during stream capture: the arena is
// sized by the caller before capturing).
swe_status plan_workspace(swe_plan* p, size_t bytes, char** out) {
    if (bytes > p->ws.bytes) {
        if (p->ws.base) {
            SWE_CHECK_CUDA(cudaDeviceSynchronize());
            cudaFree(p->ws.base);
            p->ws.base = nullptr;
            p->ws.bytes = 0;
        }
        size_t want = bytes + bytes / 8 + (1u << 20);
        p->gen += 1;
        cudaError_t e = cudaMalloc((void**)&p->ws.base, want);
        if (e != cudaSuccess) return swe_cuda_status(e, "cudaMalloc(workspace)");
        p->ws.bytes = want;
    }
    *out = p->ws.base;
    return SWE_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// extra workspace of the advective geopotential tendency (zero in the flux form)
static size_t nphi_bytes(const swe_plan* p, int S) {
    if (!p->nphi_adv) return 0;
    const size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    const size_t re = fe / 2;
    const size_t four = (size_t)(p->M + 1) * p->nlat, grid = (size_t)p->nlat * p->nlon;
    return align256(fe * p->ncx * 6 * S) + align256(fe * four * 6 * S) + align256(re * grid * 6 * S) +
           align256(fe * four * S) + align256(fe * p->ncx * S);
}

size_t nl_bytes(const swe_plan* p, int S) {
    size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    size_t four = (size_t)(p->M + 1) * p->nlat;
    return align256(sizeof(double2) * p->ncx * 4 * S) + align256(fe * four * 4 * S) +
           align256(fe * four * 5 * S) + align256(sizeof(double2) * p->ncx * 5 * S) + nphi_bytes(p, S);
}

NLBuffers nl_carve(const swe_plan* p, char* base, int S) {
    size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    size_t four = (size_t)(p->M + 1) * p->nlat;
    NLBuffers b;
    char* c = base;
    b.X = (double2*)c;
    c += align256(sizeof(double2) * p->ncx * 4 * S);
    b.Fin = c;
    c += align256(fe * four * 4 * S);
    b.Fout = c;
    c += align256(fe * four * 5 * S);
    b.Y = (double2*)c;
    c += align256(sizeof(double2) * p->ncx * 5 * S);
    b.X2 = nullptr;
    b.F2 = b.G2 = b.F3 = nullptr;
    b.Y2 = nullptr;
    if (p->nphi_adv) {
        const size_t re = fe / 2, grid = (size_t)p->nlat * p->nlon;
        b.X2 = (double2*)c;
        c += align256(fe * p->ncx * 6 * S);
        b.F2 = c;
        c += align256(fe * four * 6 * S);
        b.G2 = c;
        c += align256(re * grid * 6 * S);
        b.F3 = c;
        c += align256(fe * four * S);
        b.Y2 = (double2*)c;
    }
    return b;
}

extern "C" swe_status swe_plan_set_nphi_form(swe_plan_t p, int form) {
    if (!p || (form != SWE_NPHI_FLUX && form != SWE_NPHI_ADVECTIVE)) {
        swe_set_error("swe_plan_set_nphi_form: invalid argument");
        return SWE_EINVAL;
    }
    if (p->nphi_adv != form) {
        p->nphi_adv = form;
        p->gen += 1;          // workspace layout changed: captured graphs are stale
    }
    return SWE_OK;
}

// ---------------------------------------------------------------------------
// status word
swe_status plan_flags_fetch(const swe_plan* p, int* host, cudaStream_t st) {
    SWE_CHECK_CUDA(cudaMemcpyAsync(host, p->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    return SWE_OK;
}

swe_status plan_flags_clear(const swe_plan* p, cudaStream_t st) {
    SWE_CHECK_CUDA(cudaMemsetAsync(p->flags, 0, sizeof(int), st));
    return SWE_OK;
}

swe_status plan_flags_status(int bits, const char* where, int iter) {
    if (bits & PLAN_FLAG_TIMEOUT) {
        swe_set_error("%s: a bounded tensor-core wait gave up (iteration %d); results of that call are incomplete",
                      where, iter);
        return SWE_ETIMEOUT;
    }
    if (bits & PLAN_FLAG_NONFINITE) {
        swe_set_error("%s: non-finite value at iteration %d", where, iter);
        return SWE_EUNSTABLE;
    }
    return SWE_OK;
}

__global__ void k_or_flags(int* flags, int bits) { atomicOr(flags, bits); }

extern "C" swe_status swe_plan_check(swe_plan_t p, void* stream) {
    if (!p) {
        swe_set_error("swe_plan_check: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int bits = 0;
    SWE_CHECK(plan_flags_fetch(p, &bits, st));
    SWE_CHECK_CUDA(cudaStreamSynchronize(st));
    SWE_CHECK(plan_flags_clear(p, st));
    SWE_CHECK_CUDA(cudaStreamSynchronize(st));
    return plan_flags_status(bits, "swe_plan_check", 0);
}

extern "C" swe_status swe_plan_inject_status(swe_plan_t p, int bits, void* stream) {
    if (!p || (bits & ~(PLAN_FLAG_NONFINITE | PLAN_FLAG_TIMEOUT)) != 0) {
        swe_set_error("swe_plan_inject_status: invalid argument");
        return SWE_EINVAL;
    }
    k_or_flags<<<1, 1, 0, (cudaStream_t)stream>>>(p->flags, bits);
    SWE_CHECK_LAUNCH("k_or_flags");
    return SWE_OK;
}

extern "C" swe_status swe_wait_selftest(swe_plan_t p, long long polls, void* stream) {
    if (!p || polls < 1) {
        swe_set_error("swe_wait_selftest: invalid argument");
        return SWE_EINVAL;
    }
    return wait_selftest_launch(p, polls, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// scalar transforms (ABI)
extern "C" swe_status sht_inverse(swe_plan_t p, const void* spec, void* grid, int batch, void* stream) {
    if (!p || !spec || !grid || batch < 1) {
        swe_set_error("sht_inverse: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    size_t need = align256(sizeof(double2) * p->ncx * batch) + align256(fe * (size_t)(p->M + 1) * p->nlat * batch);
    char* ws;
    SWE_CHECK(plan_workspace(p, need, &ws));
    double2* X = (double2*)ws;
    void* F = ws + align256(sizeof(double2) * p->ncx * batch);
    SWE_CHECK(k_pack_scalar(p, (const double2*)spec, X, batch, st));
    SWE_CHECK(leg_inverse(p, X, F, batch, st));
    SWE_CHECK(ring_inverse(p, F, grid, batch, st));
    return SWE_OK;
}

extern "C" swe_status sht_forward(swe_plan_t p, const void* grid, void* spec, int batch, void* stream) {
    if (!p || !spec || !grid || batch < 1) {
        swe_set_error("sht_forward: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    size_t fbytes = align256(fe * (size_t)(p->M + 1) * p->nlat * batch);
    size_t need = fbytes + align256(sizeof(double2) * p->ncx * batch);
    char* ws;
    SWE_CHECK(plan_workspace(p, need, &ws));
    void* F = ws;
    double2* Y = (double2*)(ws + fbytes);
    SWE_CHECK(ring_forward(p, grid, F, batch, st));
    SWE_CHECK(leg_forward(p, F, Y, batch, st));
    SWE_CHECK(k_unpack_scalar(p, Y, (double2*)spec, batch, st));
    return SWE_OK;
}
