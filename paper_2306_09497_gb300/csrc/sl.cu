// SL-SI-SETTLS step (§2.3.2, Eqs. 6-7), batched over S states.
//
//   (I - dt/2 L) U^{n+1} = [U^n + dt/2 L U^n + dt/2 (2 N_R^n - N_R^{n-1})]_* + dt/2 N_R^n,
//   followed by backward-Euler viscosity; N_R = (-Phi' delta, 0, 0); "_*" = value at the
//   departure point x_d of the trajectory arriving at the grid point x_a, from SETTLS:
//   x_d^{k+1} = x_a - dt/2 [2 V(t_n, x_d^k) - V(t_{n-1}, x_d^k) + V(t_n, x_a)],  x_d^0 = x_a,
//   two iterations, in 3-D Cartesian coordinates projected back on the unit sphere.
// Interpolation: bicubic Lagrange in (longitude, Gaussian latitude) with two halo
// rows beyond each pole (the rows across the pole, shifted by 180 degrees); the
// velocity is interpolated through its three Cartesian components (smooth scalar
// fields everywhere on the sphere).  The one-step variant (§3.2.4) replaces the
// t_{n-1} data by the t_n data; the first step of a chain is always one-step.
#include "swe_internal.cuh"

namespace {

__device__ __forceinline__ double2 c_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

struct SV {   // SoA spectral state view
    const double2* u;
    int64_t nc;
    int S, M;
    __device__ __forceinline__ double2 get(int f, int m, int n, int s) const {
        if (n < m || n > M) return czero();
        if (n == 0 && f > 0) return czero();
        return u[((int64_t)f * nc + st_off(m, M) + (n - m)) * S + s];
    }
};

// Transform operands, rows (m, n <= M+1), columns f*S + s.
//   full = 1: f = 0..2 X = U + h L U (h = dt/2), 3 Phi', 4 delta, 5 U_cos, 6 V_cos   (7 fields)
//   full = 0: f = 0 Phi', 1 delta, 2 U_cos, 3 V_cos                                 (4 fields)
// transform operands are complex128 on FP64 plans, complex64 on split-precision plans
__device__ __forceinline__ void put(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void put(float2* p, double2 v) { *p = d2f2(v); }
__device__ __forceinline__ double2 get2(const double2* p) { return *p; }
__device__ __forceinline__ double2 get2(const float2* p) { return f2d2(*p); }

template <typename TX>
__global__ void k_sl_operands(SV U, TX* __restrict__ X, const int* __restrict__ row_m, int64_t ncx, int nf,
                              int full, double h, double ia2, double omega, double phibar,
                              const double* __restrict__ rc) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int S = U.S, M = U.M;
    if (t >= ncx * S) return;
    const int s = (int)(t % S);
    const int64_t rx = t / S;
    const int m = row_m[rx];
    const int n = m + (int)(rx - ex_off(m, M));
    const double* c = rc + rx * RC_NUM;
    const double uc0 = c[RC_UC0], ucm = c[RC_UCM], ucp = c[RC_UCP];
    const double2 ph = U.get(0, m, n, s), xi = U.get(1, m, n, s), de = U.get(2, m, n, s);
    const double2 xim = U.get(1, m, n - 1, s), dem = U.get(2, m, n - 1, s);
    const double2 xip = U.get(1, m, n + 1, s), dep = U.get(2, m, n + 1, s);
    // U_cos, V_cos from psi = lap^{-1} xi, chi = lap^{-1} delta (coefficients folded in rc)
    double2 Uh, Vh;
    Uh.x = fma(ucm, xim.x, fma(-ucp, xip.x, -uc0 * de.y));
    Uh.y = fma(ucm, xim.y, fma(-ucp, xip.y, uc0 * de.x));
    Vh.x = fma(-ucm, dem.x, fma(ucp, dep.x, -uc0 * xi.y));
    Vh.y = fma(-ucm, dem.y, fma(ucp, dep.y, uc0 * xi.x));
    TX* row = X + rx * (int64_t)nf * S + s;
    if (n > M) {
        // the extended row n = M+1 carries only the velocity operands; every other field is
        // truncated at M (the Coriolis coupling of L U would otherwise leak into degree M+1)
        for (int f = 0; f < nf - 2; ++f) put(row + (int64_t)f * S, czero());
        put(row + (int64_t)(nf - 2) * S, Uh);
        put(row + (int64_t)(nf - 1) * S, Vh);
        return;
    }
    if (full) {
        const double w2 = 2.0 * omega, p = w2 * c[RC_P], q = w2 * c[RC_Q], r = w2 * c[RC_R];
        const double lap = (double)(n * (n + 1)) * ia2;
        const double2 L0 = c_scale(de, -phibar);
        const double2 L1 = make_double2(-fma(p, dem.x, fma(q, dep.x, r * xi.y)),
                                        -fma(p, dem.y, fma(q, dep.y, -r * xi.x)));
        const double2 L2 = make_double2(fma(lap, ph.x, fma(p, xim.x, fma(q, xip.x, -r * de.y))),
                                        fma(lap, ph.y, fma(p, xim.y, fma(q, xip.y, r * de.x))));
        put(row, make_double2(fma(h, L0.x, ph.x), fma(h, L0.y, ph.y)));
        put(row + S, make_double2(fma(h, L1.x, xi.x), fma(h, L1.y, xi.y)));
        put(row + 2 * S, make_double2(fma(h, L2.x, de.x), fma(h, L2.y, de.y)));
        put(row + 3 * S, ph);
        put(row + 4 * S, de);
        put(row + 5 * S, Uh);
        put(row + 6 * S, Vh);
    } else {
        put(row, ph);
        put(row + S, de);
        put(row + 2 * S, Uh);
        put(row + 3 * S, Vh);
    }
}

// Cartesian velocity (m/s) and N_R = -Phi' delta on the grid, from fields
// (Phi', delta, U_cos, V_cos) at field offsets (fp, fd, fu, fv) of a grid block [nf*S][nlat][nlon].
// Grid-point kernels compute in the grid type T (double for FP64 plans, float for
// mixed plans: GB300's FP64 rate is 1/64 of its FP32 rate, and the grid values are
// FP32 there anyway).  Geometry comes from a per-plan table in T (built in FP64):
//   tab[0 .. nlat+3]             extended latitudes (two halo rows beyond each pole)
//   tab[nlat+4 .. 2 nlat+3]      sin(latitude) = mu
//   tab[2 nlat+4 .. 3 nlat+3]    cos(latitude)
//   tab[3 nlat+4 + 4 i + r]      1 / prod_{q != r} (y_r - y_q), y_r = tab[i - 1 + r]: the
//                                Lagrange denominators of the stencil on extended rows
//                                i-1 .. i+2 (i in [1, nlat+1]; zero elsewhere)
__device__ __forceinline__ void sc_pi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sc_pi(float x, float* s, float* c) { sincospif(x, s, c); }

template <typename T>
__global__ void k_sl_vel(const T* __restrict__ G, int fp, int fd, int fu, int fv, T* __restrict__ Vc,
                         T* __restrict__ NR, const T* __restrict__ tab, int S, int nlat, int nlon) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t npt = (int64_t)nlat * nlon;
    if (t >= npt * S) return;
    const int s = (int)(t / npt);
    const int64_t p = t - (int64_t)s * npt;
    const int j = (int)(p / nlon), k = (int)(p - (int64_t)j * nlon);
    auto at = [&](int f) { return G[((int64_t)f * S + s) * npt + p]; };
    const T sinl = tab[nlat + 4 + j], cosl = tab[2 * nlat + 4 + j];
    const T u = at(fu) / cosl, v = at(fv) / cosl;
    T sl, cl;
    sc_pi((T)(2 * k) / (T)nlon, &sl, &cl);
    Vc[((int64_t)0 * S + s) * npt + p] = -u * sl - v * sinl * cl;
    Vc[((int64_t)1 * S + s) * npt + p] = u * cl - v * sinl * sl;
    Vc[((int64_t)2 * S + s) * npt + p] = v * cosl;
    NR[(int64_t)s * npt + p] = -at(fp) * at(fd);
}

// X_Phi += h (2 N_R^n - N_R^{n-1}) in place (field 0 of the 7-field block); when W is given,
// also the extrapolated velocity W = 2 V^n - V^{n-1} of the SETTLS trajectory (§2.3.2, Eq. 6)
// for its three Cartesian components (interpolation is linear, so interpolating W equals
// 2 V^n(x) - V^{n-1}(x) up to rounding)
template <typename T>
__global__ void k_sl_xphi(T* __restrict__ G, const T* __restrict__ NRn, const T* __restrict__ NRm, T h, int S,
                          int64_t npt, const T* __restrict__ Vn, const T* __restrict__ Vm, T* __restrict__ W) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = npt * S;
    if (t >= n) return;
    G[t] = G[t] + h * ((T)2 * NRn[t] - NRm[t]);
    if (W) {
#pragma unroll
        for (int d = 0; d < 3; ++d) W[d * n + t] = (T)2 * Vn[d * n + t] - Vm[d * n + t];
    }
}

template <typename T>
struct Stencil {
    int off[16];      // grid offset (row * nlon + wrapped column) of point (r, c) at 4 r + c
    T wl[4], wx[4];
};

// bracket + Lagrange weights of the departure point (latd, xd = longitude in grid
// cells, in [0, nlon)); tab = the geometry table (extended latitudes first, descending)
template <typename T>
__device__ __forceinline__ void make_stencil(T latd, T xd, const T* __restrict__ tab, int nlat, int nlon,
                                             Stencil<T>& st) {
    // i = (number of extended latitudes >= latd) - 1, clipped to [1, nlat+1].  Gaussian
    // colatitudes sit close to pi (4 j + 3) / (4 nlat + 2), which gives the index to within a
    // row or two; the walk below settles it (each loop is bounded by the table's ends).
    const T* thx = tab;
    const T colat = (T)(0.5 * M_PI) - latd;
    int g = (int)floor(colat * (T)((4.0 * nlat + 2.0) / (4.0 * M_PI)) - (T)0.75) + 2;
    g = g < 0 ? 0 : (g > nlat + 3 ? nlat + 3 : g);
    while (g < nlat + 3 && thx[g + 1] >= latd) ++g;
    while (g > 0 && thx[g] < latd) --g;
    const int i = g < 1 ? 1 : (g > nlat + 1 ? nlat + 1 : g);
    int i0 = (int)floor(xd);
    const T t = xd - (T)i0;
    if (i0 >= nlon) i0 -= nlon;
    T y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = i - 1 + r;               // extended index 0..nlat+3
        y[r] = thx[e];
        int rowi, sh = 0;
        if (e < 2) {
            rowi = 1 - e;
            sh = nlon / 2;
        } else if (e < nlat + 2) {
            rowi = e - 2;
        } else {
            rowi = nlat - 1 - (e - (nlat + 2));
            sh = nlon / 2;
        }
        const int b = i0 - 1 + sh;             // first column before wrapping, in [-1, 3 nlon / 2]
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int col = b + c;
            if (col < 0) col += nlon;
            if (col >= nlon) col -= nlon;
            st.off[4 * r + c] = rowi * nlon + col;
        }
    }
    // Lagrange weights: w_r = prod_{q != r} (latd - y_q) / prod_{q != r} (y_r - y_q), the
    // reciprocal denominators from the table
    const T* rden = tab + 3 * nlat + 4 + 4 * i;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        T num = (T)1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q != r) num *= latd - y[q];
        st.wl[r] = num * rden[r];
    }
    const T sixth = (T)1 / (T)6;
    st.wx[0] = -t * (t - (T)1) * (t - (T)2) * sixth;
    st.wx[1] = (t + (T)1) * (t - (T)1) * (t - (T)2) * (T)0.5;
    st.wx[2] = -(t + (T)1) * t * (t - (T)2) * (T)0.5;
    st.wx[3] = (t + (T)1) * t * (t - (T)1) * sixth;
}

template <typename T>
__device__ __forceinline__ T interp(const T* __restrict__ F, const Stencil<T>& st) {
    T acc = (T)0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        T a = (T)0;
#pragma unroll
        for (int c = 0; c < 4; ++c) a += st.wx[c] * F[st.off[4 * r + c]];
        acc += st.wl[r] * a;
    }
    return acc;
}

// departure point (latitude, longitude in grid cells) of the Cartesian point xd (any length)
template <typename T>
__device__ __forceinline__ void to_latlon(const T* xd, int nlon, T& latd, T& lonc) {
    latd = atan2(xd[2], sqrt(xd[0] * xd[0] + xd[1] * xd[1]));
    lonc = atan2(xd[1], xd[0]) * ((T)nlon / (T)(2.0 * M_PI));
    if (lonc < (T)0) lonc += (T)nlon;
    if (lonc >= (T)nlon) lonc -= (T)nlon;
}

// departure points + gather: R[f*S + s] = X_f(x_d) (+ h N_R^n(x_a) for f = 0); W = the
// extrapolated velocity 2 V^n - V^{n-1} (V^n itself in the one-step form)
template <typename T>
__global__ void __launch_bounds__(128) k_sl_depart(const T* __restrict__ G, const T* __restrict__ Vn,
                                                   const T* __restrict__ W, const T* __restrict__ NRn,
                                                   T* __restrict__ R, const T* __restrict__ tab, T h, T a, int S,
                                                   int nlat, int nlon) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t npt = (int64_t)nlat * nlon;
    if (t >= npt * S) return;
    const int s = (int)(t / npt);
    const int64_t p = t - (int64_t)s * npt;
    const int j = (int)(p / nlon), k = (int)(p - (int64_t)j * nlon);
    const T sp = tab[nlat + 4 + j], cp = tab[2 * nlat + 4 + j];
    T sl, cl;
    sc_pi((T)(2 * k) / (T)nlon, &sl, &cl);
    const T xa[3] = {cp * cl, cp * sl, sp};
    T va[3], w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        va[d] = Vn[((int64_t)d * S + s) * npt + p];
        w[d] = W[((int64_t)d * S + s) * npt + p];      // x_d^0 = x_a: grid values
    }
    const T sc = h / a;   // (dt/2) / a
    Stencil<T> st;
    T xd[3];
    for (int it = 0; it < 2; ++it) {
        if (it > 0) {
            T latd, lonc;
            to_latlon(xd, nlon, latd, lonc);
            make_stencil(latd, lonc, tab, nlat, nlon, st);
#pragma unroll
            for (int d = 0; d < 3; ++d) w[d] = interp(W + ((int64_t)d * S + s) * npt, st);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) xd[d] = xa[d] - sc * (w[d] + va[d]);
    }
    T latd, lonc;
    to_latlon(xd, nlon, latd, lonc);
    make_stencil(latd, lonc, tab, nlat, nlon, st);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        T v = interp(G + ((int64_t)f * S + s) * npt, st);
        if (f == 0) v += h * NRn[(int64_t)s * npt + p];
        R[((int64_t)f * S + s) * npt + p] = v;
    }
}

template <typename TY>
__global__ void k_sl_unpack(const TY* __restrict__ Y, double2* __restrict__ R, const int* __restrict__ srow_m,
                            int M, int64_t nc, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * S) return;
    const int s = (int)(t % S);
    const int64_t r = t / S;
    const int m = srow_m[r];
    const int n = m + (int)(r - st_off(m, M));
    const TY* y = Y + (ex_off(m, M) + (n - m)) * 3 * (int64_t)S + s;
#pragma unroll
    for (int f = 0; f < 3; ++f) R[((int64_t)f * nc + r) * S + s] = get2(y + (int64_t)f * S);
}

// extended latitude e (0..nlat+3): two rows mirrored over each pole around the Gaussian ones
__device__ inline double ext_lat(const double* __restrict__ mu, int e, int nlat) {
    if (e < 2) return M_PI - asin(mu[1 - e]);
    if (e < nlat + 2) return asin(mu[e - 2]);
    return -M_PI - asin(mu[nlat - 1 - (e - (nlat + 2))]);
}

template <typename T>
__global__ void k_sl_table(const double* __restrict__ mu, T* __restrict__ tab, int nlat) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nlat + 4) {
        tab[e] = (T)ext_lat(mu, e, nlat);
        const bool ok = e >= 1 && e <= nlat + 1;
        double y[4];
        // the nodes exactly as the kernels see them (rounded to T), so that the weights are a
        // Lagrange basis of one node set; products and reciprocal in FP64
        for (int r = 0; r < 4; ++r) y[r] = ok ? (double)(T)ext_lat(mu, e - 1 + r, nlat) : 0.0;
        for (int r = 0; r < 4; ++r) {
            double den = 1.0;
            for (int q = 0; q < 4; ++q)
                if (q != r) den *= y[r] - y[q];
            tab[3 * nlat + 4 + 4 * e + r] = ok ? (T)(1.0 / den) : (T)0;
        }
    }
    if (e < nlat) {
        tab[nlat + 4 + e] = (T)mu[e];
        tab[2 * nlat + 4 + e] = (T)sqrt((1.0 - mu[e]) * (1.0 + mu[e]));
    }
}

inline unsigned nb(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// workspace of one SL step for S columns (grid fields in the plan's real type)
size_t sl_bytes(const swe_plan* p, int S) {
    const size_t rt = (p->prec == SWE_FP64) ? 8 : 4;
    const size_t fe = (p->prec == SWE_FP64) ? 16 : 8;
    const size_t npt = (size_t)p->nlat * p->nlon;
    const size_t four = (size_t)(p->M + 1) * p->nlat;
    size_t b = 0;
    b += a256(16 * (size_t)p->ncx * 7 * S);       // X operands
    b += a256(fe * four * 7 * S);                 // Fourier
    b += a256(rt * npt * 7 * S);                  // grid fields
    b += 2 * a256(rt * npt * 3 * S);              // Vc current / previous
    b += 2 * a256(rt * npt * S);                  // N_R current / previous
    b += a256(rt * npt * 3 * S);                  // R grid
    b += a256(rt * npt * 4 * S);                  // grid fields of an explicit previous state
    b += a256(16 * (size_t)p->ncx * 3 * S);       // forward results
    b += a256(16 * 3 * (size_t)p->nc * S);        // R spectral
    return b;
}

struct SLBuf {
    double2 *X, *Y, *Rs;
    void *Fq, *G, *Vc, *Vp, *Nc, *Np, *R, *Gp;
};

static SLBuf sl_carve(const swe_plan* p, char* c, int S) {
    const size_t rt = (p->prec == SWE_FP64) ? 8 : 4;
    const size_t fe = (p->prec == SWE_FP64) ? 16 : 8;
    const size_t npt = (size_t)p->nlat * p->nlon;
    const size_t four = (size_t)(p->M + 1) * p->nlat;
    SLBuf b;
    b.X = (double2*)c; c += a256(16 * (size_t)p->ncx * 7 * S);
    b.Fq = c; c += a256(fe * four * 7 * S);
    b.G = c; c += a256(rt * npt * 7 * S);
    b.Vc = c; c += a256(rt * npt * 3 * S);
    b.Vp = c; c += a256(rt * npt * 3 * S);
    b.Nc = c; c += a256(rt * npt * S);
    b.Np = c; c += a256(rt * npt * S);
    b.R = c; c += a256(rt * npt * 3 * S);
    b.Gp = c; c += a256(rt * npt * 4 * S);
    b.Y = (double2*)c; c += a256(16 * (size_t)p->ncx * 3 * S);
    b.Rs = (double2*)c;
    return b;
}

static swe_status ensure_thx(swe_plan* p) {
    if (p->thx) return SWE_OK;
    const size_t n = 3 * (size_t)p->nlat + 4 + 4 * ((size_t)p->nlat + 4);
    p->gen += 1;
    if (p->prec == SWE_FP64) {
        SWE_CHECK_CUDA(cudaMalloc(&p->thx, sizeof(double) * n));
        k_sl_table<double><<<nb(p->nlat + 4, 64), 64>>>(p->mu, (double*)p->thx, p->nlat);
    } else {
        SWE_CHECK_CUDA(cudaMalloc(&p->thx, sizeof(float) * n));
        k_sl_table<float><<<nb(p->nlat + 4, 64), 64>>>(p->mu, (float*)p->thx, p->nlat);
    }
    SWE_CHECK_LAUNCH("k_sl_table");
    SWE_CHECK_CUDA(cudaDeviceSynchronize());
    return SWE_OK;
}

swe_status sl_prepare(swe_plan* p) { return ensure_thx(p); }

template <typename T>
static swe_status vel_launch(const swe_plan* p, const void* G, int fp, int fd, int fu, int fv, void* Vc, void* NR,
                             int S, cudaStream_t st) {
    const int64_t n = (int64_t)p->nlat * p->nlon * S;
    k_sl_vel<T><<<nb(n), 256, 0, st>>>((const T*)G, fp, fd, fu, fv, (T*)Vc, (T*)NR, (const T*)p->thx, S, p->nlat,
                                       p->nlon);
    SWE_CHECK_LAUNCH("k_sl_vel");
    return SWE_OK;
}

// One SL-SI-SETTLS step on SoA states.  Uprev == nullptr and !have_prev -> one-step form.
// have_prev: the previous step's velocity / N_R are already in the workspace (chain inside one call).
// Result written to Uout (may not alias U).
swe_status sl_step(swe_plan* p, double dt, double nu, int q, const double2* Uprev, bool have_prev, const double2* U,
                   double2* Uout, int S, char* ws, bool swap_prev, cudaStream_t st) {
    SWE_CHECK(ensure_thx(p));
    SLBuf b = sl_carve(p, ws, S);
    const double h = 0.5 * dt;
    const bool f64 = (p->prec == SWE_FP64);
    const int64_t npt = (int64_t)p->nlat * p->nlon;
    // operands of the current state (7 fields) -> grid
    SV v{U, p->nc, S, p->M};
    {
        ProfToken tk_ = prof_begin("sl_operands", st, 0.0, 16.0 * S * (3.0 * p->nc + 7.0 * p->ncx));
        if (f64)
            k_sl_operands<<<nb(p->ncx * S), 256, 0, st>>>(v, b.X, p->row_m, p->ncx, 7, 1, h, 1.0 / (p->a * p->a),
                                                          p->omega, p->phibar, p->rc);
        else
            k_sl_operands<<<nb(p->ncx * S), 256, 0, st>>>(v, reinterpret_cast<float2*>(b.X), p->row_m, p->ncx, 7, 1,
                                                          h, 1.0 / (p->a * p->a), p->omega, p->phibar, p->rc);
        prof_end(tk_, st);
    }
    SWE_CHECK_LAUNCH("k_sl_operands");
    SWE_CHECK(leg_inverse(p, b.X, b.Fq, 7 * S, st));
    SWE_CHECK(ring_inverse(p, b.Fq, b.G, 7 * S, st));
    // current velocity / N_R
    if (f64) SWE_CHECK(vel_launch<double>(p, b.G, 3, 4, 5, 6, b.Vc, b.Nc, S, st));
    else SWE_CHECK(vel_launch<float>(p, b.G, 3, 4, 5, 6, b.Vc, b.Nc, S, st));
    // previous velocity / N_R
    const void* Vm = b.Vc;
    const void* Nm = b.Nc;
    if (have_prev) {
        Vm = b.Vp;
        Nm = b.Np;
    } else if (Uprev) {
        // grid fields (Phi', delta, U_cos, V_cos) of the previous state -> previous velocity / N_R
        SV vp{Uprev, p->nc, S, p->M};
        if (f64)
            k_sl_operands<<<nb(p->ncx * S), 256, 0, st>>>(vp, b.X, p->row_m, p->ncx, 4, 0, h, 1.0 / (p->a * p->a),
                                                          p->omega, p->phibar, p->rc);
        else
            k_sl_operands<<<nb(p->ncx * S), 256, 0, st>>>(vp, reinterpret_cast<float2*>(b.X), p->row_m, p->ncx, 4,
                                                          0, h, 1.0 / (p->a * p->a), p->omega, p->phibar, p->rc);
        SWE_CHECK_LAUNCH("k_sl_operands(prev)");
        SWE_CHECK(leg_inverse(p, b.X, b.Fq, 4 * S, st));
        SWE_CHECK(ring_inverse(p, b.Fq, b.Gp, 4 * S, st));
        if (f64) SWE_CHECK(vel_launch<double>(p, b.Gp, 0, 1, 2, 3, b.Vp, b.Np, S, st));
        else SWE_CHECK(vel_launch<float>(p, b.Gp, 0, 1, 2, 3, b.Vp, b.Np, S, st));
        Vm = b.Vp;
        Nm = b.Np;
    }
    // X_Phi += h (2 N_R^n - N_R^{n-1}); W = 2 V^n - V^{n-1} into the (now free) previous-state
    // grid block, or V^n itself in the one-step form
    const bool two = Vm != b.Vc;
    const void* W = two ? b.Gp : b.Vc;
    if (f64) {
        k_sl_xphi<double><<<nb(npt * S), 256, 0, st>>>((double*)b.G, (const double*)b.Nc, (const double*)Nm, h, S,
                                                        npt, (const double*)b.Vc, (const double*)Vm,
                                                        two ? (double*)b.Gp : nullptr);
    } else {
        k_sl_xphi<float><<<nb(npt * S), 256, 0, st>>>((float*)b.G, (const float*)b.Nc, (const float*)Nm, (float)h, S,
                                                       npt, (const float*)b.Vc, (const float*)Vm,
                                                       two ? (float*)b.Gp : nullptr);
    }
    SWE_CHECK_LAUNCH("k_sl_xphi");
    if (f64) {
        {
            ProfToken tk_ = prof_begin("sl_depart", st, 0.0, (f64 ? 8.0 : 4.0) * 13.0 * npt * S);
            k_sl_depart<double><<<nb(npt * S, 128), 128, 0, st>>>((const double*)b.G, (const double*)b.Vc,
                                                              (const double*)W, (const double*)b.Nc, (double*)b.R,
                                                              (const double*)p->thx, h, p->a, S, p->nlat, p->nlon);
            prof_end(tk_, st);
        }
    } else {
        {
            ProfToken tk_ = prof_begin("sl_depart", st, 0.0, (f64 ? 8.0 : 4.0) * 13.0 * npt * S);
            k_sl_depart<float><<<nb(npt * S, 128), 128, 0, st>>>((const float*)b.G, (const float*)b.Vc,
                                                             (const float*)W, (const float*)b.Nc, (float*)b.R,
                                                             (const float*)p->thx, (float)h, (float)p->a, S,
                                                             p->nlat, p->nlon);
            prof_end(tk_, st);
        }
    }
    SWE_CHECK_LAUNCH("k_sl_depart");
    SWE_CHECK(ring_forward(p, b.R, b.Fq, 3 * S, st));
    SWE_CHECK(leg_forward(p, b.Fq, b.Y, 3 * S, st));
    {
        ProfToken tk_ = prof_begin("sl_unpack", st, 0.0, 16.0 * 6.0 * p->nc * S);
        if (f64)
            k_sl_unpack<<<nb(p->nc * S), 256, 0, st>>>(b.Y, b.Rs, p->srow_m, p->M, p->nc, S);
        else
            k_sl_unpack<<<nb(p->nc * S), 256, 0, st>>>(reinterpret_cast<const float2*>(b.Y), b.Rs, p->srow_m, p->M,
                                                       p->nc, S);
        prof_end(tk_, st);
    }
    SWE_CHECK_LAUNCH("k_sl_unpack");
    SWE_CHECK(k_implicit(p, h, 0, b.Rs, Uout, dt, nu, q, S, st));
    if (swap_prev) {
        // the current velocity / N_R become the previous ones of the next step
        const size_t rt = f64 ? 8 : 4;
        SWE_CHECK_CUDA(cudaMemcpyAsync(b.Vp, b.Vc, rt * npt * 3 * S, cudaMemcpyDeviceToDevice, st));
        SWE_CHECK_CUDA(cudaMemcpyAsync(b.Np, b.Nc, rt * npt * S, cudaMemcpyDeviceToDevice, st));
    }
    return SWE_OK;
}
