// Advective form of the geopotential tendency (Eq. 1 as written): N_Phi = -V.grad(Phi') - Phi' delta.
//
// The default nonlinear evaluation uses the analytically identical flux form -div(Phi' V)
// (mass-conserving to rounding).  With the advective form selected on a plan
// (swe_plan_set_nphi_form), every nonlinear evaluation also runs this path and takes N_Phi
// from it:
//   1. operands (one pass over the state): U, V = (u, v) cos(lat) from xi, delta (as for the
//      fused ring kernel), Phi', delta, dPhi'/dlambda = i m Phi'_mn and (1 - mu^2) dPhi'/dmu,
//      whose coefficient of degree n is -(n-1) eps_n Phi'_{n-1} + (n+2) eps_{n+1} Phi'_{n+1};
//   2. inverse Legendre contraction and inverse longitude FFT of the six fields;
//   3. on the grid: N_Phi = -[U dPhi'/dlambda + V (1 - mu^2) dPhi'/dmu] / (a (1 - mu^2)) - Phi' delta;
//   4. forward FFT and forward Legendre contraction of N_Phi (a scalar transform).
// Unlike the fused path, the six grid fields go through HBM; this is an alternative physics
// mode, not the benchmarked one.
#include "swe_internal.cuh"

namespace {

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

template <typename T>
__device__ __forceinline__ typename V2<T>::t load_state(const double2* a, const double2* b, T beta, int64_t nc, int S,
                                                        int M, int f, int m, int n, int s) {
    using C = typename V2<T>::t;
    if (n < m || n > M || (n == 0 && f > 0)) return C{0, 0};
    const int64_t i = ((int64_t)f * nc + st_off(m, M) + (n - m)) * S + s;
    double2 v = a[i];
    if (b) {
        v.x += (double)beta * b[i].x;
        v.y += (double)beta * b[i].y;
    }
    return C{(T)v.x, (T)v.y};
}

// X2[rx][6S]: U, V, Phi', delta, dPhi'/dlambda, (1 - mu^2) dPhi'/dmu   (rows n = m..M+1)
template <typename T>
__global__ void k_nphi_pre(const double2* __restrict__ Ua, const double2* __restrict__ Ub, T beta,
                           typename V2<T>::t* __restrict__ X, const int* __restrict__ row_m, int64_t ncx, int64_t nc,
                           int M, int S, const T* __restrict__ rc) {
    using C = typename V2<T>::t;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ncx * S) return;
    const int s = (int)(t % S);
    const int64_t rx = t / S;
    const int m = row_m[rx];
    const int n = m + (int)(rx - ex_off(m, M));
    const T* c = rc + rx * RC_NUM;
    auto g = [&](int f, int nn) { return load_state<T>(Ua, Ub, beta, nc, S, M, f, m, nn, s); };
    const C xi0 = g(1, n), de0 = g(2, n), xim = g(1, n - 1), dem = g(2, n - 1), xip = g(1, n + 1), dep = g(2, n + 1);
    const C ph0 = g(0, n), phm = g(0, n - 1), php = g(0, n + 1);
    const T uc0 = c[RC_UC0], ucm = c[RC_UCM], ucp = c[RC_UCP], gm = c[RC_GM], gp = c[RC_GP];
    C* row = X + rx * 6 * (int64_t)S + s;
    row[0] = C{ucm * xim.x - ucp * xip.x - uc0 * de0.y, ucm * xim.y - ucp * xip.y + uc0 * de0.x};
    row[S] = C{-ucm * dem.x + ucp * dep.x - uc0 * xi0.y, -ucm * dem.y + ucp * dep.y + uc0 * xi0.x};
    row[2 * S] = ph0;
    row[3 * S] = de0;
    row[4 * S] = C{-(T)m * ph0.y, (T)m * ph0.x};
    row[5 * S] = C{gm * phm.x + gp * php.x, gm * phm.y + gp * php.y};
}

// G[(f S + s)][j][k] grid fields -> G[s][j][k] = N_Phi
template <typename T>
__global__ void k_nphi_grid(T* __restrict__ G, const double* __restrict__ mu, int nlat, int nlon, int S, T ia) {
    const int64_t plane = (int64_t)nlat * nlon;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= plane * S) return;
    const int s = (int)(t / plane);
    const int64_t q = t - (int64_t)s * plane;
    const int j = (int)(q / nlon);
    const double muj = mu[j];
    const T ic2 = (T)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    auto at = [&](int f) { return G[((int64_t)f * S + s) * plane + q]; };
    const T u = at(0), v = at(1), ph = at(2), de = at(3), pl = at(4), pm = at(5);
    G[(int64_t)s * plane + q] = -(u * pl + v * pm) * ia * ic2 - ph * de;
}

}  // namespace

swe_status nphi_adv_eval(const swe_plan* p, const double2* Ua, const double2* Ub, double beta, const NLBuffers& b,
                         int S, cudaStream_t st) {
    if (!b.X2) {
        swe_set_error("advective geopotential tendency: workspace not carved for it");
        return SWE_EINVAL;
    }
    const int64_t plane = (int64_t)p->nlat * p->nlon;
    if (p->prec == SWE_FP64) {
        k_nphi_pre<double><<<nblk(p->ncx * S), 256, 0, st>>>(Ua, Ub, beta, b.X2, p->row_m, p->ncx, p->nc, p->M, S, p->rc);
    } else {
        k_nphi_pre<float><<<nblk(p->ncx * S), 256, 0, st>>>(Ua, Ub, (float)beta, reinterpret_cast<float2*>(b.X2),
                                                            p->row_m, p->ncx, p->nc, p->M, S, p->rcf);
    }
    SWE_CHECK_LAUNCH("k_nphi_pre");
    SWE_CHECK(leg_inverse(p, b.X2, b.F2, 6 * S, st));
    SWE_CHECK(ring_inverse(p, b.F2, b.G2, 6 * S, st));
    if (p->prec == SWE_FP64)
        k_nphi_grid<double><<<nblk(plane * S), 256, 0, st>>>((double*)b.G2, p->mu, p->nlat, p->nlon, S, 1.0 / p->a);
    else
        k_nphi_grid<float><<<nblk(plane * S), 256, 0, st>>>((float*)b.G2, p->mu, p->nlat, p->nlon, S,
                                                            (float)(1.0 / p->a));
    SWE_CHECK_LAUNCH("k_nphi_grid");
    SWE_CHECK(ring_forward(p, b.G2, b.F3, S, st));
    SWE_CHECK(leg_forward(p, b.F3, b.Y2, S, st));
    return SWE_OK;
}
