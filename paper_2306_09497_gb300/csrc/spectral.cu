// Spectral-space kernels: operand construction for the transforms, assembly of the
// nonlinear tendency, the linear operator L = L_G + L_C (Eq. 1, f = 2 Omega mu), the
// Crank-Nicolson / semi-implicit solve (I - alpha L) X = R (Eqs. 4, 7), backward-Euler
// viscosity (App. A) and the nonlinear-balance initial state.
//
// State layout inside the library ("SoA"): [3][NC][S] complex128, slice fastest,
// so that every kernel here reads and writes whole 32-slice segments.
//
// Spectral identities used (mu = sin(latitude), eps_n^m = sqrt((n^2-m^2)/(4n^2-1))):
//   mu P_n^m = eps_{n+1}^m P_{n+1}^m + eps_n^m P_{n-1}^m
//   (1 - mu^2) dP_n^m/dmu = -n eps_{n+1}^m P_{n+1}^m + (n+1) eps_n^m P_{n-1}^m
// With psi = lap^{-1} xi, chi = lap^{-1} delta, U = u cos(lat), V = v cos(lat):
//   U_n = (1/a)[i m chi_n + (n-1) eps_n psi_{n-1} - (n+2) eps_{n+1} psi_{n+1}]
//   V_n = (1/a)[i m psi_n - (n-1) eps_n chi_{n-1} + (n+2) eps_{n+1} chi_{n+1}]   (n <= M+1)
// and for a vector with components (A, B) = (a_lon, a_lat) cos(lat) whose quadrature
// projections on P_n^m of A/(1-mu^2), B/(1-mu^2) are Ahat, Bhat (n <= M+1):
//   div_n  = (1/a)[i m Ahat_n + n eps_{n+1} Bhat_{n+1} - (n+1) eps_n Bhat_{n-1}]
//   curl_n = (1/a)[i m Bhat_n - n eps_{n+1} Ahat_{n+1} + (n+1) eps_n Ahat_{n-1}]
// The Coriolis operator follows from -div(fV) = -f delta - (2 Omega/a) V and
// curl(fV) = f xi - (2 Omega/a) U:
//   (L_C U)_xi,n    = -2 Omega [p_n delta_{n-1} + q_n delta_{n+1} - i r_n xi_n]
//   (L_C U)_delta,n =  2 Omega [p_n xi_{n-1}    + q_n xi_{n+1}    + i r_n delta_n]
//   p_n = (n+1)/n eps_n,  q_n = n/(n+1) eps_{n+1},  r_n = m/(n(n+1)).
#include "swe_internal.cuh"

namespace {

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_inv(double2 a) {
    double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ double coef_p(int m, int n) { return n >= 1 ? (n + 1.0) / n * eps_nm(m, n) : 0.0; }
__device__ __forceinline__ double coef_q(int m, int n) { return n >= 1 ? n / (n + 1.0) * eps_nm(m, n + 1) : 0.0; }
__device__ __forceinline__ double coef_r(int m, int n) { return n >= 1 ? (double)m / ((double)n * (n + 1.0)) : 0.0; }

__device__ __forceinline__ void flag_nonfinite(int* flags, double2 v) {
    if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(flags, 1);
}

// ------------------------------------------------------------------ layouts
__global__ void k_aos_soa(const double2* __restrict__ in, double2* __restrict__ out, int64_t nc, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = 3 * nc * S;
    if (t >= total) return;
    int s = (int)(t % S);
    int64_t fr = t / S;          // f * nc + r
    out[t] = in[(int64_t)s * 3 * nc + fr];
}

__global__ void k_soa_aos(const double2* __restrict__ in, double2* __restrict__ out, int64_t nc, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = 3 * nc * S;
    if (t >= total) return;
    int64_t fr = t % (3 * nc);
    int s = (int)(t / (3 * nc));
    out[t] = in[fr * S + s];
}

// strided variants: state s lives at in + s * stride (stride in complex values)
__global__ void k_aos_soa_strided(const double2* __restrict__ in, int64_t stride, double2* __restrict__ out,
                                  int64_t nc, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * nc * S) return;
    int s = (int)(t % S);
    int64_t fr = t / S;
    out[t] = in[(int64_t)s * stride + fr];
}

__global__ void k_soa_aos_strided(const double2* __restrict__ in, double2* __restrict__ out, int64_t stride,
                                  const double2* __restrict__ add, int64_t add_stride, int64_t nc, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * nc * S) return;
    int64_t fr = t % (3 * nc);
    int s = (int)(t / (3 * nc));
    double2 v = in[fr * S + s];
    if (add) v = c_add(v, add[(int64_t)s * add_stride + fr]);
    out[(int64_t)s * stride + fr] = v;
}

// Tiled forms of the strided layout changes for batches of at least TT states: a TT x TT
// tile of complex values passes through shared memory, so that the per-state side and the
// batched side are both read / written as 512-byte rows (a plain element-per-thread
// transpose makes one of the two sides a 16-byte gather).  n = 3 nc values per state.
constexpr int TT = 32;

__global__ void __launch_bounds__(256) k_aos_soa_tiled(const double2* __restrict__ in, int64_t stride,
                                                       double2* __restrict__ out, int64_t n, int S) {
    __shared__ double2 tile[TT][TT + 1];
    const int64_t r0 = (int64_t)blockIdx.x * TT;
    const int s0 = blockIdx.y * TT;
    const int tx = threadIdx.x & (TT - 1), ty = threadIdx.x / TT;
#pragma unroll
    for (int i = ty; i < TT; i += 256 / TT) {
        const int s = s0 + i;
        const int64_t r = r0 + tx;
        if (s < S && r < n) tile[i][tx] = in[(int64_t)s * stride + r];
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < TT; i += 256 / TT) {
        const int64_t r = r0 + i;
        const int s = s0 + tx;
        if (s < S && r < n) out[r * S + s] = tile[tx][i];
    }
}

__global__ void __launch_bounds__(256) k_soa_aos_tiled(const double2* __restrict__ in, double2* __restrict__ out,
                                                       int64_t stride, const double2* __restrict__ add,
                                                       int64_t add_stride, int64_t n, int S) {
    __shared__ double2 tile[TT][TT + 1];
    const int64_t r0 = (int64_t)blockIdx.x * TT;
    const int s0 = blockIdx.y * TT;
    const int tx = threadIdx.x & (TT - 1), ty = threadIdx.x / TT;
#pragma unroll
    for (int i = ty; i < TT; i += 256 / TT) {
        const int64_t r = r0 + i;
        const int s = s0 + tx;
        if (s < S && r < n) tile[i][tx] = in[r * S + s];
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < TT; i += 256 / TT) {
        const int s = s0 + i;
        const int64_t r = r0 + tx;
        if (s < S && r < n) {
            double2 v = tile[tx][i];
            if (add) v = c_add(v, add[(int64_t)s * add_stride + r]);
            out[(int64_t)s * stride + r] = v;
        }
    }
}

__global__ void k_pack(const double2* __restrict__ spec, double2* __restrict__ X, const int* __restrict__ row_m, int M,
                       int64_t nc, int64_t ncx, int B) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ncx * B) return;
    int b = (int)(t % B);
    int64_t rx = t / B;
    int m = row_m[rx];
    int n = m + (int)(rx - ex_off(m, M));
    X[t] = (n <= M) ? spec[(int64_t)b * nc + st_off(m, M) + (n - m)] : czero();
}

__global__ void k_pack_f32(const double2* __restrict__ spec, float2* __restrict__ X, const int* __restrict__ row_m,
                           int M, int64_t nc, int64_t ncx, int B) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ncx * B) return;
    int b = (int)(t % B);
    int64_t rx = t / B;
    int m = row_m[rx];
    int n = m + (int)(rx - ex_off(m, M));
    X[t] = (n <= M) ? d2f2(spec[(int64_t)b * nc + st_off(m, M) + (n - m)]) : make_float2(0.f, 0.f);
}

__global__ void k_unpack_f32(const float2* __restrict__ Y, double2* __restrict__ spec, const int* __restrict__ srow_m,
                             int M, int64_t nc, int B) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * B) return;
    int64_t r = t % nc;
    int b = (int)(t / nc);
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    spec[t] = f2d2(Y[(ex_off(m, M) + (n - m)) * B + b]);
}

__global__ void k_unpack(const double2* __restrict__ Y, double2* __restrict__ spec, const int* __restrict__ srow_m,
                         int M, int64_t nc, int B) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * B) return;
    int64_t r = t % nc;
    int b = (int)(t / nc);
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    spec[t] = Y[(ex_off(m, M) + (n - m)) * B + b];
}

// ------------------------------------------------------------------ nonlinear pre / post
struct StateView {
    const double2* a;
    const double2* b;
    double beta;
    int64_t nc;
    int S;
    int M;
    __device__ __forceinline__ double2 get(int f, int m, int n, int s) const {
        if (n < m || n > M) return czero();
        if (n == 0 && f > 0) return czero();     // xi_00 = delta_00 = 0
        int64_t i = ((int64_t)f * nc + st_off(m, M) + (n - m)) * S + s;
        double2 v = a[i];
        if (b) v = c_add(v, c_scale(b[i], beta));
        return v;
    }
};

__global__ void k_nl_pre_kernel(StateView U, double2* __restrict__ X, const int* __restrict__ row_m, int64_t ncx,
                                const double* __restrict__ rc) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int S = U.S, M = U.M;
    if (t >= ncx * S) return;
    int s = (int)(t % S);
    int64_t rx = t / S;
    int m = row_m[rx];
    int n = m + (int)(rx - ex_off(m, M));
    const double* c = rc + rx * RC_NUM;
    const double uc0 = c[RC_UC0], ucm = c[RC_UCM], ucp = c[RC_UCP];
    // U = i m chi_n/a + (n-1) eps_n psi_{n-1}/a - (n+2) eps_{n+1} psi_{n+1}/a, V likewise (psi <-> chi)
    const double2 xi0 = U.get(1, m, n, s), de0 = U.get(2, m, n, s);
    const double2 xim = U.get(1, m, n - 1, s), dem = U.get(2, m, n - 1, s);
    const double2 xip = U.get(1, m, n + 1, s), dep = U.get(2, m, n + 1, s);
    double2 Uh, Vh;
    Uh.x = fma(ucm, xim.x, fma(-ucp, xip.x, -uc0 * de0.y));
    Uh.y = fma(ucm, xim.y, fma(-ucp, xip.y, uc0 * de0.x));
    Vh.x = fma(-ucm, dem.x, fma(ucp, dep.x, -uc0 * xi0.y));
    Vh.y = fma(-ucm, dem.y, fma(ucp, dep.y, uc0 * xi0.x));
    double2* row = X + rx * 4 * (int64_t)S + s;
    row[0] = U.get(0, m, n, s);
    row[S] = xi0;
    row[2 * S] = Uh;
    row[3 * S] = Vh;
}

__global__ void k_nl_post_kernel(const double2* __restrict__ Y, int mode, double dt, const double2* __restrict__ in0,
                                 const double2* __restrict__ in1, double2* __restrict__ out0,
                                 double2* __restrict__ out1, const int* __restrict__ srow_m, int M, int64_t nc, int S,
                                 double ia, const double* __restrict__ rc, int* flags,
                                 const double2* __restrict__ Yphi) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * S) return;
    int s = (int)(t % S);
    int64_t r = t / S;
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    const int64_t rx = ex_off(m, M) + (n - m);
    const int64_t C5 = 5 * (int64_t)S;
    const double2* y0 = Y + rx * C5 + s;
    const double2* yp = y0 + C5;                       // n + 1 (<= M + 1 always present)
    const bool hm = (n - 1 >= m);
    const double2* ym = y0 - C5;
    double2 A1 = y0[0], B1 = y0[S], A2 = y0[2 * S], KE = y0[4 * S];
    double2 A1p = yp[0], B1p = yp[S], B2p = yp[3 * S];
    double2 A1m = hm ? ym[0] : czero(), B1m = hm ? ym[S] : czero(), B2m = hm ? ym[3 * S] : czero();
    const double* c = rc + rx * RC_NUM;
    const double cp = c[RC_DCP], cm = c[RC_DCM], ma = m * ia;
    // div = i m A/a + n eps_{n+1} B_{n+1}/a - (n+1) eps_n B_{n-1}/a ; curl likewise (A <-> B, sign)
    double2 N[3];
    N[0] = Yphi ? Yphi[rx * S + s]       // advective form, already a scalar transform
                : make_double2(-fma(cp, B2p.x, fma(-cm, B2m.x, -ma * A2.y)), -fma(cp, B2p.y, fma(-cm, B2m.y, ma * A2.x)));
    N[1] = make_double2(-fma(cp, B1p.x, fma(-cm, B1m.x, -ma * A1.y)), -fma(cp, B1p.y, fma(-cm, B1m.y, ma * A1.x)));
    const double ke = (double)(n * (n + 1)) * ia * ia;
    N[2] = make_double2(fma(cm, A1m.x, fma(-cp, A1p.x, fma(ke, KE.x, -ma * B1.y))),
                        fma(cm, A1m.y, fma(-cp, A1p.y, fma(ke, KE.y, ma * B1.x))));
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        int64_t i = ((int64_t)f * nc + r) * S + s;
        flag_nonfinite(flags, N[f]);
        if (mode == POST_N) {
            out0[i] = N[f];
        } else if (mode == POST_STAGE1) {
            double2 ub = c_scale(N[f], dt);
            out0[i] = ub;
            out1[i] = c_add(in0[i], ub);
        } else {
            out0[i] = c_add(in0[i], c_scale(c_add(in1[i], c_scale(N[f], dt)), 0.5));
        }
    }
}

// ------------------------------------------------------------------ linear operator
// mode 0: out = L U ; mode 1: out = U + alpha L U
__global__ void k_linop(StateView U, double2* __restrict__ out, const int* __restrict__ srow_m, int mode,
                        double alpha, double ia2, double omega, double phibar, const double* __restrict__ rc) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int S = U.S, M = U.M;
    const int64_t nc = U.nc;
    if (t >= nc * S) return;
    int s = (int)(t % S);
    int64_t r = t / S;
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    double2 ph = U.get(0, m, n, s), xi = U.get(1, m, n, s), de = U.get(2, m, n, s);
    double2 xim = U.get(1, m, n - 1, s), xip = U.get(1, m, n + 1, s);
    double2 dem = U.get(2, m, n - 1, s), dep = U.get(2, m, n + 1, s);
    const double* c = rc + (ex_off(m, M) + (n - m)) * RC_NUM;
    const double w2 = 2.0 * omega;
    const double p = w2 * c[RC_P], q = w2 * c[RC_Q], rr = w2 * c[RC_R];
    const double lap = (double)(n * (n + 1)) * ia2;
    double2 L0 = c_scale(de, -phibar);
    double2 L1 = make_double2(-fma(p, dem.x, fma(q, dep.x, rr * xi.y)), -fma(p, dem.y, fma(q, dep.y, -rr * xi.x)));
    double2 L2 = make_double2(fma(lap, ph.x, fma(p, xim.x, fma(q, xip.x, -rr * de.y))),
                              fma(lap, ph.y, fma(p, xim.y, fma(q, xip.y, rr * de.x))));
    double2 o[3] = {L0, L1, L2};
    if (mode == 1) {
        o[0] = make_double2(fma(alpha, L0.x, ph.x), fma(alpha, L0.y, ph.y));
        o[1] = make_double2(fma(alpha, L1.x, xi.x), fma(alpha, L1.y, xi.y));
        o[2] = make_double2(fma(alpha, L2.x, de.x), fma(alpha, L2.y, de.y));
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) out[((int64_t)f * nc + r) * S + s] = o[f];
}

// ------------------------------------------------------------------ implicit solve
// Eliminating Phi_n = R^Phi_n - alpha Phi_bar delta_n and xi_{n+-1} from (I - alpha L) X = R
// leaves, for each m and each parity of n - m, a tridiagonal system in delta:
//   a_k delta_{n-2} + b_k delta_n + c_k delta_{n+2} = rhs_k,   n = m + par + 2k, with c = 2 Omega alpha,
//   d_j = 1 - i c r_j,  D_n = 1 + alpha^2 Phi_bar n(n+1)/a^2 - i c r_n,
//   a_k = c^2 p_n p_{n-1}/d_{n-1},  c_k = c^2 q_n q_{n+1}/d_{n+1},
//   b_k = D_n + c^2 p_n q_{n-1}/d_{n-1} + c^2 q_n p_{n+1}/d_{n+1},
//   rhs_k = R^delta_n + alpha n(n+1)/a^2 R^Phi_n + c p_n R^xi_{n-1}/d_{n-1} + c q_n R^xi_{n+1}/d_{n+1}
// (terms with xi_{n+1} only when n+1 <= M), then
//   xi_n = [R^xi_n - c (p_n delta_{n-1} + q_n delta_{n+1})] / d_n.
// The Thomas factorisation depends only on (m, n, alpha) and is precomputed:
//   fac[0] = a_k, fac[1] = 1/(b_k - a_k c'_{k-1}), fac[2] = c'_k, fac[3] = c p_n/d_{n-1},
//   fac[4] = c q_n/d_{n+1}, fac[5] = 1/d_n, fac[6] = (c p_n, c q_n [n+1<=M]),
//   fac[7] = (alpha n(n+1)/a^2, alpha Phi_bar).
__global__ void k_cn_factor(int M, double alpha, double a, double omega, double phibar, double2* __restrict__ fac) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * (M + 1)) return;
    const int m = t >> 1, par = t & 1;
    const double c = 2.0 * omega * alpha;
    auto dd = [&](int j) { return make_double2(1.0, -c * coef_r(m, j)); };
    double2 cprev = czero();
    for (int n = m + par; n <= M; n += 2) {
        const bool hm = (n - 1 >= m), hp = (n + 1 <= M);
        const double pn = coef_p(m, n), qn = coef_q(m, n);
        double2 Dn = make_double2(1.0 + alpha * alpha * phibar * n * (n + 1.0) / (a * a), -c * coef_r(m, n));
        double2 ak = czero(), ck = czero(), Em = czero(), Ep = czero();
        double2 bk = Dn;
        if (hm) {
            double2 idm = c_inv(dd(n - 1));
            ak = c_scale(idm, c * c * pn * coef_p(m, n - 1));
            bk = c_add(bk, c_scale(idm, c * c * pn * coef_q(m, n - 1)));
            Em = c_scale(idm, c * pn);
        }
        if (hp) {
            double2 idp = c_inv(dd(n + 1));
            ck = c_scale(idp, c * c * qn * coef_q(m, n + 1));
            bk = c_add(bk, c_scale(idp, c * c * qn * coef_p(m, n + 1)));
            Ep = c_scale(idp, c * qn);
        }
        double2 g = c_inv(c_sub(bk, c_mul(ak, cprev)));
        double2 cpk = c_mul(ck, g);
        double2* f = fac + (st_off(m, M) + (n - m)) * 8;
        f[0] = ak;
        f[1] = g;
        f[2] = cpk;
        f[3] = Em;
        f[4] = Ep;
        f[5] = c_inv(dd(n));
        f[6] = make_double2(c * pn, hp ? c * qn : 0.0);
        f[7] = make_double2(alpha * n * (n + 1.0) / (a * a), alpha * phibar);
        cprev = cpk;
    }
}

__device__ __forceinline__ double visc_factor(int n, double dt, double nu, int q, double a) {
    if (nu <= 0.0) return 1.0;
    double l = (double)n * (n + 1.0) / (a * a);
    double lq = 1.0;
    for (int i = 0; i < q / 2; ++i) lq *= l;
    return 1.0 / (1.0 + dt * nu * lq);
}

// One thread per (m, parity, slice).  X may alias R: the thread of parity par
// reads R^Phi, R^delta at n = m+par (mod 2) and R^xi at the other parity, and
// writes Phi, delta and xi at exactly those positions, each after its last read;
// the other parity's thread touches the complementary positions.
__global__ void k_cn_solve(const double2* __restrict__ fac, const double2* R, double2* X, int M, int64_t nc, int S,
                           double vdt, double vnu, int vq, double a) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)2 * (M + 1) * S) return;
    const int s = (int)(t % S);
    const int mp = (int)(t / S);
    const int m = mp >> 1, par = mp & 1;
    const int64_t base = st_off(m, M);
    auto idx = [&](int f, int n) { return ((int64_t)f * nc + base + (n - m)) * S + s; };
    auto rxi = [&](int n) -> double2 {           // R^xi_n with xi_00 treated as zero
        if (n < m || n > M || n == 0) return czero();
        return R[idx(1, n)];
    };
    // forward elimination over delta_n, n = m + par + 2k
    double2 dprev = czero();
    int nlast = m + par - 2;
    for (int n = m + par; n <= M; n += 2) {
        const double2* f = fac + (base + (n - m)) * 8;
        double2 rp = R[idx(0, n)];
        double2 rd = (n == 0) ? czero() : R[idx(2, n)];
        double2 rhs = c_add(rd, c_scale(rp, f[7].x));
        rhs = c_add(rhs, c_mul(f[3], rxi(n - 1)));
        rhs = c_add(rhs, c_mul(f[4], rxi(n + 1)));
        double2 dp = c_mul(c_sub(rhs, c_mul(f[0], dprev)), f[1]);
        X[idx(2, n)] = dp;
        dprev = dp;
        nlast = n;
    }
    // back substitution for delta, then Phi_n = R^Phi_n - alpha Phi_bar delta_n
    double2 dnext = czero();
    for (int n = nlast; n >= m + par; n -= 2) {
        const double2* f = fac + (base + (n - m)) * 8;
        double2 dn = c_sub(X[idx(2, n)], c_mul(f[2], dnext));
        if (n == 0) dn = czero();
        dnext = dn;
        double2 ph = c_sub(R[idx(0, n)], c_scale(dn, f[7].y));
        X[idx(2, n)] = dn;
        X[idx(0, n)] = ph;
    }
    // xi on the other parity: xi_n = [R^xi_n - c p_n delta_{n-1} - c q_n delta_{n+1}] / d_n
    for (int n = m + (par ^ 1); n <= M; n += 2) {
        const double2* f = fac + (base + (n - m)) * 8;
        double2 dm = (n - 1 >= m) ? X[idx(2, n - 1)] : czero();
        double2 dpv = (n + 1 <= M) ? X[idx(2, n + 1)] : czero();
        double2 num = c_sub(rxi(n), c_add(c_scale(dm, f[6].x), c_scale(dpv, f[6].y)));
        double2 xn = (n == 0) ? czero() : c_mul(num, f[5]);
        X[idx(1, n)] = c_scale(xn, visc_factor(n, vdt, vnu, vq, a));
    }
    // backward-Euler viscosity on delta and Phi (after xi used the unscaled delta)
    if (vnu > 0.0) {
        for (int n = m + par; n <= M; n += 2) {
            double v = visc_factor(n, vdt, vnu, vq, a);
            X[idx(2, n)] = c_scale(X[idx(2, n)], v);
            X[idx(0, n)] = c_scale(X[idx(0, n)], v);
        }
    }
}

// Warp-parallel form of the same solve, for small batches: one warp per (m, parity, slice).
// Both recurrences are affine, x_k = A_k x_{k-1} + B_k (forward elimination with
// A = -a_k g_k, B = rhs_k g_k; back substitution, walked from the top degree down, with
// A = -c'_k, B = d'_k), so each 32-element chunk is an inclusive scan of the maps
// (A, B) under composition (A2 A1, A2 B1 + B2), continued from the previous chunk's value.
__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}

__device__ __forceinline__ void affine_scan(double2& A, double2& B) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        double2 Ap = shfl_up2(A, d), Bp = shfl_up2(B, d);
        if (lane >= d) {
            B = c_add(c_mul(A, Bp), B);
            A = c_mul(A, Ap);
        }
    }
}

__global__ void k_cn_solve_warp(const double2* __restrict__ fac, const double2* R, double2* X, int M, int64_t nc,
                                int S, double vdt, double vnu, int vq, double a) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)2 * (M + 1) * S) return;          // whole warps exit together
    const int s = (int)(w % S);
    const int mp = (int)(w / S);
    const int m = mp >> 1, par = mp & 1;
    const int64_t base = st_off(m, M);
    auto idx = [&](int f, int n) { return ((int64_t)f * nc + base + (n - m)) * S + s; };
    auto rxi = [&](int n) -> double2 {
        if (n < m || n > M || n == 0) return czero();
        return R[idx(1, n)];
    };
    const int n0 = m + par;
    const int K = (n0 <= M) ? (M - n0) / 2 + 1 : 0;
    // forward elimination: d'_k into X[delta]
    double2 carry = czero();
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        double2 A = czero(), B = czero();
        if (k < K) {
            const int n = n0 + 2 * k;
            const double2* f = fac + (base + (n - m)) * 8;
            double2 rhs = c_add((n == 0) ? czero() : R[idx(2, n)], c_scale(R[idx(0, n)], f[7].x));
            rhs = c_add(rhs, c_mul(f[3], rxi(n - 1)));
            rhs = c_add(rhs, c_mul(f[4], rxi(n + 1)));
            A = c_scale(c_mul(f[0], f[1]), -1.0);
            B = c_mul(rhs, f[1]);
        }
        affine_scan(A, B);
        const double2 v = c_add(c_mul(A, carry), B);
        __syncwarp();
        if (k < K) X[idx(2, n0 + 2 * k)] = v;
        carry = make_double2(__shfl_sync(0xffffffffu, v.x, 31), __shfl_sync(0xffffffffu, v.y, 31));
    }
    __syncwarp();
    // back substitution from the top: delta_k = -c'_k delta_{k+1} + d'_k; then Phi
    carry = czero();
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = K - 1 - (k0 + lane);
        double2 A = czero(), B = czero();
        if (k >= 0) {
            const int n = n0 + 2 * k;
            const double2* f = fac + (base + (n - m)) * 8;
            A = c_scale(f[2], -1.0);
            B = X[idx(2, n)];
        }
        affine_scan(A, B);
        double2 dn = c_add(c_mul(A, carry), B);
        carry = make_double2(__shfl_sync(0xffffffffu, dn.x, 31), __shfl_sync(0xffffffffu, dn.y, 31));
        __syncwarp();
        if (k >= 0) {
            const int n = n0 + 2 * k;
            if (n == 0) dn = czero();
            const double2* f = fac + (base + (n - m)) * 8;
            const double2 ph = c_sub(R[idx(0, n)], c_scale(dn, f[7].y));
            X[idx(2, n)] = dn;
            X[idx(0, n)] = ph;
        }
    }
    __syncwarp();
    // xi on the other parity (uses the unscaled delta)
    for (int n = m + (par ^ 1) + 2 * lane; n <= M; n += 64) {
        const double2* f = fac + (base + (n - m)) * 8;
        double2 dm = (n - 1 >= m) ? X[idx(2, n - 1)] : czero();
        double2 dpv = (n + 1 <= M) ? X[idx(2, n + 1)] : czero();
        double2 num = c_sub(rxi(n), c_add(c_scale(dm, f[6].x), c_scale(dpv, f[6].y)));
        double2 xn = (n == 0) ? czero() : c_mul(num, f[5]);
        X[idx(1, n)] = c_scale(xn, visc_factor(n, vdt, vnu, vq, a));
    }
    __syncwarp();
    if (vnu > 0.0) {
        for (int n = n0 + 2 * lane; n <= M; n += 64) {
            const double v = visc_factor(n, vdt, vnu, vq, a);
            X[idx(2, n)] = c_scale(X[idx(2, n)], v);
            X[idx(0, n)] = c_scale(X[idx(0, n)], v);
        }
    }
}

// ------------------------------------------------------------------ mixed-precision variants
// On split-precision plans the spectral kernels compute in FP32 on integer-pipe conversions
// of their FP64 operands (GB300 runs FP64 arithmetic and conversions at a small fraction of
// its FP32 rate).  Whatever feeds the FP32 transforms is produced in FP32; an update of the
// FP64 state adds an FP32 increment with one FP64 addition per real number, so the state
// keeps its FP64 resolution and only the increment carries FP32 rounding.
__global__ void k_to_f32(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = d2f2(in[t]);
}

__device__ __forceinline__ float2 fz() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 dadd_f(double2 a, float2 inc) {
    return make_double2(a.x + f2d_fast(inc.x), a.y + f2d_fast(inc.y));
}

struct StateViewF {
    const double2* a;
    const double2* b;
    float beta;
    int64_t nc;
    int S;
    int M;
    __device__ __forceinline__ float2 get(int f, int m, int n, int s) const {
        if (n < m || n > M) return fz();
        if (n == 0 && f > 0) return fz();
        int64_t i = ((int64_t)f * nc + st_off(m, M) + (n - m)) * S + s;
        float2 v = d2f2(a[i]);
        if (b) {
            const float2 w = d2f2(b[i]);
            v = make_float2(fmaf(beta, w.x, v.x), fmaf(beta, w.y, v.y));
        }
        return v;
    }
};

__global__ void k_nl_pre_f32(StateViewF U, float2* __restrict__ X, const int* __restrict__ row_m, int64_t ncx,
                             const float* __restrict__ rcf) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int S = U.S, M = U.M;
    if (t >= ncx * S) return;
    int s = (int)(t % S);
    int64_t rx = t / S;
    int m = row_m[rx];
    int n = m + (int)(rx - ex_off(m, M));
    const float* c = rcf + rx * RC_NUM;
    const float uc0 = c[RC_UC0], ucm = c[RC_UCM], ucp = c[RC_UCP];
    const float2 xi0 = U.get(1, m, n, s), de0 = U.get(2, m, n, s);
    const float2 xim = U.get(1, m, n - 1, s), dem = U.get(2, m, n - 1, s);
    const float2 xip = U.get(1, m, n + 1, s), dep = U.get(2, m, n + 1, s);
    float2 Uh, Vh;
    Uh.x = fmaf(ucm, xim.x, fmaf(-ucp, xip.x, -uc0 * de0.y));
    Uh.y = fmaf(ucm, xim.y, fmaf(-ucp, xip.y, uc0 * de0.x));
    Vh.x = fmaf(-ucm, dem.x, fmaf(ucp, dep.x, -uc0 * xi0.y));
    Vh.y = fmaf(-ucm, dem.y, fmaf(ucp, dep.y, uc0 * xi0.x));
    float2* row = X + rx * 4 * (int64_t)S + s;
    row[0] = U.get(0, m, n, s);
    row[S] = xi0;
    row[2 * S] = Uh;
    row[3 * S] = Vh;
}

__device__ __forceinline__ void flag_nonfinite_f(int* flags, float2 v) {
    if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(flags, 1);
}

__global__ void k_nl_post_f32(const float2* __restrict__ Y, int mode, float dt, const double2* __restrict__ in0,
                              const double2* __restrict__ in1, double2* __restrict__ out0,
                              double2* __restrict__ out1, const int* __restrict__ srow_m, int M, int64_t nc, int S,
                              float ia, const float* __restrict__ rcf, int* flags, const float2* __restrict__ Yphi) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * S) return;
    int s = (int)(t % S);
    int64_t r = t / S;
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    const int64_t rx = ex_off(m, M) + (n - m);
    const int64_t C5 = 5 * (int64_t)S;
    const float2* y0 = Y + rx * C5 + s;
    const float2* yp = y0 + C5;
    const bool hm = (n - 1 >= m);
    const float2* ym = y0 - C5;
    const float2 A1 = y0[0], B1 = y0[S], A2 = y0[2 * S], KE = y0[4 * S];
    const float2 A1p = yp[0], B1p = yp[S], B2p = yp[3 * S];
    const float2 A1m = hm ? ym[0] : fz(), B1m = hm ? ym[S] : fz(), B2m = hm ? ym[3 * S] : fz();
    const float* c = rcf + rx * RC_NUM;
    const float cp = c[RC_DCP], cm = c[RC_DCM], ma = (float)m * ia;
    float2 N[3];
    N[0] = Yphi ? Yphi[rx * S + s]       // advective form, already a scalar transform
                : make_float2(-fmaf(cp, B2p.x, fmaf(-cm, B2m.x, -ma * A2.y)), -fmaf(cp, B2p.y, fmaf(-cm, B2m.y, ma * A2.x)));
    N[1] = make_float2(-fmaf(cp, B1p.x, fmaf(-cm, B1m.x, -ma * A1.y)), -fmaf(cp, B1p.y, fmaf(-cm, B1m.y, ma * A1.x)));
    const float ke = (float)(n * (n + 1)) * ia * ia;
    N[2] = make_float2(fmaf(cm, A1m.x, fmaf(-cp, A1p.x, fmaf(ke, KE.x, -ma * B1.y))),
                       fmaf(cm, A1m.y, fmaf(-cp, A1p.y, fmaf(ke, KE.y, ma * B1.x))));
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        int64_t i = ((int64_t)f * nc + r) * S + s;
        flag_nonfinite_f(flags, N[f]);
        if (mode == POST_N) {
            out0[i] = f2d2(N[f]);
        } else if (mode == POST_STAGE1) {
            const float2 ub = make_float2(N[f].x * dt, N[f].y * dt);
            out0[i] = f2d2(ub);
            out1[i] = dadd_f(in0[i], ub);
        } else {
            const float2 b = d2f2(in1[i]);
            out0[i] = dadd_f(in0[i], make_float2(0.5f * fmaf(N[f].x, dt, b.x), 0.5f * fmaf(N[f].y, dt, b.y)));
        }
    }
}

// Implicit solve in increment form on split-precision plans:
//   kappa = 1:  (I - alpha L) X = U       ->  X = U + D,  (I - alpha L) D = alpha L U
//   kappa = 2:  (I - alpha L) X = (I + alpha L) U (Crank-Nicolson)  ->  X = U + D,  (I - alpha L) D = 2 alpha L U
// then backward-Euler viscosity X <- X v_n written as U + [D - (U + D) w_n], w_n = 1 - v_n.
// The right-hand side kappa alpha L U, the elimination (the FP32 copy of the Thomas
// factors of k_cn_factor) and the increment are FP32; X = U + increment is one FP64 add.
// U and X must not alias.  The two Thomas recurrences run as affine scans (as in
// k_cn_solve_warp): one warp per (m, parity, group of 32/KL slices); lane = (32/KL) kl + sl,
// with sl the slice within the group (KL = 8: 4 consecutive slices, 64-byte runs) and kl the
// position in a chunk of KL consecutive unknowns of the chain.  Passes: forward scan (d' parked in
// X[delta]), backward scan (D_delta parked in X[delta], Phi final), xi of the other parity
// (final), delta (final).
__device__ __forceinline__ float2 cmf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 shfl_up_f2(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
// inclusive scan of the maps x -> A x + B over kl = 0..KL-1 (lane stride 32/KL)
template <int KL>
__device__ __forceinline__ void affine_scan_kl(float2& A, float2& B, int kl) {
#pragma unroll
    for (int d = 1; d < KL; d <<= 1) {
        const float2 Ap = shfl_up_f2(A, (32 / KL) * d), Bp = shfl_up_f2(B, (32 / KL) * d);
        if (kl >= d) {
            const float2 nb = cmf(A, Bp);
            B = make_float2(nb.x + B.x, nb.y + B.y);
            A = cmf(A, Ap);
        }
    }
}

// KL unknowns of a chain per chunk, 32/KL slices per warp (KL = 8 for batches, 32 for S <= 4)
template <int KL>
__global__ void __launch_bounds__(128) k_cn_inc_scan_f32(const float2* __restrict__ fac, const double2* __restrict__ U,
                                                         double2* __restrict__ X, int M, int64_t nc, int S,
                                                         float kalpha, float w2, float phibar, float ia2,
                                                         const float* __restrict__ rcf, float vdn, int vq) {
    constexpr int SL = 32 / KL;                            // slices per warp
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, sl = lane % SL, kl = lane / SL;
    const int SG = (S + SL - 1) / SL;
    if (wid >= (int64_t)2 * (M + 1) * SG) return;          // whole warps exit together
    const int g = (int)(wid % SG);
    const int mp = (int)(wid / SG);
    const int m = mp >> 1, par = mp & 1;
    const int s = SL * g + sl;
    const bool sok = s < S;
    const int64_t base = st_off(m, M), xbase = ex_off(m, M);
    auto idx = [&](int f, int n) { return ((int64_t)f * nc + base + (n - m)) * S + s; };
    auto coef = [&](int n, int k) { return rcf[(xbase + (n - m)) * RC_NUM + k]; };
    auto ld = [&](int f, int n, double2& raw) -> float2 {
        if (!sok || n < m || n > M || (n == 0 && f > 0)) {
            raw = make_double2(0.0, 0.0);
            return fz();
        }
        raw = U[idx(f, n)];
        return d2f2(raw);
    };
    auto visc_w = [&](int n) -> float {
        if (vdn <= 0.f) return 0.f;
        const float l = (float)(n * (n + 1)) * ia2;
        float lq = 1.f;
        for (int i = 0; i < vq / 2; ++i) lq *= l;
        const float gg = vdn * lq;
        return gg / (1.f + gg);
    };
    auto rde = [&](int n, float2 ph, float2 de, float2 xm, float2 xp) -> float2 {
        if (n == 0) return fz();
        const float p = w2 * coef(n, RC_P), q = w2 * coef(n, RC_Q), r = w2 * coef(n, RC_R);
        const float lap = (float)(n * (n + 1)) * ia2;
        return make_float2(kalpha * (lap * ph.x + p * xm.x + q * xp.x - r * de.y),
                           kalpha * (lap * ph.y + p * xm.y + q * xp.y + r * de.x));
    };
    auto rxi = [&](int n, float2 xi, float2 dm, float2 dp) -> float2 {
        if (n < m || n > M || n == 0) return fz();
        const float p = w2 * coef(n, RC_P), q = w2 * coef(n, RC_Q), r = w2 * coef(n, RC_R);
        return make_float2(kalpha * (-(p * dm.x + q * dp.x) - r * xi.y), kalpha * (-(p * dm.y + q * dp.y) + r * xi.x));
    };
    const float kp = -kalpha * phibar;
    const int n0 = m + par;
    const int K = (n0 <= M) ? (M - n0) / 2 + 1 : 0;
    double2 rw;
    // forward elimination: d'_k = (rhs_k - a_k d'_{k-1}) g_k = A_k d'_{k-1} + B_k
    float2 carry = fz();
    for (int k0 = 0; k0 < K; k0 += KL) {
        const int k = k0 + kl, n = n0 + 2 * k;
        float2 A = fz(), B = fz();
        if (k < K) {
            const float2* f = fac + (base + (n - m)) * 8;
            const float2 ph = ld(0, n, rw), de = ld(2, n, rw), dem = ld(2, n - 2, rw), dep = ld(2, n + 2, rw);
            const float2 xm = ld(1, n - 1, rw), xp = ld(1, n + 1, rw);
            float2 rhs = rde(n, ph, de, xm, xp);
            const float f7 = f[7].x;
            const float2 e3 = cmf(f[3], rxi(n - 1, xm, dem, de)), e4 = cmf(f[4], rxi(n + 1, xp, de, dep));
            rhs = make_float2(rhs.x + kp * de.x * f7 + e3.x + e4.x, rhs.y + kp * de.y * f7 + e3.y + e4.y);
            const float2 g1 = f[1], na = cmf(f[0], g1);
            A = make_float2(-na.x, -na.y);
            B = cmf(rhs, g1);
        }
        affine_scan_kl<KL>(A, B, kl);
        const float2 ca = cmf(A, carry);
        const float2 v = make_float2(ca.x + B.x, ca.y + B.y);
        if (k < K && sok) X[idx(2, n)] = f2d2(v);
        carry = make_float2(__shfl_sync(0xffffffffu, v.x, (KL - 1) * SL + sl), __shfl_sync(0xffffffffu, v.y, (KL - 1) * SL + sl));
    }
    __syncwarp();
    // back substitution from the top: D_k = -c'_k D_{k+1} + d'_k; then Phi (final)
    carry = fz();
    for (int k0 = 0; k0 < K; k0 += KL) {
        const int k = K - 1 - (k0 + kl), n = n0 + 2 * k;
        float2 A = fz(), B = fz();
        if (k >= 0) {
            const float2* f = fac + (base + (n - m)) * 8;
            const float2 c2 = f[2];
            A = make_float2(-c2.x, -c2.y);
            B = sok ? d2f2(X[idx(2, n)]) : fz();
        }
        affine_scan_kl<KL>(A, B, kl);
        const float2 ca = cmf(A, carry);
        float2 dn = make_float2(ca.x + B.x, ca.y + B.y);
        carry = make_float2(__shfl_sync(0xffffffffu, dn.x, (KL - 1) * SL + sl), __shfl_sync(0xffffffffu, dn.y, (KL - 1) * SL + sl));
        if (k >= 0 && sok) {
            if (n == 0) dn = fz();
            const float2* f = fac + (base + (n - m)) * 8;
            double2 up_raw;
            const float2 up = ld(0, n, up_raw), ud = ld(2, n, rw);
            const float2 dphi = make_float2(kp * ud.x - dn.x * f[7].y, kp * ud.y - dn.y * f[7].y);
            const float w = visc_w(n);
            X[idx(2, n)] = f2d2(dn);
            X[idx(0, n)] = dadd_f(up_raw, make_float2(dphi.x - (up.x + dphi.x) * w, dphi.y - (up.y + dphi.y) * w));
        }
    }
    __syncwarp();
    // xi on the other parity: D_xi = [rhs_xi - c p D_delta(n-1) - c q D_delta(n+1)] / d_n (final)
    const int nx0 = m + (par ^ 1);
    const int J = (nx0 <= M) ? (M - nx0) / 2 + 1 : 0;
    for (int j0 = 0; j0 < J; j0 += KL) {
        const int j = j0 + kl, n = nx0 + 2 * j;
        if (j < J && sok) {
            const float2* f = fac + (base + (n - m)) * 8;
            double2 ux_raw;
            const float2 ux = ld(1, n, ux_raw), dmu = ld(2, n - 1, rw), dpu = ld(2, n + 1, rw);
            const float2 Dm = (n - 1 >= m) ? d2f2(X[idx(2, n - 1)]) : fz();
            const float2 Dp = (n + 1 <= M) ? d2f2(X[idx(2, n + 1)]) : fz();
            const float2 rxv = rxi(n, ux, dmu, dpu);
            const float2 num = make_float2(rxv.x - (f[6].x * Dm.x + f[6].y * Dp.x), rxv.y - (f[6].x * Dm.y + f[6].y * Dp.y));
            const float2 dxi = cmf(num, f[5]);
            const float w = visc_w(n);
            X[idx(1, n)] = n == 0 ? make_double2(0.0, 0.0)
                                  : dadd_f(ux_raw, make_float2(dxi.x - (ux.x + dxi.x) * w, dxi.y - (ux.y + dxi.y) * w));
        }
    }
    __syncwarp();
    // delta (final) from the parked D_delta
    for (int k0 = 0; k0 < K; k0 += KL) {
        const int k = k0 + kl, n = n0 + 2 * k;
        if (k < K && sok) {
            double2 ud_raw;
            const float2 ud = ld(2, n, ud_raw), dn = d2f2(X[idx(2, n)]);
            const float w = visc_w(n);
            X[idx(2, n)] = n == 0 ? make_double2(0.0, 0.0)
                                  : dadd_f(ud_raw, make_float2(dn.x - (ud.x + dn.x) * w, dn.y - (ud.y + dn.y) * w));
        }
    }
}

// The same solve with one thread per (m, parity, slice) walking its chain sequentially
// (rolling registers: every value of U is converted once per sweep).  Latency-bound for
// moderate batches, but the cheapest per element once the batch alone fills the GPU.
__global__ void __launch_bounds__(128) k_cn_inc_f32(const float2* __restrict__ fac, const double2* __restrict__ U,
                                                    double2* __restrict__ X, int M, int64_t nc, int S, float kalpha,
                                                    float w2, float phibar, float ia2, const float* __restrict__ rcf,
                                                    float vdn, int vq) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)2 * (M + 1) * S) return;
    const int s = (int)(t % S);
    const int mp = (int)(t / S);
    const int m = mp >> 1, par = mp & 1;
    const int64_t base = st_off(m, M), xbase = ex_off(m, M);
    auto idx = [&](int f, int n) { return ((int64_t)f * nc + base + (n - m)) * S + s; };
    auto coef = [&](int n, int k) { return rcf[(xbase + (n - m)) * RC_NUM + k]; };
    auto visc_w = [&](int n) -> float {
        if (vdn <= 0.f) return 0.f;
        const float l = (float)(n * (n + 1)) * ia2;
        float lq = 1.f;
        for (int i = 0; i < vq / 2; ++i) lq *= l;
        const float g = vdn * lq;
        return g / (1.f + g);
    };
    auto ld = [&](int f, int n, double2& raw) -> float2 {
        if (n < m || n > M || (n == 0 && f > 0)) {
            raw = make_double2(0.0, 0.0);
            return fz();
        }
        raw = U[idx(f, n)];
        return d2f2(raw);
    };
    auto rde = [&](int n, float2 ph, float2 de, float2 xm, float2 xp) -> float2 {
        if (n == 0) return fz();
        const float p = w2 * coef(n, RC_P), q = w2 * coef(n, RC_Q), r = w2 * coef(n, RC_R);
        const float lap = (float)(n * (n + 1)) * ia2;
        return make_float2(kalpha * (lap * ph.x + p * xm.x + q * xp.x - r * de.y),
                           kalpha * (lap * ph.y + p * xm.y + q * xp.y + r * de.x));
    };
    auto rxi = [&](int n, float2 xi, float2 dm, float2 dp) -> float2 {
        if (n < m || n > M || n == 0) return fz();
        const float p = w2 * coef(n, RC_P), q = w2 * coef(n, RC_Q), r = w2 * coef(n, RC_R);
        return make_float2(kalpha * (-(p * dm.x + q * dp.x) - r * xi.y), kalpha * (-(p * dm.y + q * dp.y) + r * xi.x));
    };
    const float kp = -kalpha * phibar;
    // forward elimination (d' parked in X[delta]); de0 = delta_n, de2 = delta_{n+2}, xlo/xhi = xi_{n-1}/xi_{n+1}
    const int n0 = m + par;
    double2 rw;
    float2 de0 = ld(2, n0, rw), de2 = ld(2, n0 + 2, rw);
    float2 xlo = ld(1, n0 - 1, rw), xhi = ld(1, n0 + 1, rw);
    float2 dprev = fz();
    float2 rx_lo = rxi(n0 - 1, xlo, ld(2, n0 - 2, rw), de0);
    int nlast = n0 - 2;
    for (int n = n0; n <= M; n += 2) {
        const float2* f = fac + (base + (n - m)) * 8;
        const float2 ph = ld(0, n, rw);
        const float2 rx_hi = rxi(n + 1, xhi, de0, de2);
        float2 rhs = rde(n, ph, de0, xlo, xhi);
        const float2 e3 = cmf(f[3], rx_lo), e4 = cmf(f[4], rx_hi), e0 = cmf(f[0], dprev);
        rhs = make_float2(rhs.x + kp * de0.x * f[7].x + e3.x + e4.x - e0.x,
                          rhs.y + kp * de0.y * f[7].x + e3.y + e4.y - e0.y);
        const float2 dp = cmf(rhs, f[1]);
        X[idx(2, n)] = f2d2(dp);
        dprev = dp;
        rx_lo = rx_hi;
        nlast = n;
        xlo = xhi;
        xhi = ld(1, n + 3, rw);
        de0 = de2;
        de2 = ld(2, n + 4, rw);
    }
    // back substitution (descending): D_delta, Phi (final), and the xi just above (final);
    // dup = delta_{n+2} of U, dnext = D_delta(n+2)
    float2 dnext = fz();
    float2 dup = ld(2, nlast + 2, rw);
    for (int n = nlast; n >= n0; n -= 2) {
        const float2* f = fac + (base + (n - m)) * 8;
        double2 ud_raw, up_raw, ux_raw;
        const float2 ud = ld(2, n, ud_raw), up = ld(0, n, up_raw);
        const float2 dpark = d2f2(X[idx(2, n)]);
        const float2 e2 = cmf(f[2], dnext);
        float2 dn = make_float2(dpark.x - e2.x, dpark.y - e2.y);
        if (n == 0) dn = fz();
        const float2 dphi = make_float2(kp * ud.x - dn.x * f[7].y, kp * ud.y - dn.y * f[7].y);
        const float w = visc_w(n);
        X[idx(2, n)] = n == 0 ? make_double2(0.0, 0.0)
                              : dadd_f(ud_raw, make_float2(dn.x - (ud.x + dn.x) * w, dn.y - (ud.y + dn.y) * w));
        X[idx(0, n)] = dadd_f(up_raw, make_float2(dphi.x - (up.x + dphi.x) * w, dphi.y - (up.y + dphi.y) * w));
        const int nx = n + 1;
        if (nx <= M) {
            const float2* fx = fac + (base + (nx - m)) * 8;
            const float2 ux = ld(1, nx, ux_raw);
            const float2 rxv = rxi(nx, ux, ud, dup);
            const float2 num = make_float2(rxv.x - (fx[6].x * dn.x + fx[6].y * dnext.x),
                                           rxv.y - (fx[6].x * dn.y + fx[6].y * dnext.y));
            const float2 dxi = cmf(num, fx[5]);
            const float wx = visc_w(nx);
            X[idx(1, nx)] = dadd_f(ux_raw, make_float2(dxi.x - (ux.x + dxi.x) * wx, dxi.y - (ux.y + dxi.y) * wx));
        }
        dnext = dn;
        dup = ud;
    }
    // the xi just below the first delta (parity 1: xi_m, whose lower neighbour is outside)
    if (par == 1) {
        const int nx = m;
        const float2* fx = fac + (base + (nx - m)) * 8;
        double2 ux_raw;
        const float2 ux = ld(1, nx, ux_raw);
        const float2 rxv = rxi(nx, ux, fz(), dup);
        const float2 num = make_float2(rxv.x - fx[6].y * dnext.x, rxv.y - fx[6].y * dnext.y);
        const float2 dxi = cmf(num, fx[5]);
        const float wx = visc_w(nx);
        X[idx(1, nx)] = nx == 0 ? make_double2(0.0, 0.0)
                                : dadd_f(ux_raw, make_float2(dxi.x - (ux.x + dxi.x) * wx, dxi.y - (ux.y + dxi.y) * wx));
    }
}

__global__ void k_balance(const double2* __restrict__ xi, const double2* __restrict__ N,
                          const double2* __restrict__ add, double2* __restrict__ U, const int* __restrict__ srow_m,
                          int M, int64_t nc, int S, double a, double omega) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nc * S) return;
    int s = (int)(t % S);
    int64_t r = t / S;
    int m = srow_m[r];
    int n = m + (int)(r - st_off(m, M));
    auto X = [&](int k) -> double2 {
        if (k < m || k > M || k == 0) return czero();
        return xi[(st_off(m, M) + (k - m)) * S + s];
    };
    double2 ph = czero();
    if (n >= 1) {
        double2 lc = c_scale(c_add(c_scale(X(n - 1), coef_p(m, n)), c_scale(X(n + 1), coef_q(m, n))), 2.0 * omega);
        double2 nd = N[(2 * nc + r) * S + s];
        ph = c_scale(c_add(lc, nd), -a * a / ((double)n * (n + 1.0)));
    }
    if (add) ph = c_add(ph, add[r * S + s]);
    U[(0 * nc + r) * S + s] = ph;
    U[(1 * nc + r) * S + s] = X(n);
    U[(2 * nc + r) * S + s] = czero();
}

__global__ void k_axpy_kernel(double2* __restrict__ y, const double2* __restrict__ x, double a, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) y[t] = c_add(y[t], c_scale(x[t], a));
}

// AoS [S][3][NC(Min)] -> AoS [S][3][NC(Mout)]: keep n <= min(Min, Mout), zero the rest
__global__ void k_trunc(const double2* __restrict__ in, int Min, double2* __restrict__ out, int Mout, int S) {
    int64_t ncout = nc_state(Mout), ncin = nc_state(Min);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * ncout * S) return;
    int64_t r = t % ncout;
    int64_t sf = t / ncout;
    // locate (m, n) of r in the output truncation
    int m = 0;
    while (m < Mout && st_off(m + 1, Mout) <= r) ++m;
    int n = m + (int)(r - st_off(m, Mout));
    double2 v = czero();
    if (m <= Min && n <= Min) v = in[sf * ncin + st_off(m, Min) + (n - m)];
    out[t] = v;
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// batches of at least TT states (and at most 65535 TT, the grid's y limit) take the tiled forms
static bool tiled_ok(int S) { return S >= TT && S <= 65535 * TT; }
static dim3 tiled_grid(int64_t n, int S) { return dim3((unsigned)((n + TT - 1) / TT), (unsigned)((S + TT - 1) / TT)); }

swe_status k_aos_to_soa(const swe_plan* p, const double2* in, double2* out, int S, cudaStream_t st) {
    if (tiled_ok(S))
        k_aos_soa_tiled<<<tiled_grid(3 * p->nc, S), 256, 0, st>>>(in, 3 * p->nc, out, 3 * p->nc, S);
    else
        k_aos_soa<<<nblk(3 * p->nc * S), 256, 0, st>>>(in, out, p->nc, S);
    SWE_CHECK_LAUNCH("k_aos_soa");
    return SWE_OK;
}
swe_status k_soa_to_aos(const swe_plan* p, const double2* in, double2* out, int S, cudaStream_t st) {
    if (tiled_ok(S))
        k_soa_aos_tiled<<<tiled_grid(3 * p->nc, S), 256, 0, st>>>(in, out, 3 * p->nc, nullptr, 0, 3 * p->nc, S);
    else
        k_soa_aos<<<nblk(3 * p->nc * S), 256, 0, st>>>(in, out, p->nc, S);
    SWE_CHECK_LAUNCH("k_soa_aos");
    return SWE_OK;
}
swe_status k_pack_scalar(const swe_plan* p, const double2* spec, double2* X, int B, cudaStream_t st) {
    if (p->prec == SWE_FP64)
        k_pack<<<nblk(p->ncx * B), 256, 0, st>>>(spec, X, p->row_m, p->M, p->nc, p->ncx, B);
    else
        k_pack_f32<<<nblk(p->ncx * B), 256, 0, st>>>(spec, reinterpret_cast<float2*>(X), p->row_m, p->M, p->nc,
                                                     p->ncx, B);
    SWE_CHECK_LAUNCH("k_pack");
    return SWE_OK;
}
swe_status k_unpack_scalar(const swe_plan* p, const double2* Y, double2* spec, int B, cudaStream_t st) {
    if (p->prec == SWE_FP64)
        k_unpack<<<nblk(p->nc * B), 256, 0, st>>>(Y, spec, p->srow_m, p->M, p->nc, B);
    else
        k_unpack_f32<<<nblk(p->nc * B), 256, 0, st>>>(reinterpret_cast<const float2*>(Y), spec, p->srow_m, p->M,
                                                      p->nc, B);
    SWE_CHECK_LAUNCH("k_unpack");
    return SWE_OK;
}
swe_status k_nl_pre(const swe_plan* p, const double2* Ua, const double2* Ub, double beta, double2* X, int S,
                    cudaStream_t st) {
    const double xe = (p->prec == SWE_FP64) ? 16.0 : 8.0;   // bytes per operand element
    ProfToken tk_ = prof_begin("nl_pre", st, 0.0, S * (16.0 * 3.0 * p->nc * (Ub ? 2.0 : 1.0) + xe * 4.0 * p->ncx));
    if (p->prec == SWE_FP64) {
        StateView v{Ua, Ub, beta, p->nc, S, p->M};
        k_nl_pre_kernel<<<nblk(p->ncx * S), 256, 0, st>>>(v, X, p->row_m, p->ncx, p->rc);
    } else {
        StateViewF v{Ua, Ub, (float)beta, p->nc, S, p->M};
        k_nl_pre_f32<<<nblk(p->ncx * S), 256, 0, st>>>(v, reinterpret_cast<float2*>(X), p->row_m, p->ncx, p->rcf);
    }
    prof_end(tk_, st);
    SWE_CHECK_LAUNCH("k_nl_pre");
    return SWE_OK;
}
swe_status k_nl_post(const swe_plan* p, const double2* Y, int mode, double dt, const double2* in0, const double2* in1,
                     double2* out0, double2* out1, int S, cudaStream_t st, const double2* Yphi) {
    const double ye = (p->prec == SWE_FP64) ? 16.0 : 8.0;   // bytes per operand element
    ProfToken tk_ = prof_begin("nl_post", st, 0.0, S * (ye * 5.0 * p->ncx + 16.0 * 3.0 * p->nc * (in1 ? 4.0 : 3.0)));
    if (p->prec == SWE_FP64) {
        k_nl_post_kernel<<<nblk(p->nc * S), 256, 0, st>>>(Y, mode, dt, in0, in1, out0, out1, p->srow_m, p->M, p->nc, S,
                                                          1.0 / p->a, p->rc, p->flags, Yphi);
    } else {
        k_nl_post_f32<<<nblk(p->nc * S), 256, 0, st>>>(reinterpret_cast<const float2*>(Y), mode, (float)dt, in0, in1,
                                                       out0, out1, p->srow_m, p->M,
                                                       p->nc, S, (float)(1.0 / p->a), p->rcf, p->flags,
                                                       reinterpret_cast<const float2*>(Yphi));
    }
    prof_end(tk_, st);
    SWE_CHECK_LAUNCH("k_nl_post");
    return SWE_OK;
}
swe_status k_linear(const swe_plan* p, const double2* U, double2* LU, int S, cudaStream_t st) {
    StateView v{U, nullptr, 0.0, p->nc, S, p->M};
    k_linop<<<nblk(p->nc * S), 256, 0, st>>>(v, LU, p->srow_m, 0, 0.0, 1.0 / (p->a * p->a), p->omega, p->phibar,
                                             p->rc);
    SWE_CHECK_LAUNCH("k_linop");
    return SWE_OK;
}

swe_status plan_cn_factor(swe_plan* p, double alpha, const double2** fac, cudaStream_t st, const float2** fac32) {
    for (int i = 0; i < p->ncn; ++i)
        if (p->cn[i].alpha == alpha) {
            *fac = p->cn[i].fac;
            if (fac32) *fac32 = p->cn[i].fac32;
            return SWE_OK;
        }
    int slot = p->ncn < 16 ? p->ncn++ : 15;
    p->gen += 1;
    if (p->ncn == 16 && slot == 15 && p->cn[15].fac) {
        SWE_CHECK_CUDA(cudaStreamSynchronize(st));
        cudaFree(p->cn[15].fac);
        cudaFree(p->cn[15].fac32);
        p->cn[15].fac = nullptr;
        p->cn[15].fac32 = nullptr;
    }
    double2* f;
    SWE_CHECK_CUDA(cudaMalloc((void**)&f, sizeof(double2) * 8 * p->nc));
    k_cn_factor<<<nblk(2 * (p->M + 1), 64), 64, 0, st>>>(p->M, alpha, p->a, p->omega, p->phibar, f);
    SWE_CHECK_LAUNCH("k_cn_factor");
    float2* f32 = nullptr;
    if (p->prec != SWE_FP64) {
        SWE_CHECK_CUDA(cudaMalloc((void**)&f32, sizeof(float2) * 8 * p->nc));
        k_to_f32<<<nblk(8 * p->nc), 256, 0, st>>>(f, f32, 8 * p->nc);
        SWE_CHECK_LAUNCH("k_to_f32");
    }
    p->cn[slot].alpha = alpha;
    p->cn[slot].fac = f;
    p->cn[slot].fac32 = f32;
    *fac = f;
    if (fac32) *fac32 = f32;
    return SWE_OK;
}

swe_status k_implicit(swe_plan* p, double alpha, int with_rhs, const double2* in, double2* out, double visc_dt,
                      double visc_nu, int visc_q, int S, cudaStream_t st) {
    const double2* fac;
    const float2* fac32 = nullptr;
    SWE_CHECK(plan_cn_factor(p, alpha, &fac, st, &fac32));
    if (p->prec != SWE_FP64 && fac32 && in != out) {
        // split-precision plans: FP32 increment form (right-hand side fused for CN); also for
        // single slices (the serial chains), where it replaces two FP64-bound launches
        const float kap = with_rhs ? 2.0f : 1.0f;
        ProfToken tk = prof_begin("cn_step_f32", st, 0.0, 16.0 * p->nc * (6.0 * S + 8.0));
        const float ka = (float)(kap * alpha), w2 = (float)(2.0 * p->omega), pb = (float)p->phibar;
        const float ia2 = (float)(1.0 / (p->a * p->a)), vdn = visc_nu > 0.0 ? (float)(visc_dt * visc_nu) : 0.f;
        if (S >= 512) {
            // the batch alone fills the GPU with chains: one thread per chain
            k_cn_inc_f32<<<nblk((int64_t)2 * (p->M + 1) * S, 128), 128, 0, st>>>(fac32, in, out, p->M, p->nc, S, ka,
                                                                                w2, pb, ia2, p->rcf, vdn, visc_q);
        } else if (S > 4) {
            const int64_t nwarps = (int64_t)2 * (p->M + 1) * ((S + 3) / 4);
            k_cn_inc_scan_f32<8><<<nblk(nwarps * 32, 128), 128, 0, st>>>(fac32, in, out, p->M, p->nc, S, ka, w2, pb,
                                                                          ia2, p->rcf, vdn, visc_q);
        } else {
            // small batches (serial chains): 32 unknowns of one chain per chunk
            const int64_t nwarps = (int64_t)2 * (p->M + 1) * S;
            k_cn_inc_scan_f32<32><<<nblk(nwarps * 32, 128), 128, 0, st>>>(fac32, in, out, p->M, p->nc, S, ka, w2, pb,
                                                                           ia2, p->rcf, vdn, visc_q);
        }
        prof_end(tk, st);
        SWE_CHECK_LAUNCH("k_cn_inc_f32");
        return SWE_OK;
    }
    const double2* R = in;
    if (with_rhs) {
        if (in == out) {
            swe_set_error("k_implicit: Crank-Nicolson right-hand side needs distinct buffers");
            return SWE_EINVAL;
        }
        StateView v{in, nullptr, 0.0, p->nc, S, p->M};
        {
            ProfToken tk_ = prof_begin("linop_rhs", st, 0.0, 16.0 * 6.0 * p->nc * S);
            k_linop<<<nblk(p->nc * S), 256, 0, st>>>(v, out, p->srow_m, 1, alpha, 1.0 / (p->a * p->a), p->omega,
                                                     p->phibar, p->rc);
            prof_end(tk_, st);
        }
        SWE_CHECK_LAUNCH("k_linop(rhs)");
        R = out;
    }
    // algorithmic traffic: R (3 fields) + factors read, X written
    ProfToken tk = prof_begin("cn_solve", st, 0.0, 16.0 * p->nc * (6.0 * S + 8.0));
    if (S <= 4) {
        // small batches (serial coarse chains): one warp per (m, parity, slice), scan-based
        k_cn_solve_warp<<<nblk((int64_t)2 * (p->M + 1) * S * 32, 128), 128, 0, st>>>(fac, R, out, p->M, p->nc, S,
                                                                                  visc_dt, visc_nu, visc_q, p->a);
    } else {
        k_cn_solve<<<nblk((int64_t)2 * (p->M + 1) * S, 128), 128, 0, st>>>(fac, R, out, p->M, p->nc, S, visc_dt,
                                                                        visc_nu, visc_q, p->a);
    }
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_cn_solve");
    return SWE_OK;
}

swe_status k_balance_combine(const swe_plan* p, const double2* xi_soa, const double2* N, const double2* phi_add_soa,
                             double2* U, int S, cudaStream_t st) {
    k_balance<<<nblk(p->nc * S), 256, 0, st>>>(xi_soa, N, phi_add_soa, U, p->srow_m, p->M, p->nc, S, p->a, p->omega);
    SWE_CHECK_LAUNCH("k_balance");
    return SWE_OK;
}

swe_status k_axpy(double2* y, const double2* x, double a, int64_t n, cudaStream_t st) {
    k_axpy_kernel<<<nblk(n), 256, 0, st>>>(y, x, a, n);
    SWE_CHECK_LAUNCH("k_axpy");
    return SWE_OK;
}

swe_status k_truncate(const double2* in, int Min, double2* out, int Mout, int S, cudaStream_t st) {
    k_trunc<<<nblk(3 * nc_state(Mout) * S), 256, 0, st>>>(in, Min, out, Mout, S);
    SWE_CHECK_LAUNCH("k_trunc");
    return SWE_OK;
}

swe_status k_aos_to_soa_strided(const swe_plan* p, const double2* in, int64_t stride, double2* out, int S,
                                cudaStream_t st) {
    {
        ProfToken tk_ = prof_begin("aos_soa", st, 0.0, 16.0 * 6.0 * p->nc * S);
        if (tiled_ok(S))
            k_aos_soa_tiled<<<tiled_grid(3 * p->nc, S), 256, 0, st>>>(in, stride, out, 3 * p->nc, S);
        else
            k_aos_soa_strided<<<nblk(3 * p->nc * S), 256, 0, st>>>(in, stride, out, p->nc, S);
        prof_end(tk_, st);
    }
    SWE_CHECK_LAUNCH("k_aos_soa_strided");
    return SWE_OK;
}

swe_status k_soa_to_aos_strided(const swe_plan* p, const double2* in, double2* out, int64_t stride, const double2* add,
                                int64_t add_stride, int S, cudaStream_t st) {
    {
        ProfToken tk_ = prof_begin("soa_aos", st, 0.0, 16.0 * (add ? 9.0 : 6.0) * p->nc * S);
        if (tiled_ok(S))
            k_soa_aos_tiled<<<tiled_grid(3 * p->nc, S), 256, 0, st>>>(in, out, stride, add, add_stride, 3 * p->nc,
                                                                      S);
        else
            k_soa_aos_strided<<<nblk(3 * p->nc * S), 256, 0, st>>>(in, out, stride, add, add_stride, p->nc, S);
        prof_end(tk_, st);
    }
    SWE_CHECK_LAUNCH("k_soa_aos_strided");
    return SWE_OK;
}
