// Stability regions of the linearised test ODE u' = lambda_L u + lambda_N u (§4, Eqs. 10-20),
// evaluated on a grid of xi_N = lambda_N Delta t in the complex plane for a fixed xi_L.
//
// One thread per grid point, FP64 complex arithmetic in registers; no memory traffic beyond
// the one output value per point, so the kernel is bound by the FP64 pipe.  Per point:
//   coarse factor(s): IMEX, A = ((4 + xi_L)/(4 - xi_L))^2 (1 + xi_N (2 + xi_N)/2) (§4.1.1 with
//     the Heun reading of Eq. 5), or the two roots of the SL-SI-SETTLS quadratic (Eq. 13) for
//     every kappa s in [0, 2 pi] (n_kappa values, step 2 pi / (n_kappa - 1));
//   fine factor: IMEX at xi / cf (cf fine steps per coarse step, N_f = cf N_c);
//   method: the coarse scheme alone over n slices (A_c^{n N_c}), Parareal (Eq. 17) or two-level
//     MGRIT with F(CF)^nu relaxation (Eq. 20, upper summation limit either as printed,
//     floor(k/(nu+1)), or from path counting on Eq. 19, min(k, floor(n/(nu+1))));
//   output |A|, the maximum over the SL roots and kappa s values (the region is their
//   intersection, §4.1.2).
// Both the scaling of xi (relative to the coarse step) and the use of each SL root as the
// coarse factor inside Eqs. 17 and 20 are readings of the paper, which does not spell them out.
#include <cmath>

#include "swe_internal.cuh"

namespace {

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    // Smith's algorithm (scaled to avoid overflow)
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + b.y * r;
        return {(a.x + a.y * r) / d, (a.y - a.x * r) / d};
    }
    const double r = b.x / b.y, d = b.x * r + b.y;
    return {(a.x * r + a.y) / d, (a.y * r - a.x) / d};
}
__device__ __forceinline__ double cabs_(cd a) { return hypot(a.x, a.y); }
// principal square root: sqrt((|z| + x)/2) + i sign(y) sqrt((|z| - x)/2)
__device__ __forceinline__ cd csqrt_(cd z) {
    const double r = hypot(z.x, z.y);
    const double u = sqrt(fmax(0.0, 0.5 * (r + z.x)));
    const double v = sqrt(fmax(0.0, 0.5 * (r - z.x)));
    return {u, z.y < 0.0 ? -v : v};
}
__device__ cd cpow(cd a, int e) {
    cd r = {1.0, 0.0};
    while (e > 0) {
        if (e & 1) r = cmul(r, a);
        a = cmul(a, a);
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ cd imex_factor(cd xiL, cd xiN) {
    const cd ai = cdiv(cadd({4.0, 0.0}, xiL), csub({4.0, 0.0}, xiL));
    const cd ae = cadd({1.0, 0.0}, cscale(cmul(xiN, cadd({2.0, 0.0}, xiN)), 0.5));
    return cmul(cmul(ai, ai), ae);
}

// the two roots of (1 - xiL/2) A^2 - (e (1 + xiL/2 + xiN) + xiN/2) A + (xiN/2) e = 0, e = exp(-i ks)
__device__ __forceinline__ void sl_roots(cd xiL, cd xiN, double ks, cd* r0, cd* r1) {
    const cd e = {cos(ks), -sin(ks)};
    const cd a = csub({1.0, 0.0}, cscale(xiL, 0.5));
    const cd b = cscale(cadd(cmul(e, cadd(cadd({1.0, 0.0}, cscale(xiL, 0.5)), xiN)), cscale(xiN, 0.5)), -1.0);
    const cd c = cmul(cscale(xiN, 0.5), e);
    const cd disc = csub(cmul(b, b), cscale(cmul(a, c), 4.0));
    const cd sq = csqrt_(disc);
    const cd two_a = cscale(a, 2.0);
    *r0 = cdiv(cadd(cscale(b, -1.0), sq), two_a);
    *r1 = cdiv(csub(cscale(b, -1.0), sq), two_a);
}

struct StabParams {
    int coarse, method, n, k, cf, Nc, nu, n_kappa;
    cd xiL;
};

// |A| of the selected method for one coarse factor Ac (one step of Delta t_c) and the fine
// factor Af (one step of Delta t_c / cf)
__device__ double method_abs(const StabParams& P, cd Ac, cd Af) {
    const cd R = cpow(Ac, P.Nc);                  // A_c^{N_c}
    if (P.method == SWE_STAB_COARSE_ALONE) return cabs_(cpow(R, P.n));
    const cd F = cpow(Af, P.cf * P.Nc);           // A_f^{N_f}, N_f = cf N_c
    if (P.method == SWE_STAB_PARAREAL) {
        // sum_{i=0}^{k} C(n,i) S^i R^{n-i} = R^{n-k'} sum_i C(n,i) S^i R^{k'-i}, k' = min(k, n)
        const cd S = csub(F, R);
        const int kk = P.k < P.n ? P.k : P.n;
        cd acc = {0.0, 0.0}, Si = {1.0, 0.0};
        double binom = 1.0;
        for (int i = 0; i <= kk; ++i) {
            acc = cadd(acc, cscale(cmul(Si, cpow(R, kk - i)), binom));
            Si = cmul(Si, S);
            binom = binom * (double)(P.n - i) / (double)(i + 1);
        }
        return cabs_(cmul(acc, cpow(R, P.n - kk)));
    }
    // two-level MGRIT, F(CF)^nu: sum_i C(n - i nu, i) (F^nu (F - R))^i R^{n - i (nu+1)}
    const cd S = cmul(cpow(F, P.nu), csub(F, R));
    const int lim_printed = P.k / (P.nu + 1);
    const int lim_paths = P.k < P.n / (P.nu + 1) ? P.k : P.n / (P.nu + 1);
    const int imax = P.method == SWE_STAB_MGRIT2_PRINTED ? lim_printed : lim_paths;
    cd acc = {0.0, 0.0}, Si = {1.0, 0.0};
    for (int i = 0; i <= imax; ++i) {
        const int top = P.n - i * P.nu, ex = P.n - i * (P.nu + 1);
        if (ex < 0 || top < i) break;
        double binom = 1.0;                       // C(top, i)
        for (int j = 0; j < i; ++j) binom = binom * (double)(top - j) / (double)(j + 1);
        acc = cadd(acc, cscale(cmul(Si, cpow(R, ex)), binom));
        Si = cmul(Si, S);
    }
    return cabs_(acc);
}

__global__ void k_stability(StabParams P, double re0, double dre, int nre, double im0, double dim, int nim,
                            double* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nre * nim) return;
    const int ix = (int)(idx % nre), iy = (int)(idx / nre);
    const cd xiN = {re0 + ix * dre, im0 + iy * dim};
    const cd Af = imex_factor(cscale(P.xiL, 1.0 / P.cf), cscale(xiN, 1.0 / P.cf));
    double best = 0.0;
    if (P.coarse == SWE_IMEX) {
        best = method_abs(P, imex_factor(P.xiL, xiN), Af);
    } else {
        const int nk = P.n_kappa;
        for (int q = 0; q < nk; ++q) {
            const double ks = nk > 1 ? 2.0 * M_PI * q / (nk - 1) : 0.0;
            cd r0, r1;
            sl_roots(P.xiL, xiN, ks, &r0, &r1);
            best = fmax(best, method_abs(P, r0, Af));
            best = fmax(best, method_abs(P, r1, Af));
        }
    }
    out[idx] = best;
}

}  // namespace

extern "C" swe_status swe_stability_region(const swe_stability_desc* d, double re0, double re1, int nre, double im0,
                                           double im1, int nim, double* absA, void* stream) {
    if (!d || !absA || nre < 1 || nim < 1 || d->n < 1 || d->k < 0 || d->cf < 1 || d->Nc < 1 || d->nu < 0 ||
        (d->coarse_scheme != SWE_IMEX && d->coarse_scheme != SWE_SLSI_SETTLS) ||
        d->method < SWE_STAB_COARSE_ALONE || d->method > SWE_STAB_MGRIT2_PRINTED ||
        (d->coarse_scheme == SWE_SLSI_SETTLS && d->n_kappa < 1) ||
        (d->method == SWE_STAB_MGRIT2_PRINTED && (d->k / (d->nu + 1)) * (d->nu + 1) > d->n)) {
        swe_set_error("swe_stability_region: invalid descriptor or grid");
        return SWE_EINVAL;
    }
    StabParams P;
    P.coarse = d->coarse_scheme;
    P.method = d->method;
    P.n = d->n;
    P.k = d->k;
    P.cf = d->cf;
    P.Nc = d->Nc;
    P.nu = d->nu;
    P.n_kappa = d->n_kappa;
    P.xiL = {d->xiL_re, d->xiL_im};
    const double dre = nre > 1 ? (re1 - re0) / (nre - 1) : 0.0;
    const double dim = nim > 1 ? (im1 - im0) / (nim - 1) : 0.0;
    const int64_t npts = (int64_t)nre * nim;
    cudaStream_t st = (cudaStream_t)stream;
    ProfToken tk = prof_begin("stability", st, 0.0, 8.0 * npts);
    k_stability<<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(P, re0, dre, nre, im0, dim, nim, absA);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_stability");
    return SWE_OK;
}
