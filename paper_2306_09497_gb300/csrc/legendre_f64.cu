// Legendre contraction in FP64 (DFMA), the "FP64 plain" path of §2.2.
//
// Inverse, per zonal wavenumber m:   G_m(mu_j) = sum_{n=m}^{M+1} P_n^m(mu_j) X_{m,n}
// Forward, per m:                    Y_{m,n}   = sum_j P_n^m(mu_j) F_m(mu_j)
// (the Gauss weight and the 1/nlon of the DFT are applied by the ring kernels).
// Both use the equatorial symmetry P_n^m(-mu) = (-1)^{n-m} P_n^m(mu): the inverse
// forms E = sum over even n-m, O = sum over odd n-m at the northern latitudes and
// writes E + O (north) and E - O (south); the forward contracts even rows with
// F(mu) + F(-mu) and odd rows with F(mu) - F(-mu) over the northern latitudes.
//
// Layouts (C complex columns = 2C real columns, complex interleaved):
//   P [ncx][nlat2]            rows (m, n = m..M+1), j in the northern half
//   X, Y [ncx][2C]            same rows
//   F [M+1][nlat][2C]         all latitudes, north to south
#include "swe_internal.cuh"

namespace {

constexpr int TJ = 32;   // latitude rows per block (inverse)
constexpr int TN = 32;   // degree rows per block (forward)
constexpr int TC = 64;   // real columns per block
constexpr int KC = 16;   // contraction chunk

__global__ void __launch_bounds__(256) k_leg_inv_f64(const double* __restrict__ P, const double* __restrict__ X,
                                                     double* __restrict__ F, int M, int nlat, int nlat2, int ncol) {
    const int m = M - (int)blockIdx.z;      // heavy (small m) blocks last in z: spread evenly
    const int j0 = blockIdx.y * TJ, c0 = blockIdx.x * TC;
    if (j0 >= nlat2) return;
    const int K = M + 2 - m;
    const double* Pm = P + ex_off(m, M) * nlat2;
    const double* Xm = X + ex_off(m, M) * ncol;
    __shared__ double sP[KC][TJ];
    __shared__ double sX[KC][TC];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double e[2][4], o[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) e[r][c] = o[r][c] = 0.0;
    for (int k0 = 0; k0 < K; k0 += KC) {
        for (int i = threadIdx.x; i < KC * TJ; i += 256) {
            int kk = i / TJ, jj = i % TJ;
            int k = k0 + kk, j = j0 + jj;
            sP[kk][jj] = (k < K && j < nlat2) ? Pm[(int64_t)k * nlat2 + j] : 0.0;
        }
        for (int i = threadIdx.x; i < KC * TC; i += 256) {
            int kk = i / TC, cc = i % TC;
            int k = k0 + kk, c = c0 + cc;
            sX[kk][cc] = (k < K && c < ncol) ? Xm[(int64_t)k * ncol + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; kk += 2) {      // k0 is even: kk even <-> n - m even
            double p0 = sP[kk][ty], p1 = sP[kk][ty + 16];
            double q0 = sP[kk + 1][ty], q1 = sP[kk + 1][ty + 16];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double x = sX[kk][tx + 16 * c];
                double y = sX[kk + 1][tx + 16 * c];
                e[0][c] = fma(p0, x, e[0][c]);
                e[1][c] = fma(p1, x, e[1][c]);
                o[0][c] = fma(q0, y, o[0][c]);
                o[1][c] = fma(q1, y, o[1][c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int j = j0 + ty + 16 * r;
        if (j >= nlat2) continue;
        double* Fn = F + ((int64_t)m * nlat + j) * ncol;
        double* Fs = F + ((int64_t)m * nlat + (nlat - 1 - j)) * ncol;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int col = c0 + tx + 16 * c;
            if (col < ncol) {
                Fn[col] = e[r][c] + o[r][c];
                Fs[col] = e[r][c] - o[r][c];
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_leg_fwd_f64(const double* __restrict__ P, const double* __restrict__ F,
                                                     double* __restrict__ Y, int M, int nlat, int nlat2, int ncol) {
    const int m = M - (int)blockIdx.z;
    const int k0 = blockIdx.y * TN, c0 = blockIdx.x * TC;
    const int K = M + 2 - m;
    if (k0 >= K) return;
    const double* Pm = P + ex_off(m, M) * nlat2;
    const double* Fm = F + (int64_t)m * nlat * ncol;
    __shared__ double sP[TN][KC + 1];
    __shared__ double sS[KC][TC];
    __shared__ double sA[KC][TC];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
    for (int j0 = 0; j0 < nlat2; j0 += KC) {
        for (int i = threadIdx.x; i < TN * KC; i += 256) {
            int kk = i / KC, jj = i % KC;
            int k = k0 + kk, j = j0 + jj;
            sP[kk][jj] = (k < K && j < nlat2) ? Pm[(int64_t)k * nlat2 + j] : 0.0;
        }
        for (int i = threadIdx.x; i < KC * TC; i += 256) {
            int jj = i / TC, cc = i % TC;
            int j = j0 + jj, c = c0 + cc;
            double fn = 0.0, fs = 0.0;
            if (j < nlat2 && c < ncol) {
                fn = Fm[(int64_t)j * ncol + c];
                fs = Fm[(int64_t)(nlat - 1 - j) * ncol + c];
            }
            sS[jj][cc] = fn + fs;
            sA[jj][cc] = fn - fs;
        }
        __syncthreads();
        // rows ty and ty+16 have the parity of ty (k0 is a multiple of 32)
        const double(*src)[TC] = (ty & 1) ? sA : sS;
#pragma unroll
        for (int jj = 0; jj < KC; ++jj) {
            double p0 = sP[ty][jj], p1 = sP[ty + 16][jj];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double v = src[jj][tx + 16 * c];
                acc[0][c] = fma(p0, v, acc[0][c]);
                acc[1][c] = fma(p1, v, acc[1][c]);
            }
        }
        __syncthreads();
    }
    double* Ym = Y + ex_off(m, M) * ncol;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int k = k0 + ty + 16 * r;
        if (k >= K) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int col = c0 + tx + 16 * c;
            if (col < ncol) Ym[(int64_t)k * ncol + col] = acc[r][c];
        }
    }
}

}  // namespace

swe_status leg_inverse_f64(const swe_plan* p, const double2* X, double2* F, int C, cudaStream_t st) {
    int ncol = 2 * C;
    dim3 grid((ncol + TC - 1) / TC, (p->nlat2 + TJ - 1) / TJ, p->M + 1);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 16.0 * C * (p->ncx + (p->M + 1.0) * p->nlat) + 8.0 * p->ncx * p->nlat2;
    ProfToken tk = prof_begin("leg_inv_f64", st, fl, by);
    k_leg_inv_f64<<<grid, 256, 0, st>>>(p->P, (const double*)X, (double*)F, p->M, p->nlat, p->nlat2, ncol);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_inv_f64");
    return SWE_OK;
}

swe_status leg_forward_f64(const swe_plan* p, const double2* F, double2* Y, int C, cudaStream_t st) {
    int ncol = 2 * C;
    dim3 grid((ncol + TC - 1) / TC, (p->M + 2 + TN - 1) / TN, p->M + 1);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 16.0 * C * (p->ncx + (p->M + 1.0) * p->nlat) + 8.0 * p->ncx * p->nlat2;
    ProfToken tk = prof_begin("leg_fwd_f64", st, fl, by);
    k_leg_fwd_f64<<<grid, 256, 0, st>>>(p->P, (const double*)F, (double*)Y, p->M, p->nlat, p->nlat2, ncol);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_fwd_f64");
    return SWE_OK;
}
