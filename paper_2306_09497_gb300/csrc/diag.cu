// Diagnostics of §5: the spectral error of Eq. 21, the relative L2 error, and the kinetic-energy
// spectrum of §5.1, on batches of states [S][3][NC] (complex128, m-major triangular).
//
// Error norms: one block per (state, field).  The block streams the NC coefficients of the
// field and of its reference once (coalesced 16-byte loads) and reduces, in FP64,
//   max |psi - ref| and max |ref| over 0 <= m <= n <= R          (Eq. 21, R = R_norm)
//   sum c_m |psi - ref|^2 and sum c_m |ref|^2 over all coefficients (c_0 = 1, c_m = 2)
// The second pair is the area-weighted L2 norm on the sphere by Parseval's identity for the
// orthonormal basis (area mean of f^2 = (1/2) sum c_m |f_mn|^2); the imaginary part of every
// m = 0 coefficient is ignored, as everywhere in the library.  HBM-bound: 32 bytes per
// coefficient pair, read once.
//
// KE spectrum: one block per state; E(n) = a^2 / (4 n (n+1)) sum_{m=-n..n} (|xi_mn|^2 +
// |delta_mn|^2), where the m < 0 terms equal the m > 0 terms by conjugate symmetry, so the sum
// is sum_{m>=0} c_m (...).  With this normalisation sum_n E(n) is the area mean of |V|^2 / 2.
// The block accumulates per-degree partial sums in shared memory (FP64 shared atomics), then
// writes E(0..M) for the state.
#include <cmath>
#include <vector>

#include "swe_internal.cuh"

namespace {

constexpr int NT = 256;

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out[(s*3 + f)*4 + {0,1,2,3}] = {max_R |d|, max_R |ref|, sum c|d|^2, sum c|ref|^2}
__global__ void __launch_bounds__(NT) k_error_norms(const double2* __restrict__ U, const double2* __restrict__ R,
                                                    const int* __restrict__ srow_m, int M, int64_t nc, int Rn,
                                                    double* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * nc;
    double mx_d = 0.0, mx_r = 0.0, s_d = 0.0, s_r = 0.0;
    for (int64_t i = threadIdx.x; i < nc; i += NT) {
        const int m = srow_m[i];
        const int n = m + (int)(i - st_off(m, M));
        double2 u = U[base + i], r = R[base + i];
        if (m == 0) {
            u.y = 0.0;
            r.y = 0.0;
        }
        const double dx = u.x - r.x, dy = u.y - r.y;
        const double d2 = dx * dx + dy * dy, r2 = r.x * r.x + r.y * r.y;
        const double c = m == 0 ? 1.0 : 2.0;
        s_d += c * d2;
        s_r += c * r2;
        if (n <= Rn) {
            mx_d = fmax(mx_d, sqrt(d2));
            mx_r = fmax(mx_r, sqrt(r2));
        }
    }
    __shared__ double red[4][NT / 32];
    mx_d = warp_max(mx_d);
    mx_r = warp_max(mx_r);
    s_d = warp_sum(s_d);
    s_r = warp_sum(s_r);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = mx_d;
        red[1][w] = mx_r;
        red[2][w] = s_d;
        red[3][w] = s_r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0, d = 0;
        for (int k = 0; k < NT / 32; ++k) {
            a = fmax(a, red[0][k]);
            b = fmax(b, red[1][k]);
            c += red[2][k];
            d += red[3][k];
        }
        double* o = out + (int64_t)blockIdx.x * 4;
        o[0] = a;
        o[1] = b;
        o[2] = c;
        o[3] = d;
    }
}

// E[s][n], n = 0..M (E[s][0] = 0)
__global__ void __launch_bounds__(NT) k_ke_spectrum(const double2* __restrict__ U, const int* __restrict__ srow_m,
                                                    int M, int64_t nc, double a, double* __restrict__ E) {
    extern __shared__ double acc[];
    for (int n = threadIdx.x; n <= M; n += NT) acc[n] = 0.0;
    __syncthreads();
    const double2* xi = U + (int64_t)blockIdx.x * 3 * nc + nc;
    const double2* de = xi + nc;
    for (int64_t i = threadIdx.x; i < nc; i += NT) {
        const int m = srow_m[i];
        const int n = m + (int)(i - st_off(m, M));
        if (n == 0) continue;
        double2 x = xi[i], d = de[i];
        if (m == 0) {
            x.y = 0.0;
            d.y = 0.0;
        }
        const double c = m == 0 ? 1.0 : 2.0;
        atomicAdd(&acc[n], c * (x.x * x.x + x.y * x.y + d.x * d.x + d.y * d.y));
    }
    __syncthreads();
    for (int n = threadIdx.x; n <= M; n += NT)
        E[(int64_t)blockIdx.x * (M + 1) + n] = n == 0 ? 0.0 : acc[n] * a * a / (4.0 * n * (n + 1.0));
}

}  // namespace

extern "C" swe_status swe_error_norms(swe_plan_t p, const double* U, const double* Uref, int S, int R_norm,
                                      double* out_host, void* stream) {
    if (!p || !U || !Uref || !out_host || S < 1 || R_norm < 0 || R_norm > p->M) {
        swe_set_error("swe_error_norms: invalid argument (need 0 <= R_norm <= M, S >= 1)");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nout = (size_t)S * 3 * 4;
    char* ws;
    SWE_CHECK(plan_workspace(p, sizeof(double) * nout, &ws));
    double* dout = (double*)ws;
    ProfToken tk = prof_begin("error_norms", st, 0.0, 32.0 * 3.0 * S * p->nc);
    k_error_norms<<<3 * S, NT, 0, st>>>((const double2*)U, (const double2*)Uref, p->srow_m, p->M, p->nc, R_norm,
                                         dout);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_error_norms");
    std::vector<double> h(nout);
    SWE_CHECK_CUDA(cudaMemcpyAsync(h.data(), dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
    SWE_CHECK_CUDA(cudaStreamSynchronize(st));
    for (size_t k = 0; k < (size_t)S * 3; ++k) {
        const double* o = &h[4 * k];
        out_host[2 * k] = o[1] > 0.0 ? o[0] / o[1] : (o[0] > 0.0 ? INFINITY : 0.0);
        out_host[2 * k + 1] = o[3] > 0.0 ? sqrt(o[2] / o[3]) : (o[2] > 0.0 ? INFINITY : 0.0);
    }
    return SWE_OK;
}

extern "C" swe_status swe_ke_spectrum(swe_plan_t p, const double* U, int S, double* E, void* stream) {
    if (!p || !U || !E || S < 1) {
        swe_set_error("swe_ke_spectrum: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = sizeof(double) * (p->M + 1);
    ProfToken tk = prof_begin("ke_spectrum", st, 0.0, 32.0 * S * p->nc + 8.0 * S * (p->M + 1));
    k_ke_spectrum<<<S, NT, smem, st>>>((const double2*)U, p->srow_m, p->M, p->nc, p->a, E);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_ke_spectrum");
    return SWE_OK;
}
