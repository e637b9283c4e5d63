// Split-precision Legendre contraction for narrow batches (at most NCS = 16 real data
// columns, i.e. 8 complex columns: one state of the serial coarse chains).
//
// Same sums as the tensor-core kernels (§2.2, the per-wavenumber contraction with the
// equatorial fold):
//   inverse:  D_par(j) = sum_{r = n - m, r = par mod 2} P_n^m(mu_j) X(m, n),
//             F(mu_j) = D_0 + D_1,  F(-mu_j) = D_0 - D_1
//   forward:  Y(m, n) = sum_{j < nlat/2} P_n^m(mu_j) G_{(n - m) mod 2}(j),
//             G_0 = F(mu_j) + F(-mu_j),  G_1 = F(mu_j) - F(-mu_j)
// in FP32 with an FP32 copy of the FP64 P table (rounded once; the bf16 three-way split of
// the tensor-core path carries the same 24 significant bits).
//
// At such widths a tensor-core CTA spends its time in pipeline set-up and drain, not in
// MMAs.  Here one block of 8 warps handles one wavenumber and a tile of 32 latitudes
// (inverse) or 32 degrees (forward): every load of the tile's P block and of the data
// rows is issued at once into shared memory, warp g sums the indices of residue g mod 8
// (for the inverse, rows of one parity per warp), and the 8 partial sums are added in
// shared memory.  The longest dependent chain is one staging round trip plus ceil(K/8)
// shared-memory FMAs.
#include "swe_internal.cuh"

namespace {

constexpr int NCS = 16;          // largest number of real data columns
constexpr int NG = 8;            // warps per block (residue classes of the summed index)
constexpr int NTS = 32 * NG;
constexpr int PADC = NCS + 1;    // row stride of the partial sums (floats)

__global__ void k_p_to_f32(const double* __restrict__ P, float* __restrict__ Pf, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) Pf[i] = __double2float_rn(P[i]);
}

// grid (M+1, ceil(nlat2 / 32)); X [ncx][ncol], F [M+1][nlat][ncol]
__global__ void __launch_bounds__(NTS) k_leg_inv_small(const float* __restrict__ X, float* __restrict__ F,
                                                       const float* __restrict__ Pf, int M, int nlat, int nlat2,
                                                       int ncol) {
    extern __shared__ float sm[];
    const int m = blockIdx.x;                    // m = 0 (the most rows) is scheduled first
    const int j0 = blockIdx.y * 32;
    const int Kx = M + 2 - m;
    const int64_t row0 = ex_off(m, M);
    float* sx = sm;                              // [Kx][ncol] data rows
    float* sp = sx + (M + 2) * NCS;              // [Kx][32] P of this latitude tile
    float* sr = sp + (M + 2) * 32;               // [NG][32][PADC] partial sums
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    for (int i = tid; i < Kx * ncol; i += NTS) sx[i] = X[row0 * ncol + i];
    for (int i = tid; i < Kx * 32; i += NTS) {
        const int r = i >> 5, jj = i & 31;
        sp[i] = (j0 + jj < nlat2) ? Pf[(row0 + r) * nlat2 + j0 + jj] : 0.f;
    }
    __syncthreads();
    float acc[NCS];
#pragma unroll
    for (int c = 0; c < NCS; ++c) acc[c] = 0.f;
    for (int r = g; r < Kx; r += NG) {           // r = n - m: warp g holds one parity (NG even)
        const float pv = sp[r * 32 + lane];
        const float* xr = sx + r * ncol;
#pragma unroll
        for (int c = 0; c < NCS; ++c)
            if (c < ncol) acc[c] = fmaf(pv, xr[c], acc[c]);
    }
    float* mine = sr + (g * 32 + lane) * PADC;
#pragma unroll
    for (int c = 0; c < NCS; ++c) mine[c] = acc[c];
    __syncthreads();
    for (int i = tid; i < 32 * ncol; i += NTS) {
        const int jj = i / ncol, c = i - jj * ncol, j = j0 + jj;
        if (j >= nlat2) continue;
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int q = 0; q < NG; q += 2) {
            e += sr[(q * 32 + jj) * PADC + c];
            o += sr[((q + 1) * 32 + jj) * PADC + c];
        }
        F[((int64_t)m * nlat + j) * ncol + c] = e + o;
        F[((int64_t)m * nlat + (nlat - 1 - j)) * ncol + c] = e - o;
    }
}

// grid (M+1, ceil((M+2) / 32)); F [M+1][nlat][ncol], Y [ncx][ncol]
__global__ void __launch_bounds__(NTS) k_leg_fwd_small(const float* __restrict__ F, float* __restrict__ Y,
                                                       const float* __restrict__ Pf, int M, int nlat, int nlat2,
                                                       int ncol) {
    extern __shared__ float sm[];
    const int m = blockIdx.x;
    const int r0 = blockIdx.y * 32;
    const int Kx = M + 2 - m;
    if (r0 >= Kx) return;                        // uniform for the block, before any barrier
    const int64_t row0 = ex_off(m, M);
    float* sg = sm;                              // [2][nlat2][ncol]: G_0, G_1
    float* sp = sg + 2 * nlat2 * NCS;            // [nlat2][33]: P of rows r0 .. r0 + 31, transposed
    float* sr = sp + nlat2 * 33;                 // [NG][32][PADC] partial sums
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const float* Fm = F + (int64_t)m * nlat * ncol;
    for (int i = tid; i < nlat2 * ncol; i += NTS) {
        const int j = i / ncol, c = i - j * ncol;
        const float fn = Fm[(int64_t)j * ncol + c], fs = Fm[(int64_t)(nlat - 1 - j) * ncol + c];
        sg[i] = fn + fs;
        sg[nlat2 * ncol + i] = fn - fs;
    }
    for (int i = tid; i < 32 * nlat2; i += NTS) {
        const int rr = i / nlat2, j = i - rr * nlat2;
        sp[j * 33 + rr] = (r0 + rr < Kx) ? Pf[(row0 + r0 + rr) * nlat2 + j] : 0.f;
    }
    __syncthreads();
    const float* gp = sg + (lane & 1) * nlat2 * ncol;   // r0 is even: the parity of r = r0 + lane
    float acc[NCS];
#pragma unroll
    for (int c = 0; c < NCS; ++c) acc[c] = 0.f;
    for (int j = g; j < nlat2; j += NG) {
        const float pv = sp[j * 33 + lane];
        const float* gr = gp + j * ncol;
#pragma unroll
        for (int c = 0; c < NCS; ++c)
            if (c < ncol) acc[c] = fmaf(pv, gr[c], acc[c]);
    }
    float* mine = sr + (g * 32 + lane) * PADC;
#pragma unroll
    for (int c = 0; c < NCS; ++c) mine[c] = acc[c];
    __syncthreads();
    for (int i = tid; i < 32 * ncol; i += NTS) {
        const int rr = i / ncol, c = i - rr * ncol;
        if (r0 + rr >= Kx) continue;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < NG; ++q) s += sr[(q * 32 + rr) * PADC + c];
        Y[(row0 + r0 + rr) * ncol + c] = s;
    }
}

size_t inv_smem(const swe_plan* p) { return sizeof(float) * ((size_t)(p->M + 2) * (NCS + 32) + NG * 32 * PADC); }
size_t fwd_smem(const swe_plan* p) { return sizeof(float) * ((size_t)p->nlat2 * (2 * NCS + 33) + NG * 32 * PADC); }

}  // namespace

bool leg_small_ok(const swe_plan* p, int C) { return p->Pf != nullptr && 2 * C <= NCS; }

swe_status small_tables_build(swe_plan* p) {
    if (p->Pf) return SWE_OK;
    // shared-memory footprints must fit one block (227 KB); otherwise the tensor-core path serves all widths
    const size_t lim = 227 * 1024;
    if (inv_smem(p) > lim || fwd_smem(p) > lim) return SWE_OK;
    const int64_t n = p->ncx * p->nlat2;
    SWE_CHECK_CUDA(cudaMalloc((void**)&p->Pf, sizeof(float) * n));
    k_p_to_f32<<<(unsigned)((n + 255) / 256), 256>>>(p->P, p->Pf, n);
    SWE_CHECK_LAUNCH("k_p_to_f32");
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_inv_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem(p)));
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_fwd_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(p)));
    SWE_CHECK_CUDA(cudaDeviceSynchronize());
    return SWE_OK;
}

void small_tables_free(swe_plan* p) {
    cudaFree(p->Pf);
    p->Pf = nullptr;
}

swe_status leg_inverse_small(const swe_plan* p, const float* X, float* F, int C, cudaStream_t st) {
    const int ncol = 2 * C;
    const size_t sm = inv_smem(p);
    dim3 grid(p->M + 1, (p->nlat2 + 31) / 32);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 4.0 * ncol * (p->ncx + (p->M + 1.0) * p->nlat) + 4.0 * p->ncx * p->nlat2;
    // the dynamic shared-memory limit is a per-function attribute shared by all plans: set it per launch
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_inv_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ProfToken tk = prof_begin("leg_inv_small", st, fl, by);
    k_leg_inv_small<<<grid, NTS, sm, st>>>(X, F, p->Pf, p->M, p->nlat, p->nlat2, ncol);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_inv_small");
    return SWE_OK;
}

swe_status leg_forward_small(const swe_plan* p, const float* F, float* Y, int C, cudaStream_t st) {
    const int ncol = 2 * C;
    const size_t sm = fwd_smem(p);
    dim3 grid(p->M + 1, (p->M + 2 + 31) / 32);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 4.0 * ncol * (p->ncx + (p->M + 1.0) * p->nlat) + 4.0 * p->ncx * p->nlat2;
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_fwd_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    ProfToken tk = prof_begin("leg_fwd_small", st, fl, by);
    k_leg_fwd_small<<<grid, NTS, sm, st>>>(F, Y, p->Pf, p->M, p->nlat, p->nlat2, ncol);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_fwd_small");
    return SWE_OK;
}
