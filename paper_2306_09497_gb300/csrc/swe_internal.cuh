// Internal declarations of the GB300 shallow-water library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/swe_gb300.h"
#include "prof.cuh"

// ---------------------------------------------------------------------------
// error plumbing: thread-local message + status codes, no exceptions across the ABI
void swe_set_error(const char* fmt, ...);
swe_status swe_cuda_status(cudaError_t e, const char* what);

#define SWE_CHECK_CUDA(call)                                                   \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return swe_cuda_status(e_, #call);              \
    } while (0)

#define SWE_CHECK(call)                                                        \
    do {                                                                       \
        swe_status s_ = (call);                                                \
        if (s_ != SWE_OK) return s_;                                           \
    } while (0)

#define SWE_CHECK_LAUNCH(what)                                                 \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess) return swe_cuda_status(e_, what);               \
        prof_launch(1);                                                        \
    } while (0)

// ---------------------------------------------------------------------------
// spectral index helpers
//   "state" rows: (m, n), 0 <= m <= n <= M            -> NC(M) rows
//   "extended" rows: (m, n), 0 <= m <= M, m <= n <= M+1 -> NCX rows (transform operands)
__host__ __device__ inline int64_t st_off(int m, int M) {
    return (int64_t)m * (M + 1) - (int64_t)m * (m - 1) / 2;
}
__host__ __device__ inline int64_t ex_off(int m, int M) {
    return (int64_t)m * (M + 2) - (int64_t)m * (m - 1) / 2;
}
__host__ __device__ inline int64_t nc_state(int M) { return (int64_t)(M + 1) * (M + 2) / 2; }
__host__ __device__ inline int64_t nc_ext(int M) { return (int64_t)(M + 1) * (M + 4) / 2; }

// epsilon_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)), zero for n <= m
// Per extended row (m, n <= M+1) coefficient table, built once per plan in FP64 so that
// the spectral kernels do no division or square root per element (GB300 runs FP64 at
// 1/64 of the FP32 rate).  il_n = -a^2/(n(n+1)) for 1 <= n <= M, else 0.
enum RowCoef {
    RC_UC0 = 0,   // m il_n / a
    RC_UCM = 1,   // (n-1) eps_n il_{n-1} / a       (n-1 >= m)
    RC_UCP = 2,   // (n+2) eps_{n+1} il_{n+1} / a
    RC_DCP = 3,   // n eps_{n+1} / a
    RC_DCM = 4,   // (n+1) eps_n / a
    RC_P = 5,     // p_n = (n+1)/n eps_n
    RC_Q = 6,     // q_n = n/(n+1) eps_{n+1}
    RC_R = 7,     // r_n = m/(n(n+1))
    RC_GM = 8,    // -(n-1) eps_n        ((1 - mu^2) d/dmu of a scalar: weight of its n-1 coefficient)
    RC_GP = 9,    // (n+2) eps_{n+1}     (weight of its n+1 coefficient)
    RC_NUM = 10
};

// FP64 <-> FP32 conversions on the integer pipe.  GB300 executes the hardware conversion
// instructions at its (low) FP64 rate; these bit-level versions round to nearest (ties
// away from zero), flush results below the FP32 normal range to zero and map
// out-of-range magnitudes to infinity (NaN stays NaN).  Used on the mixed-precision path.
__device__ __forceinline__ float d2f_fast(double x) {
    const unsigned long long o = (unsigned long long)__double_as_longlong(x);
    const unsigned long long b = o + (1ull << 28);                   // round at bit 29
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    unsigned f = sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    if (e < 897) f = sign;                                           // zero / below FP32 normals
    if (e > 1150) f = sign | 0x7f800000u | (((o >> 52 & 0x7ffu) == 0x7ffu && (o & 0xfffffffffffffull)) ? 0x400000u : 0u);
    return __uint_as_float(f);
}
__device__ __forceinline__ double f2d_fast(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0) hi = sign, lo = 0;                                   // zero (FP32 subnormals flushed)
    if (e == 255) hi = sign | 0x7ff00000u | (m >> 3);                // inf / NaN
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float2 d2f2(double2 v) { return make_float2(d2f_fast(v.x), d2f_fast(v.y)); }
__device__ __forceinline__ double2 f2d2(float2 v) { return make_double2(f2d_fast(v.x), f2d_fast(v.y)); }

__host__ __device__ inline double eps_nm(int m, int n) {
    if (n <= m) return 0.0;
    double nn = (double)n, mm = (double)m;
    return sqrt((nn * nn - mm * mm) / (4.0 * nn * nn - 1.0));
}

// ---------------------------------------------------------------------------
// CN / implicit-solve factorisation for one alpha (see spectral.cu)
struct CNFactor {
    double alpha;
    double2* fac;             // [NC][8] complex coefficients per (m, n)
    float2* fac32 = nullptr;  // FP32 copy (mixed-precision plans)
};

struct Workspace {
    char* base = nullptr;
    size_t bytes = 0;
};

struct swe_plan {
    int M, nlat, nlon, nlat2;
    double a, omega, g, phibar;
    swe_precision prec;
    int device;
    int64_t nc, ncx;
    // device tables (FP64)
    double* mu = nullptr;       // [nlat] north -> south
    double* w = nullptr;        // [nlat]
    double* P = nullptr;        // [ncx][nlat2]: P_n^m(mu_j), j in the northern half
    int* row_m = nullptr;       // [ncx] m of each extended row
    int* srow_m = nullptr;      // [nc]  m of each state row
    double2* tw = nullptr;      // [nlon] e^{-2 pi i k / nlon}
    float2* twf = nullptr;      // FP32 copy
    int nrad = 0;
    int rad[32];
    // split-precision Legendre operands: pre-split bf16 tiles for the tensor-core kernels,
    // and an FP32 copy of P for narrow batches
    void* Pbf = nullptr;
    float* Pf = nullptr;        // [ncx][nlat2]
    // implicit-solve factor cache
    CNFactor cn[16];
    int ncn = 0;
    // workspace arena
    Workspace ws;
    // device status word flags[0]: PLAN_FLAG_* bits set by kernels that ran on this plan
    int* flags = nullptr;
    // row coefficients [ncx][RC_NUM] (see RowCoef), and an FP32 copy
    double* rc = nullptr;
    float* rcf = nullptr;
    // semi-Lagrangian geometry in the grid type (extended latitudes, sin and cos of the
    // Gaussian latitudes; built on first use)
    void* thx = nullptr;
    // launch configuration of the fused nonlinear ring kernel (autotuned on first large call)
    int ring_cfg = -1, ring_G = 1;
    // geopotential tendency of N: 0 flux form -div(Phi' V), 1 advective form -V.grad Phi' - Phi' delta
    int nphi_adv = 0;
    // split-precision Legendre contractions (swe_legendre_mode): 0 pick per column count by
    // measured time, 1 persistent tcgen05 kernels, 2 one CTA per tile
    int legendre_mode = 0;
    // bumped whenever a plan-owned device buffer is allocated, grown or freed after creation
    // (workspace, implicit-solve factors, SL geometry): a CUDA graph that captured pointers
    // into the plan is valid only while the generation it was captured at is current
    unsigned long long gen = 0;
};

// ---------------------------------------------------------------------------
// split-precision tensor-core operand tables (legendre_tc.cu)
swe_status split_tables_build(swe_plan* p);
void split_tables_free(swe_plan* p);
swe_status wait_selftest_launch(const swe_plan* p, long long polls, cudaStream_t st);

// status word of a plan (flags[0]); kernels OR these bits in, synchronising calls read them
enum { PLAN_FLAG_NONFINITE = 1, PLAN_FLAG_TIMEOUT = 2 };
// enqueue the copy of the status word to *host (valid once st is synchronised)
swe_status plan_flags_fetch(const swe_plan* p, int* host, cudaStream_t st);
swe_status plan_flags_clear(const swe_plan* p, cudaStream_t st);
// status for a fetched word: a timed-out wait wins over a non-finite value; sets the message
swe_status plan_flags_status(int bits, const char* where, int iter);
// narrow batches (at most 8 complex columns) on split-precision plans (legendre_small.cu)
swe_status small_tables_build(swe_plan* p);
void small_tables_free(swe_plan* p);
bool leg_small_ok(const swe_plan* p, int C);
// narrow batches: 1 FP32 SIMT kernel, 2 tensor-core path (measured on the first call per
// direction (0 inverse, 1 forward) and column count outside stream capture)
swe_status leg_narrow_choice(const swe_plan* p, int dir, int C, const void* in, void* out, cudaStream_t st,
                             int* choice);
swe_status leg_inverse_split(const swe_plan* p, const float2* X, float2* F, int C, cudaStream_t st);
swe_status leg_forward_split(const swe_plan* p, const float2* F, float2* Y, int C, cudaStream_t st);
swe_status leg_inverse_small(const swe_plan* p, const float* X, float* F, int C, cudaStream_t st);
swe_status leg_forward_small(const swe_plan* p, const float* F, float* Y, int C, cudaStream_t st);

// plan helpers (plan.cu)
swe_status plan_workspace(swe_plan* p, size_t bytes, char** out);
swe_status plan_cn_factor(swe_plan* p, double alpha, const double2** fac, cudaStream_t st,
                          const float2** fac32 = nullptr);

// workspace layout of a nonlinear evaluation / stepper for S columns
struct NLBuffers {
    double2* X;     // [ncx][4S]    transform operands (Phi', xi, U, V)
    void* Fin;      // [M+1][nlat][4S] Fourier coefficients (double2 or float2)
    void* Fout;     // [M+1][nlat][5S]
    double2* Y;     // [ncx][5S]    forward-transform results (A1, B1, A2, B2, KE)
    // advective geopotential tendency only (plan nphi_adv), else null:
    double2* X2;    // [ncx][6S]    operands U, V, Phi', delta, dPhi'/dlambda, (1 - mu^2) dPhi'/dmu
    void* F2;       // [M+1][nlat][6S] Fourier coefficients of those
    void* G2;       // [6S][nlat][nlon] grid fields (double or float); slot 0 later holds N_Phi
    void* F3;       // [M+1][nlat][S]  Fourier coefficients of N_Phi
    double2* Y2;    // [ncx][S]     N_Phi coefficients (rows n <= M used)
};
size_t nl_bytes(const swe_plan* p, int S);
NLBuffers nl_carve(const swe_plan* p, char* base, int S);

// ---------------------------------------------------------------------------
// kernel launchers (legendre.cu, ring.cu, spectral.cu)
swe_status leg_inverse(const swe_plan* p, const double2* X, void* F, int C, cudaStream_t st);
swe_status leg_forward(const swe_plan* p, const void* F, double2* Y, int C, cudaStream_t st);

swe_status ring_inverse(const swe_plan* p, const void* F, void* grid, int C, cudaStream_t st);
swe_status ring_forward(const swe_plan* p, const void* grid, void* F, int C, cudaStream_t st);
swe_status ring_nonlinear(const swe_plan* p, const void* Fin, void* Fout, int S, cudaStream_t st);

// state layout conversions: AoS [S][3][NC] <-> SoA [3][NC][S]
swe_status k_aos_to_soa(const swe_plan* p, const double2* in, double2* out, int S, cudaStream_t st);
swe_status k_soa_to_aos(const swe_plan* p, const double2* in, double2* out, int S, cudaStream_t st);

swe_status k_aos_to_soa_strided(const swe_plan* p, const double2* in, int64_t stride, double2* out, int S,
                                cudaStream_t st);
swe_status k_soa_to_aos_strided(const swe_plan* p, const double2* in, double2* out, int64_t stride, const double2* add,
                                int64_t add_stride, int S, cudaStream_t st);

// scalar spectral [B][NC] <-> transform operand [ncx][B]
swe_status k_pack_scalar(const swe_plan* p, const double2* spec, double2* X, int B, cudaStream_t st);
swe_status k_unpack_scalar(const swe_plan* p, const double2* Y, double2* spec, int B, cudaStream_t st);

// nonlinear pre/post (SoA state, S columns)
//   X <- operands of U_a + beta * U_b
swe_status k_nl_pre(const swe_plan* p, const double2* Ua, const double2* Ub, double beta,
                    double2* X, int S, cudaStream_t st);
// post modes
enum { POST_N = 0, POST_STAGE1 = 1, POST_STAGE2 = 2 };
//   POST_N:      out0 <- N
//   POST_STAGE1: out0 <- dt N (=Ubar), out1 <- in0 + dt N  (in0 = U*)
//   POST_STAGE2: out0 <- in0 + (in1 + dt N) / 2            (in0 = U*, in1 = Ubar)
swe_status k_nl_post(const swe_plan* p, const double2* Y, int mode, double dt, const double2* in0,
                     const double2* in1, double2* out0, double2* out1, int S, cudaStream_t st,
                     const double2* Yphi = nullptr);
// advective-form geopotential tendency of U_a + beta U_b into b.Y2 (nphi_adv.cu); k_nl_post then
// takes N_Phi from b.Y2 instead of the flux divergence
swe_status nphi_adv_eval(const swe_plan* p, const double2* Ua, const double2* Ub, double beta, const NLBuffers& b,
                         int S, cudaStream_t st);

// implicit solve (SoA). If with_rhs, R = (I + alpha L) U is formed first (Crank-Nicolson).
// Viscosity factor [1 + dt nu (n(n+1)/a^2)^{q/2}]^{-1} applied to the result if nu > 0.
swe_status k_implicit(swe_plan* p, double alpha, int with_rhs, const double2* in, double2* out,
                      double visc_dt, double visc_nu, int visc_q, int S, cudaStream_t st);
swe_status k_linear(const swe_plan* p, const double2* U, double2* LU, int S, cudaStream_t st);
swe_status k_balance_combine(const swe_plan* p, const double2* xi_soa, const double2* N,
                             const double2* phi_add_soa, double2* U, int S, cudaStream_t st);
swe_status k_axpy(double2* y, const double2* x, double a, int64_t n, cudaStream_t st);
swe_status k_truncate(const double2* in, int Min, double2* out, int Mout, int S, cudaStream_t st);

// semi-Lagrangian step (sl.cu)
size_t sl_bytes(const swe_plan* p, int S);
swe_status sl_prepare(swe_plan* p);
swe_status sl_step(swe_plan* p, double dt, double nu, int q, const double2* Uprev, bool have_prev, const double2* U,
                   double2* Uout, int S, char* ws, bool swap_prev, cudaStream_t st);

// stepper (stepper.cu), SoA state with S columns; U updated in place
swe_status stepper_run(swe_plan* p, const swe_stepper_desc* sd, double2* U, int S, cudaStream_t st);
size_t stepper_bytes(const swe_plan* p, int S);
// plan workspace one propagation of S states claims (batches are chunked to bound it)
size_t stepper_bytes_chunked(const swe_plan* p, int S);
// S states at in + s*in_stride (AoS, strides in states) advanced by sd; written to out + s*out_stride,
// plus add + s*add_stride when add != nullptr.  in and out may alias with equal strides.
swe_status propagate_strided(swe_plan* p, const swe_stepper_desc* sd, const double2* in, int64_t in_stride,
                             double2* out, int64_t out_stride, const double2* add, int64_t add_stride, int S,
                             cudaStream_t st);
swe_status nonlinear_soa(swe_plan* p, const double2* Ua, const double2* Ub, double beta,
                         double2* N, int S, char* ws, cudaStream_t st);

// one MGRIT cycle enqueued behind `user` without a host synchronisation (mgrit.cu); red_host: 6
// pinned words (max |du|, max |u| per field, double bits), bits_host: one status word per level
swe_status mgrit_cycle_enqueue(swe_mgrit* g, cudaStream_t user, unsigned long long* red_host, int* bits_host);

// Parareal correction of one slice boundary (pint.cu)
swe_status parareal_correct_launch(const double2* G, const double2* F, double2* Gold, double2* Unext, int64_t nc,
                                   unsigned long long* red, int* flags, cudaStream_t st);
