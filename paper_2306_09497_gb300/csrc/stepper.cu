// Time steppers and propagators (§2.3, §3.1): IMEX Strang splitting (Eqs. 3-5)
// batched over S states, the propagate_F / propagate_G entry points and the
// operator-level entry points used for parity checks.
#include "swe_internal.cuh"

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

swe_status leg_inverse_f64(const swe_plan* p, const double2* X, double2* F, int C, cudaStream_t st);
swe_status leg_forward_f64(const swe_plan* p, const double2* F, double2* Y, int C, cudaStream_t st);

// The transform operands X (into the inverse contraction) and Y (out of the forward one) hold
// complex128 on FP64 plans and complex64 on split-precision plans (the same buffers, half used).
swe_status leg_inverse(const swe_plan* p, const double2* X, void* F, int C, cudaStream_t st) {
    if (p->prec == SWE_FP64) return leg_inverse_f64(p, X, (double2*)F, C, st);
    if (leg_small_ok(p, C)) {
        int choice = 1;
        SWE_CHECK(leg_narrow_choice(p, 0, C, X, F, st, &choice));
        if (choice == 1) return leg_inverse_small(p, reinterpret_cast<const float*>(X), (float*)F, C, st);
    }
    return leg_inverse_split(p, reinterpret_cast<const float2*>(X), (float2*)F, C, st);
}

swe_status leg_forward(const swe_plan* p, const void* F, double2* Y, int C, cudaStream_t st) {
    if (p->prec == SWE_FP64) return leg_forward_f64(p, (const double2*)F, Y, C, st);
    if (leg_small_ok(p, C)) {
        int choice = 1;
        SWE_CHECK(leg_narrow_choice(p, 1, C, F, Y, st, &choice));
        if (choice == 1) return leg_forward_small(p, (const float*)F, reinterpret_cast<float*>(Y), C, st);
    }
    return leg_forward_split(p, (const float2*)F, reinterpret_cast<float2*>(Y), C, st);
}

static size_t state_bytes(const swe_plan* p, int S) { return al256(sizeof(double2) * 3 * p->nc * S); }

size_t stepper_bytes(const swe_plan* p, int S) {
    size_t imex = 3 * state_bytes(p, S) + nl_bytes(p, S);
    size_t sl = state_bytes(p, S) + sl_bytes(p, S);
    return imex > sl ? imex : sl;
}

// N(U_a + beta U_b) -> N (SoA, S columns); ws must hold nl_bytes(p, S)
swe_status nonlinear_soa(swe_plan* p, const double2* Ua, const double2* Ub, double beta, double2* N, int S, char* ws,
                         cudaStream_t st) {
    NLBuffers b = nl_carve(p, ws, S);
    SWE_CHECK(k_nl_pre(p, Ua, Ub, beta, b.X, S, st));
    SWE_CHECK(leg_inverse(p, b.X, b.Fin, 4 * S, st));
    SWE_CHECK(ring_nonlinear(p, b.Fin, b.Fout, S, st));
    SWE_CHECK(leg_forward(p, b.Fout, b.Y, 5 * S, st));
    if (p->nphi_adv) SWE_CHECK(nphi_adv_eval(p, Ua, Ub, beta, b, S, st));
    SWE_CHECK(k_nl_post(p, b.Y, POST_N, 0.0, nullptr, nullptr, N, nullptr, S, st, b.Y2));
    return SWE_OK;
}

// One IMEX step (Eqs. 3-5, Heun reading of Eq. 5) on U (SoA).  The result is
// written to *out, which is one of {U, T}; the other buffer is scratch.
static swe_status imex_step(swe_plan* p, double dt, double nu, int q, double2* U, double2* T, double2* Us,
                            double2* Ub, char* nlws, int S, cudaStream_t st, double2** out) {
    const double alpha = 0.25 * dt;
    NLBuffers b = nl_carve(p, nlws, S);
    // U* = CN(dt/4) U
    SWE_CHECK(k_implicit(p, alpha, 1, U, Us, 0.0, 0.0, 2, S, st));
    // Ubar = dt N(U*),  T = U* + Ubar
    SWE_CHECK(k_nl_pre(p, Us, nullptr, 0.0, b.X, S, st));
    SWE_CHECK(leg_inverse(p, b.X, b.Fin, 4 * S, st));
    SWE_CHECK(ring_nonlinear(p, b.Fin, b.Fout, S, st));
    SWE_CHECK(leg_forward(p, b.Fout, b.Y, 5 * S, st));
    if (p->nphi_adv) SWE_CHECK(nphi_adv_eval(p, Us, nullptr, 0.0, b, S, st));
    SWE_CHECK(k_nl_post(p, b.Y, POST_STAGE1, dt, Us, nullptr, Ub, T, S, st, b.Y2));
    // U** = U* + (Ubar + dt N(U* + Ubar)) / 2   -> written into U (no longer needed)
    SWE_CHECK(k_nl_pre(p, T, nullptr, 0.0, b.X, S, st));
    SWE_CHECK(leg_inverse(p, b.X, b.Fin, 4 * S, st));
    SWE_CHECK(ring_nonlinear(p, b.Fin, b.Fout, S, st));
    SWE_CHECK(leg_forward(p, b.Fout, b.Y, 5 * S, st));
    if (p->nphi_adv) SWE_CHECK(nphi_adv_eval(p, T, nullptr, 0.0, b, S, st));
    SWE_CHECK(k_nl_post(p, b.Y, POST_STAGE2, dt, Us, Ub, U, nullptr, S, st, b.Y2));
    // U^{n+1} = CN(dt/4) U**, then backward-Euler viscosity
    SWE_CHECK(k_implicit(p, alpha, 1, U, T, dt, nu, q, S, st));
    *out = T;
    return SWE_OK;
}

static swe_status check_stepper(const swe_stepper_desc* sd) {
    if (!sd) {
        swe_set_error("stepper descriptor is NULL");
        return SWE_EINVAL;
    }
    if (sd->nsteps < 0 || !(sd->dt > 0.0) || sd->visc_nu < 0.0 || (sd->visc_nu > 0.0 && (sd->visc_q < 2 || (sd->visc_q & 1)))) {
        swe_set_error("stepper: need nsteps >= 0, dt > 0, nu >= 0 and even q >= 2 (got nsteps=%d dt=%g nu=%g q=%d)",
                      sd->nsteps, sd->dt, sd->visc_nu, sd->visc_q);
        return SWE_EINVAL;
    }
    if (sd->scheme != SWE_IMEX && sd->scheme != SWE_SLSI_SETTLS && sd->scheme != SWE_SLSI_SETTLS_1STEP) {
        swe_set_error("stepper: unknown scheme %d", sd->scheme);
        return SWE_EINVAL;
    }
    return SWE_OK;
}

// Runs sd->nsteps steps on U (SoA, S columns) in place; ws holds stepper_bytes(p, S).
static swe_status run_soa(swe_plan* p, const swe_stepper_desc* sd, double2* U, int S, char* ws, cudaStream_t st) {
    size_t sb = state_bytes(p, S);
    double2* T = (double2*)ws;
    double2* Us = (double2*)(ws + sb);
    double2* Ub = (double2*)(ws + 2 * sb);
    char* nlws = ws + 3 * sb;
    double2* cur = U;
    double2* oth = T;
    if (sd->scheme != SWE_IMEX) {
        // SL-SI-SETTLS: the first step is one-step; later steps of the two-step scheme reuse
        // the previous step's velocity and N_R (kept in the SL workspace)
        char* slws = ws + sb;
        SWE_CHECK(sl_prepare(p));
        const bool two = (sd->scheme == SWE_SLSI_SETTLS);
        for (int k = 0; k < sd->nsteps; ++k) {
            SWE_CHECK(sl_step(p, sd->dt, sd->visc_nu, sd->visc_q, nullptr, two && k > 0, cur, oth, S, slws,
                              two && k + 1 < sd->nsteps, st));
            double2* t = cur;
            cur = oth;
            oth = t;
        }
        if (cur != U) SWE_CHECK_CUDA(cudaMemcpyAsync(U, cur, sizeof(double2) * 3 * p->nc * S, cudaMemcpyDeviceToDevice, st));
        return SWE_OK;
    }
    for (int k = 0; k < sd->nsteps; ++k) {
        double2* res;
        SWE_CHECK(imex_step(p, sd->dt, sd->visc_nu, sd->visc_q, cur, oth, Us, Ub, nlws, S, st, &res));
        oth = cur;
        cur = res;
    }
    if (cur != U) SWE_CHECK_CUDA(cudaMemcpyAsync(U, cur, sizeof(double2) * 3 * p->nc * S, cudaMemcpyDeviceToDevice, st));
    return SWE_OK;
}

swe_status stepper_run(swe_plan* p, const swe_stepper_desc* sd, double2* U, int S, cudaStream_t st) {
    SWE_CHECK(check_stepper(sd));
    char* ws;
    SWE_CHECK(plan_workspace(p, stepper_bytes(p, S), &ws));
    return run_soa(p, sd, U, S, ws, st);
}

// Columns per chunk so that one chunk's workspace stays below ~24 GB.
static int chunk_cols(const swe_plan* p, int S) {
    size_t per = state_bytes(p, 1) + stepper_bytes(p, 1);
    size_t budget = (size_t)24 << 30;
    int c = (int)(budget / per);
    if (c < 1) c = 1;
    return S < c ? S : c;
}

// plan workspace one propagation of S states claims (one chunk's staging and stepper buffers)
size_t stepper_bytes_chunked(const swe_plan* p, int S) {
    const int cols = chunk_cols(p, S);
    return state_bytes(p, cols) + stepper_bytes(p, cols);
}

static swe_status propagate_impl(swe_plan* p, const swe_stepper_desc* sd, const double* U_in, double* U_out, int S,
                                 cudaStream_t st) {
    SWE_CHECK(check_stepper(sd));
    if (!U_in || !U_out || S < 1) {
        swe_set_error("propagate: invalid state pointers or S < 1");
        return SWE_EINVAL;
    }
    const int cols = chunk_cols(p, S);
    const size_t sb = state_bytes(p, cols);
    char* ws;
    SWE_CHECK(plan_workspace(p, sb + stepper_bytes(p, cols), &ws));
    double2* Ut = (double2*)ws;
    char* sws = ws + sb;
    const int64_t per = 3 * p->nc;
    for (int s0 = 0; s0 < S; s0 += cols) {
        const int c = (S - s0) < cols ? (S - s0) : cols;
        const double2* in = (const double2*)U_in + per * s0;
        double2* out = (double2*)U_out + per * s0;
        if (c == 1) {
            SWE_CHECK_CUDA(cudaMemcpyAsync(Ut, in, sizeof(double2) * per, cudaMemcpyDeviceToDevice, st));
        } else {
            SWE_CHECK(k_aos_to_soa(p, in, Ut, c, st));
        }
        SWE_CHECK(run_soa(p, sd, Ut, c, sws, st));
        if (c == 1) {
            SWE_CHECK_CUDA(cudaMemcpyAsync(out, Ut, sizeof(double2) * per, cudaMemcpyDeviceToDevice, st));
        } else {
            SWE_CHECK(k_soa_to_aos(p, Ut, out, c, st));
        }
    }
    return SWE_OK;
}

swe_status propagate_strided(swe_plan* p, const swe_stepper_desc* sd, const double2* in, int64_t in_stride,
                             double2* out, int64_t out_stride, const double2* add, int64_t add_stride, int S,
                             cudaStream_t st) {
    SWE_CHECK(check_stepper(sd));
    if (S < 1) return SWE_OK;
    const int cols = chunk_cols(p, S);
    const size_t sb = state_bytes(p, cols);
    char* ws;
    SWE_CHECK(plan_workspace(p, sb + stepper_bytes(p, cols), &ws));
    double2* Ut = (double2*)ws;
    char* sws = ws + sb;
    const int64_t per = 3 * p->nc;
    for (int s0 = 0; s0 < S; s0 += cols) {
        const int c = (S - s0) < cols ? (S - s0) : cols;
        SWE_CHECK(k_aos_to_soa_strided(p, in + per * in_stride * s0, per * in_stride, Ut, c, st));
        SWE_CHECK(run_soa(p, sd, Ut, c, sws, st));
        SWE_CHECK(k_soa_to_aos_strided(p, Ut, out + per * out_stride * s0, per * out_stride,
                                       add ? add + per * add_stride * s0 : nullptr, per * add_stride, c, st));
    }
    return SWE_OK;
}

extern "C" swe_status propagate_F(swe_plan_t p, const swe_stepper_desc* sd, const double* U_in, double* U_out, int S,
                                  void* stream) {
    if (!p) {
        swe_set_error("propagate_F: plan is NULL");
        return SWE_EINVAL;
    }
    return propagate_impl(p, sd, U_in, U_out, S, (cudaStream_t)stream);
}

extern "C" swe_status propagate_G(swe_plan_t coarse, swe_plan_t fine, const swe_stepper_desc* sd, const double* U_in,
                                  double* U_out, int S, void* stream) {
    if (!coarse) {
        swe_set_error("propagate_G: coarse plan is NULL");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!fine || fine == coarse || fine->M == coarse->M) return propagate_impl(coarse, sd, U_in, U_out, S, st);
    // spatial coarsening: truncate to the coarse T_M, propagate, zero-pad back
    if (!U_in || !U_out || S < 1) {
        swe_set_error("propagate_G: invalid state pointers or S < 1");
        return SWE_EINVAL;
    }
    size_t cb = al256(sizeof(double2) * 3 * coarse->nc * S);
    double2* tmp;
    SWE_CHECK_CUDA(cudaMallocAsync((void**)&tmp, cb, st));
    swe_status s = k_truncate((const double2*)U_in, fine->M, tmp, coarse->M, S, st);
    if (s == SWE_OK) s = propagate_impl(coarse, sd, (const double*)tmp, (double*)tmp, S, st);
    if (s == SWE_OK) s = k_truncate(tmp, coarse->M, (double2*)U_out, fine->M, S, st);
    cudaFreeAsync(tmp, st);
    return s;
}

// ---------------------------------------------------------------------------
// operator-level entry points (AoS in/out)
template <typename F>
static swe_status with_soa(swe_plan* p, const double* in, double* out, int S, size_t extra, cudaStream_t st, F body) {
    if (!p || !in || !out || S < 1) {
        swe_set_error("invalid argument (plan, pointers or S)");
        return SWE_EINVAL;
    }
    size_t sb = state_bytes(p, S);
    char* ws;
    SWE_CHECK(plan_workspace(p, 2 * sb + extra, &ws));
    double2* A = (double2*)ws;
    double2* B = (double2*)(ws + sb);
    SWE_CHECK(k_aos_to_soa(p, (const double2*)in, A, S, st));
    SWE_CHECK(body(A, B, ws + 2 * sb));
    SWE_CHECK(k_soa_to_aos(p, B, (double2*)out, S, st));
    return SWE_OK;
}

extern "C" swe_status swe_nonlinear(swe_plan_t p, const double* U, double* N, int S, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    return with_soa(p, U, N, S, p ? nl_bytes(p, S) : 0, st, [&](double2* A, double2* B, char* ws) {
        return nonlinear_soa(p, A, nullptr, 0.0, B, S, ws, st);
    });
}

extern "C" swe_status swe_linear(swe_plan_t p, const double* U, double* LU, int S, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    return with_soa(p, U, LU, S, 0, st, [&](double2* A, double2* B, char*) { return k_linear(p, A, B, S, st); });
}

extern "C" swe_status swe_implicit_solve(swe_plan_t p, double alpha, const double* R, double* X, int S, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    return with_soa(p, R, X, S, 0, st, [&](double2* A, double2* B, char*) {
        return k_implicit(p, alpha, 0, A, B, 0.0, 0.0, 2, S, st);
    });
}

extern "C" swe_status swe_balance(swe_plan_t p, const double* xi, const double* phi_add, double* U, int S,
                                  void* stream) {
    if (!p || !xi || !U || S < 1) {
        swe_set_error("swe_balance: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    size_t sb = state_bytes(p, S);
    size_t fb = al256(sizeof(double2) * p->nc * S);
    char* ws;
    SWE_CHECK(plan_workspace(p, 2 * sb + 2 * fb + nl_bytes(p, S), &ws));
    double2* A = (double2*)ws;                 // (0, xi, 0) in SoA
    double2* N = (double2*)(ws + sb);
    double2* xs = (double2*)(ws + 2 * sb);     // xi [NC][S]
    double2* ps = (double2*)(ws + 2 * sb + fb);
    char* nlws = ws + 2 * sb + 2 * fb;
    // stage xi (and phi_add) [S][NC] as AoS states (0, xi, 0) and transpose to SoA
    double2* stage;
    SWE_CHECK_CUDA(cudaMallocAsync((void**)&stage, sb, st));
    SWE_CHECK_CUDA(cudaMemsetAsync(stage, 0, sb, st));
    for (int s = 0; s < S; ++s)
        SWE_CHECK_CUDA(cudaMemcpyAsync(stage + (int64_t)s * 3 * p->nc + p->nc, (const double2*)xi + (int64_t)s * p->nc,
                                       sizeof(double2) * p->nc, cudaMemcpyDeviceToDevice, st));
    SWE_CHECK(k_aos_to_soa(p, stage, A, S, st));
    SWE_CHECK(nonlinear_soa(p, A, nullptr, 0.0, N, S, nlws, st));
    SWE_CHECK_CUDA(cudaMemcpyAsync(xs, A + p->nc * S, sizeof(double2) * p->nc * S, cudaMemcpyDeviceToDevice, st));
    const double2* padd = nullptr;
    if (phi_add) {
        SWE_CHECK_CUDA(cudaMemsetAsync(stage, 0, sb, st));
        for (int s = 0; s < S; ++s)
            SWE_CHECK_CUDA(cudaMemcpyAsync(stage + (int64_t)s * 3 * p->nc, (const double2*)phi_add + (int64_t)s * p->nc,
                                           sizeof(double2) * p->nc, cudaMemcpyDeviceToDevice, st));
        SWE_CHECK(k_aos_to_soa(p, stage, A, S, st));
        SWE_CHECK_CUDA(cudaMemcpyAsync(ps, A, sizeof(double2) * p->nc * S, cudaMemcpyDeviceToDevice, st));
        padd = ps;
    }
    SWE_CHECK(k_balance_combine(p, xs, N, padd, A, S, st));
    SWE_CHECK(k_soa_to_aos(p, A, (double2*)U, S, st));
    cudaFreeAsync(stage, st);
    return SWE_OK;
}
