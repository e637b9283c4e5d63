/*
 * swe_gb300.h -- C ABI of the GB300 (sm_103a) Parareal/MGRIT shallow-water hot path.
 *
 * Method: arXiv 2306.09497, "Parallel-in-time integration of the shallow water
 * equations on the rotating sphere using Parareal and MGRIT".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Spectral coefficients: complex128 stored as interleaved (re, im) doubles,
 *   triangular truncation T_M, m-major: for m = 0..M the entries n = m..M are
 *   contiguous, so coefficient (m, n) sits at m(M+1) - m(m-1)/2 + (n - m);
 *   NC(M) = (M+1)(M+2)/2 complex values per field.  Associated Legendre
 *   functions are normalised to unit square integral over mu in [-1, 1], with
 *   no Condon-Shortley phase; a real field is
 *   f = sum_n f_{0n} P_n^0 + 2 Re sum_{m>=1} sum_n f_{mn} P_n^m(mu) e^{i m lambda}
 *   (the imaginary part of every m = 0 coefficient is ignored) (§2.2, Eq. 2).
 * Grid: Gauss-Legendre latitudes ordered north to south, longitudes
 *   lambda_k = 2 pi k / nlon; fields are [batch][nlat][nlon], longitude fastest.
 * State vector U = (Phi', xi, delta): geopotential perturbation (the mean
 *   Phi_bar is a plan constant), vorticity, divergence (§2.1, Eq. 1); a batch of
 *   S states is [S][3][NC] complex128.  The n = 0 coefficients of xi and delta
 *   are zero for every flow and are ignored on input.
 * Memory: every array argument is a DEVICE pointer owned by the caller unless
 *   the comment says "host".  The library owns its tables and workspace.
 * Streams: every call is asynchronous on the given stream (NULL = legacy
 *   default stream) unless its comment says it synchronises.  Calls on one
 *   plan must not overlap in time (the plan's workspace is shared).  On
 *   split-precision plans the first call that runs a Legendre contraction at a
 *   new batch width outside stream capture times the kernel variants once and
 *   synchronises its stream (swe_plan_set_legendre_mode).
 * Errors: functions return a swe_status; SWE_OK is 0.  swe_last_error()
 *   returns a thread-local message describing the last failure.  No C++
 *   exception crosses this boundary.
 */
#ifndef SWE_GB300_H
#define SWE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SWE_OK = 0,
    SWE_EINVAL = 1,      /* invalid argument (sizes, pointers, descriptor fields) */
    SWE_ENOMEM = 2,      /* device allocation failed */
    SWE_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    SWE_EUNSTABLE = 4,   /* a non-finite value appeared in the state */
    SWE_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    SWE_ENOTCONV = 6     /* iteration limit reached before the tolerance */
} swe_status;

typedef enum {
    SWE_FP64 = 0,          /* every step in double precision */
    SWE_SPLIT_BF16X3 = 1   /* Legendre GEMM on tcgen05 tensor cores with operands split
                              into three bf16 terms (six partial products) and FP32
                              accumulation; batches of at most 8 complex columns use an
                              FP32 contraction with an FP32-rounded P table instead;
                              longitude FFT, grid products, SL interpolation and the
                              implicit-solve increments in FP32; Gauss nodes, P recurrence,
                              spectral state and PinT correction in FP64 */
} swe_precision;

typedef enum {
    SWE_IMEX = 0,                /* IMEX Strang splitting, §2.3.1 Eqs. 3-5 */
    SWE_SLSI_SETTLS = 1,         /* SL-SI-SETTLS two-step, §2.3.2 Eqs. 6-7 */
    SWE_SLSI_SETTLS_1STEP = 2    /* one-step variant used inside PinT, §3.2.4 */
} swe_scheme;

/* Spatial discretisation of one truncation (§2.2). nlat must be even,
 * nlat >= M + 2, nlon > 2(M+1) and nlon = 2^a 3^b. */
typedef struct {
    int M, nlat, nlon;
    double a;        /* sphere radius, m */
    double omega;    /* rotation rate, 1/s; Coriolis parameter f = 2 omega mu */
    double g;        /* gravity, m/s^2 (used by diagnostics only) */
    double phibar;   /* mean geopotential Phi_bar, m^2/s^2 */
    swe_precision prec;
} swe_plan_desc;

/* One propagator phi: nsteps steps of length dt of a scheme, each followed by
 * backward-Euler (hyper)viscosity of order visc_q (even, >= 2) and coefficient
 * visc_nu >= 0 (§2.3, App. A). */
typedef struct {
    int scheme;      /* swe_scheme */
    double dt;       /* s */
    int nsteps;
    int visc_q;
    double visc_nu;
} swe_stepper_desc;

typedef struct swe_plan* swe_plan_t;
typedef struct swe_pint* swe_pint_t;

/* Library version string (static storage). */
const char* swe_version(void);

/* Message of the last failure on the calling thread ("" if none). */
const char* swe_last_error(void);

/* Number of complex coefficients per field for truncation M: (M+1)(M+2)/2. */
int64_t swe_ncoef(int M);

/* Creates a plan on the current CUDA device: Gauss-Legendre nodes/weights
 * (Newton iteration), normalised associated Legendre table for n <= M+1 at
 * the northern Gauss latitudes (three-term recurrence), FFT twiddles.  All
 * generated on the device in FP64 (§2.2).  Synchronises.  *out receives the
 * plan; destroy it with swe_plan_destroy. */
swe_status swe_plan_create(const swe_plan_desc* desc, swe_plan_t* out);
swe_status swe_plan_destroy(swe_plan_t plan);

/* Form of the geopotential tendency in N (Eq. 1).  SWE_NPHI_FLUX (the default): the
 * analytically identical flux form -div(Phi' V), which conserves the global mean Phi'_00 to
 * rounding.  SWE_NPHI_ADVECTIVE: Eq. 1 as written, -V.grad(Phi') - Phi' delta, with
 * grad Phi' synthesised from its spectral derivatives and the products taken on the grid;
 * it costs six extra inverse scalar transforms and one forward transform per nonlinear
 * evaluation, with the grid fields in device memory.  Applies to every later nonlinear
 * evaluation on the plan (swe_nonlinear, the IMEX stepper, propagate_*, PinT); the
 * SL-SI-SETTLS scheme uses N_R = -Phi' delta only and is unaffected.  Host-side setting. */
typedef enum { SWE_NPHI_FLUX = 0, SWE_NPHI_ADVECTIVE = 1 } swe_nphi_form;
swe_status swe_plan_set_nphi_form(swe_plan_t plan, int form);

/* Kernel variant of the split-precision tensor-core Legendre contractions (§2.2) of a plan:
 *   SWE_LEGENDRE_AUTO (default): per direction and column count, the first call outside CUDA
 *     stream capture runs both variants twice on its own operands, times them with CUDA events
 *     on the call's stream (it synchronises that stream once) and keeps the faster; a call
 *     under capture before that takes the persistent kernel;
 *   SWE_LEGENDRE_PERSISTENT: one CTA per SM walks all (column tile, m, N tile) work items,
 *     with two TMEM accumulator sets so that one item's epilogue overlaps the next's MMAs;
 *   SWE_LEGENDRE_PER_TILE: one CTA per work item.
 * Both variants issue the same MMAs in the same order per item: their results are identical.
 * Host-side setting; SWE_EINVAL for another value. */
typedef enum { SWE_LEGENDRE_AUTO = 0, SWE_LEGENDRE_PERSISTENT = 1, SWE_LEGENDRE_PER_TILE = 2 } swe_legendre_mode;
swe_status swe_plan_set_legendre_mode(swe_plan_t plan, int mode);

/* Launch configurations the plan has chosen so far (fused ring kernel; per direction and
 * column count the tensor-core Legendre variant, and for batches of at most 8 complex columns
 * the SIMT or tensor-core contraction, each with the measured times), as a NUL-terminated text
 * in the HOST buffer buf of len bytes (truncated to fit).  SWE_EINVAL for a null plan or buffer. */
swe_status swe_plan_tuning(swe_plan_t plan, char* buf, size_t len);

/* Copies the Gauss-Legendre nodes mu_j (north to south) and weights w_j into
 * HOST arrays of nlat doubles.  Synchronises. */
swe_status swe_plan_gauss(swe_plan_t plan, double* mu_host, double* w_host);

/* Inverse scalar spherical-harmonic transform (§2.2): spec [batch][NC] complex128
 * -> grid [batch][nlat][nlon].  grid is double for SWE_FP64 plans and float
 * for split-precision plans. */
swe_status sht_inverse(swe_plan_t plan, const void* spec, void* grid, int batch, void* stream);

/* Forward scalar transform: grid [batch][nlat][nlon] (double or float as above)
 * -> spec [batch][NC] complex128, by FFT in longitude and Gauss quadrature in mu. */
swe_status sht_forward(swe_plan_t plan, const void* grid, void* spec, int batch, void* stream);

/* Nonlinear tendency N(U) = N_A(U) + N_R(U) of Eq. 1 for S states, evaluated
 * pseudospectrally on the Gaussian grid (the geopotential part in the
 * equivalent flux form -div(Phi' V)).  U, N: [S][3][NC] complex128. */
swe_status swe_nonlinear(swe_plan_t plan, const double* U, double* N, int S, void* stream);

/* Linear tendency L U = L_G U + L_C U of Eq. 1 (f = 2 omega mu), exact in
 * spectral space.  U, LU: [S][3][NC] complex128. */
swe_status swe_linear(swe_plan_t plan, const double* U, double* LU, int S, void* stream);

/* Solves (I - alpha L) X = R for S right-hand sides, one banded system per
 * zonal wavenumber m (Eq. 4 / Eq. 7 implicit part).  R, X: [S][3][NC]. */
swe_status swe_implicit_solve(swe_plan_t plan, double alpha, const double* R, double* X,
                              int S, void* stream);

/* Balanced initial state: given vorticity xi [S][NC] and a geopotential
 * increment phi_add [S][NC] (may be NULL), writes U = (Phi', xi, 0) with
 * Phi' = lap^{-1}([L_C U + N U]_delta) + phi_add, i.e. d(delta)/dt = 0 for the
 * non-divergent flow (nonlinear balance).  U: [S][3][NC]. */
swe_status swe_balance(swe_plan_t plan, const double* xi, const double* phi_add, double* U,
                       int S, void* stream);

/* Propagator phi_f (§3.1): applies the stepper to S independent states at once.
 * U_in, U_out: [S][3][NC]; may alias.  For the two-step SL-SI-SETTLS scheme
 * the first step of each state uses the one-step form (§3.2.4). */
swe_status propagate_F(swe_plan_t plan, const swe_stepper_desc* st, const double* U_in,
                       double* U_out, int S, void* stream);

/* Coarse propagator phi_c: runs the stepper on the coarse plan.  When the two
 * plans have different truncations the input is truncated from `fine` to
 * `coarse` and the result zero-padded back (spatial coarsening, §5.1).
 * fine may be NULL or equal to coarse.  U_in, U_out use the fine plan's NC. */
swe_status propagate_G(swe_plan_t coarse, swe_plan_t fine, const swe_stepper_desc* st,
                       const double* U_in, double* U_out, int S, void* stream);

/* Parallel-in-time problem on [0, S * slice] with S slices. */
typedef struct {
    swe_plan_t fine_plan;          /* level-0 spatial plan */
    swe_plan_t coarse_plan;        /* coarse plan (may equal fine_plan) */
    swe_stepper_desc fine;         /* phi_f over one slice (nsteps fine steps) */
    swe_stepper_desc coarse;       /* phi_c over one slice */
    int S;                         /* number of time slices N */
    int use_graphs;                /* 1: capture the serial coarse chain in a CUDA graph */
} swe_pint_desc;

swe_status swe_pint_create(const swe_pint_desc* desc, swe_pint_t* out);
swe_status swe_pint_destroy(swe_pint_t p);

/* Sets U_0 (device, [3][NC]) and computes the Parareal initial guess
 * U^0_{n+1} = phi_c(U^0_n), n = 0..S-1 (§3.1). */
swe_status swe_pint_init(swe_pint_t p, const double* U0, void* stream);

/* Runs up to kmax Parareal iterations (Eq. 9):
 * U^{k+1}_{n+1} = phi_c(U^{k+1}_n) + phi_f(U^k_n) - phi_c(U^k_n).
 * After each iteration the FP64 norm max_n ||U^{k+1}_n - U^k_n||_inf /
 * max_n ||U^{k+1}_n||_inf is written to norm_hist_host[k] (HOST, kmax doubles,
 * may be NULL); iterations stop early when it falls below tol (tol <= 0: never).
 * *k_done (HOST) receives the number of iterations run.  Synchronises once per
 * iteration (norm readback).  Returns SWE_EUNSTABLE if a non-finite value
 * appeared. */
swe_status parareal_iterate(swe_pint_t p, int kmax, double tol, int* k_done,
                            double* norm_hist_host, void* stream);

/* Copies the slice-boundary states U^k_n, n = 0..S, into U_out (device,
 * [S+1][3][NC]). */
swe_status swe_pint_solution(swe_pint_t p, double* U_out, void* stream);

/* MGRIT (§3.2): L levels, coarsening factor cf (Delta t_{l+1} = cf Delta t_l), F(CF)^nu
 * relaxation, full approximation scheme with injection at C-points, spectral
 * truncation / zero padding between the levels' truncations (level l+1 may be coarser
 * in space), and either V-cycles or F-cycles followed by one V-cycle per level
 * (§3.2.3).  step[l] is ONE time step of level l (nsteps is ignored).  On the coarsest
 * level the two-step SL-SI-SETTLS scheme keeps its previous state (the serial coarse
 * solve); relaxations and restriction steps use the one-step form (§3.2.4).
 * N0 level-0 steps must be divisible by cf^(L-1).  All time points of all levels live in
 * device memory. */
typedef struct swe_mgrit* swe_mgrit_t;
typedef struct {
    int L;                       /* number of levels, 2..8 */
    int cf;                      /* coarsening factor >= 2 */
    int nu;                      /* number of CF relaxations after the first F relaxation */
    int N0;                      /* level-0 time steps */
    int cycle;                   /* 0: V-cycle, 1: F-cycle + one V-cycle */
    swe_plan_t plan[8];          /* spatial plan of each level (truncation non-increasing) */
    swe_stepper_desc step[8];    /* one step of each level: scheme, dt, viscosity */
} swe_mgrit_desc;

swe_status swe_mgrit_create(const swe_mgrit_desc* desc, swe_mgrit_t* out);
swe_status swe_mgrit_destroy(swe_mgrit_t g);
/* Sets U_0 (device, [3][NC_0]) and builds the initial guess: serial propagation on the
 * coarsest level, injected to every finer level followed by F-relaxation. */
swe_status swe_mgrit_init(swe_mgrit_t g, const double* U0, void* stream);
/* Runs up to ncycles MGRIT iterations; after each, the FP64 per-field norm
 * max_i ||u_{cf i} - u_{cf i}^{prev}||_inf / max_i ||u_{cf i}||_inf over the level-0
 * C-points goes to norm_hist_host[k] (HOST, may be NULL); stops when it is below tol
 * (tol <= 0: never).  *k_done (HOST) = cycles run.  Synchronises once per cycle.
 * Returns SWE_EUNSTABLE if a non-finite value appeared. */
swe_status mgrit_cycle(swe_mgrit_t g, int ncycles, double tol, int* k_done, double* norm_hist_host,
                       void* stream);
/* Copies the level-0 C-point values u_{cf i}, i = 0..N0/cf, into U_out ([N0/cf+1][3][NC_0],
 * host or device). */
swe_status swe_mgrit_cpoints(swe_mgrit_t g, double* U_out, void* stream);

/* Continuous-batching forecast server.  A request is a Parareal (§3.1) or two-level
 * MGRIT (§3.2) solve of one initial state; requests queue FIFO and are admitted at the start
 * of a swe_server_step call while fewer than max_active run and the device memory they are
 * charged (swe_request_bytes: their state, staging for their slices and the plan workspace
 * their batched propagations need) fits in hbm_budget_bytes.  Each step advances every
 * active request by one iteration / cycle and synchronises once.  Requests that share a plan
 * run in one lane (one CUDA stream, in order); lanes run concurrently, so requests of
 * different truncations with their own plans overlap on the device (give coarse levels plan
 * objects of their own for that).  Parareal requests with the same plans and steppers
 * share their launches: all their slices go through one fine propagation, their serial
 * coarse chains advance together (one batched coarse step per chain position), and the
 * initial coarse chains of requests admitted together are batched the same way.  State
 * stays in device memory from admission until swe_server_result.  On FP64 plans a result
 * equals the request's result alone up to rounding (relative 1e-12); on split-precision
 * plans the batch width selects the Legendre kernel (narrow FP32 contraction for at most 8
 * complex columns, tcgen05 GEMM above) and the implicit-solve kernel, so a result in a mix
 * equals the result alone within the split-precision tolerance (full height 1e-6), not bit
 * for bit.  A non-finite value or a timed-out wait in any active request fails the step
 * (SWE_EUNSTABLE / SWE_ETIMEOUT). */
typedef struct swe_server* swe_server_t;
typedef enum { SWE_METHOD_PARAREAL = 0, SWE_METHOD_MGRIT2 = 1 } swe_method;
typedef struct {
    size_t hbm_budget_bytes;     /* admission budget for the requests' device state */
    int max_active;              /* slots */
} swe_server_desc;
typedef struct {
    swe_plan_t fine_plan, coarse_plan;
    int method;                  /* swe_method */
    swe_stepper_desc fine;       /* Parareal: fine propagator over one slice; MGRIT: one level-0 step */
    swe_stepper_desc coarse;     /* Parareal: coarse propagator over one slice; MGRIT: one level-1 step */
    int S;                       /* Parareal: slices; MGRIT: C-intervals (N0 = S * cf) */
    int cf;                      /* MGRIT coarsening factor */
    int nu_relax;                /* MGRIT F(CF)^nu */
    int iters;                   /* Parareal iterations / MGRIT cycles */
    const double* U0_host;       /* HOST [3][NC] initial state, copied by swe_server_submit */
} swe_request_desc;

swe_status swe_server_create(const swe_server_desc* desc, swe_server_t* out);
/* Device memory the server charges to a request while it is held (HOST *bytes). */
swe_status swe_request_bytes(const swe_request_desc* req, size_t* bytes);
swe_status swe_server_destroy(swe_server_t s);
/* Queues a request; *id receives its handle.  Host-side only. */
swe_status swe_server_submit(swe_server_t s, const swe_request_desc* req, long long* id);
/* Admits what fits, advances every active request by one iteration and synchronises.
 * Outputs (HOST, may be NULL): active, queued, and finished-in-this-step counts. */
swe_status swe_server_step(swe_server_t s, int* n_active, int* n_queued, int* n_done);
/* Result of a finished request: Parareal slice-boundary states [S+1][3][NC], MGRIT
 * C-points [S+1][3][NC] (HOST, may be NULL); timing_host[3] = latency (s, submit to
 * finish), queueing (s, submit to admission), iterations.  Frees the request. */
swe_status swe_server_result(swe_server_t s, long long id, double* U_host, double* timing_host);
/* Per-iteration FP64 convergence norms of a request (HOST array of max_norms); *n = count. */
swe_status swe_server_norms(swe_server_t s, long long id, double* norms_host, int max_norms, int* n);

/* Checkpoint / resume of the Parareal state: the iterate U^k_n, n = 0..S
 * ([S+1][3][NC]) and the coarse results phi_c(U^k_n), n = 0..S-1 ([S][3][NC]),
 * which is all the next iteration needs.  U and Gold may be HOST (pageable or
 * pinned) or device pointers.  swe_pint_load with Gold == NULL recomputes
 * phi_c(U^k_n) serially.  Asynchronous on `stream`. */
swe_status swe_pint_load(swe_pint_t p, const double* U, const double* Gold, void* stream);
swe_status swe_pint_save(swe_pint_t p, double* U, double* Gold, void* stream);

/* Inverse scalar transform for callers that cannot allocate device memory at
 * call time -- for example real-time loops that forbid allocator calls (an
 * allocation can block and synchronise the device), or applications whose
 * device memory belongs entirely to their own pool allocator, so that a
 * library allocation would fail or break their accounting.  Same arguments,
 * layouts and result as sht_inverse (the paper has no counterpart: this is a
 * library-usage variant).  Like sht_inverse, the first call at a new batch
 * width may time the plan's kernel variants once, synchronising `stream`.
 * Scratch comes from a fixed static device array of SWE_NOALLOC_SCRATCH_BYTES
 * (64 MiB) that every GPU which loads the library holds until the process
 * exits; nothing is allocated or freed by the call.  The scratch needed is
 * 16 * NCX + e * (M+1) * nlat bytes per field (NCX = (M+1)(M+4)/2, e = 16 for
 * SWE_FP64 plans, 8 otherwise), rounded up to 256-byte multiples; a batch that
 * does not fit returns SWE_EINVAL with the limit in swe_last_error() (for T255
 * on 384 x 768 in FP64: at most 31 fields per call).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it: make that first call before any stream
 * capture.  Every call on a device shares the one array, so calls that overlap
 * on the GPU (other streams, other threads) race and must be serialised by the
 * caller.  Nothing in the array needs to start at zero: each call writes every
 * scratch element it reads before reading it. */
#define SWE_NOALLOC_SCRATCH_BYTES (64u << 20)
swe_status sht_inverse_noalloc(swe_plan_t plan, const void* spec, void* grid, int batch, void* stream);

/* Error norms of §5 between S states U and S reference states Uref (device,
 * [S][3][NC] each, same plan).  For every state s and field f (Phi', xi, delta)
 * out_host[(3 s + f) * 2 + 0] = E_{psi,R} of Eq. 21: max |psi_mn - ref_mn| over
 *   0 <= m <= n <= R_norm divided by the same maximum of |ref_mn|;
 * out_host[(3 s + f) * 2 + 1] = relative L2 error over the sphere,
 *   sqrt(sum c_m |psi_mn - ref_mn|^2 / sum c_m |ref_mn|^2), c_0 = 1, c_m = 2: the area-weighted
 *   L2 norm of the grid fields by Parseval's identity (the paper's physical-space L2 uses an
 *   unweighted grid mean; on band-limited fields both measure the same error, with different
 *   latitude weights).
 * A zero reference norm gives 0 (equal fields) or +inf.  0 <= R_norm <= M.  out_host is HOST
 * ([S][3][2] doubles).  Uses the plan workspace; synchronises `stream`. */
swe_status swe_error_norms(swe_plan_t plan, const double* U, const double* Uref, int S, int R_norm,
                           double* out_host, void* stream);

/* Kinetic-energy spectrum of §5.1: for S states U (device, [S][3][NC]) writes
 * E[s][n] = a^2 / (4 n (n+1)) * sum_{m=-n..n} (|xi_mn|^2 + |delta_mn|^2), n = 0..M (device,
 * [S][M+1] doubles; E[s][0] = 0), the m < 0 terms being the conjugates of m > 0.  With the
 * library's normalisation sum_n E(n) is the area mean of |V|^2 / 2.  Asynchronous. */
swe_status swe_ke_spectrum(swe_plan_t plan, const double* U, int S, double* E, void* stream);

/* Stability regions of the linearised test ODE u' = lambda_L u + lambda_N u (§4, Eqs.
 * 10-20): |A| on a uniform grid of xi_N = lambda_N Delta t_c, Re xi_N in [re0, re1] (nre
 * points, fastest index) and Im xi_N in [im0, im1] (nim points), for a fixed xi_L =
 * lambda_L Delta t_c; the stability region is where |A| <= 1.  Delta t_c is the coarse
 * scheme's step; the fine scheme is IMEX with Delta t_f = Delta t_c / cf and N_f = cf N_c
 * steps per slice (§4.2).  Factors: IMEX A = ((4 + xi_L)/(4 - xi_L))^2 (1 + xi_N (2 + xi_N)/2)
 * (§4.1.1, Heun reading of Eq. 5); SL-SI-SETTLS: both roots of Eq. 13 for n_kappa values of
 * kappa s evenly spaced over [0, 2 pi] (21 for the paper's step pi/10), |A| being the largest
 * over roots and kappa s (the region is their intersection, §4.1.2), each root taken as the
 * coarse factor of Eqs. 17 / 20.  Methods:
 *   SWE_STAB_COARSE_ALONE   |A_c^{n N_c}| (n = 1: the serial scheme's factor, Fig. of §4.1);
 *   SWE_STAB_PARAREAL       Eq. 17 at slice n, iteration k;
 *   SWE_STAB_MGRIT2         two-level MGRIT with F(CF)^nu, Eq. 20 with the summation limit
 *                           min(k, floor(n/(nu+1))) that path counting on Eq. 19 gives;
 *   SWE_STAB_MGRIT2_PRINTED Eq. 20 with the printed limit floor(k/(nu+1)) (requires
 *                           floor(k/(nu+1)) (nu+1) <= n).
 * absA: DEVICE array [nim][nre] of doubles, written asynchronously on `stream`. */
typedef enum {
    SWE_STAB_COARSE_ALONE = 0,
    SWE_STAB_PARAREAL = 1,
    SWE_STAB_MGRIT2 = 2,
    SWE_STAB_MGRIT2_PRINTED = 3
} swe_stab_method;
typedef struct {
    int coarse_scheme;     /* SWE_IMEX or SWE_SLSI_SETTLS */
    int method;            /* swe_stab_method */
    int n, k;              /* slice index n >= 1 and iteration k >= 0 */
    int cf, Nc, nu;        /* coarsening factor, coarse steps per slice, CF relaxations */
    int n_kappa;           /* SL-SI-SETTLS: number of kappa s values in [0, 2 pi] */
    double xiL_re, xiL_im; /* xi_L = lambda_L Delta t_c */
} swe_stability_desc;
swe_status swe_stability_region(const swe_stability_desc* desc, double re0, double re1, int nre, double im0,
                                double im1, int nim, double* absA, void* stream);

/* Status word of a plan: kernels that run on the plan record two conditions in it
 * without stopping the stream -- a non-finite tendency (the unstable runs that the
 * paper reports as stopped, §5.2) and a bounded device-side wait of a tensor-core
 * Legendre kernel that gave up (that launch's output is incomplete; the kernel returned
 * instead of hanging).  parareal_iterate, mgrit_cycle and swe_server_step clear the
 * words of their plans, read them after every iteration and return SWE_ETIMEOUT (which
 * wins) or SWE_EUNSTABLE.  Callers of the asynchronous entry points (sht_*, propagate_*,
 * swe_nonlinear, ...) call swe_plan_check: it synchronises `stream`, reads and clears
 * the word and returns SWE_ETIMEOUT, SWE_EUNSTABLE or SWE_OK. */
swe_status swe_plan_check(swe_plan_t plan, void* stream);

/* Host-side fault injection for tests of the error paths: ORs `bits` (1 = non-finite,
 * 2 = wait timeout) into the plan's status word, asynchronously on `stream`.  No kernel
 * of the numerical path is disturbed.  Other bits return SWE_EINVAL. */
swe_status swe_plan_inject_status(swe_plan_t plan, int bits, void* stream);

/* Diagnostic of the bounded waits: one warp polls, at most `polls` times (capped at the
 * tensor-core kernels' own limit of 2^22 polls), an mbarrier that nothing completes, then
 * records a timeout in the plan's status word the way a tensor-core kernel does, and
 * returns.  Asynchronous; swe_plan_check then returns SWE_ETIMEOUT.  The paper has no
 * counterpart (failure handling of this library). */
swe_status swe_wait_selftest(swe_plan_t plan, long long polls, void* stream);

/* Instrumentation (host side, no GPU work).
 * swe_launch_count: kernels launched by the library so far (replays of a
 *   captured CUDA graph count every kernel node).
 * swe_prof_enable(on): when on, the Legendre, ring and implicit-solve kernels are
 *   bracketed by CUDA events on their own launch stream (launches inside a stream
 *   capture are not timed); returns the previous setting.
 * swe_prof_read(i, ...): statistics of the i-th timed kernel (name, timed launches,
 *   total milliseconds, algorithmic FLOPs and bytes summed over those launches);
 *   synchronises on the recorded events; returns 0 when i is out of range.
 * swe_prof_reset: drops all statistics. */
long long swe_launch_count(void);
int swe_prof_enable(int on);
void swe_prof_reset(void);
int swe_prof_read(int i, char* name, int namelen, long long* launches, double* total_ms, double* flops,
                  double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* SWE_GB300_H */
