// Longitude transforms on latitude rings (§2.2, "Fast Fourier"), in shared memory.
//
// Every real field of length N = nlon gets its own complex Stockham FFT (radix
// 4/3/2) of length H = N/2 on z_n = x_{2n} + i x_{2n+1}: the spectra of even and
// odd samples of ONE field are untangled with the twiddles e^{-2 pi i k / N}, so
// fields of very different magnitude never share a transform (packing two
// fields into one complex FFT would add the rounding of the larger one to the
// smaller one).  Fourier coefficients are kept for m = 0..M (M < H).
//
//   inverse:  g(lambda_k) = Re F_0 + 2 Re sum_{m>=1} F_m e^{i m lambda_k}
//   forward:  F_m = (w_j / N) sum_k g(lambda_k) e^{-i m lambda_k}   (Gauss weight folded in)
//
// k_ring_nl fuses, for one (slice, latitude) ring, the inverse FFTs of
// (Phi', xi, U, V), the grid products of the nonlinear terms (Eq. 1) and the
// forward FFTs of (xi U, xi V, Phi' U, Phi' V)/(1 - mu^2) and (U^2 + V^2)/(2 (1 - mu^2)),
// so that no grid field is ever written to HBM.
#include "swe_internal.cuh"

namespace {

template <typename T> struct CT;
template <> struct CT<double> { using V = double2; };
template <> struct CT<float> { using V = float2; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
// multiply by s * i  (s = +1 or -1)
template <int S, typename V> __device__ __forceinline__ V cmul_si(V a) {
    return S > 0 ? V{-a.y, a.x} : V{a.y, -a.x};
}

struct FFTPlan {
    int n, nrad;     // transform length (H = nlon / 2) and radices
    int tws;         // stride into the nlon-point twiddle table (2)
    int rad[32];
};

// One Stockham pass of radix R over nfft sequences of length N stored at stride `stride`.
// S = -1 forward, +1 inverse.  tw[k * tws] = e^{-2 pi i k / N}.
template <typename T, int S>
__device__ void fft_pass(const typename CT<T>::V* __restrict__ src, typename CT<T>::V* __restrict__ dst, int N, int R,
                         int Ns, const typename CT<T>::V* __restrict__ tw, int tws, int nfft, int stride) {
    using V = typename CT<T>::V;
    const int nb = N / R;
    const int tstep = N / (Ns * R);
    const int total = nb * nfft;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int f = t / nb;
        const int j = t - f * nb;
        const V* x = src + (int64_t)f * stride;
        V* y = dst + (int64_t)f * stride;
        const int k = j % Ns;
        const int idx = (j / Ns) * Ns * R + k;
        V v0 = x[j], v1 = x[j + nb];
        if (R == 2) {
            if (k) {
                V w1 = tw[k * tstep * tws];
                if (S > 0) w1 = cconj(w1);
                v1 = cmul(v1, w1);
            }
            y[idx] = cadd(v0, v1);
            y[idx + Ns] = csub(v0, v1);
        } else if (R == 3) {
            V v2 = x[j + 2 * nb];
            if (k) {
                V w1 = tw[k * tstep * tws], w2 = tw[((2 * k * tstep) % N) * tws];
                if (S > 0) {
                    w1 = cconj(w1);
                    w2 = cconj(w2);
                }
                v1 = cmul(v1, w1);
                v2 = cmul(v2, w2);
            }
            const T h = (T)0.86602540378443864676;   // sqrt(3)/2
            V t1 = cadd(v1, v2), t2 = csub(v1, v2);
            V a = V{v0.x - (T)0.5 * t1.x, v0.y - (T)0.5 * t1.y};
            V b = cmul_si<S>(V{h * t2.x, h * t2.y});
            y[idx] = cadd(v0, t1);
            y[idx + Ns] = cadd(a, b);
            y[idx + 2 * Ns] = csub(a, b);
        } else {   // R == 4
            V v2 = x[j + 2 * nb], v3 = x[j + 3 * nb];
            if (k) {
                V w1 = tw[k * tstep * tws], w2 = tw[((2 * k * tstep) % N) * tws], w3 = tw[((3 * k * tstep) % N) * tws];
                if (S > 0) {
                    w1 = cconj(w1);
                    w2 = cconj(w2);
                    w3 = cconj(w3);
                }
                v1 = cmul(v1, w1);
                v2 = cmul(v2, w2);
                v3 = cmul(v3, w3);
            }
            V a0 = cadd(v0, v2), a1 = csub(v0, v2), b0 = cadd(v1, v3), b1 = cmul_si<S>(csub(v1, v3));
            y[idx] = cadd(a0, b0);
            y[idx + Ns] = cadd(a1, b1);
            y[idx + 2 * Ns] = csub(a0, b0);
            y[idx + 3 * Ns] = csub(a1, b1);
        }
    }
}

// Full FFT of nfft sequences; data starts in `a`, `b` is scratch; returns the buffer holding the result.
template <typename T, int S>
__device__ typename CT<T>::V* fft_block(typename CT<T>::V* a, typename CT<T>::V* b, const FFTPlan& fp,
                                        const typename CT<T>::V* tw, int nfft, int stride) {
    using V = typename CT<T>::V;
    V* src = a;
    V* dst = b;
    int Ns = 1;
    for (int p = 0; p < fp.nrad; ++p) {
        const int R = fp.rad[p];
        fft_pass<T, S>(src, dst, fp.n, R, Ns, tw, fp.tws, nfft, stride);
        __syncthreads();
        V* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// c2r preparation, in place on one sequence z[0..H): on entry z holds the half
// spectrum X_k (k <= M, zero above, X_0 real part only); on exit
//   Z_k = (X_k + conj X_{H-k}) + i e^{+2 pi i k/N} (X_k - conj X_{H-k}),  k = 0..H-1,
// whose inverse H-point DFT is z_n = x_{2n} + i x_{2n+1}.  twN[k] = e^{-2 pi i k / N}.
template <typename V>
__device__ __forceinline__ void c2r_prepare(V* z, int H, int k, const V* twN) {
    V a = z[k];
    V b = (k == 0) ? V{0, 0} : z[H - k];
    V e = cconj(twN[k]);                       // e^{+i theta_k}
    V s1 = cadd(a, cconj(b)), d1 = csub(a, cconj(b));
    z[k] = cadd(s1, cmul_si<1>(cmul(e, d1)));
    if (k > 0 && k < H - k) {
        V s2 = cadd(b, cconj(a)), d2 = csub(b, cconj(a));
        V e2 = V{-twN[k].x, -twN[k].y};        // e^{+i theta_{H-k}} = -e^{-i theta_k}
        z[H - k] = cadd(s2, cmul_si<1>(cmul(e2, d2)));
    }
}

// r2c untangling: X_k = (Z_k + conj Z_{H-k})/2 - (i/2) e^{-2 pi i k/N} (Z_k - conj Z_{H-k}), scaled.
template <typename T, typename V>
__device__ __forceinline__ V r2c_mode(const V* Z, int H, int k, const V* twN, T scale) {
    V zk = Z[k % H], zn = cconj(Z[(H - k) % H]);
    V s1 = cadd(zk, zn), d1 = csub(zk, zn);
    V t = cmul_si<-1>(cmul(twN[k], d1));       // -i e^{-i theta_k} (Z_k - conj Z_{H-k})
    return V{(T)0.5 * (s1.x + t.x) * scale, (T)0.5 * (s1.y + t.y) * scale};
}

// Per-ring fused nonlinear kernel (one slice, one latitude per block): Fin [M+1][nlat][4S] (Phi', xi, U, V), Fout [M+1][nlat][5S]
// (A1 = xi U/c2, B1 = xi V/c2, A2 = Phi' U/c2, B2 = Phi' V/c2, KE = (U^2+V^2)/(2 c2)), c2 = 1 - mu^2.
template <typename T>
__global__ void __launch_bounds__(256) k_ring_nl_1(const typename CT<T>::V* __restrict__ Fin,
                                                 typename CT<T>::V* __restrict__ Fout, int M, int nlat, int S,
                                                 FFTPlan fp, const typename CT<T>::V* __restrict__ twg,
                                                 const double* __restrict__ mu, const double* __restrict__ w) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = fp.n;
    V* d = reinterpret_cast<V*>(smem_raw);   // 5 sequences
    V* sc = d + 5 * H;                        // 5 scratch sequences
    V* tw = sc + 5 * H;                       // twiddle table staged in shared memory
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) tw[k] = twg[k];
    const int s = blockIdx.x;
    const int j = blockIdx.y;
    for (int k = threadIdx.x; k < 4 * H; k += blockDim.x) d[k] = V{0, 0};
    __syncthreads();
    const int64_t C4 = 4 * (int64_t)S;
    for (int t = threadIdx.x; t < 4 * (M + 1); t += blockDim.x) {
        int f = t / (M + 1), m = t - f * (M + 1);
        V x = Fin[((int64_t)m * nlat + j) * C4 + (int64_t)f * S + s];
        if (m == 0) x.y = 0;
        d[f * H + m] = x;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * (H / 2 + 1); t += blockDim.x) {
        int f = t / (H / 2 + 1), k = t - f * (H / 2 + 1);
        c2r_prepare(d + f * H, H, k, tw);
    }
    __syncthreads();
    V* r = fft_block<T, +1>(d, sc, fp, tw, 4, H);
    const double muj = mu[j];
    const T ic2 = (T)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    for (int n = threadIdx.x; n < H; n += blockDim.x) {
        // each complex element carries two grid points (2n, 2n+1) of the same field
        V ph = r[n], xi = r[H + n], U = r[2 * H + n], Vv = r[3 * H + n];
        r[n] = V{xi.x * U.x * ic2, xi.y * U.y * ic2};
        r[H + n] = V{xi.x * Vv.x * ic2, xi.y * Vv.y * ic2};
        r[2 * H + n] = V{ph.x * U.x * ic2, ph.y * U.y * ic2};
        r[3 * H + n] = V{ph.x * Vv.x * ic2, ph.y * Vv.y * ic2};
        r[4 * H + n] = V{(T)0.5 * (U.x * U.x + Vv.x * Vv.x) * ic2, (T)0.5 * (U.y * U.y + Vv.y * Vv.y) * ic2};
    }
    __syncthreads();
    V* other = (r == d) ? sc : d;
    V* q = fft_block<T, -1>(r, other, fp, tw, 5, H);
    const T scale = (T)(w[j] / (double)(2 * H));
    const int64_t C5 = 5 * (int64_t)S;
    for (int t = threadIdx.x; t < 5 * (M + 1); t += blockDim.x) {
        int f = t / (M + 1), m = t - f * (M + 1);
        Fout[((int64_t)m * nlat + j) * C5 + (int64_t)f * S + s] = r2c_mode<T>(q + f * H, H, m, tw, scale);
    }
}

// In-place Stockham pass: every thread first loads the inputs of all its butterflies
// (at most W of them) into registers, the block synchronises, and the outputs are
// written back into the same buffer.  Needs nfft * N / R <= W * blockDim.x.
template <typename T, int S, int R, int W>
__device__ __forceinline__ void fft_pass_inplace(typename CT<T>::V* __restrict__ x, int N, int Ns,
                                                 const typename CT<T>::V* __restrict__ tw, int tws, int nfft) {
    using V = typename CT<T>::V;
    const int nb = N / R;
    const int tstep = N / (Ns * R);
    const int total = nb * nfft;
    V v[W][R];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int t = threadIdx.x + w * blockDim.x;
        if (t < total) {
            const int f = t / nb, j = t - f * nb;
            const V* xs = x + (int64_t)f * N;
#pragma unroll
            for (int r = 0; r < R; ++r) v[w][r] = xs[j + r * nb];
        }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int t = threadIdx.x + w * blockDim.x;
        if (t < total) {
            const int f = t / nb, j = t - f * nb;
            const int k = j % Ns;
            const int idx = (j / Ns) * Ns * R + k;
            V* y = x + (int64_t)f * N;
            if (k) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    V wr = tw[((r * k * tstep) % N) * tws];
                    if (S > 0) wr = cconj(wr);
                    v[w][r] = cmul(v[w][r], wr);
                }
            }
            if (R == 2) {
                y[idx] = cadd(v[w][0], v[w][1]);
                y[idx + Ns] = csub(v[w][0], v[w][1]);
            } else if (R == 3) {
                const T h = (T)0.86602540378443864676;
                V t1 = cadd(v[w][1], v[w][2]), t2 = csub(v[w][1], v[w][2]);
                V a = V{v[w][0].x - (T)0.5 * t1.x, v[w][0].y - (T)0.5 * t1.y};
                V b = cmul_si<S>(V{h * t2.x, h * t2.y});
                y[idx] = cadd(v[w][0], t1);
                y[idx + Ns] = cadd(a, b);
                y[idx + 2 * Ns] = csub(a, b);
            } else {
                V a0 = cadd(v[w][0], v[w][2]), a1 = csub(v[w][0], v[w][2]);
                V b0 = cadd(v[w][1], v[w][3]), b1 = cmul_si<S>(csub(v[w][1], v[w][3]));
                y[idx] = cadd(a0, b0);
                y[idx + Ns] = cadd(a1, b1);
                y[idx + 2 * Ns] = csub(a0, b0);
                y[idx + 3 * Ns] = csub(a1, b1);
            }
        }
    }
    __syncthreads();
}

// W = butterflies per thread for radix 4 (radix 3: 3W/2, radix 2: 2W)
template <typename T, int S, int W>
__device__ __forceinline__ void fft_inplace(typename CT<T>::V* x, const FFTPlan& fp, const typename CT<T>::V* tw,
                                            int nfft) {
    int Ns = 1;
    for (int p = 0; p < fp.nrad; ++p) {
        const int R = fp.rad[p];
        if (R == 4) fft_pass_inplace<T, S, 4, W>(x, fp.n, Ns, tw, fp.tws, nfft);
        else if (R == 3) fft_pass_inplace<T, S, 3, (3 * W + 1) / 2>(x, fp.n, Ns, tw, fp.tws, nfft);
        else fft_pass_inplace<T, S, 2, 2 * W>(x, fp.n, Ns, tw, fp.tws, nfft);
        Ns *= R;
    }
}

// Grouped fused nonlinear ring: one latitude j, G consecutive slices per block (every
// (field, m) access touches G contiguous columns).  Shared memory: G x 5 sequences of H.
// NT threads, W radix-4 butterflies per thread and pass: requires 5 G H / 4 <= W NT.
template <typename T, int NT, int W, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_ring_nl_g(const typename CT<T>::V* __restrict__ Fin,
                                                   typename CT<T>::V* __restrict__ Fout, int M, int nlat, int S, int G,
                                                   FFTPlan fp, const typename CT<T>::V* __restrict__ twg,
                                                   const double* __restrict__ mu, const double* __restrict__ w) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = fp.n;
    V* d = reinterpret_cast<V*>(smem_raw);      // [g][5][H]
    V* tw = d + (size_t)G * 5 * H;              // twiddle table staged in shared memory
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) tw[k] = twg[k];
    const int s0 = blockIdx.x * G;
    const int Gv = min(G, S - s0);
    const int j = blockIdx.y;
    for (int k = threadIdx.x; k < G * 5 * H; k += blockDim.x) d[k] = V{0, 0};
    __syncthreads();
    const int64_t C4 = 4 * (int64_t)S;
    for (int t = threadIdx.x; t < 4 * (M + 1) * G; t += blockDim.x) {
        const int g = t % G;
        const int fm = t / G;
        const int f = fm / (M + 1), m = fm - f * (M + 1);
        if (g < Gv) {
            V x = Fin[((int64_t)m * nlat + j) * C4 + (int64_t)f * S + s0 + g];
            if (m == 0) x.y = 0;
            d[(g * 5 + f) * H + m] = x;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * G * (H / 2 + 1); t += blockDim.x) {
        const int q = t / (H / 2 + 1), k = t - q * (H / 2 + 1);
        const int g = q / 4, f = q - g * 4;
        c2r_prepare(d + (g * 5 + f) * H, H, k, tw);
    }
    __syncthreads();
    // inverse FFTs of the 4 input sequences of every slice: run over all 5G sequences
    // (the fifth of each slice is zero and unused)
    fft_inplace<T, +1, W>(d, fp, tw, 5 * G);
    const double muj = mu[j];
    const T ic2 = (T)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    for (int t = threadIdx.x; t < G * H; t += blockDim.x) {
        const int g = t / H, n = t - g * H;
        V* b = d + (g * 5) * H;
        V ph = b[n], xi = b[H + n], U = b[2 * H + n], Vv = b[3 * H + n];
        b[n] = V{xi.x * U.x * ic2, xi.y * U.y * ic2};
        b[H + n] = V{xi.x * Vv.x * ic2, xi.y * Vv.y * ic2};
        b[2 * H + n] = V{ph.x * U.x * ic2, ph.y * U.y * ic2};
        b[3 * H + n] = V{ph.x * Vv.x * ic2, ph.y * Vv.y * ic2};
        b[4 * H + n] = V{(T)0.5 * (U.x * U.x + Vv.x * Vv.x) * ic2, (T)0.5 * (U.y * U.y + Vv.y * Vv.y) * ic2};
    }
    __syncthreads();
    fft_inplace<T, -1, W>(d, fp, tw, 5 * G);
    const T scale = (T)(w[j] / (double)(2 * H));
    const int64_t C5 = 5 * (int64_t)S;
    for (int t = threadIdx.x; t < 5 * (M + 1) * G; t += blockDim.x) {
        const int g = t % G;
        const int fm = t / G;
        const int f = fm / (M + 1), m = fm - f * (M + 1);
        if (g < Gv)
            Fout[((int64_t)m * nlat + j) * C5 + (int64_t)f * S + s0 + g] = r2c_mode<T>(d + (g * 5 + f) * H, H, m, tw, scale);
    }
}

// ---------------------------------------------------------------------------
// Lane-group FP32 path for H = nlon/2 = 12 T, T in {8, 16, 32}: T lanes of one warp own
// one ring and every lane holds 12 values in registers.  Each H-point transform is a
// Stockham sequence of passes (radix R, span Ns): butterfly j reads x[j + r H/R],
// applies e^{-+2 pi i r (j mod Ns) / (Ns R)} and writes y[(j - j mod Ns) R + j mod Ns + r Ns];
// lane t takes the butterflies j = t + T b.  Between passes the values go through a
// padded per-ring shared-memory buffer (index i + i/16 against bank conflicts), with
// a warp barrier only, since a ring never leaves its warp.
//   inverse radices T = 32: 4 4 2 12 | 16: 4 4 12 | 8: 4 2 12 (every span Ns a power of
//     two); the first pass takes the c2r-prepared spectrum straight from the staged modes,
//     the last (radix 12, span T) keeps its outputs in registers (lane t, register q: grid
//     pair n = t + T q);
//   forward radices T = 32: 2 4 4 12 | 16: 4 4 12 | 8: 2 4 12; its first pass reads the
//     same grid pairs after a compile-time register permutation, and its last (radix 12,
//     span T) leaves X_{t + T r} in register r, whose r2c partner X_{H-k} is register
//     11 - r of lane T - t (one shuffle per r).
// The grid products of the nonlinear terms are taken in registers.  Twiddles of each
// pass live in a shared table ordered by (j mod Ns, r).  Each block holds G = 128 / T
// rings (G consecutive slices of one latitude), so every (mode, field) access of the
// block touches G contiguous columns.
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
template <int S> __device__ __forceinline__ float2 twd(float2 w) { return S > 0 ? f2(w.x, -w.y) : w; }

template <int R, int S> __device__ __forceinline__ void bfly(float2 (&v)[R]) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const float h = 0.86602540378443864676f;
        float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        float2 a = f2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
        float2 b = cmul_si<S>(f2(h * t2.x, h * t2.y));
        v[0] = cadd(v[0], t1);
        v[1] = cadd(a, b);
        v[2] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = cmul_si<S>(csub(v[1], v[3]));
        v[0] = cadd(a0, b0);
        v[1] = cadd(a1, b1);
        v[2] = csub(a0, b0);
        v[3] = csub(a1, b1);
    } else {   // R == 12 = 4 x 3: radix-4 over stride 3, twiddles e^{-+2 pi i q p / 12}, radix-3 over stride 1
        const float c = 0.86602540378443864676f;
        float2 u[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float2 w4[4] = {v[q], v[q + 3], v[q + 6], v[q + 9]};
            bfly<4, S>(w4);
#pragma unroll
            for (int p = 0; p < 4; ++p) u[4 * q + p] = w4[p];
        }
        // twiddle e^{S 2 pi i q p / 12} for q = 1, 2 and p = 1..3 (angles 30, 60, 90, 120, 180 degrees)
        const float2 w30 = f2(c, S * 0.5f), w60 = f2(0.5f, S * c);
        u[5] = cmul(u[5], w30);
        u[6] = cmul(u[6], w60);
        u[7] = cmul_si<S>(u[7]);
        u[9] = cmul(u[9], w60);
        u[10] = cmul(u[10], f2(-0.5f, S * c));
        u[11] = f2(-u[11].x, -u[11].y);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float2 w3[3] = {u[p], u[4 + p], u[8 + p]};
            bfly<3, S>(w3);
            v[p] = w3[0];
            v[p + 4] = w3[1];
            v[p + 8] = w3[2];
        }
    }
}

constexpr int EL = 12;                 // values per lane
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// One Stockham pass over a ring of H = 12 T values.  Register b R + r holds input
// x[j_b + r H/R] (LOAD: read from buf first) and receives output y[(j_b - k) R + k + r Ns]
// (STORE: written to buf instead).
// Position of element i of a ring buffer.  SW < 0: one padding element per 16 (i + i/16).
// SW >= 0 (T = 32 passes): i stays in its 16-element row (128 bytes, all 32 banks) and its
// position in the row is XORed with a mask of the row index, chosen per pass so that the
// pass's strided stores hit 16 different bank pairs in every half-warp; the next pass reads
// whole rows, which any in-row permutation leaves conflict-free.
template <int SW> __device__ __forceinline__ int bidx(int i) {
    if constexpr (SW < 0) {
        return padi(i);
    } else {
        const int q = i >> 4;
        int x = 0;
        if constexpr (SW == 1) x = q & 1;                  // forward (2, Ns 1)
        else if constexpr (SW == 2) x = q & 3;             // inverse (4, Ns 1)
        else if constexpr (SW == 3) x = (q & 7) << 1;      // forward (4, Ns 2)
        else if constexpr (SW == 4) x = (q & 3) << 2;      // inverse (4, Ns 4)
        else if constexpr (SW == 5) x = ((q >> 1) & 1) << 3;   // forward (4, Ns 8)
        return i ^ x;
    }
}

// Barrier of the T lanes that own one ring (lane group): a warp barrier for T <= 32; for T = 64
// (two warps per group, groups of 64 consecutive threads, at most 7 per block) the named
// barrier 1 + group index over 64 threads (the index is warp-uniform; the ids are immediates).
template <int T> __device__ __forceinline__ void ring_sync() {
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        switch (threadIdx.x >> 6) {
            case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
            case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
            case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
            case 3: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
            case 4: asm volatile("bar.sync 5, 64;" ::: "memory"); break;
            case 5: asm volatile("bar.sync 6, 64;" ::: "memory"); break;
            default: asm volatile("bar.sync 7, 64;" ::: "memory"); break;
        }
    }
}

// Period of a layout: bidx<SW>(i + P) = bidx<SW>(i) + P (+ P / 16 for the padded layout).
template <int SW> __host__ __device__ constexpr int bperiod() {
    return SW < 0 ? 16 : (SW == 1 ? 32 : (SW == 3 ? 128 : 64));
}
// Position of element L + C, with L the lane's part and C >= 0 a constant of the unrolled
// loop: only bidx<SW>(L + C mod P) depends on the lane, and accesses whose C agree mod P
// share it; the rest is an immediate offset of the shared-memory access.
template <int SW> __device__ __forceinline__ int bidx_at(int L, int C) {
    constexpr int P = bperiod<SW>();
    const int c = C % P, hi = C - c;
    return bidx<SW>(L + c) + (SW < 0 ? hi + hi / 16 : hi);
}

// SWL: layout the previous pass stored with; SWS: layout this pass stores with
template <int T, int R, int Ns, int S, bool LOAD, bool STORE, int SWL = -1, int SWS = -1>
__device__ __forceinline__ void spass(float2 (&a)[EL], float2* buf, const float2* twp, int t) {
    constexpr int H = EL * T, NB = EL / R;
    if constexpr (LOAD) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) a[b * R + r] = buf[bidx_at<SWL>(t, T * b + r * (H / R))];
        if constexpr (STORE) ring_sync<T>();
    }
    // when Ns divides T (every lane-group pass), k = j mod Ns = t mod Ns for all of the lane's
    // butterflies: its R - 1 twiddles are loaded once
    constexpr bool kLane = (Ns > 1) && (T % Ns == 0);
    float2 twl[R > 1 ? R - 1 : 1];
    const int kl = t & (Ns - 1);                 // j mod Ns of every butterfly when kLane
    if constexpr (kLane) {
#pragma unroll
        for (int r = 1; r < R; ++r) twl[r - 1] = twd<S>(twp[kl * (R - 1) + r - 1]);
    }
    // store position (j - k) R + k + r Ns of butterfly j = t + T b: lane part (t - k) R + k,
    // constant part T b R + r Ns (when k = j mod Ns is the lane's own kl)
    const int Ls = (t - kl) * R + kl;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + T * b;
        const int k = (Ns == 1) ? 0 : (kLane ? kl : j % Ns);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = a[b * R + r];
        if constexpr (kLane) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twl[r - 1]);
        } else if constexpr (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twd<S>(twp[k * (R - 1) + r - 1]));
        }
        bfly<R, S>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (STORE) {
                if constexpr (Ns == 1 || kLane) buf[bidx_at<SWS>(Ls, T * b * R + r * Ns)] = v[r];
                else buf[bidx<SWS>((j - k) * R + k + r * Ns)] = v[r];
            } else {
                a[b * R + r] = v[r];
            }
        }
    }
}

// twiddle-table layout per T: offsets of the passes' tables (entries (Ns)(R-1)).  The inverse
// runs the radices 4 4 2 12 (T = 32), 4 4 12 (16), 4 2 12 (8), so that every span Ns is a
// power of two (j mod Ns is a mask); the radix-12 pass, last in the inverse and in the forward,
// shares one table (the inverse takes the conjugates).
template <int T> struct RingTw;
template <> struct RingTw<32> { static constexpr int i1 = 0, i2 = 12, i3 = 28, f1 = 380, f2 = 386, f3 = 28, n = 410; };
template <> struct RingTw<16> { static constexpr int i1 = 0, i2 = 12, f1 = 0, f2 = 12, n = 188; };
template <> struct RingTw<8> { static constexpr int i1 = 0, i2 = 4, f1 = 92, f2 = 4, n = 98; };
template <> struct RingTw<64> { static constexpr int i1 = 0, i2 = 12, i3 = 60, f1 = 0, f2 = 12, f3 = 60, n = 764; };

// entries e^{-2 pi i r k / (Ns R)}, k < Ns, r = 1..R-1, from the 2H-point table twg
__device__ __forceinline__ void fill_tw(float2* dst, int R, int Ns, int H, const float2* twg) {
    const int n = Ns * (R - 1);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int k = e / (R - 1), r = e - k * (R - 1) + 1;
        dst[e] = twg[2 * ((r * k * (H / (Ns * R))) % H)];
    }
}
template <int T> __device__ __forceinline__ void fill_ring_tw(float2* tws, const float2* twg) {
    constexpr int H = EL * T;
    using L = RingTw<T>;
    if constexpr (T == 32) {
        fill_tw(tws + L::i1, 4, 4, H, twg);
        fill_tw(tws + L::i2, 2, 16, H, twg);
        fill_tw(tws + L::i3, 12, 32, H, twg);     // also f3
        fill_tw(tws + L::f1, 4, 2, H, twg);
        fill_tw(tws + L::f2, 4, 8, H, twg);
    } else if constexpr (T == 64) {
        fill_tw(tws + L::i1, 4, 4, H, twg);       // also f1
        fill_tw(tws + L::i2, 4, 16, H, twg);      // also f2
        fill_tw(tws + L::i3, 12, 64, H, twg);     // also f3
    } else if constexpr (T == 16) {
        fill_tw(tws + L::i1, 4, 4, H, twg);       // also f1
        fill_tw(tws + L::i2, 12, 16, H, twg);     // also f2
    } else {
        fill_tw(tws + L::i1, 2, 4, H, twg);
        fill_tw(tws + L::i2, 12, 8, H, twg);      // also f2
        fill_tw(tws + L::f1, 4, 2, H, twg);
    }
}

// Register order of the grid pairs a lane holds: the inverse leaves grid pair n = t + T q in
// register q; the forward's first pass (radix 2 for T = 32 and 8, radix 4 for T = 16, span 1)
// wants register b R + r to hold x[t + T b + r H / R], i.e. inverse register b + (12 / R) r.
template <int T> __device__ __forceinline__ void grid_to_forward_order(float2 (&a)[EL]) {
    constexpr int R = (T == 16 || T == 64) ? 4 : 2;
    float2 w[EL];
#pragma unroll
    for (int q = 0; q < EL; ++q) w[q] = a[q];
#pragma unroll
    for (int b = 0; b < EL / R; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) a[b * R + r] = w[b + (EL / R) * r];
}

// Twiddle e^{-2 pi i k / (2H)} of mode k = t + T c, H = 12 T: e^{-i pi t / H} (the lane's own
// entry of the table) times e^{-i pi c / 12} (cos and sin of multiples of 15 degrees, exact
// values of the unit circle rounded to FP32): one shared-memory load per transform instead
// of one per mode.
__device__ __forceinline__ float2 tw_mode(float2 wt, int c) {
    // cos(15 c degrees), c = 0..11; sin(15 c degrees) = cos(15 |6 - c| degrees)
    constexpr float C15[12] = {1.0f, 0.96592582628906829f, 0.86602540378443865f, 0.70710678118654752f, 0.5f,
                               0.25881904510252076f, 0.0f, -0.25881904510252076f, -0.5f, -0.70710678118654752f,
                               -0.86602540378443865f, -0.96592582628906829f};
    if (c == 0) return wt;
    if (c == 6) return f2(wt.y, -wt.x);                  // times -i
    const float cr = C15[c], si = -C15[c < 6 ? 6 - c : c - 6];   // e^{-i pi c / 12} = cos - i sin
    return f2(wt.x * cr - wt.y * si, wt.x * si + wt.y * cr);
}

// MP: M + 1 fixed at compile time (0: the runtime M).  With MP a multiple of T, whether mode
// k = t + T c exists is decided per c at compile time, for every lane at once.
template <int T, int MP>
__device__ __forceinline__ bool mode_in(int k, int c, int M) {
    if constexpr (MP > 0) {
        if (T * (c + 1) <= MP) return true;
        if (T * c >= MP) return false;
    }
    return k <= M;
}
// whether H - k <= M for k = t + T c, k > 0 (the conjugate partner of mode k exists)
template <int T, int MP>
__device__ __forceinline__ bool partner_in(int k, int c, int M) {
    constexpr int H = EL * T;
    if constexpr (MP > 0) {
        if (T * c >= H - MP + 1) return true;           // every k of this c
        if (T * c + T - 1 < H - MP + 1) return false;   // none
    }
    return k > 0 && H - k <= M;
}

// inverse transform of one field: modes X[0..M] (staged) -> grid pairs in registers
template <int T, int MP = 0>
__device__ __forceinline__ void ring_inverse_regs(const float2* X, int M, const float2* twN, const float2* tws,
                                                  float2* buf, int t, float2 (&a)[EL]) {
    constexpr int H = EL * T;
    using L = RingTw<T>;
    // c2r-prepared spectrum Z_k in the first pass's order: register b 4 + r holds
    // x[t + T b + r H/4], i.e. k = t + T (b + 3 r)
    const float2 wt = twN[t];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int c = b + 3 * r;
            const int k = t + T * c;
            float2 xa = mode_in<T, MP>(k, c, M) ? X[k] : f2(0.f, 0.f);
            if (c == 0 && t == 0) xa.y = 0.f;               // the m = 0 mode is real
            const float2 xb = partner_in<T, MP>(k, c, M) ? X[H - k] : f2(0.f, 0.f);
            const float2 wk = tw_mode(wt, c);
            const float2 e = f2(wk.x, -wk.y);               // e^{+i theta_k}, theta_k = 2 pi k / (2H)
            const float2 s1 = cadd(xa, cconj(xb)), d1 = csub(xa, cconj(xb));
            a[b * 4 + r] = cadd(s1, cmul_si<1>(cmul(e, d1)));
        }
    ring_sync<T>();                                          // buf free (previous transform done)
    if constexpr (T == 32) {
        spass<T, 4, 1, +1, false, true, -1, 2>(a, buf, nullptr, t);
        ring_sync<T>();
        spass<T, 4, 4, +1, true, true, 2, 4>(a, buf, tws + L::i1, t);
        ring_sync<T>();
        spass<T, 2, 16, +1, true, true, 4, 0>(a, buf, tws + L::i2, t);
        ring_sync<T>();
        spass<T, 12, 32, +1, true, false, 0, -1>(a, buf, tws + L::i3, t);
        return;
    }
    spass<T, 4, 1, +1, false, true>(a, buf, nullptr, t);
    ring_sync<T>();
    if constexpr (T == 64) {
        spass<T, 4, 4, +1, true, true>(a, buf, tws + L::i1, t);
        ring_sync<T>();
        spass<T, 4, 16, +1, true, true>(a, buf, tws + L::i2, t);
        ring_sync<T>();
        spass<T, 12, 64, +1, true, false>(a, buf, tws + L::i3, t);
    } else if constexpr (T == 16) {
        spass<T, 4, 4, +1, true, true>(a, buf, tws + L::i1, t);
        ring_sync<T>();
        spass<T, 12, 16, +1, true, false>(a, buf, tws + L::i2, t);
    } else {
        spass<T, 2, 4, +1, true, true>(a, buf, tws + L::i1, t);
        ring_sync<T>();
        spass<T, 12, 8, +1, true, false>(a, buf, tws + L::i2, t);
    }
    // register q now holds grid pair n = t + T q
}

// forward transform of one field from the grid pairs in registers -> modes X[0..M] (scaled)
template <int T, int MP = 0>
__device__ __forceinline__ void ring_forward_regs(float2 (&a)[EL], int M, const float2* twN, const float2* tws,
                                                  float2* buf, int t, float scale, float2* X) {
    using L = RingTw<T>;
    grid_to_forward_order<T>(a);                           // a arrives in grid order (n = t + T q)
    ring_sync<T>();
    if constexpr (T == 32) {
        spass<T, 2, 1, -1, false, true, -1, 1>(a, buf, nullptr, t);
        ring_sync<T>();
        spass<T, 4, 2, -1, true, true, 1, 3>(a, buf, tws + L::f1, t);
        ring_sync<T>();
        spass<T, 4, 8, -1, true, true, 3, 5>(a, buf, tws + L::f2, t);
        ring_sync<T>();
        spass<T, 12, 32, -1, true, false, 5, -1>(a, buf, tws + L::f3, t);
    } else if constexpr (T == 64) {
        spass<T, 4, 1, -1, false, true>(a, buf, nullptr, t);
        ring_sync<T>();
        spass<T, 4, 4, -1, true, true>(a, buf, tws + L::f1, t);
        ring_sync<T>();
        spass<T, 4, 16, -1, true, true>(a, buf, tws + L::f2, t);
        ring_sync<T>();
        spass<T, 12, 64, -1, true, false>(a, buf, tws + L::f3, t);
    } else if constexpr (T == 16) {
        spass<T, 4, 1, -1, false, true>(a, buf, nullptr, t);
        ring_sync<T>();
        spass<T, 4, 4, -1, true, true>(a, buf, tws + L::f1, t);
        ring_sync<T>();
        spass<T, 12, 16, -1, true, false>(a, buf, tws + L::f2, t);
    } else {
        spass<T, 2, 1, -1, false, true>(a, buf, nullptr, t);
        ring_sync<T>();
        spass<T, 4, 2, -1, true, true>(a, buf, tws + L::f1, t);
        ring_sync<T>();
        spass<T, 12, 8, -1, true, false>(a, buf, tws + L::f2, t);
    }
    const int partner = (T - t) & (T - 1);
    const float2 wt = twN[t];
    if constexpr (T > 32) {
        // the partner lane is in the other warp of the ring: exchange through the ring buffer
        // (after the last pass's loads from it)
        ring_sync<T>();
#pragma unroll
        for (int r = 0; r < EL; ++r) buf[padi(t + T * r)] = a[r];
        ring_sync<T>();
    }
#pragma unroll
    for (int r = 0; r < EL; ++r) {
        if constexpr (MP > 0) {
            if (T * r >= MP) continue;                      // no lane keeps a mode of this r
        }
        // Z_{H-k}: lane T - t, register 11 - r (t >= 1); lane 0: its own register (12 - r) mod 12
        float2 zp;
        if constexpr (T > 32) {
            zp = buf[padi(t == 0 ? T * ((EL - r) % EL) : partner + T * (EL - 1 - r))];
        } else {
            zp.x = __shfl_sync(0xffffffffu, a[EL - 1 - r].x, partner, T);
            zp.y = __shfl_sync(0xffffffffu, a[EL - 1 - r].y, partner, T);
            if (t == 0) zp = a[(EL - r) % EL];
        }
        const int k = t + T * r;
        if (mode_in<T, MP>(k, r, M)) {
            const float2 zk = a[r], zn = cconj(zp);
            const float2 s1 = cadd(zk, zn), d1 = csub(zk, zn);
            const float2 tt = cmul_si<-1>(cmul(tw_mode(wt, r), d1));
            X[k] = f2(0.5f * (s1.x + tt.x) * scale, 0.5f * (s1.y + tt.y) * scale);
        }
    }
}

// stride of the per-ring staging regions: n float2 rounded up to 1 mod 16, so that the rings
// of a block (up to 16) fall on different shared-memory banks at the same offset
__host__ __device__ constexpr int ring_stride(int n) { return n + (17 - n % 16) % 16; }
// T = 32 (one ring per warp, 4 rings per block): the transforms never mix rings within a
// warp, but the staging and output loops do (lane q: ring q mod 4, mode q / 4); a stride of
// 4 mod 16 puts the 16 (ring, mode) pairs of a half-warp on 16 different bank pairs
template <int T> __host__ __device__ constexpr int ring_stride_t(int n) {
    return T == 32 ? n + (20 - n % 16) % 16 : ring_stride(n);
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(pred ? 8 : 0)
                 : "memory");
}

template <int T, int MP>
__global__ void __launch_bounds__(128, 3) k_ring_nl_lg(const float2* __restrict__ Fin, float2* __restrict__ Fout, int M,
                                                    int nlat, int S, const float2* __restrict__ twg,
                                                    const double* __restrict__ mu, const double* __restrict__ w) {
    constexpr int H = EL * T, G = 128 / T, HB = H + H / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* twN = reinterpret_cast<float2*>(smem_raw);     // 2H entries e^{-2 pi i k / (2H)}
    float2* tws = twN + 2 * H;                              // pass tables
    float2* fbuf = tws + RingTw<T>::n;                      // [G][HB]
    float2* reg = fbuf + G * HB;                            // [G][5][M+1], ring stride RS
    if constexpr (MP > 0) M = MP - 1;
    const int Mp = M + 1, RS = ring_stride_t<T>(5 * Mp);
    const int s0 = blockIdx.x * G;
    const int j = blockIdx.y;
    const int64_t C4 = 4 * (int64_t)S, C5 = 5 * (int64_t)S;
    // stage the 4 input fields of the G rings: every copy in flight at once (fields outermost,
    // so that the mode index needs no division by M+1)
#pragma unroll
    for (int f = 0; f < 4; ++f)
        for (int q = threadIdx.x; q < Mp * G; q += blockDim.x) {
            const int g = q % G, m = q / G;
            const bool ok = s0 + g < S;
            cp_async8(&reg[g * RS + f * Mp + m],
                      ok ? (const void*)&Fin[((int64_t)m * nlat + j) * C4 + (int64_t)f * S + s0 + g] : (const void*)Fin,
                      ok);
        }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) twN[k] = twg[k];
    fill_ring_tw<T>(tws, twg);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int t = threadIdx.x & (T - 1), g = threadIdx.x / T;
    float2* R = reg + g * RS;
    float2* buf = fbuf + g * HB;
    const double muj = mu[j];
    const float ic2 = (float)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    const float scale = (float)(w[j] / (double)(2 * H));
    // Inputs (slots): 0 Phi', 1 xi, 2 U, 3 V, 4 free.  Inverse order U, V, xi, Phi'.  With p
    // = xi (then Phi') in registers: p V / c2 is parked lane-privately in slots 2-3 (free once
    // U and V are in registers), p U / c2 is transformed, then the parked product:
    //   xi:   A1 = xi U -> slot 1, B1 = xi V -> slot 4
    //   Phi': A2 = Phi' U -> slot 0, B2 = Phi' V -> slot 3, KE = (U^2 + V^2)/2 -> slot 2
    // Rolled loops keep one copy of each transform in the instruction stream.
    float2 u[EL], v[EL], a[EL];
    float2* park = R + 2 * Mp;                               // 2 (M+1) >= H entries
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const int in_slot = i == 0 ? 2 : (i == 1 ? 3 : (i == 2 ? 1 : 0));
        ring_inverse_regs<T, MP>(R + in_slot * Mp, M, twN, tws, buf, t, a);
        if (i < 2) {
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                if (i == 0) u[e] = a[e];
                else v[e] = a[e];
            }
            continue;
        }
        ring_sync<T>();                                      // slots 2-3 no longer read
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            park[e * T + t] = f2(a[e].x * v[e].x * ic2, a[e].y * v[e].y * ic2);
            a[e] = f2(a[e].x * u[e].x * ic2, a[e].y * u[e].y * ic2);
        }
        const int nout = (i == 3) ? 3 : 2;
#pragma unroll 1
        for (int o = 0; o < nout; ++o) {
            if (o == 1) {
#pragma unroll
                for (int e = 0; e < EL; ++e) a[e] = park[e * T + t];
            } else if (o == 2) {
#pragma unroll
                for (int e = 0; e < EL; ++e)
                    a[e] = f2(0.5f * (u[e].x * u[e].x + v[e].x * v[e].x) * ic2,
                              0.5f * (u[e].y * u[e].y + v[e].y * v[e].y) * ic2);
            }
            const int out_slot = (i == 2) ? (o == 0 ? 1 : 4) : (o == 0 ? 0 : (o == 1 ? 3 : 2));
            ring_forward_regs<T, MP>(a, M, twN, tws, buf, t, scale, R + out_slot * Mp);
        }
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const int slot = f == 0 ? 1 : (f == 1 ? 4 : (f == 2 ? 0 : (f == 3 ? 3 : 2)));
        for (int q = threadIdx.x; q < Mp * G; q += blockDim.x) {
            const int gg = q % G, m = q / G;
            if (s0 + gg < S)
                Fout[((int64_t)m * nlat + j) * C5 + (int64_t)f * S + s0 + gg] = reg[gg * RS + slot * Mp + m];
        }
    }
}

// Latency form of the fused nonlinear ring kernel for few slices (the serial coarse chains run
// one state): one ring (slice, latitude) per block and five lane groups of T lanes, T in
// {32, 64}.  Groups 0-3 take the four inverse transforms (Phi', xi, U, V) at once and leave
// the grid pairs in shared memory; after one block barrier group f forms product f (xi U,
// xi V, Phi' U, Phi' V, KE, each over cos^2) from them and runs its forward transform.  The
// dependent chain is one inverse and one forward transform instead of nine.
constexpr int NLW_GROUPS = 5;

template <int T, int MP>
__global__ void __launch_bounds__(NLW_GROUPS * T) k_ring_nl_w(const float2* __restrict__ Fin, float2* __restrict__ Fout,
                                                             int M, int nlat, int S, const float2* __restrict__ twg,
                                                             const double* __restrict__ mu,
                                                             const double* __restrict__ w) {
    constexpr int H = EL * T, HB = H + H / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* twN = reinterpret_cast<float2*>(smem_raw);     // 2H entries e^{-2 pi i k / (2H)}
    float2* tws = twN + 2 * H;                              // pass tables
    float2* fbuf = tws + RingTw<T>::n;                      // [5][HB] exchange buffers
    float2* gp = fbuf + NLW_GROUPS * HB;                    // [4][H] grid pairs: Phi', xi, U, V
    float2* spin = gp + 4 * H;                              // [4][M+1] input modes
    if constexpr (MP > 0) M = MP - 1;
    const int Mp = M + 1;
    float2* spout = spin + 4 * Mp;                          // [5][M+1] output modes
    const int s = blockIdx.x, j = blockIdx.y;
    const int64_t C4 = 4 * (int64_t)S, C5 = 5 * (int64_t)S;
    for (int q = threadIdx.x; q < 4 * Mp; q += blockDim.x) {
        const int f = q / Mp, m = q - f * Mp;
        cp_async8(&spin[q], &Fin[((int64_t)m * nlat + j) * C4 + (int64_t)f * S + s], true);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) twN[k] = twg[k];
    fill_ring_tw<T>(tws, twg);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int t = threadIdx.x & (T - 1), g = threadIdx.x / T;
    float2* buf = fbuf + g * HB;
    float2 a[EL];
    if (g < 4) {
        // input slots: 0 Phi', 1 xi, 2 U, 3 V (grid pair n = t + T q in register q)
        ring_inverse_regs<T, MP>(spin + g * Mp, M, twN, tws, buf, t, a);
#pragma unroll
        for (int q = 0; q < EL; ++q) gp[g * H + t + T * q] = a[q];
    }
    __syncthreads();
    const double muj = mu[j];
    const float ic2 = (float)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    const float scale = (float)(w[j] / (double)(2 * H));
    // product g: 0 xi U, 1 xi V, 2 Phi' U, 3 Phi' V, 4 KE = (U^2 + V^2) / 2, each / cos^2
#pragma unroll
    for (int q = 0; q < EL; ++q) {
        const int n = t + T * q;
        const float2 u = gp[2 * H + n], v = gp[3 * H + n];
        if (g == 4) {
            a[q] = f2(0.5f * (u.x * u.x + v.x * v.x) * ic2, 0.5f * (u.y * u.y + v.y * v.y) * ic2);
        } else {
            const float2 p = gp[(g < 2 ? 1 : 0) * H + n];
            const float2 o = (g & 1) ? v : u;
            a[q] = f2(p.x * o.x * ic2, p.y * o.y * ic2);
        }
    }
    ring_forward_regs<T, MP>(a, M, twN, tws, buf, t, scale, spout + g * Mp);
    __syncthreads();
    for (int q = threadIdx.x; q < 5 * Mp; q += blockDim.x) {
        const int f = q / Mp, m = q - f * Mp;
        Fout[((int64_t)m * nlat + j) * C5 + (int64_t)f * S + s] = spout[q];
    }
}

// Plain transforms on the lane-group path (FP32, H = 12 T): one ring per T lanes, G = 128/T
// consecutive columns of one latitude per block.
//   inverse: Fourier [M+1][nlat][C] -> grid [C][nlat][nlon]; modes staged with cp.async,
//            grid pairs stored straight from registers (lane t holds n = t + T i: coalesced)
//   forward: grid -> Fourier; grid pairs loaded straight into the forward's register layout,
//            modes staged in shared memory for a coalesced write (G columns per mode)
template <int T, int MP>
__global__ void __launch_bounds__(128) k_ring_inv_lg(const float2* __restrict__ F, float* __restrict__ grid, int M,
                                                     int nlat, int C, const float2* __restrict__ twg) {
    constexpr int H = EL * T, G = 128 / T, HB = H + H / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* twN = reinterpret_cast<float2*>(smem_raw);
    float2* tws = twN + 2 * H;
    float2* fbuf = tws + RingTw<T>::n;                      // [G][HB]
    float2* reg = fbuf + G * HB;                            // [G][M+1], ring stride RS
    if constexpr (MP > 0) M = MP - 1;
    const int Mp = M + 1, RS = ring_stride_t<T>(Mp);
    const int c0 = blockIdx.x * G;
    const int j = blockIdx.y;
    for (int q = threadIdx.x; q < Mp * G; q += blockDim.x) {
        const int g = q % G, m = q / G;
        const bool ok = c0 + g < C;
        cp_async8(&reg[g * RS + m], ok ? (const void*)&F[((int64_t)m * nlat + j) * C + c0 + g] : (const void*)F, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) twN[k] = twg[k];
    fill_ring_tw<T>(tws, twg);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int t = threadIdx.x & (T - 1), g = threadIdx.x / T;
    float2 a[EL];
    ring_inverse_regs<T, MP>(reg + g * RS, M, twN, tws, fbuf + g * HB, t, a);
    if (c0 + g < C) {
        float2* row = reinterpret_cast<float2*>(grid + ((int64_t)(c0 + g) * nlat + j) * (2 * H));
#pragma unroll
        for (int q = 0; q < EL; ++q) row[t + T * q] = a[q];  // register q: grid pair t + T q
    }
}

template <int T, int MP>
__global__ void __launch_bounds__(128) k_ring_fwd_lg(const float* __restrict__ grid, float2* __restrict__ F, int M,
                                                     int nlat, int C, const float2* __restrict__ twg,
                                                     const double* __restrict__ w) {
    constexpr int H = EL * T, G = 128 / T, HB = H + H / 16 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* twN = reinterpret_cast<float2*>(smem_raw);
    float2* tws = twN + 2 * H;
    float2* fbuf = tws + RingTw<T>::n;
    float2* reg = fbuf + G * HB;                            // [G][M+1], ring stride RS
    if constexpr (MP > 0) M = MP - 1;
    const int Mp = M + 1, RS = ring_stride_t<T>(Mp);
    const int c0 = blockIdx.x * G;
    const int j = blockIdx.y;
    const int t = threadIdx.x & (T - 1), g = threadIdx.x / T;
    float2 a[EL];
    {
        const bool ok = c0 + g < C;
        const float2* row = reinterpret_cast<const float2*>(grid + ((int64_t)(ok ? c0 + g : 0) * nlat + j) * (2 * H));
#pragma unroll
        for (int q = 0; q < EL; ++q) a[q] = ok ? row[t + T * q] : f2(0.f, 0.f);   // grid order
    }
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) twN[k] = twg[k];
    fill_ring_tw<T>(tws, twg);
    __syncthreads();
    const float scale = (float)(w[j] / (double)(2 * H));
    ring_forward_regs<T, MP>(a, M, twN, tws, fbuf + g * HB, t, scale, reg + g * RS);
    __syncthreads();
    for (int q = threadIdx.x; q < Mp * G; q += blockDim.x) {
        const int gg = q % G, m = q / G;
        if (c0 + gg < C) F[((int64_t)m * nlat + j) * C + c0 + gg] = reg[gg * RS + m];
    }
}

template <int T, int MP>
static swe_status ring_plain_lg_mp(const swe_plan* p, const void* in, void* out, int C, bool inverse, cudaStream_t st) {
    constexpr int H = EL * T, G = 128 / T, HB = H + H / 16 + 1;
    const size_t sm = (2 * (size_t)H + RingTw<T>::n + (size_t)G * HB + (size_t)G * ring_stride_t<T>(p->M + 1)) * sizeof(float2);
    dim3 g((C + G - 1) / G, p->nlat);
    if (inverse) {
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_ring_inv_lg<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_ring_inv_lg<T, MP><<<g, 128, sm, st>>>((const float2*)in, (float*)out, p->M, p->nlat, C, p->twf);
        SWE_CHECK_LAUNCH("k_ring_inv_lg");
    } else {
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_ring_fwd_lg<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_ring_fwd_lg<T, MP><<<g, 128, sm, st>>>((const float*)in, (float2*)out, p->M, p->nlat, C, p->twf, p->w);
        SWE_CHECK_LAUNCH("k_ring_fwd_lg");
    }
    return SWE_OK;
}

// the 3/2-rule truncation of the grid (M + 1 = 2 H / 3 = 8 T) is compiled with M fixed
template <int T>
static swe_status ring_plain_lg(const swe_plan* p, const void* in, void* out, int C, bool inverse, cudaStream_t st) {
    if (p->M + 1 == 8 * T) return ring_plain_lg_mp<T, 8 * T>(p, in, out, C, inverse, st);
    return ring_plain_lg_mp<T, 0>(p, in, out, C, inverse, st);
}

// the lane-group kernels serve FP32 plans with nlon / 2 = 12 T whose two mode slots cover a ring
static int ring_lg_T(const swe_plan* p) {
    if (p->prec == SWE_FP64) return 0;
    const int H = p->nlon / 2;
    if (2 * (p->M + 1) < H) return 0;
    return H == 96 ? 8 : (H == 192 ? 16 : (H == 384 ? 32 : (H == 768 ? 64 : 0)));
}

constexpr int RING_G = 4;   // columns per block in the plain transforms

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_ring_inv(const typename CT<T>::V* __restrict__ F, T* __restrict__ grid, int M,
                                                  int nlat, int C, FFTPlan fp, const typename CT<T>::V* __restrict__ twg) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = fp.n;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + RING_G * H;
    V* tw = b + RING_G * H;                        // twiddle table staged in shared memory
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) tw[k] = twg[k];
    const int j = blockIdx.y;
    const int c0 = RING_G * blockIdx.x;
    const int G = min(RING_G, C - c0);
    for (int k = threadIdx.x; k < RING_G * H; k += blockDim.x) a[k] = V{0, 0};
    __syncthreads();
    for (int t = threadIdx.x; t < G * (M + 1); t += blockDim.x) {
        int m = t / G, g = t - m * G;                 // columns fastest: contiguous loads
        V x = F[((int64_t)m * nlat + j) * C + c0 + g];
        if (m == 0) x.y = 0;
        a[g * H + m] = x;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < G * (H / 2 + 1); t += blockDim.x) {
        int g = t / (H / 2 + 1), k = t - g * (H / 2 + 1);
        c2r_prepare(a + g * H, H, k, tw);
    }
    __syncthreads();
    V* r = fft_block<T, +1>(a, b, fp, tw, RING_G, H);
    for (int t = threadIdx.x; t < G * H; t += blockDim.x) {
        int g = t / H, n = t - g * H;
        V z = r[g * H + n];
        T* row = grid + ((int64_t)(c0 + g) * nlat + j) * (2 * H);
        row[2 * n] = z.x;
        row[2 * n + 1] = z.y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ring_fwd(const T* __restrict__ grid, typename CT<T>::V* __restrict__ F, int M,
                                                  int nlat, int C, FFTPlan fp, const typename CT<T>::V* __restrict__ twg,
                                                  const double* __restrict__ w) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = fp.n;
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + RING_G * H;
    V* tw = b + RING_G * H;                        // twiddle table staged in shared memory
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) tw[k] = twg[k];
    const int j = blockIdx.y;
    const int c0 = RING_G * blockIdx.x;
    const int G = min(RING_G, C - c0);
    for (int t = threadIdx.x; t < RING_G * H; t += blockDim.x) {
        int g = t / H, n = t - g * H;
        V z = V{0, 0};
        if (g < G) {
            const T* row = grid + ((int64_t)(c0 + g) * nlat + j) * (2 * H);
            z = V{row[2 * n], row[2 * n + 1]};
        }
        a[t] = z;
    }
    __syncthreads();
    V* r = fft_block<T, -1>(a, b, fp, tw, RING_G, H);
    const T scale = (T)(w[j] / (double)(2 * H));
    for (int t = threadIdx.x; t < G * (M + 1); t += blockDim.x) {
        int m = t / G, g = t - m * G;                 // columns fastest: contiguous stores
        F[((int64_t)m * nlat + j) * C + c0 + g] = r2c_mode<T>(r + g * H, H, m, tw, scale);
    }
}

FFTPlan make_fft_plan(const swe_plan* p) {
    FFTPlan fp;
    fp.n = p->nlon / 2;
    fp.tws = 2;
    fp.nrad = p->nrad;
    for (int i = 0; i < p->nrad; ++i) fp.rad[i] = p->rad[i];
    return fp;
}

template <typename K>
swe_status set_smem(K kernel, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return swe_cuda_status(e, "cudaFuncSetAttribute(smem)");
    return SWE_OK;
}

}  // namespace

swe_status ring_inverse(const swe_plan* p, const void* F, void* grid, int C, cudaStream_t st) {
    if (const int lgT = ring_lg_T(p)) {
        ProfToken tk = prof_begin("ring_inv", st, 0.0, 4.0 * (double)C * p->nlat * (2.0 * (p->M + 1) + p->nlon));
        const swe_status r = lgT == 8    ? ring_plain_lg<8>(p, F, grid, C, true, st)
                             : lgT == 16 ? ring_plain_lg<16>(p, F, grid, C, true, st)
                             : lgT == 32 ? ring_plain_lg<32>(p, F, grid, C, true, st)
                                         : ring_plain_lg<64>(p, F, grid, C, true, st);
        prof_end(tk, st);
        return r;
    }
    FFTPlan fp = make_fft_plan(p);
    dim3 g((C + RING_G - 1) / RING_G, p->nlat);
    const double fe_ = p->prec == SWE_FP64 ? 8.0 : 4.0;   // bytes per real element
    ProfToken tk = prof_begin("ring_inv", st, 0.0, fe_ * (double)C * p->nlat * (2.0 * (p->M + 1) + p->nlon));
    if (p->prec == SWE_FP64) {
        size_t sm = (2 * RING_G + 2) * sizeof(double2) * fp.n;
        SWE_CHECK(set_smem(k_ring_inv<double>, sm));
        k_ring_inv<double><<<g, 256, sm, st>>>((const double2*)F, (double*)grid, p->M, p->nlat, C, fp, p->tw);
    } else {
        size_t sm = (2 * RING_G + 2) * sizeof(float2) * fp.n;
        SWE_CHECK(set_smem(k_ring_inv<float>, sm));
        k_ring_inv<float><<<g, 256, sm, st>>>((const float2*)F, (float*)grid, p->M, p->nlat, C, fp, p->twf);
    }
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_ring_inv");
    return SWE_OK;
}

swe_status ring_forward(const swe_plan* p, const void* grid, void* F, int C, cudaStream_t st) {
    if (const int lgT = ring_lg_T(p)) {
        ProfToken tk = prof_begin("ring_fwd", st, 0.0, 4.0 * (double)C * p->nlat * (2.0 * (p->M + 1) + p->nlon));
        const swe_status r = lgT == 8    ? ring_plain_lg<8>(p, grid, F, C, false, st)
                             : lgT == 16 ? ring_plain_lg<16>(p, grid, F, C, false, st)
                             : lgT == 32 ? ring_plain_lg<32>(p, grid, F, C, false, st)
                                         : ring_plain_lg<64>(p, grid, F, C, false, st);
        prof_end(tk, st);
        return r;
    }
    FFTPlan fp = make_fft_plan(p);
    dim3 g((C + RING_G - 1) / RING_G, p->nlat);
    const double fe_ = p->prec == SWE_FP64 ? 8.0 : 4.0;   // bytes per real element
    ProfToken tk = prof_begin("ring_fwd", st, 0.0, fe_ * (double)C * p->nlat * (2.0 * (p->M + 1) + p->nlon));
    if (p->prec == SWE_FP64) {
        size_t sm = (2 * RING_G + 2) * sizeof(double2) * fp.n;
        SWE_CHECK(set_smem(k_ring_fwd<double>, sm));
        k_ring_fwd<double><<<g, 256, sm, st>>>((const double*)grid, (double2*)F, p->M, p->nlat, C, fp, p->tw, p->w);
    } else {
        size_t sm = (2 * RING_G + 2) * sizeof(float2) * fp.n;
        SWE_CHECK(set_smem(k_ring_fwd<float>, sm));
        k_ring_fwd<float><<<g, 256, sm, st>>>((const float*)grid, (float2*)F, p->M, p->nlat, C, fp, p->twf, p->w);
    }
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_ring_fwd");
    return SWE_OK;
}

namespace {

// ----------------------------------------------------------------------------- launch configs
// Candidate (slices per block, threads, butterflies per thread, min blocks per SM) of the
// fused nonlinear ring kernel; the first call of a plan with S >= 8 slices times every
// candidate that fits (5 G H / 4 <= W NT) on its real operands and keeps the fastest.
struct RingCfg {
    int G, NT, W;
};
template <typename T>
struct RingLaunch {
    static void launch(int id, dim3 g, size_t sm, cudaStream_t st, const void* Fin, void* Fout, int M, int nlat, int S,
                       int G, const FFTPlan& fp, const void* tw, const double* mu, const double* w) {
        using V = typename CT<T>::V;
        const V* fi = (const V*)Fin;
        V* fo = (V*)Fout;
        const V* t = (const V*)tw;
        switch (id) {
            case 0: k_ring_nl_g<T, 512, 4, 1><<<g, 512, sm, st>>>(fi, fo, M, nlat, S, G, fp, t, mu, w); break;
            case 1: k_ring_nl_g<T, 512, 2, 2><<<g, 512, sm, st>>>(fi, fo, M, nlat, S, G, fp, t, mu, w); break;
            case 2: k_ring_nl_g<T, 256, 4, 2><<<g, 256, sm, st>>>(fi, fo, M, nlat, S, G, fp, t, mu, w); break;
            case 3: k_ring_nl_g<T, 256, 2, 3><<<g, 256, sm, st>>>(fi, fo, M, nlat, S, G, fp, t, mu, w); break;
            default: k_ring_nl_1<T><<<g, 256, sm, st>>>(fi, fo, M, nlat, S, fp, t, mu, w); break;
        }
    }
    static swe_status set_attr(int id, size_t sm) {
        switch (id) {
            case 0: return set_smem(k_ring_nl_g<T, 512, 4, 1>, sm);
            case 1: return set_smem(k_ring_nl_g<T, 512, 2, 2>, sm);
            case 2: return set_smem(k_ring_nl_g<T, 256, 4, 2>, sm);
            case 3: return set_smem(k_ring_nl_g<T, 256, 2, 3>, sm);
            default: return set_smem(k_ring_nl_1<T>, sm);
        }
    }
};
const int kRingNT[5] = {512, 512, 256, 256, 256};
const int kRingW[5] = {4, 2, 4, 2, 0};
constexpr int kRingCandidates = 5;

// candidate 4 is the per-ring kernel with a scratch buffer (one slice per block)
bool ring_fits(int id, int G, int H) {
    if (id == 4) return G == 1;
    return 5 * G * H <= 4 * kRingW[id] * kRingNT[id];
}

template <typename T>
swe_status ring_run(const swe_plan* p, int id, int G, const void* Fin, void* Fout, int S, cudaStream_t st) {
    FFTPlan fp = make_fft_plan(p);
    dim3 g((S + G - 1) / G, p->nlat);
    size_t sm = (id == 4 ? (size_t)12 : (size_t)G * 5 + 2) * sizeof(typename CT<T>::V) * fp.n;
    SWE_CHECK(RingLaunch<T>::set_attr(id, sm));
    const void* tw = (p->prec == SWE_FP64) ? (const void*)p->tw : (const void*)p->twf;
    RingLaunch<T>::launch(id, g, sm, st, Fin, Fout, p->M, p->nlat, S, G, fp, tw, p->mu, p->w);
    SWE_CHECK_LAUNCH("k_ring_nl_g");
    return SWE_OK;
}

}  // namespace

// lane-group FP32 kernel for H = 12 T, T in {8, 16, 32}
template <int T, int MP>
static swe_status ring_lg_launch_mp(const swe_plan* p, const void* Fin, void* Fout, int S, cudaStream_t st) {
    constexpr int H = EL * T, G = 128 / T, HB = H + H / 16 + 1;
    const size_t sm =
        (2 * (size_t)H + RingTw<T>::n + (size_t)G * HB + (size_t)G * ring_stride_t<T>(5 * (p->M + 1))) * sizeof(float2);
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_ring_nl_lg<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 g((S + G - 1) / G, p->nlat);
    k_ring_nl_lg<T, MP><<<g, 128, sm, st>>>((const float2*)Fin, (float2*)Fout, p->M, p->nlat, S, p->twf, p->mu, p->w);
    SWE_CHECK_LAUNCH("k_ring_nl_lg");
    return SWE_OK;
}

template <int T, int MP>
static swe_status ring_w_launch_mp(const swe_plan* p, const void* Fin, void* Fout, int S, cudaStream_t st) {
    constexpr int H = EL * T, HB = H + H / 16 + 1;
    const size_t sm = (2 * (size_t)H + RingTw<T>::n + (size_t)NLW_GROUPS * HB + 4 * (size_t)H +
                       9 * (size_t)(p->M + 1)) * sizeof(float2);
    SWE_CHECK_CUDA(cudaFuncSetAttribute(k_ring_nl_w<T, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 g(S, p->nlat);
    k_ring_nl_w<T, MP><<<g, NLW_GROUPS * T, sm, st>>>((const float2*)Fin, (float2*)Fout, p->M, p->nlat, S, p->twf,
                                                       p->mu, p->w);
    SWE_CHECK_LAUNCH("k_ring_nl_w");
    return SWE_OK;
}

// batches of at most this many slices take the one-ring-per-block latency form (T >= 32)
constexpr int RING_W_MAX_S = 4;

template <int T>
static swe_status ring_lg_launch(const swe_plan* p, const void* Fin, void* Fout, int S, cudaStream_t st) {
    if constexpr (T >= 32) {
        if (S <= RING_W_MAX_S) {
            if (p->M + 1 == 8 * T) return ring_w_launch_mp<T, 8 * T>(p, Fin, Fout, S, st);
            return ring_w_launch_mp<T, 0>(p, Fin, Fout, S, st);
        }
    }
    if (p->M + 1 == 8 * T) return ring_lg_launch_mp<T, 8 * T>(p, Fin, Fout, S, st);
    return ring_lg_launch_mp<T, 0>(p, Fin, Fout, S, st);
}

swe_status ring_nonlinear(const swe_plan* pc, const void* Fin, void* Fout, int S, cudaStream_t st) {
    swe_plan* p = const_cast<swe_plan*>(pc);
    const bool f64 = (p->prec == SWE_FP64);
    const int H = p->nlon / 2;
    // lane-group kernel (its parking area, two mode slots, must hold a ring of H values)
    if (ring_lg_T(p)) {
        const double by = 8.0 * 9.0 * (p->M + 1.0) * p->nlat * S;
        const double fl = ((9.0 * 2.5 * log2((double)p->nlon)) + 30.0) * p->nlon * (double)p->nlat * S;
        ProfToken tk = prof_begin("ring_nl_f32", st, fl, by);
        swe_status r = H == 96    ? ring_lg_launch<8>(p, Fin, Fout, S, st)
                       : H == 192 ? ring_lg_launch<16>(p, Fin, Fout, S, st)
                       : H == 384 ? ring_lg_launch<32>(p, Fin, Fout, S, st)
                                  : ring_lg_launch<64>(p, Fin, Fout, S, st);
        prof_end(tk, st);
        return r;
    }
    int id = p->ring_cfg, G = p->ring_G;
    if (id < 0 || G > S) {
        // default: the largest group that fits the first candidate with room, else 1 slice
        id = -1;
        G = 1;
        for (int gg = 4; gg >= 1 && id < 0; gg >>= 1)
            for (int c = 0; c < kRingCandidates && id < 0; ++c)
                if (gg <= S && ring_fits(c, gg, H)) {
                    id = c;
                    G = gg;
                }
        if (id < 0) {
            swe_set_error("ring_nonlinear: nlon = %d too large for the ring kernels", p->nlon);
            return SWE_EINVAL;
        }
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (S >= 8 && cs == cudaStreamCaptureStatusNone && p->ring_cfg < 0) {
            // autotune on the real operands (the kernel only reads Fin and writes Fout)
            float best = 1e30f;
            int bid = id, bG = G;
            cudaEvent_t e0, e1;
            SWE_CHECK_CUDA(cudaEventCreate(&e0));
            SWE_CHECK_CUDA(cudaEventCreate(&e1));
            for (int gg = 1; gg <= 4; gg <<= 1)
                for (int c = 0; c < kRingCandidates; ++c) {
                    if (!ring_fits(c, gg, H)) continue;
                    float ms = 0.f;
                    for (int rep = 0; rep < 2; ++rep) {      // first run warms up, second is timed
                        SWE_CHECK_CUDA(cudaEventRecord(e0, st));
                        if (f64) SWE_CHECK(ring_run<double>(p, c, gg, Fin, Fout, S, st));
                        else SWE_CHECK(ring_run<float>(p, c, gg, Fin, Fout, S, st));
                        SWE_CHECK_CUDA(cudaEventRecord(e1, st));
                        SWE_CHECK_CUDA(cudaEventSynchronize(e1));
                        SWE_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    }
                    if (ms < best) {
                        best = ms;
                        bid = c;
                        bG = gg;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            p->ring_cfg = bid;
            p->ring_G = bG;
            id = bid;
            G = bG;
        }
    }
    // algorithmic traffic: read 4 and write 5 Fourier rows of (M+1) modes per ring;
    // 9 real FFTs of length nlon (2.5 N log2 N each) + ~30 flops per grid point
    const double fe = f64 ? 16.0 : 8.0;
    const double by = fe * 9.0 * (p->M + 1.0) * p->nlat * S;
    const double fl = ((9.0 * 2.5 * log2((double)p->nlon)) + 30.0) * p->nlon * (double)p->nlat * S;
    ProfToken tk = prof_begin(f64 ? "ring_nl_f64" : "ring_nl_f32", st, fl, by);
    swe_status r = f64 ? ring_run<double>(p, id, G, Fin, Fout, S, st) : ring_run<float>(p, id, G, Fin, Fout, S, st);
    prof_end(tk, st);
    return r;
}
