// Longitude transforms on latitude rings (§2.2, "Fast Fourier"), in shared memory.
//
// A real DFT of length N = nlon is done as a complex Stockham FFT (radix 4/3/2)
// of two real sequences packed as z = a + i b.  Fourier coefficients are kept
// for m = 0..M only (M + 1 < N / 2).
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
    int n, nrad;
    int rad[32];
};

// One Stockham pass of radix R over nfft sequences of length N stored at stride `stride`.
// S = -1 forward, +1 inverse.  tw[k] = e^{-2 pi i k / N}.
template <typename T, int S>
__device__ void fft_pass(const typename CT<T>::V* __restrict__ src, typename CT<T>::V* __restrict__ dst, int N, int R,
                         int Ns, const typename CT<T>::V* __restrict__ tw, int nfft, int stride) {
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
                V w1 = tw[k * tstep];
                if (S > 0) w1 = cconj(w1);
                v1 = cmul(v1, w1);
            }
            y[idx] = cadd(v0, v1);
            y[idx + Ns] = csub(v0, v1);
        } else if (R == 3) {
            V v2 = x[j + 2 * nb];
            if (k) {
                V w1 = tw[k * tstep], w2 = tw[(2 * k * tstep) % N];
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
                V w1 = tw[k * tstep], w2 = tw[(2 * k * tstep) % N], w3 = tw[(3 * k * tstep) % N];
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
        fft_pass<T, S>(src, dst, fp.n, R, Ns, tw, nfft, stride);
        __syncthreads();
        V* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// Hermitian synthesis input for the pair (A, B) of half spectra, m = 0..M.
template <typename V>
__device__ __forceinline__ void put_pair(V* z, int N, int m, V A, V B) {
    if (m == 0) {
        z[0] = V{A.x, B.x};
    } else {
        z[m] = V{A.x - B.y, A.y + B.x};          // A + i B
        z[N - m] = V{A.x + B.y, B.x - A.y};      // conj(A) + i conj(B)
    }
}

// Split the spectrum of z = a + i b into the spectra of a and b at mode m, scaled.
template <typename T, typename V>
__device__ __forceinline__ void get_pair(const V* Z, int N, int m, T scale, V& A, V& B) {
    V zm = Z[m], zn = Z[m == 0 ? 0 : N - m];
    A = V{(T)0.5 * (zm.x + zn.x) * scale, (T)0.5 * (zm.y - zn.y) * scale};
    B = V{(T)0.5 * (zm.y + zn.y) * scale, (T)-0.5 * (zm.x - zn.x) * scale};
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_ring_inv(const typename CT<T>::V* __restrict__ F, T* __restrict__ grid, int M,
                                                  int nlat, int C, FFTPlan fp, const typename CT<T>::V* __restrict__ tw) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + fp.n;
    const int N = fp.n;
    const int j = blockIdx.y;
    const int c0 = 2 * blockIdx.x;
    const bool two = (c0 + 1) < C;
    for (int k = threadIdx.x; k < N; k += blockDim.x) a[k] = V{0, 0};
    __syncthreads();
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        const V* row = F + ((int64_t)m * nlat + j) * C;
        V A = row[c0];
        V B = two ? row[c0 + 1] : V{0, 0};
        put_pair(a, N, m, A, B);
    }
    __syncthreads();
    V* r = fft_block<T, +1>(a, b, fp, tw, 1, N);
    T* g0 = grid + ((int64_t)c0 * nlat + j) * N;
    T* g1 = grid + ((int64_t)(c0 + 1) * nlat + j) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        g0[k] = r[k].x;
        if (two) g1[k] = r[k].y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ring_fwd(const T* __restrict__ grid, typename CT<T>::V* __restrict__ F, int M,
                                                  int nlat, int C, FFTPlan fp, const typename CT<T>::V* __restrict__ tw,
                                                  const double* __restrict__ w) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* a = reinterpret_cast<V*>(smem_raw);
    V* b = a + fp.n;
    const int N = fp.n;
    const int j = blockIdx.y;
    const int c0 = 2 * blockIdx.x;
    const bool two = (c0 + 1) < C;
    const T* g0 = grid + ((int64_t)c0 * nlat + j) * N;
    const T* g1 = grid + ((int64_t)(c0 + 1) * nlat + j) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) a[k] = V{g0[k], two ? g1[k] : (T)0};
    __syncthreads();
    V* r = fft_block<T, -1>(a, b, fp, tw, 1, N);
    const T scale = (T)(w[j] / (double)N);
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        V A, B;
        get_pair<T>(r, N, m, scale, A, B);
        V* row = F + ((int64_t)m * nlat + j) * C;
        row[c0] = A;
        if (two) row[c0 + 1] = B;
    }
}

// Fused nonlinear ring: Fin [M+1][nlat][4S] (Phi', xi, U, V), Fout [M+1][nlat][5S]
// (A1 = xi U/c2, B1 = xi V/c2, A2 = Phi' U/c2, B2 = Phi' V/c2, KE = (U^2+V^2)/(2 c2)), c2 = 1 - mu^2.
template <typename T>
__global__ void __launch_bounds__(256) k_ring_nl(const typename CT<T>::V* __restrict__ Fin,
                                                 typename CT<T>::V* __restrict__ Fout, int M, int nlat, int S,
                                                 FFTPlan fp, const typename CT<T>::V* __restrict__ tw,
                                                 const double* __restrict__ mu, const double* __restrict__ w) {
    using V = typename CT<T>::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = fp.n;
    V* d = reinterpret_cast<V*>(smem_raw);   // 3 data sequences
    V* sc = d + 3 * N;                        // 3 scratch sequences
    const int s = blockIdx.x;
    const int j = blockIdx.y;
    for (int k = threadIdx.x; k < 2 * N; k += blockDim.x) d[k] = V{0, 0};
    __syncthreads();
    const int64_t C4 = 4 * (int64_t)S;
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        const V* row = Fin + ((int64_t)m * nlat + j) * C4 + s;
        V ph = row[0], xi = row[S], uu = row[2 * S], vv = row[3 * S];
        put_pair(d, N, m, ph, xi);
        put_pair(d + N, N, m, uu, vv);
    }
    __syncthreads();
    V* r = fft_block<T, +1>(d, sc, fp, tw, 2, N);
    const double muj = mu[j];
    const T ic2 = (T)(1.0 / ((1.0 - muj) * (1.0 + muj)));
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        V z1 = r[k], z2 = r[N + k];
        T ph = z1.x, xi = z1.y, U = z2.x, Vv = z2.y;
        r[k] = V{xi * U * ic2, xi * Vv * ic2};
        r[N + k] = V{ph * U * ic2, ph * Vv * ic2};
        r[2 * N + k] = V{(T)0.5 * (U * U + Vv * Vv) * ic2, (T)0};
    }
    __syncthreads();
    V* other = (r == d) ? sc : d;
    V* q = fft_block<T, -1>(r, other, fp, tw, 3, N);
    const T scale = (T)(w[j] / (double)N);
    const int64_t C5 = 5 * (int64_t)S;
    for (int m = threadIdx.x; m <= M; m += blockDim.x) {
        V a1, b1, a2, b2, ke, zero;
        get_pair<T>(q, N, m, scale, a1, b1);
        get_pair<T>(q + N, N, m, scale, a2, b2);
        get_pair<T>(q + 2 * N, N, m, scale, ke, zero);
        V* row = Fout + ((int64_t)m * nlat + j) * C5 + s;
        row[0] = a1;
        row[S] = b1;
        row[2 * S] = a2;
        row[3 * S] = b2;
        row[4 * S] = ke;
    }
}

FFTPlan make_fft_plan(const swe_plan* p) {
    FFTPlan fp;
    fp.n = p->nlon;
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
    FFTPlan fp = make_fft_plan(p);
    dim3 g((C + 1) / 2, p->nlat);
    if (p->prec == SWE_FP64) {
        size_t sm = 2 * sizeof(double2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_inv<double>, sm));
        k_ring_inv<double><<<g, 256, sm, st>>>((const double2*)F, (double*)grid, p->M, p->nlat, C, fp, p->tw);
    } else {
        size_t sm = 2 * sizeof(float2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_inv<float>, sm));
        k_ring_inv<float><<<g, 256, sm, st>>>((const float2*)F, (float*)grid, p->M, p->nlat, C, fp, p->twf);
    }
    SWE_CHECK_LAUNCH("k_ring_inv");
    return SWE_OK;
}

swe_status ring_forward(const swe_plan* p, const void* grid, void* F, int C, cudaStream_t st) {
    FFTPlan fp = make_fft_plan(p);
    dim3 g((C + 1) / 2, p->nlat);
    if (p->prec == SWE_FP64) {
        size_t sm = 2 * sizeof(double2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_fwd<double>, sm));
        k_ring_fwd<double><<<g, 256, sm, st>>>((const double*)grid, (double2*)F, p->M, p->nlat, C, fp, p->tw, p->w);
    } else {
        size_t sm = 2 * sizeof(float2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_fwd<float>, sm));
        k_ring_fwd<float><<<g, 256, sm, st>>>((const float*)grid, (float2*)F, p->M, p->nlat, C, fp, p->twf, p->w);
    }
    SWE_CHECK_LAUNCH("k_ring_fwd");
    return SWE_OK;
}

swe_status ring_nonlinear(const swe_plan* p, const void* Fin, void* Fout, int S, cudaStream_t st) {
    FFTPlan fp = make_fft_plan(p);
    dim3 g(S, p->nlat);
    if (p->prec == SWE_FP64) {
        size_t sm = 6 * sizeof(double2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_nl<double>, sm));
        k_ring_nl<double><<<g, 256, sm, st>>>((const double2*)Fin, (double2*)Fout, p->M, p->nlat, S, fp, p->tw, p->mu,
                                              p->w);
    } else {
        size_t sm = 6 * sizeof(float2) * p->nlon;
        SWE_CHECK(set_smem(k_ring_nl<float>, sm));
        k_ring_nl<float><<<g, 256, sm, st>>>((const float2*)Fin, (float2*)Fout, p->M, p->nlat, S, fp, p->twf, p->mu,
                                             p->w);
    }
    SWE_CHECK_LAUNCH("k_ring_nl");
    return SWE_OK;
}
