// Allocation-free inverse spherical-harmonic transform.
//
// sht_inverse() takes its scratch (the transform operands and the Fourier
// coefficients) from the plan's workspace arena, which grows with cudaMalloc on
// demand.  Some callers cannot allocate device memory at call time: real-time
// loops that forbid allocator calls (an allocation can block and synchronise the
// device), and applications whose device memory is fully owned by their own pool
// allocator, where a library allocation would fail or escape their accounting.  For them
// sht_inverse_noalloc() uses a fixed scratch array that lives in this file as a
// static __device__ variable: SWE_NOALLOC_SCRATCH_BYTES (64 MiB) on every GPU
// that loads the library, held until the process exits.
#include <mutex>

#include "swe_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[SWE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device; looked up once per
// device (the host-side symbol is only a stand-in and must never reach a kernel).
swe_status scratch_address(void** out) {
    int dev = 0;
    SWE_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        swe_set_error("sht_inverse_noalloc: device index %d out of range", dev);
        return SWE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return swe_cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SWE_OK;
}

// scratch bytes of a batch: the same expression the admission check below uses
size_t noalloc_need(const swe_plan* p, size_t batch) {
    const size_t fe = (p->prec == SWE_FP64) ? sizeof(double2) : sizeof(float2);
    return a256(sizeof(double2) * p->ncx * batch) + a256(fe * (size_t)(p->M + 1) * p->nlat * batch);
}

// largest batch whose scratch fits the static array (binary search on noalloc_need)
size_t noalloc_max_batch(const swe_plan* p) {
    size_t lo = 0, hi = SWE_NOALLOC_SCRATCH_BYTES;
    while (lo < hi) {
        const size_t mid = (lo + hi + 1) / 2;
        if (noalloc_need(p, mid) <= (size_t)SWE_NOALLOC_SCRATCH_BYTES) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace

extern "C" swe_status sht_inverse_noalloc(swe_plan_t p, const void* spec, void* grid, int batch, void* stream) {
    if (!p || !spec || !grid || batch < 1) {
        swe_set_error("sht_inverse_noalloc: invalid argument");
        return SWE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t xbytes = a256(sizeof(double2) * p->ncx * (size_t)batch);
    if (noalloc_need(p, (size_t)batch) > (size_t)SWE_NOALLOC_SCRATCH_BYTES) {
        swe_set_error("sht_inverse_noalloc: batch %d needs %zu bytes of scratch, more than the %zu-byte "
                      "static array (at most %zu fields for this plan)",
                      batch, noalloc_need(p, (size_t)batch), (size_t)SWE_NOALLOC_SCRATCH_BYTES,
                      noalloc_max_batch(p));
        return SWE_EINVAL;
    }
    void* base = nullptr;
    SWE_CHECK(scratch_address(&base));
    double2* X = (double2*)base;
    void* F = (char*)base + xbytes;
    // every scratch element read below is written earlier in the same call:
    // the pack writes all ncx x batch operands (zeros for n = M+1), the Legendre
    // kernel writes all (M+1) x nlat x batch Fourier coefficients
    SWE_CHECK(k_pack_scalar(p, (const double2*)spec, X, batch, st));
    SWE_CHECK(leg_inverse(p, X, F, batch, st));
    SWE_CHECK(ring_inverse(p, F, grid, batch, st));
    return SWE_OK;
}
