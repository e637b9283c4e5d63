// Split-precision Legendre contraction on the 5th-generation tensor cores (tcgen05).
//
// The contraction of §2.2 ("Fast Legendre") per zonal wavenumber m is a small
// dense GEMM; all slices and fields are batched into its column dimension.  Both
// directions are written with the data columns as the MMA M dimension (128 per CTA):
//
//   inverse:  D_par[c, j] = sum_k X[(m, n = m+par+2k), c] P_n^m(mu_j)      (j: northern latitudes)
//             F(mu_j)  = D_0 + D_1,  F(-mu_j) = D_0 - D_1                     (equatorial symmetry)
//   forward:  D_par[c, k] = sum_j G_par[j, c] P_{m+par+2k}^m(mu_j),
//             G_0 = F(mu_j) + F(-mu_j),  G_1 = F(mu_j) - F(-mu_j)
//
// Precision: every operand value v (FP64 / FP32) is split into three bf16 terms
// v = v0 + v1 + v2 (24 significant bits), and each product is formed from the six
// largest partial products a0 b0 + a0 b1 + a1 b0 + a0 b2 + a2 b0 + a1 b1 with FP32
// accumulation in tensor memory (relative error ~1e-8 per contraction, below the
// FP32 rounding of the Fourier data this path carries).
//
// Data movement: the Legendre operand (B) is pre-split and pre-tiled on the device
// into the canonical no-swizzle K-major core-matrix layout and streamed into shared
// memory by the bulk-copy engine (cp.async.bulk + mbarrier transaction counts);
// the FP32 rows of the data operand (A) arrive a few chunks ahead as 2-D TMA tensor
// tiles issued by the control lane (per-thread cp.async when the row pitch is not a
// multiple of 16 bytes), and the converter warps split them in registers (4 threads
// per column, each a quarter of the chunk) and store the same layout.  One elected thread issues
// tcgen05.mma (kind::f16, bf16 x bf16 -> f32, M = 128, K = 16) into two TMEM
// accumulators (one per parity); a two-stage ring overlaps the split of chunk q+1
// with the MMAs of chunk q; the epilogue reads TMEM with tcgen05.ld (16 warps,
// each a lane quarter and a quarter of the accumulator columns) and writes
// coalesced rows.  Every mbarrier wait is bounded: on
// timeout the kernel sets an error flag, stops issuing work, releases its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <string>
#include <vector>

#include "swe_internal.cuh"

namespace {

constexpr int BM = 128;          // data columns per CTA (MMA M)
constexpr int NCV = 512;         // converter threads: 4 per data column, each a quarter of a K chunk
constexpr int NTH = NCV + 32;    // + one control warp (table copies and MMA issue)
constexpr int KQ = 4;            // K values per thread per chunk
constexpr int KC = 16;           // K per chunk (one MMA)
constexpr int NPLANE = 3;        // bf16 split terms
constexpr int NTERMS = 6;        // partial products kept
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_LIMIT = 1ull << 22;   // bounded polling (about a second)
constexpr int NR_INV = 4;        // raw data-operand prefetch depth, inverse (FP32 rows)
constexpr int NR_FWD = 4;        // raw data-operand prefetch depth, forward (FP32 rows)
constexpr int NT_MAX = 224;      // largest N tile (two parity accumulators + a 32-column read fit in 512)
constexpr int NB_MAX = 4;        // table-tile ring depth (set per plan from the shared-memory budget)


// ----------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 2-D tensor tile (TMA) into shared memory, completion on an mbarrier's transaction count
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// per-thread asynchronous global -> shared copies (zero-filled when !pred)
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor, no swizzle, K-major core matrices (8 rows x 16 bytes)
__device__ __forceinline__ uint64_t smem_desc(const void* base, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(base) & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: kind::f16 with bf16 A/B, f32 accumulate, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t make_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------------------- operand helpers
// three-term bf16 split of a value already rounded to FP32 (24 significant bits)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(a);
    b = __float2bfloat16_rn(r);
    r = r - __bfloat162float(b);
    c = __float2bfloat16_rn(r);
}

// byte offset of element (row, k) in a K-major no-swizzle tile with 16 K-elements:
// core matrices of 8 rows x 8 elements; K-adjacent core matrices 128 B apart (LBO),
// row-group-adjacent ones 256 B apart (SBO)
__host__ __device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Writes one thread's 4 consecutive K values (k0..k0+3, k0 a multiple of 4) of its row
// as three bf16 planes (8-byte stores).
// (packed bf16x2 conversions: the same round-to-nearest split as split3, two values at a time)
__device__ __forceinline__ void split3x2(float a, float b, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
    const __nv_bfloat162 p0 = __float22bfloat162_rn(make_float2(a, b));
    const float2 q0 = __bfloat1622float2(p0);
    const float2 r1 = make_float2(a - q0.x, b - q0.y);
    const __nv_bfloat162 p1 = __float22bfloat162_rn(r1);
    const float2 q1 = __bfloat1622float2(p1);
    const __nv_bfloat162 p2 = __float22bfloat162_rn(make_float2(r1.x - q1.x, r1.y - q1.y));
    memcpy(&h0, &p0, 4);
    memcpy(&h1, &p1, 4);
    memcpy(&h2, &p2, 4);
}

__device__ __forceinline__ void store_quad_planes(unsigned char* plane0, uint32_t plane_bytes, int row, int k0,
                                                  const float* v) {
    uint32_t a0, a1, a2, b0, b1, b2;
    split3x2(v[0], v[1], a0, a1, a2);
    split3x2(v[2], v[3], b0, b1, b2);
    const uint32_t off = tile_off(row, k0);
    *reinterpret_cast<uint2*>(plane0 + off) = make_uint2(a0, b0);
    *reinterpret_cast<uint2*>(plane0 + plane_bytes + off) = make_uint2(a1, b1);
    *reinterpret_cast<uint2*>(plane0 + 2 * plane_bytes + off) = make_uint2(a2, b2);
}

struct TCShape {
    int M, nlat, nlat2, ncol;    // ncol: real data columns
    int nt;                      // N tile (multiple of 16, <= 256)
};

// Both kernels run one warp-specialised pipeline over 16-deep K chunks q:
//   converter warps 0-15 (4 threads per data column): wait for the raw FP32 rows of chunk
//     q (TMA path: mbarrier "r_full" of raw stage q mod NR; cp.async path: each thread
//     copies its own column NR - 1 chunks ahead, so only it reads it back), wait for the
//     MMAs of chunk q - 2 to release bf16 stage q mod 2 (mbarrier "a_empty", signalled by
//     tcgen05.commit), split chunk q into three bf16 planes there, fence the async proxy
//     and arrive on "a_full" (one lane per warp);
//   control warp 16, one lane: on the TMA path issues the raw tiles of chunks 0 .. NR-1 and
//     then those of chunk q + NR once "a_full" of chunk q shows stage q mod NR consumed;
//     keeps the table tiles NB - 2 chunks ahead in an NB-deep ring (bulk copies on
//     "b_full"; a stage is reused once "b_empty" says its MMAs are done), waits for
//     "a_full" and "b_full" of chunk q, issues the 2 x 6 MMAs and commits them to
//     "a_empty" and "b_empty"; after the last chunk it commits to "acc_full";
//   then the converter warps read the accumulators (tcgen05.ld) and write the result.
// There is no block barrier inside the loop.  Every wait is bounded; a thread that
// gives up raises a shared abort flag that makes every other wait return at once, the
// control lane drains the copies and MMAs it has in flight (bounded), and the CTA
// reports the timeout and releases its tensor memory.
constexpr int NR_MAX = 4;

struct WS {
    uint64_t a_full[2], a_empty[2], b_full[NB_MAX], b_empty[NB_MAX], acc_full;
    uint64_t r_full[NR_MAX];          // raw data-operand stages filled by TMA
    int abort;
    uint32_t tmem_slot;
};

// bounded wait (at most `limit` polls) that also gives up once another thread raised the
// abort flag
__device__ __forceinline__ bool ws_wait_n(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          unsigned long long limit) {
    const uint32_t a = smem_u32(bar);
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n"
            " .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return ws_wait_n(bar, parity, abort, WAIT_LIMIT);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 2 parities x 6 partial products of one chunk into the two accumulators
// (the descriptors' start-address field is the shared-memory address / 16, 14 bits: the
// planes' descriptors are the stage's plus the plane offset / 16, which never carries out)
__device__ __forceinline__ void issue_mmas(const unsigned char* sA, uint32_t a_plane, const unsigned char* sB,
                                           uint32_t b_plane, uint32_t tmem, int acc_stride, uint32_t idesc,
                                           bool first) {
    constexpr int ta[NTERMS] = {0, 0, 1, 0, 2, 1}, tb[NTERMS] = {0, 1, 0, 2, 0, 1};
    const uint64_t da = smem_desc(sA, 128, 256), db = smem_desc(sB, 128, 256);
#pragma unroll
    for (int par = 0; par < 2; ++par) {
#pragma unroll
        for (int t = 0; t < NTERMS; ++t) {
            const uint64_t a = da + (uint64_t)(((uint32_t)(par * NPLANE + ta[t]) * a_plane) >> 4);
            const uint64_t b = db + (uint64_t)(((uint32_t)(par * NPLANE + tb[t]) * b_plane) >> 4);
            mma_bf16(tmem + par * acc_stride, a, b, idesc, (!first || t > 0) ? 1u : 0u);
        }
    }
}

__device__ __forceinline__ uint32_t ws_setup(WS* ws, int tid) {
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ws->a_full[i], NCV / 32);
            mbar_init(&ws->a_empty[i], 1);
        }
        for (int i = 0; i < NB_MAX; ++i) {
            mbar_init(&ws->b_full[i], 1);
            mbar_init(&ws->b_empty[i], 1);
        }
        mbar_init(&ws->acc_full, 1);
        for (int i = 0; i < NR_MAX; ++i) mbar_init(&ws->r_full[i], 1);
        ws->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ws->tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return ws->tmem_slot;
}

__device__ __forceinline__ void tmem_release(uint32_t tmem, int tid) {
    tc_fence_before();
    __syncthreads();
    if ((tid >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// control lane: table-tile ring + MMA issue for chunks 0..nq-1 (see above)
// Data-operand producers for the control lane.  NoTma: the converter warps load their own
// columns with cp.async.  TmaA: the control lane loads each chunk's raw FP32 rows as 2-D
// tensor tiles (128 columns wide) into raw stage c mod NR; a stage is refilled once the
// converters' a_full arrival for the chunk that used it has been observed.
struct NoTma {
    int issued = 0;
    __device__ __forceinline__ void issue(int) {}
    __device__ __forceinline__ int nr() const { return 0; }
    __device__ __forceinline__ uint64_t* full(int) const { return nullptr; }
};
struct TmaA {
    const CUtensorMap* map;
    unsigned char* raw;
    uint32_t stage_bytes;
    uint64_t* r_full;
    int NR, nq, x;
    int fwd;                 // 0: inverse, one 32-row tile at y0 + 32 c; 1: forward, north + south 16-row tiles
    int y0, nlat;
    int issued = 0;
    __device__ __forceinline__ int nr() const { return NR; }
    __device__ __forceinline__ uint64_t* full(int c) const { return &r_full[c % NR]; }
    __device__ __forceinline__ void issue(int c) {
        if (c >= nq) return;
        uint64_t* bar = &r_full[c % NR];
        unsigned char* dst = raw + (size_t)(c % NR) * stage_bytes;
        mbar_expect_tx(bar, stage_bytes);
        if (!fwd) {
            tma_load_2d(dst, map, x, y0 + 32 * c, bar);
        } else {
            tma_load_2d(dst, map, x, y0 + 16 * c, bar);
            tma_load_2d(dst + stage_bytes / 2, map, x, y0 + nlat - 16 * (c + 1), bar);
        }
        issued = c + 1;
    }
};

// (b_stride: byte distance of the ring's stages; b_bytes: bytes of one chunk's table tile)
template <typename AProd>
__device__ __forceinline__ void ws_control(WS* ws, unsigned char* sA0, uint32_t a_stage, uint32_t a_plane,
                                           unsigned char* sB0,
                                           uint32_t b_stride, uint32_t b_bytes, uint32_t b_plane, int NB,
                                           const unsigned char* Bm, int64_t bchunk, int nq, uint32_t tmem,
                                           int acc_stride, uint32_t idesc, AProd& ap) {
    volatile int* ab = &ws->abort;
    for (int c = 0; c < ap.nr(); ++c) ap.issue(c);          // data operand: the first NR chunks
    int a_seen = 0;                                          // chunks whose converters have finished
    const int D = NB - 2;                                   // table chunks in flight ahead of the MMAs
    int issued_b = 0, last_mma = -1;
    auto copy_b = [&](int c) {
        mbar_expect_tx(&ws->b_full[c % NB], b_bytes);
        bulk_g2s(sB0 + (size_t)(c % NB) * b_stride, Bm + (int64_t)c * bchunk, b_bytes, &ws->b_full[c % NB]);
        issued_b = c + 1;
    };
    for (int c = 0; c < D && c < nq; ++c) copy_b(c);
    bool ok = true;
    for (int q = 0; q < nq && ok; ++q) {
        const int c = q + D;
        if (c < nq) {
            if (c >= NB) ok = ws_wait(&ws->b_empty[c % NB], ((c / NB) - 1) & 1, ab);
            if (!ok) break;
            copy_b(c);
        }
        ok = ws_wait(&ws->a_full[q & 1], (q >> 1) & 1, ab);
        if (!ok) break;
        a_seen = q + 1;
        if (ap.nr()) ap.issue(q + ap.nr());                  // raw stage of chunk q is free again
        ok = ws_wait(&ws->b_full[q % NB], (q / NB) & 1, ab);
        if (!ok) break;
        tc_fence_after();
        issue_mmas(sA0 + (q & 1) * a_stage, a_plane, sB0 + (size_t)(q % NB) * b_stride, b_plane, tmem, acc_stride,
                   idesc, q == 0);
        mma_commit(&ws->a_empty[q & 1]);
        mma_commit(&ws->b_empty[q % NB]);
        last_mma = q;
    }
    if (ok) {
        mma_commit(&ws->acc_full);
        return;
    }
    *ab = 1;
    // bounded drain of this CTA's own work in flight: the MMAs (their last commit) and
    // the table copies not yet consumed
    volatile int zero = 0;
    if (last_mma >= 0) ws_wait(&ws->a_empty[last_mma & 1], (last_mma >> 1) & 1, &zero);
    for (int c = last_mma + 1; c < issued_b; ++c) ws_wait(&ws->b_full[c % NB], (c / NB) & 1, &zero);
    for (int c = a_seen; c < ap.issued; ++c) ws_wait(ap.full(c), (c / ap.nr()) & 1, &zero);
}

// converter side of chunk q, after its planes are stored: make them visible to the
// tensor core and signal (one lane per warp)
template <typename W>
__device__ __forceinline__ void ws_planes_ready(W* ws, int q, int lane) {
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ws->a_full[q & 1]);
}

// converter warp: wait (lane 0) for a barrier phase, broadcast the outcome
template <typename W>
__device__ __forceinline__ bool ws_warp_wait(W* ws, uint64_t* bar, uint32_t parity, int lane) {
    bool ok = true;
    if (lane == 0) ok = ws_wait(bar, parity, &ws->abort);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// converter warp: every lane waits for a TMA-filled raw stage (each lane then sees the
// tile's bytes); the warp gives up together if any lane does
template <typename W>
__device__ __forceinline__ bool ws_raw_wait(W* ws, uint64_t* bar, uint32_t parity) {
    const bool ok = ws_wait(bar, parity, &ws->abort);
    return __all_sync(0xffffffffu, ok) != 0;
}

// ----------------------------------------------------------------------------- inverse
// grid: (ceil(ncol/128), M+1, n-tiles over j).  Table Binv: for each m, chunk q, parity,
// N-tile: a [nt x 16] bf16 tile x 3 planes, contiguous (offsets from inv_off[m]).
// TMA: the raw rows of a chunk arrive as one 32 x 128 tensor tile (rows xrow0 + 32 q ..,
// raw row t = extended row 32 q + t) issued by the control lane; otherwise each converter
// thread copies its own column with cp.async into [parity][k][column].
template <bool TMA>
__global__ void __launch_bounds__(NTH, 1) k_leg_inv_tc(const float* __restrict__ X, float* __restrict__ F,
                                                       const unsigned char* __restrict__ Binv,
                                                       const long long* __restrict__ inv_off,
                                                       const int* __restrict__ inv_nq, TCShape sh, int NB, int* err,
                                                       const __grid_constant__ CUtensorMap tmX) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nt = sh.nt;
    const uint32_t a_plane = BM * KC * 2;                 // 4 KB
    const uint32_t b_plane = (uint32_t)nt * KC * 2;
    const uint32_t a_stage = 2 * NPLANE * a_plane;        // two parities
    const uint32_t b_stage = 2 * NPLANE * b_plane;
    unsigned char* const sA0 = smem;                       // bf16 stages: sA0 + (q & 1) a_stage
    unsigned char* sB0 = smem + 2 * a_stage;
    float* raw = reinterpret_cast<float*>(sB0 + (size_t)NB * b_stage);   // [NR][2][KC][BM]
    WS* ws = reinterpret_cast<WS*>(raw + NR_INV * 2 * KC * BM);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int col = tid & (BM - 1), sub = (tid >> 7) & 3;
    const int M = sh.M;
    const int m = M - (int)blockIdx.y;
    const int c0 = blockIdx.x * BM;
    const int jt0 = blockIdx.z * nt;
    const int nq = inv_nq[m];
    const int Kx = M + 2 - m;                              // extended rows of this m
    const int64_t xrow0 = ex_off(m, M);
    const int c = c0 + col;
    const bool cin = c < sh.ncol;
    const bool conv = tid < NCV;

    // raw prefetch of chunk qq (rows n = m + par + 2k, k in [16 qq, 16 qq + 16)): this thread's
    // column and quarter
    auto prefetch = [&](int qq) {
        if (!TMA && qq < nq) {
            float* r = raw + (qq % NR_INV) * (2 * KC * BM);
#pragma unroll
            for (int par = 0; par < 2; ++par)
#pragma unroll
                for (int i = 0; i < KQ; ++i) {
                    const int kk = KQ * sub + i;
                    const int rr = par + 2 * (KC * qq + kk);
                    const bool pr = cin && rr < Kx;
                    cp_async4(&r[(par * KC + kk) * BM + col], pr ? (const void*)&X[(xrow0 + rr) * sh.ncol + c] : X,
                              pr);
                }
        }
        cp_async_commit();
    };
    if (conv && !TMA) {
#pragma unroll
        for (int qq = 0; qq < NR_INV - 1; ++qq) prefetch(qq);
    }
    const uint32_t tmem = ws_setup(ws, tid);
    const uint32_t idesc = make_idesc(nt);
    if (!conv) {
        if (lane == 0) {
            const unsigned char* Bm = Binv + inv_off[m] + (int64_t)blockIdx.z * 2 * NPLANE * b_plane;
            const int64_t bchunk = (int64_t)gridDim.z * 2 * NPLANE * b_plane;   // bytes per chunk, all n-tiles
            if constexpr (TMA) {
                TmaA ap{&tmX, reinterpret_cast<unsigned char*>(raw), 2 * KC * BM * 4, ws->r_full, NR_INV, nq, c0, 0,
                        (int)xrow0, 0};
                ws_control(ws, sA0, a_stage, a_plane, sB0, b_stage, b_stage, b_plane, NB, Bm, bchunk, nq, tmem, nt,
                           idesc, ap);
            } else {
                NoTma ap;
                ws_control(ws, sA0, a_stage, a_plane, sB0, b_stage, b_stage, b_plane, NB, Bm, bchunk, nq, tmem, nt,
                           idesc, ap);
            }
        }
    } else {
        for (int q = 0; q < nq; ++q) {
            if constexpr (TMA) {
                if (!ws_raw_wait(ws, &ws->r_full[q % NR_INV], (q / NR_INV) & 1)) break;
            } else {
                prefetch(q + NR_INV - 1);
                cp_async_wait<NR_INV - 1>();
            }
            if (q >= 2 && !ws_warp_wait(ws, &ws->a_empty[q & 1], ((q - 2) >> 1) & 1, lane)) break;
            const float* r = raw + (q % NR_INV) * (2 * KC * BM);
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                float v[KQ];
#pragma unroll
                for (int i = 0; i < KQ; ++i) {
                    const int kk = KQ * sub + i;
                    if constexpr (TMA) {
                        // rows past this wavenumber's Kx belong to the next one (or are the tile's zero fill)
                        const float x = r[(par + 2 * kk) * BM + col];
                        v[i] = par + 2 * (KC * q + kk) < Kx ? x : 0.f;
                    } else {
                        v[i] = r[(par * KC + kk) * BM + col];
                    }
                }
                store_quad_planes(sA0 + (q & 1) * a_stage + par * NPLANE * a_plane, a_plane, col, KQ * sub, v);
            }
            ws_planes_ready(ws, q, lane);
        }
        cp_async_wait<0>();
        ws_warp_wait(ws, &ws->acc_full, 0, lane);
    }
    __syncthreads();
    tc_fence_after();
    if (!ws->abort) {
        if (conv) {
            // epilogue: warp w reads TMEM lanes (= data columns) 32 (w mod 4) .. + 31, and the
            // 32-column groups j0 = 32 sub + 128 i of the accumulators
            const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
            for (int j0 = 32 * sub; j0 < nt; j0 += 128) {
                float e[32], o[32];
                tmem_ld32(tmem + lane_base + (uint32_t)j0, e);
                tmem_ld32(tmem + lane_base + (uint32_t)(nt + j0), o);
                if (cin) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int j = jt0 + j0 + i;
                        if (j0 + i < nt && j < sh.nlat2) {
                            F[((int64_t)m * sh.nlat + j) * sh.ncol + c] = e[i] + o[i];
                            F[((int64_t)m * sh.nlat + (sh.nlat - 1 - j)) * sh.ncol + c] = e[i] - o[i];
                        }
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(err, PLAN_FLAG_TIMEOUT);
    }
    tmem_release(tmem, tid);
}

// ----------------------------------------------------------------------------- forward
// grid: (ceil(ncol/128), M+1, max n-tiles over k).  Table Bfwd: for each m, j-chunk q,
// n-tile z, parity: a [nt_m x 16] tile x 3 planes (rows k = degree index within the
// parity); nt_m = fwd_nt[m] follows the number of degrees of m (multiple of 16).
// TMA: chunk q arrives as two 16 x 128 tensor tiles, the northern rows j = 16 q + t (raw
// row t) and the southern rows nlat - 16 (q + 1) + t (raw row 16 + t, i.e. the mirror of
// j = 16 q + 15 - t); otherwise each converter thread copies its own column with cp.async.
template <bool TMA>
__global__ void __launch_bounds__(NTH, 1) k_leg_fwd_tc(const float* __restrict__ F, float* __restrict__ Y,
                                                       const unsigned char* __restrict__ Bfwd,
                                                       const long long* __restrict__ fwd_off,
                                                       const int* __restrict__ fwd_ntiles,
                                                       const int* __restrict__ fwd_nt, TCShape sh, int NB, int* err,
                                                       const __grid_constant__ CUtensorMap tmF) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int M = sh.M;
    const int m = M - (int)blockIdx.y;
    const int nz = fwd_ntiles[m];
    if ((int)blockIdx.z >= nz) return;                     // uniform for the CTA: before any barrier
    const int nt = fwd_nt[m];
    const int acc = (nt + 31) & ~31;                       // TMEM column offset of the parity-1 accumulator
    const uint32_t a_plane = BM * KC * 2;
    const uint32_t b_plane = (uint32_t)nt * KC * 2;
    const uint32_t a_stage = 2 * NPLANE * a_plane;
    const uint32_t b_stage = 2 * NPLANE * b_plane;
    const uint32_t b_stage_max = 2 * NPLANE * (uint32_t)sh.nt * KC * 2;
    unsigned char* const sA0 = smem;                       // bf16 stages: sA0 + (q & 1) a_stage
    unsigned char* sB0 = smem + 2 * a_stage;               // NB stages of b_stage_max bytes
    float* raw = reinterpret_cast<float*>(sB0 + (size_t)NB * b_stage_max);   // [NR][2 KC][BM]
    WS* ws = reinterpret_cast<WS*>(raw + NR_FWD * 2 * KC * BM);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int col = tid & (BM - 1), sub = (tid >> 7) & 3;
    const int c0 = blockIdx.x * BM;
    const int kt0 = blockIdx.z * nt;
    const int nq = (sh.nlat2 + KC - 1) / KC;
    const int Kx = M + 2 - m;
    const int64_t yrow0 = ex_off(m, M);
    const int c = c0 + col;
    const bool cin = c < sh.ncol;
    const bool conv = tid < NCV;
    const float* Fm = F + (int64_t)m * sh.nlat * sh.ncol;

    // raw prefetch of chunk qq: rows j = 16 qq + jj (north) and nlat-1-j (south), this thread's
    // column and quarter
    auto prefetch = [&](int qq) {
        if (!TMA && qq < nq) {
            float* r = raw + (qq % NR_FWD) * (2 * KC * BM);
#pragma unroll
            for (int i = 0; i < KQ; ++i) {
                const int jj = KQ * sub + i;
                const int j = KC * qq + jj;
                const bool pr = cin && j < sh.nlat2;
                cp_async4(&r[jj * BM + col], pr ? (const void*)&Fm[(int64_t)j * sh.ncol + c] : F, pr);
                cp_async4(&r[(KC + jj) * BM + col],
                          pr ? (const void*)&Fm[(int64_t)(sh.nlat - 1 - j) * sh.ncol + c] : F, pr);
            }
        }
        cp_async_commit();
    };
    if (conv && !TMA) {
#pragma unroll
        for (int qq = 0; qq < NR_FWD - 1; ++qq) prefetch(qq);
    }
    const uint32_t tmem = ws_setup(ws, tid);
    const uint32_t idesc = make_idesc(nt);
    if (!conv) {
        if (lane == 0) {
            // the ring's stages are b_stage_max apart so that every wavenumber's tiles fit;
            // the copies move this wavenumber's b_stage bytes
            const unsigned char* Bm = Bfwd + fwd_off[m] + (int64_t)blockIdx.z * b_stage;
            const int64_t bchunk = (int64_t)nz * b_stage;
            if constexpr (TMA) {
                TmaA ap{&tmF, reinterpret_cast<unsigned char*>(raw), 2 * KC * BM * 4, ws->r_full, NR_FWD, nq, c0, 1,
                        m * sh.nlat, sh.nlat};
                ws_control(ws, sA0, a_stage, a_plane, sB0, b_stage_max, b_stage, b_plane, NB, Bm, bchunk, nq, tmem,
                           acc, idesc, ap);
            } else {
                NoTma ap;
                ws_control(ws, sA0, a_stage, a_plane, sB0, b_stage_max, b_stage, b_plane, NB, Bm, bchunk, nq, tmem,
                           acc, idesc, ap);
            }
        }
    } else {
        for (int q = 0; q < nq; ++q) {
            if constexpr (TMA) {
                if (!ws_raw_wait(ws, &ws->r_full[q % NR_FWD], (q / NR_FWD) & 1)) break;
            } else {
                prefetch(q + NR_FWD - 1);
                cp_async_wait<NR_FWD - 1>();
            }
            if (q >= 2 && !ws_warp_wait(ws, &ws->a_empty[q & 1], ((q - 2) >> 1) & 1, lane)) break;
            const float* r = raw + (q % NR_FWD) * (2 * KC * BM);
            float vs[KQ], va[KQ];
#pragma unroll
            for (int i = 0; i < KQ; ++i) {
                const int jj = KQ * sub + i;
                float fn, fs;
                if constexpr (TMA) {
                    // rows j >= nlat/2 of the last chunk are the other hemisphere's: dropped
                    const bool in = KC * q + jj < sh.nlat2;
                    fn = in ? r[jj * BM + col] : 0.f;
                    fs = in ? r[(2 * KC - 1 - jj) * BM + col] : 0.f;
                } else {
                    fn = r[jj * BM + col];
                    fs = r[(KC + jj) * BM + col];
                }
                vs[i] = fn + fs;
                va[i] = fn - fs;
            }
            store_quad_planes(sA0 + (q & 1) * a_stage, a_plane, col, KQ * sub, vs);
            store_quad_planes(sA0 + (q & 1) * a_stage + NPLANE * a_plane, a_plane, col, KQ * sub, va);
            ws_planes_ready(ws, q, lane);
        }
        cp_async_wait<0>();
        ws_warp_wait(ws, &ws->acc_full, 0, lane);
    }
    __syncthreads();
    tc_fence_after();
    if (!ws->abort) {
        if (conv) {
            const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
            for (int k0 = 32 * sub; k0 < nt; k0 += 128) {
                float d0[32], d1[32];
                tmem_ld32(tmem + lane_base + (uint32_t)k0, d0);
                tmem_ld32(tmem + lane_base + (uint32_t)(acc + k0), d1);
                if (cin) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int k = kt0 + k0 + i;
                        const int r0 = 2 * k, r1 = 2 * k + 1;        // extended-row offsets of parities 0 / 1
                        if (k0 + i < nt) {
                            if (r0 < Kx) Y[(yrow0 + r0) * sh.ncol + c] = d0[i];
                            if (r1 < Kx) Y[(yrow0 + r1) * sh.ncol + c] = d1[i];
                        }
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(err, PLAN_FLAG_TIMEOUT);
    }
    tmem_release(tmem, tid);
}

// ----------------------------------------------------------------------------- persistent kernels
// One CTA per SM walks a list of work items (column tile, wavenumber m, N tile) round-robin
// (CTA b takes items b, b + G, b + 2G, ...; the items are ordered by decreasing K so that the
// longest come first).  The K chunks of all its items form one continuous pipeline:
//   converter warps 0-15: as in the per-tile kernels, chunk after chunk across items;
//   control warp 16, one lane: raw TMA tiles NR chunks ahead and table tiles NB - 2 chunks
//     ahead across item boundaries; the MMAs of item i go to accumulator set i mod nsets
//     (see below), after "acc_empty" of that set shows the epilogue of the item that used it
//     last done; after the item's last chunk it commits to "acc_full" of the set;
//   epilogue warps 17-20 (TMEM lane quarter = warp mod 4): wait "acc_full" of item i, read
//     the accumulators, write the result, fence, arrive on "acc_empty".
// So (with two sets) the epilogue of one item overlaps the MMAs of the next, and the CTA's
// prologue (barriers, TMEM allocation, first copies) is paid once per SM.  Every wait is
// bounded as in the per-tile kernels.
constexpr int NEPI = 4;                       // epilogue warps
constexpr int NTHP = NCV + 32 + 32 * NEPI;    // 672 threads
// Accumulator sets: two of 256 TMEM columns when both parities of an item fit in 256 (N tile
// <= 128), else one set of all 512 (then item i + 1's MMAs wait for item i's epilogue, while
// its copies and conversions still run ahead).  Item i uses set i mod nsets.

struct WSP {
    uint64_t a_full[2], a_empty[2], b_full[NB_MAX], b_empty[NB_MAX];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t r_full[NR_MAX];
    int abort;
    uint32_t tmem_slot;
};

__device__ __forceinline__ uint32_t wsp_setup(WSP* ws, int tid) {
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ws->a_full[i], NCV / 32);
            mbar_init(&ws->a_empty[i], 1);
            mbar_init(&ws->acc_full[i], 1);
            mbar_init(&ws->acc_empty[i], NEPI);
        }
        for (int i = 0; i < NB_MAX; ++i) {
            mbar_init(&ws->b_full[i], 1);
            mbar_init(&ws->b_empty[i], 1);
        }
        for (int i = 0; i < NR_MAX; ++i) mbar_init(&ws->r_full[i], 1);
        ws->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ws->tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return ws->tmem_slot;
}

// Work item of a persistent launch: pair list entry (m | z << 16) and column tile x.
struct PItem {
    int m, z, x, nq;
};

// Per-direction parameters the control lane needs for item `it`.
struct PInv {
    const unsigned char* B;
    const long long* off;
    const int* nqm;
    const int* pairs;
    int nx, M, nt, ntl;
    __device__ __forceinline__ PItem item(int it) const {
        const int pr = pairs[it / nx];
        PItem r{pr & 0xFFFF, pr >> 16, it % nx, 0};
        r.nq = nqm[r.m];
        return r;
    }
    __device__ __forceinline__ uint32_t nt_of(const PItem&) const { return (uint32_t)nt; }
    __device__ __forceinline__ int acc_of(const PItem&) const { return nt; }
    // table tile of chunk q: tiles ordered (q, z, par, plane), ntl tiles per chunk
    __device__ __forceinline__ const unsigned char* btile(const PItem& w, int q, uint32_t& bytes) const {
        const uint32_t bs = 2 * NPLANE * (uint32_t)nt * KC * 2;
        bytes = bs;
        return B + off[w.m] + ((int64_t)q * ntl + w.z) * bs;
    }
    __device__ __forceinline__ void raw(const CUtensorMap* map, unsigned char* dst, const PItem& w, int q,
                                        uint64_t* bar) const {
        tma_load_2d(dst, map, w.x * BM, (int)ex_off(w.m, M) + 32 * q, bar);
    }
};
struct PFwd {
    const unsigned char* B;
    const long long* off;
    const int* nzm;
    const int* ntm;
    const int* pairs;
    int nx, M, nlat, nq;
    __device__ __forceinline__ PItem item(int it) const {
        const int pr = pairs[it / nx];
        return PItem{pr & 0xFFFF, pr >> 16, it % nx, nq};
    }
    __device__ __forceinline__ uint32_t nt_of(const PItem& w) const { return (uint32_t)ntm[w.m]; }
    __device__ __forceinline__ int acc_of(const PItem& w) const { return (ntm[w.m] + 31) & ~31; }
    __device__ __forceinline__ const unsigned char* btile(const PItem& w, int q, uint32_t& bytes) const {
        const uint32_t bs = 2 * NPLANE * (uint32_t)ntm[w.m] * KC * 2;
        bytes = bs;
        return B + off[w.m] + ((int64_t)q * nzm[w.m] + w.z) * bs;
    }
    __device__ __forceinline__ void raw(const CUtensorMap* map, unsigned char* dst, const PItem& w, int q,
                                        uint64_t* bar) const {
        tma_load_2d(dst, map, w.x * BM, w.m * nlat + 16 * q, bar);
        tma_load_2d(dst + KC * BM * 4, map, w.x * BM, w.m * nlat + nlat - 16 * (q + 1), bar);
    }
};

// Walks the (item, chunk) sequence of this CTA: items blockIdx.x + i gridDim.x, chunks 0..nq-1.
template <typename D>
struct PCursor {
    const D* d;
    int nitems, i = 0, q = 0, g = 0;
    PItem w{};
    bool done = false;
    __device__ __forceinline__ void start(const D* dd, int n) {
        d = dd;
        nitems = n;
        load();
    }
    // (every item has at least one chunk: the host builds no other)
    __device__ __forceinline__ void load() {
        const int it = (int)blockIdx.x + i * (int)gridDim.x;
        if (it >= nitems) {
            done = true;
            return;
        }
        w = d->item(it);
    }
    __device__ __forceinline__ void next() {
        ++g;
        if (++q >= w.nq) {
            q = 0;
            ++i;
            load();
        }
    }
};

// control lane of a persistent launch
template <typename D>
__device__ __forceinline__ void wsp_control(WSP* ws, const D& d, int nitems, const CUtensorMap* map,
                                            unsigned char* sA0, uint32_t a_stage, uint32_t a_plane, unsigned char* sB0,
                                            uint32_t b_stride, int NB, unsigned char* raw, uint32_t raw_stage, int NR,
                                            uint32_t tmem, int nsets) {
    volatile int* ab = &ws->abort;
    PCursor<D> rc, bc, mc;               // raw tiles, table tiles, MMAs
    rc.start(&d, nitems);
    bc.start(&d, nitems);
    mc.start(&d, nitems);
    auto issue_raw = [&]() {
        uint64_t* bar = &ws->r_full[rc.g % NR];
        mbar_expect_tx(bar, raw_stage);
        d.raw(map, raw + (size_t)(rc.g % NR) * raw_stage, rc.w, rc.q, bar);
        rc.next();
    };
    for (int c = 0; c < NR && !rc.done; ++c) issue_raw();
    const int D_AHEAD = NB - 2;
    bool ok = true;
    auto issue_b = [&]() {
        if (bc.g >= NB) {
            ok = ws_wait(&ws->b_empty[bc.g % NB], ((bc.g / NB) - 1) & 1, ab);
            if (!ok) return;
        }
        uint32_t bytes;
        const unsigned char* src = d.btile(bc.w, bc.q, bytes);
        mbar_expect_tx(&ws->b_full[bc.g % NB], bytes);
        bulk_g2s(sB0 + (size_t)(bc.g % NB) * b_stride, src, bytes, &ws->b_full[bc.g % NB]);
        bc.next();
    };
    while (ok && !bc.done && bc.g < D_AHEAD) issue_b();
    int last_mma = -1, item_i = -1;
    uint32_t idesc = 0, acc_base = 0;
    int acc_stride = 0;
    while (ok && !mc.done) {
        if (mc.q == 0) {                                  // first chunk of local item mc.i
            item_i = mc.i;
            const int s = item_i % nsets;
            if (item_i >= nsets) {
                ok = ws_wait(&ws->acc_empty[s], ((item_i / nsets) - 1) & 1, ab);
                if (!ok) break;
            }
            idesc = make_idesc((int)d.nt_of(mc.w));
            acc_stride = d.acc_of(mc.w);
            acc_base = tmem + (uint32_t)s * (TMEM_COLS / nsets);
        }
        const int g = mc.g;
        while (ok && !bc.done && bc.g < g + D_AHEAD + 1) issue_b();
        if (!ok) break;
        ok = ws_wait(&ws->a_full[g & 1], (g >> 1) & 1, ab);
        if (!ok) break;
        if (!rc.done) issue_raw();                        // raw stage of chunk g is free again
        ok = ws_wait(&ws->b_full[g % NB], (g / NB) & 1, ab);
        if (!ok) break;
        tc_fence_after();
        issue_mmas(sA0 + (g & 1) * a_stage, a_plane, sB0 + (size_t)(g % NB) * b_stride,
                   d.nt_of(mc.w) * KC * 2, acc_base, acc_stride, idesc, mc.q == 0);
        mma_commit(&ws->a_empty[g & 1]);
        mma_commit(&ws->b_empty[g % NB]);
        last_mma = g;
        const bool last_of_item = (mc.q + 1 >= mc.w.nq);
        mc.next();
        if (last_of_item) mma_commit(&ws->acc_full[item_i % nsets]);
    }
    if (ok) return;
    *ab = 1;
    // bounded drain of this CTA's own work in flight: the last MMAs, the table tiles and raw
    // tiles issued but not consumed
    volatile int zero = 0;
    if (last_mma >= 0) ws_wait(&ws->a_empty[last_mma & 1], (last_mma >> 1) & 1, &zero);
    for (int c = last_mma + 1; c < bc.g; ++c) ws_wait(&ws->b_full[c % NB], (c / NB) & 1, &zero);
    for (int c = last_mma + 1; c < rc.g; ++c) ws_wait(&ws->r_full[c % NR], (c / NR) & 1, &zero);
}

// epilogue warp: wait for item i's accumulators (lane 0, broadcast)
__device__ __forceinline__ bool wsp_acc_wait(WSP* ws, int i, int nsets, int lane) {
    bool ok = true;
    if (lane == 0) ok = ws_wait(&ws->acc_full[i % nsets], (i / nsets) & 1, &ws->abort);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    tc_fence_after();
    return ok;
}
__device__ __forceinline__ void wsp_acc_release(WSP* ws, int i, int nsets, int lane) {
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ws->acc_empty[i % nsets]);
}

__global__ void __launch_bounds__(NTHP, 1) k_leg_inv_tcp(float* __restrict__ F, PInv d, int nitems, int ncol,
                                                        int nlat, int nlat2, int NB, int nsets, int* err,
                                                        const __grid_constant__ CUtensorMap tmX) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nt = d.nt;
    const uint32_t a_plane = BM * KC * 2;
    const uint32_t b_plane = (uint32_t)nt * KC * 2;
    const uint32_t a_stage = 2 * NPLANE * a_plane;
    const uint32_t b_stage = 2 * NPLANE * b_plane;
    const uint32_t raw_stage = 2 * KC * BM * 4;
    unsigned char* const sA0 = smem;
    unsigned char* sB0 = smem + 2 * a_stage;
    float* raw = reinterpret_cast<float*>(sB0 + (size_t)NB * b_stage);   // [NR][32 rows][BM]
    WSP* ws = reinterpret_cast<WSP*>(raw + NR_INV * 2 * KC * BM);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem = wsp_setup(ws, tid);
    if (warp == NCV / 32) {
        if (lane == 0)
            wsp_control(ws, d, nitems, &tmX, sA0, a_stage, a_plane, sB0, b_stage, NB,
                        reinterpret_cast<unsigned char*>(raw), raw_stage, NR_INV, tmem, nsets);
    } else if (warp < NCV / 32) {
        const int col = tid & (BM - 1), sub = (tid >> 7) & 3;
        PCursor<PInv> cc;
        cc.start(&d, nitems);
        while (!cc.done) {
            const int g = cc.g, q = cc.q;
            const int Kx = d.M + 2 - cc.w.m;
            if (!ws_raw_wait(ws, &ws->r_full[g % NR_INV], (g / NR_INV) & 1)) break;
            if (g >= 2 && !ws_warp_wait(ws, &ws->a_empty[g & 1], ((g - 2) >> 1) & 1, lane)) break;
            const float* r = raw + (g % NR_INV) * (2 * KC * BM);
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                float v[KQ];
#pragma unroll
                for (int i = 0; i < KQ; ++i) {
                    const int kk = KQ * sub + i;
                    const float x = r[(par + 2 * kk) * BM + col];
                    v[i] = par + 2 * (KC * q + kk) < Kx ? x : 0.f;
                }
                store_quad_planes(sA0 + (g & 1) * a_stage + par * NPLANE * a_plane, a_plane, col, KQ * sub, v);
            }
            ws_planes_ready(ws, g, lane);
            cc.next();
        }
    } else {
        // epilogue warps: TMEM lanes (= data columns) 32 (warp mod 4) .. + 31
        const int quarter = warp & 3;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        for (int i = 0;; ++i) {
            const int it = (int)blockIdx.x + i * (int)gridDim.x;
            if (it >= nitems) break;
            const PItem w = d.item(it);
            if (!wsp_acc_wait(ws, i, nsets, lane)) break;
            const uint32_t base = tmem + (uint32_t)(i % nsets) * (TMEM_COLS / nsets) + lane_base;
            const int c = w.x * BM + quarter * 32 + lane;
            const bool cin = c < ncol;
            const int jt0 = w.z * nt;
            float* Fm = F + (int64_t)w.m * nlat * ncol + c;
            for (int j0 = 0; j0 < nt; j0 += 32) {
                float e[32], o[32];
                tmem_ld32(base + (uint32_t)j0, e);
                tmem_ld32(base + (uint32_t)(nt + j0), o);
                if (cin) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int j = jt0 + j0 + k;
                        if (j < nlat2) {
                            Fm[(int64_t)j * ncol] = e[k] + o[k];
                            Fm[(int64_t)(nlat - 1 - j) * ncol] = e[k] - o[k];
                        }
                    }
                }
            }
            wsp_acc_release(ws, i, nsets, lane);
        }
    }
    __syncthreads();
    if (ws->abort && tid == 0) atomicOr(err, PLAN_FLAG_TIMEOUT);
    tmem_release(tmem, tid);
}

__global__ void __launch_bounds__(NTHP, 1) k_leg_fwd_tcp(float* __restrict__ Y, PFwd d, int nitems, int ncol,
                                                        int nlat2, int b_stage_max, int NB, int nsets, int* err,
                                                        const __grid_constant__ CUtensorMap tmF) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t a_plane = BM * KC * 2;
    const uint32_t a_stage = 2 * NPLANE * a_plane;
    const uint32_t raw_stage = 2 * KC * BM * 4;
    unsigned char* const sA0 = smem;
    unsigned char* sB0 = smem + 2 * a_stage;               // NB stages of b_stage_max bytes
    float* raw = reinterpret_cast<float*>(sB0 + (size_t)NB * b_stage_max);   // [NR][2 KC][BM]
    WSP* ws = reinterpret_cast<WSP*>(raw + NR_FWD * 2 * KC * BM);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem = wsp_setup(ws, tid);
    if (warp == NCV / 32) {
        if (lane == 0)
            wsp_control(ws, d, nitems, &tmF, sA0, a_stage, a_plane, sB0, (uint32_t)b_stage_max, NB,
                        reinterpret_cast<unsigned char*>(raw), raw_stage, NR_FWD, tmem, nsets);
    } else if (warp < NCV / 32) {
        const int col = tid & (BM - 1), sub = (tid >> 7) & 3;
        PCursor<PFwd> cc;
        cc.start(&d, nitems);
        while (!cc.done) {
            const int g = cc.g, q = cc.q;
            if (!ws_raw_wait(ws, &ws->r_full[g % NR_FWD], (g / NR_FWD) & 1)) break;
            if (g >= 2 && !ws_warp_wait(ws, &ws->a_empty[g & 1], ((g - 2) >> 1) & 1, lane)) break;
            const float* r = raw + (g % NR_FWD) * (2 * KC * BM);
            float vs[KQ], va[KQ];
#pragma unroll
            for (int i = 0; i < KQ; ++i) {
                const int jj = KQ * sub + i;
                // rows j >= nlat/2 of the last chunk are the other hemisphere's: dropped
                const bool in = KC * q + jj < nlat2;
                const float fn = in ? r[jj * BM + col] : 0.f;
                const float fs = in ? r[(2 * KC - 1 - jj) * BM + col] : 0.f;
                vs[i] = fn + fs;
                va[i] = fn - fs;
            }
            store_quad_planes(sA0 + (g & 1) * a_stage, a_plane, col, KQ * sub, vs);
            store_quad_planes(sA0 + (g & 1) * a_stage + NPLANE * a_plane, a_plane, col, KQ * sub, va);
            ws_planes_ready(ws, g, lane);
            cc.next();
        }
    } else {
        const int quarter = warp & 3;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        for (int i = 0;; ++i) {
            const int it = (int)blockIdx.x + i * (int)gridDim.x;
            if (it >= nitems) break;
            const PItem w = d.item(it);
            if (!wsp_acc_wait(ws, i, nsets, lane)) break;
            const int nt = (int)d.nt_of(w), acc = d.acc_of(w);
            const uint32_t base = tmem + (uint32_t)(i % nsets) * (TMEM_COLS / nsets) + lane_base;
            const int c = w.x * BM + quarter * 32 + lane;
            const bool cin = c < ncol;
            const int kt0 = w.z * nt;
            const int Kx = d.M + 2 - w.m;
            float* Ym = Y + ex_off(w.m, d.M) * (int64_t)ncol + c;
            for (int k0 = 0; k0 < nt; k0 += 32) {
                float d0[32], d1[32];
                tmem_ld32(base + (uint32_t)k0, d0);
                tmem_ld32(base + (uint32_t)(acc + k0), d1);
                if (cin) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int kk = kt0 + k0 + k;
                        const int r0 = 2 * kk, r1 = 2 * kk + 1;   // extended-row offsets of parities 0 / 1
                        if (k0 + k < nt) {
                            if (r0 < Kx) Ym[(int64_t)r0 * ncol] = d0[k];
                            if (r1 < Kx) Ym[(int64_t)r1 * ncol] = d1[k];
                        }
                    }
                }
            }
            wsp_acc_release(ws, i, nsets, lane);
        }
    }
    __syncthreads();
    if (ws->abort && tid == 0) atomicOr(err, PLAN_FLAG_TIMEOUT);
    tmem_release(tmem, tid);
}

// ----------------------------------------------------------------------------- table builders
// Inverse table: element (j, kk) of tile (m, q, tile z, par, plane) = P_{m+par+2(16q+kk)}(mu_{16... j})
__global__ void k_build_inv_table(const double* __restrict__ P, unsigned char* __restrict__ T,
                                  const long long* __restrict__ inv_off, const int* __restrict__ inv_nq, int M,
                                  int nlat2, int nt, int ntiles) {
    const int m = blockIdx.y;
    const int nq = inv_nq[m];
    const uint32_t b_plane = (uint32_t)nt * KC * 2;
    const int64_t total = (int64_t)nq * ntiles * 2 * nt * KC;
    const int Kx = M + 2 - m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int kk = (int)(t % KC);
        int64_t r = t / KC;
        int row = (int)(r % nt);
        r /= nt;
        int par = (int)(r % 2);
        r /= 2;
        int z = (int)(r % ntiles);
        int q = (int)(r / ntiles);
        int j = z * nt + row;
        int rr = par + 2 * (KC * q + kk);
        double v = (j < nlat2 && rr < Kx) ? P[(ex_off(m, M) + rr) * nlat2 + j] : 0.0;
        __nv_bfloat16 h0, h1, h2;
        split3((float)v, h0, h1, h2);
        unsigned char* tile = T + inv_off[m] + (((int64_t)q * ntiles + z) * 2 + par) * NPLANE * b_plane;
        uint32_t off = tile_off(row, kk);
        *reinterpret_cast<__nv_bfloat16*>(tile + off) = h0;
        *reinterpret_cast<__nv_bfloat16*>(tile + b_plane + off) = h1;
        *reinterpret_cast<__nv_bfloat16*>(tile + 2 * b_plane + off) = h2;
    }
}

// Forward table: element (k, jj) of tile (m, q, tile z, par, plane) = P_{m+par+2k}(mu_{16q+jj}),
// k = z*nt_m + row
__global__ void k_build_fwd_table(const double* __restrict__ P, unsigned char* __restrict__ T,
                                  const long long* __restrict__ fwd_off, const int* __restrict__ fwd_ntiles,
                                  const int* __restrict__ fwd_nt, int M, int nlat2) {
    const int m = blockIdx.y;
    const int nz = fwd_ntiles[m];
    const int nt = fwd_nt[m];
    const int nq = (nlat2 + KC - 1) / KC;
    const uint32_t b_plane = (uint32_t)nt * KC * 2;
    const int64_t total = (int64_t)nq * nz * 2 * nt * KC;
    const int Kx = M + 2 - m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int jj = (int)(t % KC);
        int64_t r = t / KC;
        int row = (int)(r % nt);
        r /= nt;
        int par = (int)(r % 2);
        r /= 2;
        int z = (int)(r % nz);
        int q = (int)(r / nz);
        int k = z * nt + row;
        int j = KC * q + jj;
        int rr = par + 2 * k;
        double v = (j < nlat2 && rr < Kx) ? P[(ex_off(m, M) + rr) * nlat2 + j] : 0.0;
        __nv_bfloat16 h0, h1, h2;
        split3((float)v, h0, h1, h2);
        unsigned char* tile = T + fwd_off[m] + (((int64_t)q * nz + z) * 2 + par) * NPLANE * b_plane;
        uint32_t off = tile_off(row, jj);
        *reinterpret_cast<__nv_bfloat16*>(tile + off) = h0;
        *reinterpret_cast<__nv_bfloat16*>(tile + b_plane + off) = h1;
        *reinterpret_cast<__nv_bfloat16*>(tile + 2 * b_plane + off) = h2;
    }
}

}  // namespace

// ----------------------------------------------------------------------------- host side
struct SplitTables {
    int nt_inv, ntiles_inv, nt_fwd, nz_fwd;   // nt_fwd, nz_fwd: largest over m
    int* inv_pairs = nullptr;                 // persistent work lists: m | z << 16, m ascending
    int* fwd_pairs = nullptr;
    int n_inv_pairs = 0, n_fwd_pairs = 0;
    size_t smem_inv_p = 0, smem_fwd_p = 0;    // persistent kernels
    int nb_inv_p = 2, nb_fwd_p = 2;
    // autotuned choice per direction and real column count: 1 persistent, 2 per tile, with the
    // two measured times (ms; 0 when not measured)
    struct Tune {
        int ncol, choice;
        float ms_persist, ms_tile;
    };
    std::vector<Tune> tune[2];                // [0] inverse, [1] forward
    // batches of at most 8 complex columns: 1 the FP32 SIMT kernel, 2 the tensor-core path
    // (ms_persist: SIMT time, ms_tile: tensor-core time)
    std::vector<Tune> narrow[2];
    unsigned char* inv = nullptr;
    unsigned char* fwd = nullptr;
    long long* inv_off = nullptr;
    int* inv_nq = nullptr;
    long long* fwd_off = nullptr;
    int* fwd_ntiles = nullptr;
    int* fwd_nt = nullptr;
    size_t smem_inv = 0, smem_fwd = 0;
    int nb_inv = 2, nb_fwd = 2;               // table-tile ring depths
};

static int round16(int x) { return (x + 15) / 16 * 16; }

constexpr size_t SMEM_LIMIT = 227 * 1024;

// planes (2 stages) + table tiles (nb stages) + raw prefetch ring + barriers
static size_t tc_smem(int nt, size_t raw_stage, int nr, int nb) {
    size_t a_stage = 2 * NPLANE * BM * KC * 2, b_stage = 2 * NPLANE * (size_t)nt * KC * 2;
    return 2 * a_stage + (size_t)nb * b_stage + (size_t)nr * raw_stage + sizeof(WS) + 64;
}

// deepest table-tile ring (<= NB_MAX) that fits the shared-memory limit; 0 if even 2 do not
static int tc_nb(int nt, size_t raw_stage, int nr) {
    for (int nb = NB_MAX; nb >= 2; --nb)
        if (tc_smem(nt, raw_stage, nr, nb) <= SMEM_LIMIT) return nb;
    return 0;
}
static size_t tcp_smem(int nt, size_t raw_stage, int nr, int nb) {
    return tc_smem(nt, raw_stage, nr, nb) - sizeof(WS) + sizeof(WSP);
}
static int tcp_nb(int nt, size_t raw_stage, int nr) {
    for (int nb = NB_MAX; nb >= 2; --nb)
        if (tcp_smem(nt, raw_stage, nr, nb) <= SMEM_LIMIT) return nb;
    return 0;
}

swe_status split_tables_build(swe_plan* p) {
    if (p->Pbf) return SWE_OK;
    SplitTables* t = new SplitTables();
    const int M = p->M;
    // inverse: N tiles over the northern latitudes, at most 192 (equal tiles, multiples of 32
    // for the epilogue's 32-column reads), so that the table stages and the raw prefetch ring
    // fit in shared memory
    int ntiles = (p->nlat2 + 191) / 192;
    t->ntiles_inv = ntiles;
    t->nt_inv = round16((p->nlat2 + ntiles - 1) / ntiles);
    if (t->nt_inv % 32) t->nt_inv = (t->nt_inv + 31) / 32 * 32;   // epilogue reads 32 columns at a time
    // forward: N tiles over the degree index within a parity, sized per m to its
    // K_par = ceil((M + 2 - m) / 2) degrees (multiple of 16, at most NT_MAX)
    std::vector<long long> ioff(M + 1), foff(M + 1);
    std::vector<int> inq(M + 1), fnt(M + 1), fnz(M + 1);
    const int nqf = (p->nlat2 + KC - 1) / KC;
    t->nt_fwd = 16;
    t->nz_fwd = 1;
    long long oi = 0, of = 0;
    const long long binv = 2LL * NPLANE * t->nt_inv * KC * 2;
    for (int m = 0; m <= M; ++m) {
        int Kx = M + 2 - m;                 // extended rows
        int Kpar = (Kx + 1) / 2;            // rows in the larger parity
        inq[m] = (Kpar + KC - 1) / KC;
        ioff[m] = oi;
        oi += (long long)inq[m] * ntiles * binv;
        fnz[m] = (Kpar + NT_MAX - 1) / NT_MAX;
        fnt[m] = round16((Kpar + fnz[m] - 1) / fnz[m]);
        t->nt_fwd = std::max(t->nt_fwd, fnt[m]);
        t->nz_fwd = std::max(t->nz_fwd, fnz[m]);
        foff[m] = of;
        of += (long long)nqf * fnz[m] * 2LL * NPLANE * fnt[m] * KC * 2;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->inv, oi);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->fwd, of);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->inv_off, sizeof(long long) * (M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->inv_nq, sizeof(int) * (M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->fwd_off, sizeof(long long) * (M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->fwd_ntiles, sizeof(int) * (M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->fwd_nt, sizeof(int) * (M + 1));
    if (e == cudaSuccess) e = cudaMemcpy(t->inv_off, ioff.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->inv_nq, inq.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->fwd_off, foff.data(), sizeof(long long) * (M + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->fwd_ntiles, fnz.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->fwd_nt, fnt.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice);
    // work lists of the persistent kernels, m ascending (the inverse's longest K first)
    std::vector<int> ipairs, fpairs;
    for (int m = 0; m <= M; ++m) {
        for (int z = 0; z < ntiles; ++z) ipairs.push_back(m | (z << 16));
        for (int z = 0; z < fnz[m]; ++z) fpairs.push_back(m | (z << 16));
    }
    t->n_inv_pairs = (int)ipairs.size();
    t->n_fwd_pairs = (int)fpairs.size();
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->inv_pairs, sizeof(int) * ipairs.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->fwd_pairs, sizeof(int) * fpairs.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(t->inv_pairs, ipairs.data(), sizeof(int) * ipairs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->fwd_pairs, fpairs.data(), sizeof(int) * fpairs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(t->inv);
        cudaFree(t->fwd);
        cudaFree(t->inv_off);
        cudaFree(t->inv_nq);
        cudaFree(t->fwd_off);
        cudaFree(t->fwd_ntiles);
        cudaFree(t->fwd_nt);
        cudaFree(t->inv_pairs);
        cudaFree(t->fwd_pairs);
        delete t;
        return swe_cuda_status(e, "split tables");
    }
    k_build_inv_table<<<dim3(256, M + 1), 256>>>(p->P, t->inv, t->inv_off, t->inv_nq, M, p->nlat2, t->nt_inv,
                                                  ntiles);
    k_build_fwd_table<<<dim3(256, M + 1), 256>>>(p->P, t->fwd, t->fwd_off, t->fwd_ntiles, t->fwd_nt, M, p->nlat2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    t->nb_inv = tc_nb(t->nt_inv, 2 * KC * BM * sizeof(float), NR_INV);
    t->nb_fwd = tc_nb(t->nt_fwd, 2 * KC * BM * sizeof(float), NR_FWD);
    if (t->nb_inv == 0 || t->nb_fwd == 0) {
        p->Pbf = t;
        swe_set_error("split tables: shared-memory footprint of the tensor-core kernels exceeds 227 KB");
        return SWE_EINVAL;
    }
    t->smem_inv = tc_smem(t->nt_inv, 2 * KC * BM * sizeof(float), NR_INV, t->nb_inv);
    t->smem_fwd = tc_smem(t->nt_fwd, 2 * KC * BM * sizeof(float), NR_FWD, t->nb_fwd);
    // at least ~116 KB of shared memory so that a single CTA (holding all 512 TMEM columns) runs per SM
    const size_t one_per_sm = 116 * 1024;
    if (t->smem_inv < one_per_sm) t->smem_inv = one_per_sm;
    if (t->smem_fwd < one_per_sm) t->smem_fwd = one_per_sm;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_leg_inv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_inv);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_leg_inv_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_inv);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_leg_fwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_fwd);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_leg_fwd_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_fwd);
    t->nb_inv_p = tcp_nb(t->nt_inv, 2 * KC * BM * sizeof(float), NR_INV);
    t->nb_fwd_p = tcp_nb(t->nt_fwd, 2 * KC * BM * sizeof(float), NR_FWD);
    t->smem_inv_p = t->nb_inv_p ? tcp_smem(t->nt_inv, 2 * KC * BM * sizeof(float), NR_INV, t->nb_inv_p) : 0;
    t->smem_fwd_p = t->nb_fwd_p ? tcp_smem(t->nt_fwd, 2 * KC * BM * sizeof(float), NR_FWD, t->nb_fwd_p) : 0;
    if (t->smem_inv_p && t->smem_inv_p < one_per_sm) t->smem_inv_p = one_per_sm;
    if (t->smem_fwd_p && t->smem_fwd_p < one_per_sm) t->smem_fwd_p = one_per_sm;
    p->Pbf = t;
    if (e != cudaSuccess) return swe_cuda_status(e, "split table kernels");
    return SWE_OK;
}

void split_tables_free(swe_plan* p) {
    SplitTables* t = (SplitTables*)p->Pbf;
    if (!t) return;
    cudaFree(t->inv);
    cudaFree(t->fwd);
    cudaFree(t->inv_off);
    cudaFree(t->inv_nq);
    cudaFree(t->fwd_off);
    cudaFree(t->fwd_ntiles);
    cudaFree(t->fwd_nt);
    cudaFree(t->inv_pairs);
    cudaFree(t->fwd_pairs);
    delete t;
    p->Pbf = nullptr;
}

// ----------------------------------------------------------------------------- tensor maps
// cuTensorMapEncodeTiled is a driver entry point; it is looked up once through the runtime so
// that the library needs no link-time dependency on the driver library.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Row-major FP32 matrix [rows][ncol] read in boxes of 128 columns x box_rows rows.  Usable when
// the row pitch and the base are multiples of 16 bytes (the tensor-map rules); out-of-range
// rows and columns read as zero.  Returns false (map untouched) when TMA cannot be used.
static bool encode_rows(CUtensorMap* map, const float* base, int ncol, long long rows, int box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || ncol % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || rows <= 0 || rows >= (1LL << 31))
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ncol, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ncol * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)BM, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            v = 0;
        return v > 0 ? v : 1;
    }();
    return n;
}

// Kernel variant for one direction and real column count.  Mode 1 / 2 force the persistent /
// per-tile kernel.  Mode 0: the first call with this column count outside stream capture runs
// both variants twice on the call's own operands (the kernels only read the input and write
// the output), times the second run of each with CUDA events on the call's stream and keeps
// the faster; a call under capture before that takes the persistent kernel untimed.
template <typename A, typename B>
static swe_status legendre_choice(const swe_plan* p, SplitTables* t, int dir, int ncol, cudaStream_t st, A& persistent,
                                  B& per_tile, int* choice) {
    if (p->legendre_mode == 1 || p->legendre_mode == 2) {
        *choice = p->legendre_mode;
        return SWE_OK;
    }
    for (const auto& e : t->tune[dir])
        if (e.ncol == ncol) {
            *choice = e.choice;
            return SWE_OK;
        }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SWE_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        *choice = 1;
        return SWE_OK;
    }
    cudaEvent_t e0, e1;
    SWE_CHECK_CUDA(cudaEventCreate(&e0));
    SWE_CHECK_CUDA(cudaEventCreate(&e1));
    float ms[2] = {0.f, 0.f};
    swe_status r = SWE_OK;
    for (int v = 0; v < 2 && r == SWE_OK; ++v)
        for (int rep = 0; rep < 2 && r == SWE_OK; ++rep) {
            cudaEventRecord(e0, st);
            r = v == 0 ? persistent() : per_tile();
            cudaEventRecord(e1, st);
            if (r == SWE_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms[v], e0, e1);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SWE_CHECK(r);
    *choice = ms[0] <= ms[1] ? 1 : 2;
    t->tune[dir].push_back(SplitTables::Tune{ncol, *choice, ms[0], ms[1]});
    return SWE_OK;
}

swe_status leg_inverse_split(const swe_plan* p, const float2* X, float2* F, int C, cudaStream_t st) {
    SplitTables* t = (SplitTables*)p->Pbf;
    if (!t) {
        swe_set_error("split-precision tables missing");
        return SWE_EINVAL;
    }
    TCShape sh{p->M, p->nlat, p->nlat2, 2 * C, t->nt_inv};
    dim3 grid((sh.ncol + BM - 1) / BM, p->M + 1, t->ntiles_inv);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 8.0 * C * p->ncx + 8.0 * C * (p->M + 1.0) * p->nlat;
    alignas(64) CUtensorMap tm{};
    const bool tma = p->nlat2 >= KC && encode_rows(&tm, (const float*)X, sh.ncol, p->ncx, 2 * KC);
    const int nx = (sh.ncol + BM - 1) / BM;
    auto persistent = [&]() -> swe_status {
        // one CTA per SM over (column tile, m, N tile) items
        const int nitems = nx * t->n_inv_pairs;
        const int grid_p = nitems < sm_count() ? nitems : sm_count();
        PInv d{t->inv, t->inv_off, t->inv_nq, t->inv_pairs, nx, p->M, t->nt_inv, t->ntiles_inv};
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_inv_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)t->smem_inv_p));
        const int nsets = 2 * t->nt_inv <= (int)TMEM_COLS / 2 ? 2 : 1;
        k_leg_inv_tcp<<<grid_p, NTHP, t->smem_inv_p, st>>>((float*)F, d, nitems, sh.ncol, p->nlat, p->nlat2,
                                                            t->nb_inv_p, nsets, p->flags, tm);
        SWE_CHECK_LAUNCH("k_leg_inv_tcp");
        return SWE_OK;
    };
    auto per_tile = [&]() -> swe_status {
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_inv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)t->smem_inv));
        k_leg_inv_tc<true><<<grid, NTH, t->smem_inv, st>>>((const float*)X, (float*)F, t->inv, t->inv_off, t->inv_nq,
                                                            sh, t->nb_inv, p->flags, tm);
        SWE_CHECK_LAUNCH("k_leg_inv_tc");
        return SWE_OK;
    };
    if (tma && t->smem_inv_p) {
        int choice = 0;
        SWE_CHECK(legendre_choice(p, t, 0, sh.ncol, st, persistent, per_tile, &choice));
        ProfToken tk = prof_begin("leg_inv_tc", st, fl, by);
        const swe_status r = choice == 1 ? persistent() : per_tile();
        prof_end(tk, st);
        return r;
    }
    auto kern = tma ? k_leg_inv_tc<true> : k_leg_inv_tc<false>;
    // the dynamic shared-memory limit is a per-function attribute shared by all plans: set it per launch
    SWE_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_inv));
    ProfToken tk = prof_begin("leg_inv_tc", st, fl, by);
    kern<<<grid, NTH, t->smem_inv, st>>>((const float*)X, (float*)F, t->inv, t->inv_off, t->inv_nq, sh, t->nb_inv,
                                         p->flags, tm);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_inv_tc");
    return SWE_OK;
}

swe_status leg_forward_split(const swe_plan* p, const float2* F, float2* Y, int C, cudaStream_t st) {
    SplitTables* t = (SplitTables*)p->Pbf;
    if (!t) {
        swe_set_error("split-precision tables missing");
        return SWE_EINVAL;
    }
    TCShape sh{p->M, p->nlat, p->nlat2, 2 * C, t->nt_fwd};
    dim3 grid((sh.ncol + BM - 1) / BM, p->M + 1, t->nz_fwd);
    const double fl = (double)C * p->nlat * (p->M + 1.0) * (p->M + 2.0);
    const double by = 8.0 * C * (p->M + 1.0) * p->nlat + 8.0 * C * p->ncx;
    alignas(64) CUtensorMap tm{};
    const bool tma =
        p->nlat2 >= KC && encode_rows(&tm, (const float*)F, sh.ncol, (long long)(p->M + 1) * p->nlat, KC);
    const int nx = (sh.ncol + BM - 1) / BM;
    auto persistent = [&]() -> swe_status {
        const int nitems = nx * t->n_fwd_pairs;
        const int grid_p = nitems < sm_count() ? nitems : sm_count();
        PFwd d{t->fwd, t->fwd_off, t->fwd_ntiles, t->fwd_nt, t->fwd_pairs, nx, p->M, p->nlat, (p->nlat2 + KC - 1) / KC};
        const int b_stage_max = 2 * NPLANE * t->nt_fwd * KC * 2;
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_fwd_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)t->smem_fwd_p));
        const int nsets = 2 * ((t->nt_fwd + 31) & ~31) <= (int)TMEM_COLS / 2 ? 2 : 1;
        k_leg_fwd_tcp<<<grid_p, NTHP, t->smem_fwd_p, st>>>((float*)Y, d, nitems, sh.ncol, p->nlat2, b_stage_max,
                                                            t->nb_fwd_p, nsets, p->flags, tm);
        SWE_CHECK_LAUNCH("k_leg_fwd_tcp");
        return SWE_OK;
    };
    auto per_tile = [&]() -> swe_status {
        SWE_CHECK_CUDA(cudaFuncSetAttribute(k_leg_fwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)t->smem_fwd));
        k_leg_fwd_tc<true><<<grid, NTH, t->smem_fwd, st>>>((const float*)F, (float*)Y, t->fwd, t->fwd_off,
                                                            t->fwd_ntiles, t->fwd_nt, sh, t->nb_fwd, p->flags, tm);
        SWE_CHECK_LAUNCH("k_leg_fwd_tc");
        return SWE_OK;
    };
    if (tma && t->smem_fwd_p) {
        int choice = 0;
        SWE_CHECK(legendre_choice(p, t, 1, sh.ncol, st, persistent, per_tile, &choice));
        ProfToken tk = prof_begin("leg_fwd_tc", st, fl, by);
        const swe_status r = choice == 1 ? persistent() : per_tile();
        prof_end(tk, st);
        return r;
    }
    auto kern = tma ? k_leg_fwd_tc<true> : k_leg_fwd_tc<false>;
    SWE_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem_fwd));
    ProfToken tk = prof_begin("leg_fwd_tc", st, fl, by);
    kern<<<grid, NTH, t->smem_fwd, st>>>((const float*)F, (float*)Y, t->fwd, t->fwd_off, t->fwd_ntiles, t->fwd_nt,
                                         sh, t->nb_fwd, p->flags, tm);
    prof_end(tk, st);
    SWE_CHECK_LAUNCH("k_leg_fwd_tc");
    return SWE_OK;
}

// Diagnostic of the bounded wait: one warp waits at most `polls` polls on an mbarrier that
// nothing completes, then records the timeout in the plan's status word, as the tensor-core
// kernels do when a copy or an MMA never signals.
__global__ void k_wait_selftest(int* flags, unsigned long long polls) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        abort = 0;
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!ws_wait_n(&bar, 0, &abort, polls)) atomicOr(flags, PLAN_FLAG_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
}

swe_status wait_selftest_launch(const swe_plan* p, long long polls, cudaStream_t st) {
    const unsigned long long n = polls < 1 ? 1ull : (polls > (long long)WAIT_LIMIT ? WAIT_LIMIT : (unsigned long long)polls);
    k_wait_selftest<<<1, 32, 0, st>>>(p->flags, n);
    SWE_CHECK_LAUNCH("k_wait_selftest");
    return SWE_OK;
}

// Batches of at most 8 complex columns (the serial chains) can take the FP32 SIMT contraction
// or the tensor-core path: which is faster depends on the truncation (the SIMT kernel wins at
// T255, the tensor cores at T511).  The first call per direction and column count outside
// stream capture runs both twice on its own operands, times the second run of each and keeps
// the faster; a call under capture before that takes the SIMT kernel.
swe_status leg_narrow_choice(const swe_plan* p, int dir, int C, const void* in, void* out, cudaStream_t st,
                             int* choice) {
    *choice = 1;
    SplitTables* t = (SplitTables*)p->Pbf;
    if (!t) return SWE_OK;
    for (const auto& e : t->narrow[dir])
        if (e.ncol == 2 * C) {
            *choice = e.choice;
            return SWE_OK;
        }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SWE_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SWE_OK;
    cudaEvent_t e0, e1;
    SWE_CHECK_CUDA(cudaEventCreate(&e0));
    SWE_CHECK_CUDA(cudaEventCreate(&e1));
    float ms[2] = {0.f, 0.f};
    swe_status r = SWE_OK;
    for (int v = 0; v < 2 && r == SWE_OK; ++v)
        for (int rep = 0; rep < 2 && r == SWE_OK; ++rep) {
            cudaEventRecord(e0, st);
            if (dir == 0)
                r = v == 0 ? leg_inverse_small(p, (const float*)in, (float*)out, C, st)
                           : leg_inverse_split(p, (const float2*)in, (float2*)out, C, st);
            else
                r = v == 0 ? leg_forward_small(p, (const float*)in, (float*)out, C, st)
                           : leg_forward_split(p, (const float2*)in, (float2*)out, C, st);
            cudaEventRecord(e1, st);
            if (r == SWE_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms[v], e0, e1);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SWE_CHECK(r);
    *choice = ms[0] <= ms[1] ? 1 : 2;
    t->narrow[dir].push_back(SplitTables::Tune{2 * C, *choice, ms[0], ms[1]});
    return SWE_OK;
}

// ----------------------------------------------------------------------------- C ABI: tuning
extern "C" swe_status swe_plan_set_legendre_mode(swe_plan_t p, int mode) {
    if (!p || mode < SWE_LEGENDRE_AUTO || mode > SWE_LEGENDRE_PER_TILE) {
        swe_set_error("swe_plan_set_legendre_mode: invalid argument");
        return SWE_EINVAL;
    }
    p->legendre_mode = mode;
    return SWE_OK;
}

extern "C" swe_status swe_plan_tuning(swe_plan_t p, char* buf, size_t len) {
    if (!p || !buf || len == 0) {
        swe_set_error("swe_plan_tuning: invalid argument");
        return SWE_EINVAL;
    }
    std::string out;
    char tmp[160];
    snprintf(tmp, sizeof tmp, "ring_nl: cfg %d G %d", p->ring_cfg, p->ring_G);
    out += tmp;
    const SplitTables* t = (const SplitTables*)p->Pbf;
    if (t) {
        snprintf(tmp, sizeof tmp, "; legendre mode %d, tiles inv nt %d x %d, fwd nt <= %d", p->legendre_mode, t->nt_inv,
                 t->ntiles_inv, t->nt_fwd);
        out += tmp;
        for (int dir = 0; dir < 2; ++dir)
            for (const auto& e : t->tune[dir]) {
                snprintf(tmp, sizeof tmp, "; %s ncol %d: %s (persistent %.3f ms, per tile %.3f ms)",
                         dir == 0 ? "inverse" : "forward", e.ncol, e.choice == 1 ? "persistent" : "per tile",
                         e.ms_persist, e.ms_tile);
                out += tmp;
            }
        for (int dir = 0; dir < 2; ++dir)
            for (const auto& e : t->narrow[dir]) {
                snprintf(tmp, sizeof tmp, "; %s ncol %d: %s (SIMT %.3f ms, tensor cores %.3f ms)",
                         dir == 0 ? "inverse" : "forward", e.ncol, e.choice == 1 ? "SIMT" : "tensor cores",
                         e.ms_persist, e.ms_tile);
                out += tmp;
            }
    }
    snprintf(buf, len, "%s", out.c_str());
    return SWE_OK;
}
