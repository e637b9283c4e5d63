// Kernel-launch accounting and optional per-kernel CUDA-event timing.
//
// Every launch site of the library calls prof_launch(); when timing is enabled
// the hot kernels are bracketed with events recorded on their own launch stream
// (launches inside a stream capture are counted but not timed).  Each timed
// launch also records its algorithmic FLOPs and bytes, so that a caller can
// form achieved TFLOP/s or GB/s per kernel.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "swe_internal.cuh"
#include "prof.cuh"

namespace {

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};

struct Pending {
    int kid;
    cudaEvent_t a, b;
    double flops, bytes;
};

struct KStat {
    std::string name;
    long long launches = 0;
    double ms = 0, flops = 0, bytes = 0;
};

std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<KStat> g_stats;

int kernel_id(const char* name) {
    for (size_t i = 0; i < g_stats.size(); ++i)
        if (g_stats[i].name == name) return (int)i;
    g_stats.push_back(KStat{name});
    return (int)g_stats.size() - 1;
}

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return true;
    return cs != cudaStreamCaptureStatusNone;
}

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            KStat& s = g_stats[p.kid];
            s.launches += 1;
            s.ms += ms;
            s.flops += p.flops;
            s.bytes += p.bytes;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

}  // namespace

bool prof_enabled() { return g_enabled.load() != 0; }


void prof_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfToken prof_begin(const char* name, cudaStream_t st, double flops, double bytes) {
    ProfToken t{-1, nullptr, nullptr, 0, 0};
    if (!g_enabled.load(std::memory_order_relaxed) || capturing(st)) return t;
    std::lock_guard<std::mutex> lk(g_mu);
    t.kid = kernel_id(name);
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    cudaEventRecord(t.a, st);
    t.flops = flops;
    t.bytes = bytes;
    return t;
}

void prof_end(const ProfToken& t, cudaStream_t st) {
    if (t.kid < 0) return;
    cudaEventRecord(t.b, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(Pending{t.kid, t.a, t.b, t.flops, t.bytes});
    if (g_pending.size() > 4096) drain_locked();
}

extern "C" long long swe_launch_count(void) { return g_launches.load(); }

extern "C" int swe_prof_enable(int on) {
    int old = g_enabled.exchange(on ? 1 : 0);
    return old;
}

extern "C" void swe_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    g_stats.clear();
}

extern "C" int swe_prof_read(int idx, char* name, int namelen, long long* launches, double* total_ms, double* flops,
                             double* bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    if (idx < 0 || idx >= (int)g_stats.size()) return 0;
    const KStat& s = g_stats[idx];
    if (name && namelen > 0) {
        strncpy(name, s.name.c_str(), namelen - 1);
        name[namelen - 1] = 0;
    }
    if (launches) *launches = s.launches;
    if (total_ms) *total_ms = s.ms;
    if (flops) *flops = s.flops;
    if (bytes) *bytes = s.bytes;
    return 1;
}
