// Launch accounting / event timing used by every launch site (see prof.cu).
#pragma once
#include <cuda_runtime.h>

struct ProfToken {
    int kid;
    cudaEvent_t a, b;
    double flops, bytes;
};

void prof_launch(long long n = 1);
// true while per-kernel event timing is on (captured launches cannot be timed)
bool prof_enabled();
ProfToken prof_begin(const char* name, cudaStream_t st, double flops, double bytes);
void prof_end(const ProfToken& t, cudaStream_t st);
