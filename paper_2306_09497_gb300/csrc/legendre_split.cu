// Split-precision Legendre contraction (placeholder until the tcgen05 kernels land).
#include "swe_internal.cuh"

swe_status leg_inverse_split(const swe_plan*, const double2*, float2*, int, cudaStream_t) {
    swe_set_error("split-precision Legendre transform is not built yet");
    return SWE_EINVAL;
}

swe_status leg_forward_split(const swe_plan*, const float2*, double2*, int, cudaStream_t) {
    swe_set_error("split-precision Legendre transform is not built yet");
    return SWE_EINVAL;
}
