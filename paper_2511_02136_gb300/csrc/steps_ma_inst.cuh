// steps_ma_inst.cuh -- instantiates the several-agents step kernel of one
// capacity class (K = LOB_K slots per lane per side), plain and traced, in
// the wide register budget, in a translation unit of its own.
#include "lob_device.cuh"
#include "lob_steps.h"

#define LOB_CAT2(a, b) a##b
#define LOB_CAT(a, b) LOB_CAT2(a, b)

namespace lobk {
cudaError_t LOB_CAT(launch_steps_ma_, LOB_K)(bool trace, int blocks, int threads, size_t smem, cudaStream_t s,
                                             const KParams &p) {
    if (trace) k_env_steps_wide<LOB_K, true, true, true><<<blocks, threads, smem, s>>>(p);
    else k_env_steps_wide<LOB_K, false, true, true><<<blocks, threads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t LOB_CAT(optin_steps_ma_, LOB_K)(size_t smem) {
    const int b = (int)smem;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_env_steps_wide<LOB_K, true, true, true>, A, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_wide<LOB_K, false, true, true>, A, b);
    return e;
}
}  // namespace lobk
