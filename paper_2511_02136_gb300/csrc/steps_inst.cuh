// steps_inst.cuh -- instantiates the step kernel of one capacity class
// (K = LOB_K slots per lane per side) in a translation unit of its own so
// that the classes compile in parallel: the plain kernel, the extended one
// (episode mode, reward variants) and the traced extended one.
#include "lob_device.cuh"
#include "lob_steps.h"

#define LOB_CAT2(a, b) a##b
#define LOB_CAT(a, b) LOB_CAT2(a, b)

namespace lobk {
cudaError_t LOB_CAT(launch_steps_, LOB_K)(bool trace, bool ext, int blocks, int threads, size_t smem,
                                          cudaStream_t s, const KParams &p) {
    if (trace) k_env_steps<LOB_K, true, true><<<blocks, threads, smem, s>>>(p);
    else if (ext) k_env_steps<LOB_K, false, true><<<blocks, threads, smem, s>>>(p);
    else k_env_steps<LOB_K, false, false><<<blocks, threads, smem, s>>>(p);
    return cudaGetLastError();
}
cudaError_t LOB_CAT(optin_steps_, LOB_K)(size_t smem) {
    const int b = (int)smem;
    cudaError_t e = cudaFuncSetAttribute(k_env_steps<LOB_K, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env_steps<LOB_K, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env_steps<LOB_K, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}
}  // namespace lobk
