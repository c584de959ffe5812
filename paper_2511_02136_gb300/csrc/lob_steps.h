// lob_steps.h -- launch interface of the per-class step-kernel translation
// units (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include "lob_device.cuh"

namespace lobk {
#define LOB_DECL_CLASS(k)                                                                              \
    cudaError_t launch_steps_##k(bool trace, bool ext, bool wide, int blocks, int threads, size_t smem,\
                                 cudaStream_t s, const KParams &p);                                    \
    int wide_blocks_per_sm_##k(bool ext, int threads, size_t smem);                                    \
    cudaError_t optin_steps_##k(size_t smem);                                                          \
    cudaError_t launch_steps_ma_##k(bool trace, int blocks, int threads, size_t smem, cudaStream_t s,  \
                                    const KParams &p);                                                 \
    cudaError_t optin_steps_ma_##k(size_t smem);
LOB_DECL_CLASS(1)
LOB_DECL_CLASS(2)
LOB_DECL_CLASS(4)
LOB_DECL_CLASS(8)
LOB_DECL_CLASS(16)
LOB_DECL_CLASS(32)
#undef LOB_DECL_CLASS
}  // namespace lobk
