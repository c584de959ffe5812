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
// one persistent kernel over the classes K = 1 .. 16 (steps_multi.cu): warp w
// of a block owns a carve-out of class cls[w] at byte off[w]; class c's envs
// are env_list[begin[c] .. begin[c] + count[c]) with work counter queue[c]
constexpr int MULTI_CLASSES = 5;
struct MultiLayout {
    int cls[8];
    int off[9];
    int begin[MULTI_CLASSES], count[MULTI_CLASSES];
    int steal;
};
cudaError_t launch_steps_multi(int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p,
                               const MultiLayout &m);
cudaError_t optin_steps_multi(size_t smem);
int multi_blocks_per_sm(int threads, size_t smem);
// two warps per env (lob_split.cuh; classes K = 2, 4, 8; the plain benchmark configuration)
cudaError_t launch_steps_split(int K, int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p);
cudaError_t optin_steps_split(int K, size_t smem);
size_t split_pair_bytes(int K);
// fused BF16 rollout (classes K = 4 and 8)
cudaError_t launch_fused_4(int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p, const FusedParams &f);
cudaError_t optin_fused_4(size_t smem);
cudaError_t launch_fused_8(int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p, const FusedParams &f);
cudaError_t optin_fused_8(size_t smem);
LOB_DECL_CLASS(1)
LOB_DECL_CLASS(2)
LOB_DECL_CLASS(4)
LOB_DECL_CLASS(8)
LOB_DECL_CLASS(16)
LOB_DECL_CLASS(32)
#undef LOB_DECL_CLASS
}  // namespace lobk
