// steps_split.cu -- the two-warps-per-env step kernel (lob_split.cuh) of the
// register-pool classes K = 2, 4 and 8, in a translation unit of its own.
#include "lob_split.cuh"
#include "lob_steps.h"

namespace lobk {
cudaError_t launch_steps_split(int K, int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p) {
    switch (K) {
        case 2: k_env_steps_split<2><<<blocks, threads, smem, s>>>(p); break;
        case 4: k_env_steps_split<4><<<blocks, threads, smem, s>>>(p); break;
        case 8: k_env_steps_split<8><<<blocks, threads, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
// The shared memory a block may take, and the largest shared-memory carve-out
// of the SM: a block is small (one env), so without it the default carve-out
// bounds the resident blocks before the registers do.
template <int KK>
static cudaError_t optin_one(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_env_steps_split<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env_steps_split<KK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}
cudaError_t optin_steps_split(int K, size_t smem) {
    switch (K) {
        case 2: return optin_one<2>(smem);
        case 4: return optin_one<4>(smem);
        case 8: return optin_one<8>(smem);
        default: return cudaErrorInvalidValue;
    }
}
size_t split_pair_bytes(int K) {
    switch (K) {
        case 2: return sizeof(WarpSmem<2>) + sizeof(SplitSmem);
        case 4: return sizeof(WarpSmem<4>) + sizeof(SplitSmem);
        default: return sizeof(WarpSmem<8>) + sizeof(SplitSmem);
    }
}
}  // namespace lobk
