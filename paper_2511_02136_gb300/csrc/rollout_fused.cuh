// rollout_fused.cuh -- the fused BF16 rollout kernel of one capacity class
// (K = LOB_K slots per lane per side), in a translation unit of its own: one
// CTA runs one env per warp for the whole rollout with the books on chip and
// evaluates both agents' networks on the tensor cores after every step
// (fused.cuh), so observations and actions never go through HBM.
#include "lob_device.cuh"
#include "lob_steps.h"

#define LOB_CAT2(a, b) a##b
#define LOB_CAT(a, b) LOB_CAT2(a, b)

namespace lobk {

static_assert(sizeof(WarpSmem<LOB_K>) % 16 == 0, "the policy's tiles after the warps' areas stay 16-byte aligned");

template <int K>
__global__ void __launch_bounds__(FWMAX * 32, 1) k_rollout_fused(const KParams p, const FusedParams f) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int nw = blockDim.x >> 5;
    WarpSmem<K> &sm = reinterpret_cast<WarpSmem<K> *>(smem_raw)[wib];
    unsigned char *after = smem_raw + nw * sizeof(WarpSmem<K>);
    LadBlock<K> *lb = ladder_class<K>() ? reinterpret_cast<LadBlock<K> *>(after) + wib : nullptr;
    after += nw * ladder_bytes<K>();
    FusedSmem &fz = *reinterpret_cast<FusedSmem *>(after);
    if (lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    fused_setup(fz, f, nw, tid);
    FusedCtx fc{&fz, &f, 0u, nw, tid, wib};
    const int e = blockIdx.x * nw + wib;
    const bool active = e < p.n_envs;
    // the first actions: both networks on every env's current observation
    if (active) {
        const float *ob = p.obs_in + (long long)e * 2 * f.D;
        for (int a = 0; a < 2; a++)
            for (int k = lane; k < f.D; k += 32) fused_put_obs(fz, f, a, wib, k, ob[a * f.D + k]);
    }
    __syncwarp();
    fused_policy(fz, f, fc.phase, nw, tid);
    if (active) {
        MsgPipe pipe{0u, nullptr};
        run_env<K, false, false, false, true>(p, e, sm, nullptr, lb, pipe, lane, &fc);
    } else {
        for (int i = 0; i < p.n_steps; i++) fused_policy(fz, f, fc.phase, nw, tid);   // keep the CTA in step
    }
    fused_teardown(fz, f, tid);
}

cudaError_t LOB_CAT(launch_fused_, LOB_K)(int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p,
                                          const FusedParams &f) {
    k_rollout_fused<LOB_K><<<blocks, threads, smem, s>>>(p, f);
    return cudaGetLastError();
}
cudaError_t LOB_CAT(optin_fused_, LOB_K)(size_t smem) {
    return cudaFuncSetAttribute(k_rollout_fused<LOB_K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
}  // namespace lobk
