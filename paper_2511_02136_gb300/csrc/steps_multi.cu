// steps_multi.cu -- one persistent step kernel for envs of several capacity
// classes at once (the uneven batch: book capacities drawn from {50, 100,
// 200, 500}, messages per step Poisson with per-env rates).
//
// Each warp of a block owns a shared-memory carve-out sized for one class
// (the host picks how many warps of each class a block holds); a warp takes
// envs of its own class from that class's work queue (envs ordered longest
// first when costs are set) and, once that queue is empty, steals envs of the
// smaller classes, whose books fit its carve-out.  So no class's leftover
// work waits for SMs that another class's launch holds, and the whole
// rollout is one launch (capturable in a CUDA graph).  The plain env step
// only (no trace, extended options or several agents per type).
#include "lob_device.cuh"
#include "lob_steps.h"

namespace lobk {

static_assert(offsetof(WarpSmem<1>, bar) == offsetof(WarpSmem<16>, bar) &&
                  offsetof(WarpSmem<2>, bar) == offsetof(WarpSmem<8>, bar) &&
                  offsetof(WarpSmem<4>, bar) == offsetof(WarpSmem<1>, bar),
              "the tile barriers sit at one offset in every class's per-warp block");

template <int K>
__device__ __forceinline__ void run_class(const KParams &p, int e, unsigned char *carve, MsgPipe &pipe, int lane) {
    LadBlock<K> *lb = ladder_class<K>() ? reinterpret_cast<LadBlock<K> *>(carve + sizeof(WarpSmem<K>)) : nullptr;
    run_env<K, false, false, false>(p, e, *reinterpret_cast<WarpSmem<K> *>(carve), nullptr, lb, pipe, lane);
}

__global__ void __launch_bounds__(256, 1) k_env_steps_multi(const KParams p, const MultiLayout m) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int own = m.cls[wib];
    unsigned char *carve = smem_raw + m.off[wib];
    unsigned long long *bar = reinterpret_cast<WarpSmem<1> *>(carve)->bar;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    MsgPipe pipe{0u, nullptr};
    for (;;) {
        int c = own, w = 0;
        bool got = false;
        for (; c >= 0; c--) {   // its own class first, then (stealing) the smaller ones
            if (m.count[c] == 0) continue;
            if (lane == 0) w = atomicAdd(p.queue + c, 1);
            w = __shfl_sync(FULL, w, 0);
            if (w < m.count[c]) { got = true; break; }
            if (!m.steal) break;
        }
        if (!got) break;
        const int e = p.env_list[m.begin[c] + w];
        switch (c) {
            case 0: run_class<1>(p, e, carve, pipe, lane); break;
            case 1: run_class<2>(p, e, carve, pipe, lane); break;
            case 2: run_class<4>(p, e, carve, pipe, lane); break;
            case 3: run_class<8>(p, e, carve, pipe, lane); break;
            default: run_class<16>(p, e, carve, pipe, lane); break;
        }
    }
}

cudaError_t launch_steps_multi(int blocks, int threads, size_t smem, cudaStream_t s, const KParams &p,
                               const MultiLayout &m) {
    k_env_steps_multi<<<blocks, threads, smem, s>>>(p, m);
    return cudaGetLastError();
}
cudaError_t optin_steps_multi(size_t smem) {
    return cudaFuncSetAttribute(k_env_steps_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
int multi_blocks_per_sm(int threads, size_t smem) {
    int nb = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_steps_multi, threads, smem) == cudaSuccess ? nb : 0;
}
}  // namespace lobk
