// steps_inst.cuh -- instantiates the step kernel of one capacity class
// (K = LOB_K slots per lane per side) in a translation unit of its own so
// that the classes compile in parallel: the plain kernel, the extended one
// (episode mode, reward variants, other action spaces) and the traced
// extended one, in the register budgets below.
#include "lob_device.cuh"
#include "lob_steps.h"

#define LOB_CAT2(a, b) a##b
#define LOB_CAT(a, b) LOB_CAT2(a, b)

namespace lobk {
// K >= 8: every instance in the wide register budget; K <= 4: the plain and
// extended kernels in both budgets (the host picks by batch size), the traced
// one wide.  For launches of several waves K = 4 takes a fixed budget: 168
// registers for the extended kernel (three 4-warp blocks per SM), 128 for the
// plain one (16 warps per SM instead of the 12 its own 158 registers leave;
// it spills a few hundred bytes and still measured 2.7 % faster at 16,384 envs).  The dispatch is a template so that the branches of the other
// case are never instantiated.
template <int KK, bool ALWAYS_WIDE = (KK >= 8)>
struct StepLaunch {
    static cudaError_t launch(bool trace, bool ext, bool wide, int blocks, int threads, size_t smem, cudaStream_t s,
                              const KParams &p) {
        // other message-tile sizes: the plain kernel in the wide budget
        // (p.tile is set only for launches that take it)
        if (!trace && !ext && p.tile == 16) k_env_steps_wide<KK, false, false, false, 16><<<blocks, threads, smem, s>>>(p);
        else if (!trace && !ext && p.tile == TILE_MAX)
            k_env_steps_wide<KK, false, false, false, TILE_MAX><<<blocks, threads, smem, s>>>(p);
        else if (trace) k_env_steps_wide<KK, true, true><<<blocks, threads, smem, s>>>(p);
        else if constexpr (ALWAYS_WIDE) {
            if (ext) k_env_steps_wide<KK, false, true><<<blocks, threads, smem, s>>>(p);
            else k_env_steps_wide<KK, false, false><<<blocks, threads, smem, s>>>(p);
        } else {
            if (ext && wide) k_env_steps_wide<KK, false, true><<<blocks, threads, smem, s>>>(p);
            else if (ext) {
                if constexpr (KK == 4) k_env_steps_nreg<KK, false, true, false, 168><<<blocks, threads, smem, s>>>(p);
                else k_env_steps<KK, false, true><<<blocks, threads, smem, s>>>(p);
            }
            else if (wide) k_env_steps_wide<KK, false, false><<<blocks, threads, smem, s>>>(p);
            else if constexpr (KK == 4) k_env_steps_nreg<KK, false, false, false, 128><<<blocks, threads, smem, s>>>(p);
            else k_env_steps<KK, false, false><<<blocks, threads, smem, s>>>(p);
        }
        return cudaGetLastError();
    }
    static cudaError_t optin(size_t smem) {
        const int b = (int)smem;
        const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(k_env_steps_wide<KK, true, true>, A, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_wide<KK, false, true>, A, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_wide<KK, false, false>, A, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_wide<KK, false, false, false, 16>, A, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_wide<KK, false, false, false, TILE_MAX>, A, b);
        if constexpr (!ALWAYS_WIDE) {
            if constexpr (KK == 4) {
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_nreg<KK, false, true, false, 168>, A, b);
            } else {
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps<KK, false, true>, A, b);
            }
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps<KK, false, false>, A, b);
            if constexpr (KK == 4)
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k_env_steps_nreg<KK, false, false, false, 128>, A, b);
        }
        return e;
    }
};

cudaError_t LOB_CAT(launch_steps_, LOB_K)(bool trace, bool ext, bool wide, int blocks, int threads, size_t smem,
                                          cudaStream_t s, const KParams &p) {
    return StepLaunch<LOB_K>::launch(trace, ext, wide, blocks, threads, smem, s, p);
}

// Resident blocks per SM of the wide plain / extended kernel at this shape.
int LOB_CAT(wide_blocks_per_sm_, LOB_K)(bool ext, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = ext ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_steps_wide<LOB_K, false, true>,
                                                                        threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_steps_wide<LOB_K, false, false>,
                                                                        threads, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t LOB_CAT(optin_steps_, LOB_K)(size_t smem) { return StepLaunch<LOB_K>::optin(smem); }
}  // namespace lobk
