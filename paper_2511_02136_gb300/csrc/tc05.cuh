// tc05.cuh -- shared-memory layouts and inline-PTX wrappers of the 5th-
// generation tensor cores (tcgen05: TMEM allocation, MMA with FP32
// accumulation in tensor memory, loads), mbarriers and bulk copies, used by
// the policy forward (policy.cuh), the fused rollout (fused.cuh) and the
// IPPO update (ppo.cuh); plus the network's fixed shapes and input scale.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include "lob.h"

namespace pol {

constexpr int H = 128;        // hidden width
constexpr int NOUT = 13;      // 12 logits + value
constexpr int NA = 12;        // actions
constexpr int DMAX = 128;     // max observation length (padded to a multiple of 16)
constexpr int PT = 256;       // threads per CTA of the BF16 forward

// Input scale of feature f of an observation with L levels per side.
__host__ __device__ inline float obs_scale(int f, int L) {
    if (f < 4 * L) return (f & 1) ? 1e-3f : 0.1f;   // level (px - anchor, qty)
    const int g = f - 4 * L;
    if (g == 0) return 1e-2f;      // inventory
    if (g == 1) return 1e-6f;      // cash
    if (g == 2) return 1.0f;       // time left
    return 1e-2f;                  // remaining target, own resting quantity
}

// Byte offset of element (row, k) in a K-major core-matrix tile with Kp
// columns: core matrix (row / 8, k / 8) is 128 contiguous bytes (8 rows of
// 8 bf16); core matrices run along K first (leading byte offset 128), then
// along rows (stride byte offset Kp / 8 * 128).
__host__ __device__ inline unsigned cm_off(int row, int k, int Kp) {
    return (unsigned)((((row >> 3) * (Kp >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

struct PolicyParams {
    const float *obs;               // [n_envs][A][D]
    int n_envs, A, D, Dp, L;
    const unsigned char *wpack;     // per agent: bf16 W1 [128 x Dp], W2 [128 x 128], W3 [16 x 128] in core layout
    long long wpack_stride;         // bytes per agent
    const float *wf32;              // per agent: W1 [128][D], b1, W2 [128][128], b2, W3 [13][128], b3
    long long wf32_stride;          // floats per agent
    float *logits;                  // [n_envs][A][12] or NULL
    float *values;                  // [n_envs][A] or NULL
    int *actions;                   // [n_envs][A] or NULL
    int *status;
    long long wait_budget;
};

__device__ __forceinline__ unsigned s_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---- tcgen05 / mbarrier helpers (inline PTX)
__device__ __forceinline__ void tm_alloc(unsigned *dst_smem, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(dst_smem)),
                 "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major.
__device__ __forceinline__ unsigned long long sdesc(const void *base, unsigned lbo, unsigned sbo) {
    const unsigned long long a = (s_u32(base) >> 4) & 0x3FFFu;
    return a | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) | ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);   // descriptor version for this architecture; base offset 0, layout 0 (no swizzle)
}
// Instruction descriptor of kind::f16: BF16 x BF16 -> F32, both K-major.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4)          // accumulator format F32
         | (1u << 7)          // A format BF16
         | (1u << 10)         // B format BF16
         | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long da, unsigned long long db, unsigned idesc,
                                         int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void pbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that expects `bytes` of bulk-copy data, then the copies.
__device__ __forceinline__ void pbar_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                     "r"(s_u32(dst)), "l"(src), "r"(bytes), "r"(s_u32(bar)) : "memory");
}
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ bool pbar_wait(unsigned long long *bar, unsigned phase, long long budget) {
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(s_u32(bar)), "r"(phase) : "memory");
        if (ok) return true;
        if (clock64() - t0 > budget) return false;
    }
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tm_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tm_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
// Zero 16 consecutive FP32 columns of the warp's 32 TMEM lanes (completes
// before the call returns).
__device__ __forceinline__ void tm_zero16(unsigned taddr) {
    const unsigned z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z), "r"(z),
        "r"(z), "r"(z), "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

}  // namespace pol
