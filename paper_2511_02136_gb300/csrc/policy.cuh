// policy.cuh -- per-agent actor-critic MLP forward for the rollout (IPPO
// networks of JaxMARL-HFT Sec. 4.2: separate weights per agent).
//
//   x = obs * s                  (fixed per-feature input scale)
//   h1 = tanh(W1 x + b1)         W1: 128 x D
//   h2 = tanh(W2 h1 + b2)        W2: 128 x 128
//   y  = W3 h2 + b3              W3: 13 x 128 -> 12 logits + 1 value
//   action = argmax(logits), ties to the lowest index
//
// k_policy_bf16: BF16 operands on the 5th-generation tensor cores
// (tcgen05.mma, kind::f16, FP32 accumulation in tensor memory).  One CTA of
// 256 threads handles 128 envs of one agent: the three layers are M=128
// GEMMs (N = 128, 128, 16) whose operands sit in shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix).
// The agent's packed weights arrive by bulk copy while the threads stage
// the observation tile with coalesced loads; in the bias + tanh epilogues
// warp w reads TMEM lanes 32 (w mod 4) .. +31 (env rows) and column half
// w / 4, with the tensor-core-era tanh.approx (its error, below 2^-10.9
// relative, is under the BF16 rounding of the activations that follows).
// k_policy_fp32: the same forward with FP32 FMAs on the CUDA cores.
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

struct __align__(128) Bf16Smem {
    unsigned char w1[H * DMAX * 2];   // [128 x Dp]
    unsigned char w2[H * H * 2];      // [128 x 128]
    unsigned char w3[16 * H * 2];     // [16 x 128]
    unsigned char x[128 * DMAX * 2];  // [128 x Dp]
    unsigned char h[128 * H * 2];     // [128 x 128], h1 then h2
    float b1[H], b2[H], b3[16];
    unsigned long long bar;    // MMA completion
    unsigned long long wbar;   // weight bulk copies
    unsigned tmem_base;
};

// Greedy action and the outputs of one row.
__device__ __forceinline__ void write_outputs(const PolicyParams &p, int env, int a, const float (&y)[16]) {
    if (env >= p.n_envs) return;
    const long long r = (long long)env * p.A + a;
    int best = 0;
    float bv = y[0];
#pragma unroll
    for (int j = 1; j < NA; j++)
        if (y[j] > bv) { bv = y[j]; best = j; }
    if (p.logits) {
#pragma unroll
        for (int j = 0; j < NA; j++) p.logits[r * NA + j] = y[j];
    }
    if (p.values) p.values[r] = y[NA];
    if (p.actions) p.actions[r] = best;
}

__global__ void __launch_bounds__(PT) k_policy_bf16(const PolicyParams p) {
    extern __shared__ __align__(1024) unsigned char praw[];
    Bf16Smem &sm = *reinterpret_cast<Bf16Smem *>(praw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int a = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    const int Dp = p.Dp;
    if (warp == 0) tm_alloc(&sm.tmem_base, 128);
    if (tid == 0) {
        pbar_init(&sm.bar);
        pbar_init(&sm.wbar);
        // weights of agent a, already bf16 in core layout: three bulk copies
        const unsigned char *src = p.wpack + (long long)a * p.wpack_stride;
        const unsigned n1 = (unsigned)(H * Dp * 2), n2 = H * H * 2, n3 = 16 * H * 2;
        pbar_expect(&sm.wbar, n1 + n2 + n3);
        bulk_g2s(sm.w1, src, n1, &sm.wbar);
        bulk_g2s(sm.w2, src + n1, n2, &sm.wbar);
        bulk_g2s(sm.w3, src + n1 + n2, n3, &sm.wbar);
    }
    {
        const float *wf = p.wf32 + (long long)a * p.wf32_stride;
        const float *b1 = wf + H * p.D, *b2 = b1 + H + H * H, *b3 = b2 + H + NOUT * H;
        if (tid < H) sm.b1[tid] = b1[tid];
        else sm.b2[tid - H] = b2[tid - H];
        if (tid < 16) sm.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
    }
    // X tile [128 x Dp]: warp w stages rows w, w + 8, ..., its lanes along the
    // features (coalesced); all of a thread's loads are in flight at once
    {
        constexpr int RPW = 128 / (PT / 32);   // rows per warp
        const int lane = tid & 31;
        float v[DMAX / 32][RPW];
#pragma unroll
        for (int c = 0; c < DMAX / 32; c++) {
            const int k = 32 * c + lane;
#pragma unroll
            for (int j = 0; j < RPW; j++) {
                const int env = row0 + warp + (PT / 32) * j;
                v[c][j] = (k < p.D && env < p.n_envs)
                              ? p.obs[((long long)env * p.A + a) * p.D + k] * obs_scale(k, p.L) : 0.0f;
            }
        }
#pragma unroll
        for (int c = 0; c < DMAX / 32; c++) {
            const int k = 32 * c + lane;
            if (k < Dp) {
#pragma unroll
                for (int j = 0; j < RPW; j++)
                    *reinterpret_cast<__nv_bfloat16 *>(sm.x + cm_off(warp + (PT / 32) * j, k, Dp)) =
                        __float2bfloat16_rn(v[c][j]);
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sm.tmem_base;
    const int row = 32 * (warp & 3) + (tid & 31);   // TMEM lane = env row
    const int half = warp >> 2;                     // column half of the epilogues
    const unsigned lane_addr = tmem + ((unsigned)(32 * (warp & 3)) << 16);
    bool ok = true;
    unsigned phase = 0;
    // the weights, before the first MMA reads them
    {
        const bool landed = pbar_wait(&sm.wbar, 0, p.wait_budget);
        if (__syncthreads_or(!landed)) {
            ok = false;
            if (tid == 0) atomicOr(p.status, 4);
            pbar_wait(&sm.wbar, 0, p.wait_budget);   // let the copies in flight land
        }
    }
    // ---- three layers
    for (int layer = 0; layer < 3 && ok; layer++) {
        if (tid == 0) {
            const int K = layer == 0 ? Dp : H;
            const int N = layer == 2 ? 16 : H;
            const unsigned char *A_ = layer == 0 ? sm.x : sm.h;
            const unsigned char *B_ = layer == 0 ? sm.w1 : (layer == 1 ? sm.w2 : sm.w3);
            const unsigned idesc = idesc_bf16(128, N);
            for (int kk = 0; kk < K / 16; kk++) {
                const unsigned long long da = sdesc(A_ + kk * 256, 128, (unsigned)(K / 8) * 128);
                const unsigned long long db = sdesc(B_ + kk * 256, 128, (unsigned)(K / 8) * 128);
                mma_bf16(tmem, da, db, idesc, kk > 0);
            }
            mma_commit(&sm.bar);
        }
        const bool arrived = pbar_wait(&sm.bar, phase, p.wait_budget);
        if (__syncthreads_or(!arrived)) {   // the same decision in every thread
            ok = false;
            if (tid == 0) atomicOr(p.status, 4);
            pbar_wait(&sm.bar, phase, p.wait_budget);  // let the tensor core finish before freeing TMEM
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        if (layer < 2) {
            const float *bias = layer == 0 ? sm.b1 : sm.b2;
#pragma unroll
            for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 32) {
                float v[32];
                tm_ld32(lane_addr + c0, v);
#pragma unroll
                for (int j = 0; j < 32; j += 8) {
                    unsigned w[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const __nv_bfloat162 t = __floats2bfloat162_rn(tanh_approx(v[j + 2 * q] + bias[c0 + j + 2 * q]),
                                                                       tanh_approx(v[j + 2 * q + 1] + bias[c0 + j + 2 * q + 1]));
                        w[q] = *reinterpret_cast<const unsigned *>(&t);
                    }
                    *reinterpret_cast<uint4 *>(sm.h + cm_off(row, c0 + j, H)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        } else if (half == 0) {
            float v[32];
            tm_ld32(lane_addr, v);
            float y[16];
#pragma unroll
            for (int j = 0; j < 16; j++) y[j] = v[j] + sm.b3[j];
            write_outputs(p, row0 + row, a, y);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tm_dealloc(tmem, 128);
    }
}

// FP32 reference forward on the CUDA cores: 64 envs of one agent per CTA,
// weights and activations in shared memory (activations stored [unit][row]).
struct F32Smem {
    float w1[H * DMAX];
    float w2[H * H];
    float w3[NOUT * H];
    float b1[H], b2[H], b3[16];
    float h1[H * 64];
    float h2[H * 64];
};

__global__ void __launch_bounds__(64) k_policy_fp32(const PolicyParams p) {
    extern __shared__ __align__(16) unsigned char fraw[];
    F32Smem &sm = *reinterpret_cast<F32Smem *>(fraw);
    const int tid = threadIdx.x;
    const int a = blockIdx.y;
    const int env = blockIdx.x * 64 + tid;
    const int D = p.D;
    const float *wf = p.wf32 + (long long)a * p.wf32_stride;
    for (int i = tid; i < H * D; i += 64) sm.w1[i] = wf[i];
    const float *b1 = wf + H * D, *w2 = b1 + H, *b2 = w2 + H * H, *w3 = b2 + H, *b3 = w3 + NOUT * H;
    for (int i = tid; i < H * H; i += 64) sm.w2[i] = w2[i];
    for (int i = tid; i < NOUT * H; i += 64) sm.w3[i] = w3[i];
    for (int i = tid; i < H; i += 64) { sm.b1[i] = b1[i]; sm.b2[i] = b2[i]; }
    if (tid < 16) sm.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
    float x[DMAX];
    const float *o = p.obs + ((long long)(env < p.n_envs ? env : 0) * p.A + a) * D;
#pragma unroll
    for (int k = 0; k < DMAX; k++) x[k] = (k < D && env < p.n_envs) ? o[k] * obs_scale(k, p.L) : 0.0f;
    __syncthreads();
    for (int j = 0; j < H; j++) {
        float acc = sm.b1[j];
#pragma unroll 4
        for (int k = 0; k < D; k++) acc = fmaf(sm.w1[j * D + k], x[k], acc);
        sm.h1[j * 64 + tid] = tanhf(acc);
    }
    for (int j = 0; j < H; j++) {
        float acc = sm.b2[j];
#pragma unroll 8
        for (int k = 0; k < H; k++) acc = fmaf(sm.w2[j * H + k], sm.h1[k * 64 + tid], acc);
        sm.h2[j * 64 + tid] = tanhf(acc);
    }
    float y[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        float acc = sm.b3[j];
        if (j < NOUT)
            for (int k = 0; k < H; k++) acc = fmaf(sm.w3[j * H + k], sm.h2[k * 64 + tid], acc);
        y[j] = acc;
    }
    write_outputs(p, env, a, y);
}

}  // namespace pol
