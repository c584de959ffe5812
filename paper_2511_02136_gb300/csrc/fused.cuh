// fused.cuh -- the per-agent actor-critic forward inside the rollout kernel
// (JaxMARL-HFT Sec. 4.2: separate networks per agent; the benchmark's
// 45 -> 128 -> 128 -> 13 MLP in BF16 with FP32 accumulation).
//
// A CTA of the fused rollout runs one env per warp for the whole rollout
// (books on chip); after every step its warps write their observation rows,
// scaled and rounded to BF16, into a small shared-memory tile per agent and
// the CTA evaluates both agents' networks on the tensor cores before the
// next step.  The contraction is turned around so that the weights are the
// operand that stays put: the weights are the A operand held in tensor
// memory for the whole launch (each warp of the epilogue writes its 32 rows
// with tcgen05.st), the CTA's envs are the N = 16 columns, and the products
//     H1^T = W1 X^T,  H2^T = W2 H1^T,  Y^T = W3 H2^T
// land in TMEM as [128 units x 16 envs] FP32.  Shared memory then holds only
// the 16-row B tiles, which leaves the books their full room.  The greedy
// action (argmax of the 12 logits, ties to the lowest index) of every
// (env, agent) is the next step's action; observations and actions never
// leave the chip between steps.
#pragma once
#include "tc05.cuh"

namespace lobk {

constexpr int FN = 16;          // envs per CTA tile (the MMA's N)
constexpr int FDMAX = 96;       // widest padded observation of the fused forward

// TMEM columns of the fused forward (512 allocated): per agent a, W1 at
// 48 a (Dp / 2 <= 48 columns: each lane holds a row, 2 bf16 per column), W2 at
// 96 + 64 a, W3 at 224 + 64 a, the [128 x 16] accumulator at 352 + 16 a.
__host__ __device__ constexpr unsigned fz_w1(int a) { return (unsigned)(48 * a); }
__host__ __device__ constexpr unsigned fz_w2(int a) { return 96u + 64u * (unsigned)a; }
__host__ __device__ constexpr unsigned fz_w3(int a) { return 224u + 64u * (unsigned)a; }
__host__ __device__ constexpr unsigned fz_acc(int a) { return 352u + 16u * (unsigned)a; }

struct __align__(16) FusedSmem {
    unsigned char x[2][FN * FDMAX * 2];   // per agent: scaled observations, B operand [16 envs x Dp]
    unsigned char h[2][FN * 128 * 2];     // per agent: hidden activations, B operand [16 envs x 128]
    float b1[2][128], b2[2][128], b3[2][16];
    float ys[2][FN][16];                  // outputs per agent and env
    int acts[FN][2];                      // the actions of the next step
    unsigned long long bar;
    unsigned tmem_base;
    int failed;                           // a bounded tensor-core wait expired (then actions stay 0)
};

// Policy weights for the fused forward: per agent row-major bf16 W1 [128 x
// Dp], W2 [128 x 128], W3 [16 x 128] (rows >= 13 zero), and FP32 biases.
struct FusedParams {
    const unsigned char *wrow;
    long long wrow_stride;    // bytes per agent
    const float *wf32;        // per agent parameter block (biases)
    long long wf32_stride;
    int D, Dp, L;
    int *status;
    long long wait_budget;
};

__device__ __forceinline__ void tm_st8(unsigned taddr, const unsigned (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tm_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
// D (+)= A B^T with A [128 x K] in TMEM (bf16 pairs per column) and B [16 x K]
// in shared memory (K-major core layout), one thread.
__device__ __forceinline__ void mma_ta(unsigned tmem_d, unsigned tmem_a, const unsigned char *B_, int K) {
    const unsigned idesc = pol::idesc_bf16(128, FN);
    for (int kk = 0; kk < K / 16; kk++) {
        const unsigned long long db = pol::sdesc(B_ + kk * 256, 128, (unsigned)(K / 8) * 128);
        const unsigned ta = tmem_a + (unsigned)(8 * kk);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
            "r"(ta), "l"(db), "r"(idesc), "r"(kk > 0 ? 1 : 0) : "memory");
    }
}

// Set-up by every thread of the CTA (nw >= 4 warps): TMEM, the mbarrier,
// biases, zeroed B tiles, and each agent's weights into TMEM (warp w writes
// lanes 32 (w mod 4) .. +31, agent w / 4 when nw >= 8, else both).
__device__ __forceinline__ void fused_setup(FusedSmem &fz, const FusedParams &f, int nw, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == 0) pol::tm_alloc(&fz.tmem_base, 512);
    if (tid == 0) {
        pol::pbar_init(&fz.bar);
        fz.failed = 0;
    }
    for (int i = tid; i < 2 * FN * FDMAX * 2 / 4; i += nw * 32) reinterpret_cast<unsigned *>(&fz.x[0][0])[i] = 0u;
    for (int i = tid; i < 2 * FN * 128 * 2 / 4; i += nw * 32) reinterpret_cast<unsigned *>(&fz.h[0][0])[i] = 0u;
    for (int i = tid; i < 2 * FN * 2; i += nw * 32) (&fz.acts[0][0])[i] = 0;
    for (int i = tid; i < 2 * 272; i += nw * 32) {
        const int a = i / 272, j = i % 272;
        const float *wf = f.wf32 + (long long)a * f.wf32_stride;
        const float *b1 = wf + 128 * f.D, *b2 = b1 + 128 + 128 * 128, *b3 = b2 + 128 + 13 * 128;
        if (j < 128) fz.b1[a][j] = b1[j];
        else if (j < 256) fz.b2[a][j - 128] = b2[j - 128];
        else fz.b3[a][j - 256] = j - 256 < 13 ? b3[j - 256] : 0.0f;
    }
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    const unsigned tm = fz.tmem_base;
    if (warp < (nw >= 8 ? 8 : 4)) {
        const int row = 32 * (warp & 3) + lane;
        const unsigned lrow = tm + ((unsigned)(32 * (warp & 3)) << 16);
        for (int a = (nw >= 8 ? warp >> 2 : 0); a < 2; a += (nw >= 8 ? 2 : 1)) {
            const unsigned char *w = f.wrow + (long long)a * f.wrow_stride;
            const unsigned *w1 = reinterpret_cast<const unsigned *>(w) + (long long)row * (f.Dp / 2);
            const unsigned *w2 = reinterpret_cast<const unsigned *>(w + 128 * f.Dp * 2) + row * 64;
            const unsigned *w3 = reinterpret_cast<const unsigned *>(w + 128 * f.Dp * 2 + 128 * 128 * 2) + row * 64;
            for (int c = 0; c < f.Dp / 2; c += 8) {
                unsigned v[8];
#pragma unroll
                for (int i = 0; i < 8; i++) v[i] = w1[c + i];
                tm_st8(lrow + fz_w1(a) + c, v);
            }
            for (int c = 0; c < 64; c += 8) {
                unsigned v[8], u[8];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    v[i] = w2[c + i];
                    u[i] = row < 16 ? w3[c + i] : 0u;   // W3 rows >= 16 are zero
                }
                tm_st8(lrow + fz_w2(a) + c, v);
                tm_st8(lrow + fz_w3(a) + c, u);
            }
        }
        tm_wait_st();
    }
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
}

// One warp's observation row of agent a (D floats, already computed) into
// the B tile: entry k scaled like the network's input, rounded to BF16.
__device__ __forceinline__ void fused_put_obs(FusedSmem &fz, const FusedParams &f, int a, int row, int k, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(fz.x[a] + pol::cm_off(row, k, f.Dp)) =
        __float2bfloat16_rn(v * pol::obs_scale(k, f.L));
}

// Both agents' networks on the observation tiles and the greedy actions into
// fz.acts; every thread of the CTA calls it (nw >= 4 warps).
__device__ __forceinline__ void fused_policy(FusedSmem &fz, const FusedParams &f, unsigned &phase, int nw, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    const unsigned tm = fz.tmem_base;
    pol::fence_async_smem();
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    const bool epi = warp < (nw >= 8 ? 8 : 4);
    const int row = 32 * (warp & 3) + lane;   // TMEM lane = hidden unit / output
    const unsigned lrow = tm + ((unsigned)(32 * (warp & 3)) << 16);
    for (int layer = 0; layer < 3; layer++) {
        const bool live = fz.failed == 0;
        if (tid == 0 && live) {
            for (int a = 0; a < 2; a++) {
                if (layer == 0) mma_ta(tm + fz_acc(a), tm + fz_w1(a), fz.x[a], f.Dp);
                else mma_ta(tm + fz_acc(a), tm + (layer == 1 ? fz_w2(a) : fz_w3(a)), fz.h[a], 128);
            }
            pol::mma_commit(&fz.bar);
        }
        if (live) {
            const bool arrived = pol::pbar_wait(&fz.bar, phase, f.wait_budget);
            if (__syncthreads_or(!arrived)) {
                if (tid == 0) { fz.failed = 1; atomicOr(f.status, 4); }
                pol::pbar_wait(&fz.bar, phase, f.wait_budget);   // let the tensor core finish
            }
            phase ^= 1u;
            pol::tc_fence_after();
        }
        if (epi && live) {
            for (int a = (nw >= 8 ? warp >> 2 : 0); a < 2; a += (nw >= 8 ? 2 : 1)) {
                float v[16];
                tm_ld16(lrow + fz_acc(a), v);
                if (layer < 2) {
                    const float b = layer == 0 ? fz.b1[a][row] : fz.b2[a][row];
#pragma unroll
                    for (int n = 0; n < FN; n++)
                        *reinterpret_cast<__nv_bfloat16 *>(fz.h[a] + pol::cm_off(n, row, 128)) =
                            __float2bfloat16_rn(pol::tanh_approx(v[n] + b));
                } else if (row < 16) {
#pragma unroll
                    for (int n = 0; n < FN; n++) fz.ys[a][n][row] = v[n] + fz.b3[a][row];
                }
            }
        }
        pol::fence_async_smem();
        pol::tc_fence_before();
        __syncthreads();
        pol::tc_fence_after();
    }
    if (tid < 2 * FN) {
        const int n = tid >> 1, a = tid & 1;
        int best = 0;
        float bv = fz.ys[a][n][0];
#pragma unroll
        for (int j = 1; j < 12; j++)
            if (fz.ys[a][n][j] > bv) { bv = fz.ys[a][n][j]; best = j; }
        fz.acts[n][a] = fz.failed ? 0 : best;
    }
    __syncthreads();
}

__device__ __forceinline__ void fused_teardown(FusedSmem &fz, int tid) {
    pol::tc_fence_before();
    __syncthreads();
    if ((tid >> 5) == 0) {
        pol::tc_fence_after();
        pol::tm_dealloc(fz.tmem_base, 512);
    }
}

}  // namespace lobk
