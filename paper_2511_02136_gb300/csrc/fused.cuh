// fused.cuh -- the per-agent actor-critic forward inside the rollout kernel
// (JaxMARL-HFT Sec. 4.2: a separate network per agent; the benchmark's
// obs -> 128 -> 128 -> 13 MLP, tanh hidden units, in BF16 with FP32
// accumulation).
//
// A CTA of the fused rollout runs one env per warp for the whole rollout
// with the books on chip.  After every step its warps write their
// observation rows, scaled and rounded to BF16, into a 16-row tile per agent
// and the CTA evaluates both agents' networks before the next step.  The
// hidden layers run on the tensor cores with the roles turned around: the
// weights are the A operand (M = 128 units, loaded into shared memory once
// per launch by bulk copy, in the same K-major core layout the batched
// forward uses) and the CTA's envs are the N = 16 columns, so
//     H1^T = W1 X^T,   H2^T = W2 H1^T
// land in tensor memory as [128 units x 16 envs] FP32 and the activation
// tiles stay 16 rows.  The 13-output head is 13 x 128 dot products per
// (env, agent) on the CUDA cores.  The greedy action (argmax of the 12
// logits, ties to the lowest index) of every (env, agent) is the next step's
// action, so observations and actions never leave the chip between steps.
#pragma once
#include "tc05.cuh"

namespace lobk {

constexpr int FN = 16;          // envs per CTA tile (the MMA's N)
constexpr int FDMAX = 48;       // widest padded observation of the fused forward
constexpr int FWMAX = 12;       // env warps per CTA at most (the kernel's register budget is sized for it)

struct __align__(16) FusedSmem {
    unsigned char w1[2][128 * FDMAX * 2];   // per agent: W1 [128 x Dp], core layout (A operand)
    unsigned char w2[2][128 * 128 * 2];     // per agent: W2 [128 x 128]
    unsigned char w3[2][16 * 128 * 2];      // per agent: W3 [16 x 128] (rows >= 13 zero)
    unsigned char x[2][FN * FDMAX * 2];     // per agent: scaled observations, B operand [16 envs x Dp]
    unsigned char h[2][FN * 128 * 2];       // per agent: hidden activations, B operand [16 envs x 128]
    float b1[2][128], b2[2][128], b3[2][16];
    float ys[2][FN][16];                    // head outputs per agent and env
    int acts[FN][2];                        // the actions of the next step
    unsigned long long bar, wbar;
    unsigned tmem_base;
    int failed;                             // a bounded wait ran out (actions then stay 0)
    int bad;                                // an observation index out of range (recorded, skipped)
};

// Tensor-memory columns (64 allocated): agent a's [128 x 16] accumulator at 32 a.
__host__ __device__ constexpr unsigned fz_acc(int a) { return 32u * (unsigned)a; }

// Weights and shapes of the fused forward.
struct FusedParams {
    const unsigned char *wpack;   // per agent: W1 [128 x Dp], W2 [128 x 128], W3 [16 x 128], bf16 core layout
    long long wpack_stride;       // bytes per agent
    const float *wf32;            // per agent FP32 parameter block (biases)
    long long wf32_stride;
    int D, Dp, L;
    int *status;
    long long wait_budget;
};

// Set-up by every thread of the CTA: tensor memory, the barriers, biases,
// zeroed B tiles and both agents' weights by bulk copy (waited for).
__device__ __forceinline__ void fused_setup(FusedSmem &fz, const FusedParams &f, int nw, int tid) {
    const int warp = tid >> 5;
    if (warp == 0) {
        __syncwarp();
        pol::tm_alloc(&fz.tmem_base, 64);
    }
    if (tid == 0) {
        pol::pbar_init(&fz.bar);
        pol::pbar_init(&fz.wbar);
        fz.failed = 0;
        fz.bad = 0;
        const unsigned n1 = (unsigned)(128 * f.Dp * 2), n2 = 128 * 128 * 2, n3 = 16 * 128 * 2;
        pol::pbar_expect(&fz.wbar, 2 * (n1 + n2 + n3));
        for (int a = 0; a < 2; a++) {
            const unsigned char *src = f.wpack + (long long)a * f.wpack_stride;
            pol::bulk_g2s(fz.w1[a], src, n1, &fz.wbar);
            pol::bulk_g2s(fz.w2[a], src + n1, n2, &fz.wbar);
            pol::bulk_g2s(fz.w3[a], src + n1 + n2, n3, &fz.wbar);
        }
    }
    for (int i = tid; i < (int)(sizeof(fz.x) / 4); i += nw * 32) reinterpret_cast<unsigned *>(&fz.x[0][0])[i] = 0u;
    for (int i = tid; i < (int)(sizeof(fz.h) / 4); i += nw * 32) reinterpret_cast<unsigned *>(&fz.h[0][0])[i] = 0u;
    for (int i = tid; i < 2 * FN; i += nw * 32) (&fz.acts[0][0])[i] = 0;
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
    const bool landed = pol::pbar_wait(&fz.wbar, 0, f.wait_budget);
    if (__syncthreads_or(!landed)) {
        if (tid == 0) { fz.failed = 1; atomicOr(f.status, 4); }
        pol::pbar_wait(&fz.wbar, 0, f.wait_budget);   // let the copies in flight land
    }
    __syncthreads();
}

// Entry k of one env's observation row of agent a into the B tile, scaled
// like the network's input and rounded to BF16.  An index out of range is
// recorded and not written.
__device__ __forceinline__ void fused_put_obs(FusedSmem &fz, const FusedParams &f, int a, int row, int k, float v) {
    if ((unsigned)row >= (unsigned)FN || (unsigned)k >= (unsigned)f.D || (unsigned)a > 1u) {
        fz.bad = 1;
        return;
    }
    *reinterpret_cast<__nv_bfloat16 *>(fz.x[a] + pol::cm_off(row, k, f.Dp)) =
        __float2bfloat16_rn(v * pol::obs_scale(k, f.L));
}

// Both agents' networks on the observation tiles, the greedy actions into
// fz.acts.  Every thread of the CTA calls it (nw >= 4 warps).
__device__ __forceinline__ void fused_policy(FusedSmem &fz, const FusedParams &f, unsigned &phase, int nw, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    const unsigned tm = fz.tmem_base;
    pol::fence_async_smem();
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    const int unit = 32 * (warp & 3) + lane;                              // tensor-memory lane = hidden unit
    const unsigned lrow = tm + ((unsigned)(32 * (warp & 3)) << 16);
    const unsigned idesc = pol::idesc_bf16(128, FN);
    const int ew = nw >= 8 ? 8 : 4;                                       // epilogue warps
    for (int layer = 0; layer < 2; layer++) {
        const bool live = fz.failed == 0;                                 // the same in every thread
        if (live) {
            if (tid == 0) {
                for (int a = 0; a < 2; a++) {
                    const unsigned char *A_ = layer == 0 ? fz.w1[a] : fz.w2[a];
                    const unsigned char *B_ = layer == 0 ? fz.x[a] : fz.h[a];
                    const int K = layer == 0 ? f.Dp : 128;
                    for (int kk = 0; kk < K / 16; kk++) {
                        const unsigned long long da = pol::sdesc(A_ + kk * 256, 128, (unsigned)(K / 8) * 128);
                        const unsigned long long db = pol::sdesc(B_ + kk * 256, 128, (unsigned)(K / 8) * 128);
                        pol::mma_bf16(tm + fz_acc(a), da, db, idesc, kk > 0);
                    }
                }
                pol::mma_commit(&fz.bar);
            }
            const bool arrived = pol::pbar_wait(&fz.bar, phase, f.wait_budget);
            const bool late = __syncthreads_or(!arrived);
            if (late) {
                if (tid == 0) { fz.failed = 1; atomicOr(f.status, 4); }
                pol::pbar_wait(&fz.bar, phase, f.wait_budget);        // let the tensor core finish
            }
            phase ^= 1u;
            pol::tc_fence_after();
            // h = tanh(acc + b) into the agent's [16 envs x 128] tile
            if (warp < ew && !late) {
                for (int a = ew == 8 ? warp >> 2 : 0; a < 2; a += ew == 8 ? 2 : 1) {
                    float v[32];
                    pol::tm_ld32(lrow + fz_acc(a), v);                  // columns 0..15: this agent's envs
                    const float b = layer == 0 ? fz.b1[a][unit] : fz.b2[a][unit];
#pragma unroll
                    for (int n = 0; n < FN; n++)
                        *reinterpret_cast<__nv_bfloat16 *>(fz.h[a] + pol::cm_off(n, unit, 128)) =
                            __float2bfloat16_rn(pol::tanh_approx(v[n] + b));
                }
            }
        }
        pol::fence_async_smem();
        pol::tc_fence_before();
        __syncthreads();
        pol::tc_fence_after();
    }
    // the head: y[o] = b3[o] + sum_u W3[o][u] h2[u], one (agent, env, output) per thread
    for (int i = tid; i < 2 * FN * 13; i += nw * 32) {
        const int a = i / (FN * 13), r = i % (FN * 13), n = r / 13, o = r % 13;
        float acc = fz.b3[a][o];
        for (int u = 0; u < 128; u += 8) {
            const uint4 hw = *reinterpret_cast<const uint4 *>(fz.h[a] + pol::cm_off(n, u, 128));
            const uint4 ww = *reinterpret_cast<const uint4 *>(fz.w3[a] + pol::cm_off(o, u, 128));
            const unsigned hv[4] = {hw.x, hw.y, hw.z, hw.w}, wv[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const __nv_bfloat162 hp = *reinterpret_cast<const __nv_bfloat162 *>(&hv[q]);
                const __nv_bfloat162 wp = *reinterpret_cast<const __nv_bfloat162 *>(&wv[q]);
                acc = fmaf(__low2float(hp), __low2float(wp), acc);
                acc = fmaf(__high2float(hp), __high2float(wp), acc);
            }
        }
        fz.ys[a][n][o] = acc;
    }
    __syncthreads();
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

// Frees the tensor memory; reports a recorded index fault (status bit 8).
__device__ __forceinline__ void fused_teardown(FusedSmem &fz, const FusedParams &f, int tid) {
    pol::tc_fence_before();
    __syncthreads();
    if (tid == 0 && fz.bad) atomicOr(f.status, 8);
    if ((tid >> 5) == 0) {
        __syncwarp();
        pol::tc_fence_after();
        pol::tm_dealloc(fz.tmem_base, 64);
    }
}

}  // namespace lobk
