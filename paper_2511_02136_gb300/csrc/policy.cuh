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
#include "tc05.cuh"

namespace pol {

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

// FP32 forward on the CUDA cores, register-tiled: one CTA of 256 threads per
// (128-env tile, agent).  Every layer is a [128 x K] x [K x N] product whose
// operands sit in shared memory k-major (activations as [k][row], weights as
// [k][unit]), so a thread's 8 x 8 output tile reads two float4 of each per k
// and does 64 FMAs; the hidden activations are written back over their input
// after a barrier (the observations occupy the same buffer before layer 1).
constexpr int FT = 256;         // threads per CTA of the FP32 forward
constexpr int FDP = DMAX;       // widest (padded) observation
struct F32Smem {
    float w1t[FDP][H];          // W1^T
    float ht[H][128];           // scaled observations [feature][env row], then h1, then h2 [unit][env row]
    float w2t[H][H];            // W2^T
    float w3t[H][16];           // W3^T (outputs 13..15 zero)
    float b1[H], b2[H], b3[16];
};

__global__ void __launch_bounds__(FT, 1) k_policy_fp32(const PolicyParams p) {
    extern __shared__ __align__(16) unsigned char fraw[];
    F32Smem &sm = *reinterpret_cast<F32Smem *>(fraw);
    const int tid = threadIdx.x;
    const int a = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    const int D = p.D, Dp = (D + 3) & ~3;
    const float *wf = p.wf32 + (long long)a * p.wf32_stride;
    const float *w1 = wf, *b1 = wf + H * D, *w2 = b1 + H, *b2 = w2 + H * H, *w3 = b2 + H, *b3 = w3 + NOUT * H;
    for (int i = tid; i < H * D; i += FT) sm.w1t[i % D][i / D] = w1[i];
    for (int i = tid; i < H * (Dp - D); i += FT) sm.w1t[D + i / H][i % H] = 0.0f;
    for (int i = tid; i < H * H; i += FT) sm.w2t[i % H][i / H] = w2[i];
    for (int i = tid; i < H * 16; i += FT) {
        const int o = i / H, k = i % H;
        sm.w3t[k][o] = o < NOUT ? w3[o * H + k] : 0.0f;
    }
    if (tid < H) { sm.b1[tid] = b1[tid]; sm.b2[tid] = b2[tid]; }
    if (tid < 16) sm.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
    for (int i = tid; i < 128 * Dp; i += FT) {
        const int r = i / Dp, k = i % Dp, env = row0 + r;
        sm.ht[k][r] = (k < D && env < p.n_envs) ? p.obs[((long long)env * p.A + a) * D + k] * obs_scale(k, p.L) : 0.0f;
    }
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;   // rows 8 ty .. 8 ty + 7, units 8 tx .. 8 tx + 7
    float acc[8][8];
    // ---- two hidden layers: ht = tanh(W x + b), x = xt (layer 1) or ht (layer 2)
    for (int layer = 0; layer < 2; layer++) {
        const int K = layer == 0 ? Dp : H;
        const float *bias = layer == 0 ? sm.b1 : sm.b2;
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int j = 0; j < 8; j++) acc[i][j] = bias[8 * tx + j];
        for (int k = 0; k < K; k++) {
            const float *xa = &sm.ht[k][8 * ty];
            const float *wb = layer == 0 ? &sm.w1t[k][8 * tx] : &sm.w2t[k][8 * tx];
            const float4 a0 = *reinterpret_cast<const float4 *>(xa), a1 = *reinterpret_cast<const float4 *>(xa + 4);
            const float4 c0 = *reinterpret_cast<const float4 *>(wb), c1 = *reinterpret_cast<const float4 *>(wb + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();   // every read of the layer's input is done
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float4 t0, t1;
            t0.x = tanhf(acc[0][j]); t0.y = tanhf(acc[1][j]); t0.z = tanhf(acc[2][j]); t0.w = tanhf(acc[3][j]);
            t1.x = tanhf(acc[4][j]); t1.y = tanhf(acc[5][j]); t1.z = tanhf(acc[6][j]); t1.w = tanhf(acc[7][j]);
            *reinterpret_cast<float4 *>(&sm.ht[8 * tx + j][8 * ty]) = t0;
            *reinterpret_cast<float4 *>(&sm.ht[8 * tx + j][8 * ty + 4]) = t1;
        }
        __syncthreads();
    }
    // ---- output layer: 128 rows x 16 outputs, a thread 8 rows x 1 output
    {
        float y[8];
#pragma unroll
        for (int i = 0; i < 8; i++) y[i] = sm.b3[tx];
        for (int k = 0; k < H; k++) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sm.ht[k][8 * ty]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sm.ht[k][8 * ty + 4]);
            const float w = sm.w3t[k][tx];
            y[0] = fmaf(a0.x, w, y[0]); y[1] = fmaf(a0.y, w, y[1]); y[2] = fmaf(a0.z, w, y[2]); y[3] = fmaf(a0.w, w, y[3]);
            y[4] = fmaf(a1.x, w, y[4]); y[5] = fmaf(a1.y, w, y[5]); y[6] = fmaf(a1.z, w, y[6]); y[7] = fmaf(a1.w, w, y[7]);
        }
        __syncthreads();   // ht is free: stage the outputs [row][output] for the per-row epilogue
        float *ys = &sm.ht[0][0];
#pragma unroll
        for (int i = 0; i < 8; i++) ys[(8 * ty + i) * 16 + tx] = y[i];
        __syncthreads();
        if (tid < 128) {
            float yr[16];
#pragma unroll
            for (int j = 0; j < 16; j++) yr[j] = ys[tid * 16 + j];
            write_outputs(p, row0 + tid, a, yr);
        }
    }
}

}  // namespace pol
