// ppo.cuh -- the IPPO update on the GPU (JaxMARL-HFT Sec. 4.2: independent
// PPO, every agent its own actor-critic network and its own data).
//
// The update is the textbook one: generalised advantage estimation
// (Schulman et al. 2016), the clipped surrogate with value and entropy terms
// (Schulman et al. 2017), the gradient through the network of policy.cuh,
// clipping to a global L2 norm and Adam (Kingma & Ba 2015).  Per minibatch:
//
//   k_ppo_gae      (once per update) advantages and value targets per
//                  (agent, env), backwards over the rollout as a chunked scan;
//   k_ppo_stats    (once per update) mean and 1 / (std + 1e-8) of every
//                  minibatch's advantages;
//   k_ppo_grad     forward, loss gradient and backward of 128-sample tiles on
//                  the tensor cores (tcgen05, BF16 operands, FP32 TMEM
//                  accumulators) in two tile streams per CTA, the weight
//                  gradients accumulated in TMEM over all tiles a CTA takes,
//                  then stored into the CTA's slice of a partial buffer;
//   k_ppo_reduce   the slices summed into the gradient, and its squared
//                  global norm per agent;
//   k_ppo_adam     clip, Adam, and the BF16 repack of the new weights for
//                  both this update and the rollout's forward.
//
// The eight contractions of a tile (M = 128 everywhere; operands in the
// no-swizzle core-matrix layout of policy.cuh):
//   U1 = X W1^T,  U2 = H1 W2^T,  Y = H2 W3^T                  (forward)
//   dH2 = dY W3,  dH1 = dU2 W2                                (input gradients)
//   dW3^T += H2^T dY,  dW2 += dU2^T [H1 | 1],  dW1 += dU1^T [X | 1]
// Every tile is stored once, row by row (samples by units, or outputs by
// units for the weights), and read either K-major or MN-major: a transposed
// operand (W2^T, W3^T, and the sample-contracted H2^T, dY^T, dU2^T, [H1 | 1]^T,
// dU1^T, [X | 1]^T) is the same tile read MN-major, so no epilogue writes a
// transposed copy.  A column of ones after the inputs (X's column D, whose W1
// column is zero) and after H1 (column 128 of [H1 | 1]) gives db1 and db2 as
// the last columns of dW1 and dW2; db3 is a 16-wide sum.
#pragma once
#include "tc05.cuh"

namespace ppo {

using pol::H;
using pol::NA;
using pol::NOUT;
using pol::cm_off;

// Two tile streams per CTA: each stream of SPT threads (8 warps) takes every
// other of the CTA's tiles and runs its contractions and epilogues on its own
// operand tiles, TMEM accumulator, mbarrier and named barrier, so that one
// stream's epilogues overlap the other's contractions; the weights and the
// weight-gradient accumulators (TMEM, zeroed at the start) are shared.
constexpr int NS = 2;            // tile streams per CTA
constexpr int SPT = 256;         // threads per stream (a multiple of 128)
constexpr int PPT = NS * SPT;    // threads per CTA of the gradient kernel
constexpr int NQ = SPT / 128;    // warps of a stream per TMEM lane quarter: the column parts of an epilogue
static_assert(SPT % 128 == 0 && (128 / NQ) % 32 == 0, "an epilogue's column parts are whole 32-column loads");
constexpr int DPMAX = 48;       // widest padded input (obs dim + 1 <= 48: up to 10 levels)
constexpr int H1W = 144;        // row length of [H1 | 1]: 128 units, the ones column, padding to 16

struct GradParams {
    int A, D, Dp;                // Dp = padded (D + 1)
    int L;
    int n_envs;
    long long n_samples;         // T * n_envs (per agent)
    const float *obs;            // [T][n_envs][A][D]
    const int *actions;          // [T][n_envs][A]
    const float *logp_old;       // [T][n_envs][A]
    const float *adv;            // [A][n_samples]
    const float *ret;            // [A][n_samples]
    const int *perm;             // [A][n_samples] sample order
    long long mb_begin;          // this minibatch: perm positions [mb_begin, mb_begin + mb_size)
    int mb_size;
    const float *stats;          // [A][2]: mean, 1 / (std + 1e-8) of the minibatch's advantages
    const unsigned char *wpk;    // per agent: W1 [128 x Dp], W2 [128 x 128], W3 [16 x 128], bf16 core layout
    long long wpk_stride;        // bytes per agent
    const float *wf32;           // per agent parameter block (biases read from here)
    long long wf32_stride;
    float *gpart;                // [A][gpart_ct][P] FP32: CTA x writes all of its agent's weight gradients to slice x
    int gpart_ct;                // slices per agent (>= gridDim.x)
    float clip_eps, vf_coef, ent_coef;
    int *status;
    long long wait_budget;
};

// One stream's operand tiles and per-row data.
struct __align__(128) StreamSmem {
    unsigned char x[128 * DPMAX * 2];       // [X | 1] [128 samples x Dp]
    unsigned char r1[128 * H * 2];          // H2, then dU2, then dU1 [128 samples x 128]
    unsigned char r2[128 * H1W * 2];        // [H1 | 1] [128 samples x 144]
    unsigned char dy[128 * 16 * 2];         // dY [128 samples x 16]
    int act[128];
    float lpo[128], an[128], rt[128];
    long long orow[128];                    // the tile's samples: observation row index, or -1 past the minibatch
    unsigned long long bar;
};
// Shared memory of the gradient kernel (one CTA per SM).
struct __align__(1024) GradSmem {
    unsigned char w1[H * DPMAX * 2];        // W1 [128 x Dp] (its column D zero)
    unsigned char w2[H * H * 2];            // W2 [128 out x 128 in]; read MN-major as W2^T
    unsigned char w3[16 * H * 2];           // W3 [16 x 128]; read MN-major as W3^T
    StreamSmem st[NS];
    float b1[H], b2[H], b3[16];
    float db3[16];
    unsigned long long wbar;
    unsigned tmem_base;
};
static_assert(sizeof(GradSmem) <= 227 * 1024, "one CTA's shared memory");

// TMEM columns of the gradient kernel (512 allocated): the shared
// weight-gradient accumulators, then per stream the forward / input-gradient
// accumulator and Y.
constexpr unsigned TC_DW3 = 0;      // 16: dW3^T [128 h2 units x 16 outputs]
constexpr unsigned TC_DW1 = 16;     // Dp <= 48: dW1 [128 u1 units x Dp]
constexpr unsigned TC_DW2 = 64;     // 144: dW2 [128 u2 units x (128 + ones + pad)]
constexpr unsigned TC_STREAMS = 208;
__host__ __device__ constexpr unsigned tc_acc(int s) { return TC_STREAMS + 144u * (unsigned)s; }   // 128: U1, U2, dH2, dH1
__host__ __device__ constexpr unsigned tc_y(int s) { return tc_acc(s) + 128u; }                   // 16: Y
static_assert(TC_DW1 + DPMAX <= TC_DW2 && TC_DW2 + H1W <= TC_STREAMS && tc_y(NS - 1) + 16 <= 512,
              "TMEM regions within the 512 columns");

__device__ __forceinline__ void st_bf16(unsigned char *tile, unsigned off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(tile + off) = __float2bfloat16_rn(v);
}

// Descriptors of step kk (16 along K) of an operand held in a tile of rows
// of length Kp (element (r, c) at cm_off(r, c, Kp)): K-major when the tile's
// rows are the operand's rows (K along a row), MN-major when the tile's rows
// run along K (the operand is the tile transposed: leading offset between
// groups of 8 rows, stride offset between groups of 8 columns).
__device__ __forceinline__ unsigned long long kdesc(const unsigned char *t, int Kp, int kk) {
    return pol::sdesc(t + kk * 256, 128, (unsigned)Kp * 16);
}
__device__ __forceinline__ unsigned long long mdesc(const unsigned char *t, int Kp, int kk) {
    return pol::sdesc(t + kk * 32 * Kp, (unsigned)Kp * 16, 128);
}
// Issue C (+)= A B^T over K in steps of 16 (one thread); A [128 x K] and B
// [N x K], each from its tile (row length a_kp / b_kp) K-major or MN-major.
__device__ __forceinline__ void gemm(unsigned tmem_d, const unsigned char *A_, int a_kp, bool a_mn,
                                     const unsigned char *B_, int b_kp, bool b_mn, int K, int N, bool acc) {
    const unsigned idesc = pol::idesc_bf16(128, N) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u);
    for (int kk = 0; kk < K / 16; kk++) {
        const unsigned long long da = a_mn ? mdesc(A_, a_kp, kk) : kdesc(A_, a_kp, kk);
        const unsigned long long db = b_mn ? mdesc(B_, b_kp, kk) : kdesc(B_, b_kp, kk);
        pol::mma_bf16(tmem_d, da, db, idesc, (acc || kk > 0) ? 1 : 0);
    }
}

// Stream s's named barrier (ids 1 and 2; 0 is the whole CTA's): its SPT
// threads only.  stream_sync_or also returns whether any of them passed true.
__device__ __forceinline__ void stream_sync(int s) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + s), "r"(SPT) : "memory");
}
__device__ __forceinline__ bool stream_sync_or(int s, bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r) : "r"(v ? 1u : 0u), "r"(1 + s), "r"(SPT) : "memory");
    return r != 0;
}
// Commit the MMAs the stream's issuing thread (ts == 0) issued and wait for
// them (all the stream's threads); false on timeout.
__device__ __forceinline__ bool mma_round(StreamSmem &S, int s, unsigned &phase, const GradParams &p, int ts) {
    if (ts == 0) pol::mma_commit(&S.bar);
    const bool arrived = pol::pbar_wait(&S.bar, phase, p.wait_budget);
    if (stream_sync_or(s, !arrived)) {
        if (ts == 0) atomicOr(p.status, 4);
        pol::pbar_wait(&S.bar, phase, p.wait_budget);   // let the tensor core finish before TMEM is freed
        return false;
    }
    phase ^= 1u;
    pol::tc_fence_after();
    return true;
}
// Make the stream's shared-memory writes visible to the tensor core.
__device__ __forceinline__ void to_async(int s) {
    pol::fence_async_smem();
    pol::tc_fence_before();
    stream_sync(s);
    pol::tc_fence_after();
}

// Sample smp's observation row index and per-row data (smp < 0: past the
// minibatch): the action, the behaviour log-probability, the normalised
// advantage and the value target.
struct RowData {
    long long ra;
    int act;
    float lpo, an, rt;
};
__device__ __forceinline__ RowData row_data(const GradParams &p, int a, const float *advp, const float *retp,
                                            float mean, float istd, int smp) {
    RowData d{-1, 0, 0.0f, 0.0f, 0.0f};
    if (smp >= 0) {
        const int t = smp / p.n_envs, e = smp - t * p.n_envs;
        d.ra = ((long long)t * p.n_envs + e) * p.A + a;
        d.act = p.actions[d.ra];
        d.lpo = p.logp_old[d.ra];
        d.an = (advp[smp] - mean) * istd;
        d.rt = retp[smp];
    }
    return d;
}
__device__ __forceinline__ void put_row_data(StreamSmem &sm, int i, const RowData &d) {
    sm.orow[i] = d.ra;
    sm.act[i] = d.act;
    sm.lpo[i] = d.lpo;
    sm.an[i] = d.an;
    sm.rt[i] = d.rt;
}
constexpr int RPW = 128 / (SPT / 32);   // tile rows per warp of a stream
// This warp's observation rows (sw, sw + 8, ...) of the tile sm.orow names,
// features 2 lane and 2 lane + 1, all loads issued before any is used.
__device__ __forceinline__ void load_rows(const GradParams &p, const StreamSmem &sm, int sw, int lane,
                                          float (&va)[RPW], float (&vb)[RPW]) {
    const int D = p.D;
#pragma unroll
    for (int j = 0; j < RPW; j++) {
        const long long ra = sm.orow[sw + (SPT / 32) * j];
        const float *o = p.obs + (ra < 0 ? 0 : ra) * (long long)D;
        va[j] = (ra >= 0 && 2 * lane < D) ? o[2 * lane] : 0.0f;
        vb[j] = (ra >= 0 && 2 * lane + 1 < D) ? o[2 * lane + 1] : 0.0f;
    }
}

__global__ void __launch_bounds__(PPT, 1) k_ppo_grad(const GradParams p) {
    extern __shared__ __align__(1024) unsigned char graw[];
    GradSmem &sm = *reinterpret_cast<GradSmem *>(graw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int a = blockIdx.y;
    const int Dp = p.Dp, D = p.D;
    const int n_tiles = (p.mb_size + 127) / 128;
    if (warp == 0) pol::tm_alloc(&sm.tmem_base, 512);
    if (tid == 0) {
        for (int s = 0; s < NS; s++) pol::pbar_init(&sm.st[s].bar);
        pol::pbar_init(&sm.wbar);
        const unsigned char *src = p.wpk + (long long)a * p.wpk_stride;
        const unsigned n1 = (unsigned)(H * Dp * 2), n2 = H * H * 2, n3 = 16 * H * 2;
        pol::pbar_expect(&sm.wbar, n1 + n2 + n3);
        pol::bulk_g2s(sm.w1, src, n1, &sm.wbar);
        pol::bulk_g2s(sm.w2, src + n1, n2, &sm.wbar);
        pol::bulk_g2s(sm.w3, src + n1 + n2, n3, &sm.wbar);
    }
    {
        const float *wf = p.wf32 + (long long)a * p.wf32_stride;
        const float *b1 = wf + H * D, *b2 = b1 + H + H * H, *b3 = b2 + H + NOUT * H;
        if (tid < H) sm.b1[tid] = b1[tid];
        else if (tid < 2 * H) sm.b2[tid - H] = b2[tid - H];
        if (tid < 16) {
            sm.b3[tid] = tid < NOUT ? b3[tid] : 0.0f;
            sm.db3[tid] = 0.0f;
        }
    }
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    const unsigned tmem = sm.tmem_base;
    // the weight-gradient accumulators start at zero (both streams accumulate
    // into them from their first tile): 13 groups of 16 columns per lane
    // quarter, spread over the four warps of each quarter
    {
        const unsigned qrow = tmem + ((unsigned)(32 * (warp & 3)) << 16);
        for (int g = warp >> 2; g < (int)(TC_STREAMS / 16); g += PPT / 128) pol::tm_zero16(qrow + 16u * (unsigned)g);
    }
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    // this thread's stream, its thread and warp within the stream
    const int s = warp / (SPT / 32), ts = tid - s * SPT, sw = warp - s * (SPT / 32);
    StreamSmem &S = sm.st[s];
    const unsigned TA = tc_acc(s), TY = tc_y(s);
    const int row = 32 * (warp & 3) + lane;         // TMEM lane = sample row (or unit row for dW)
    const int part = sw >> 2;                       // this warp's column part of an epilogue
    const int cb = part * (H / NQ), ce = cb + H / NQ;   // its columns of a 128-wide accumulator
    const unsigned lrow = tmem + ((unsigned)(32 * (warp & 3)) << 16);
    bool ok = true;
    unsigned phase = 0;
    {
        const bool landed = pol::pbar_wait(&sm.wbar, 0, p.wait_budget);
        if (__syncthreads_or(!landed)) {
            ok = false;
            if (tid == 0) atomicOr(p.status, 4);
            pol::pbar_wait(&sm.wbar, 0, p.wait_budget);
        }
    }
    const float mean = p.stats[2 * a], istd = p.stats[2 * a + 1];
    const float inv_b = 1.0f / (float)p.mb_size;
    const float *advp = p.adv + (long long)a * p.n_samples, *retp = p.ret + (long long)a * p.n_samples;
    const int *perm = p.perm + (long long)a * p.n_samples + p.mb_begin;
    // Stream s takes tiles blockIdx.x + (s + NS k) gridDim.x.  Its samples are
    // gathered one tile ahead: while a tile's contractions run, the next
    // tile's sample indices, per-row data and observation rows are loaded, so
    // their latency stays off the tile's chain.
    const int tile0 = (int)blockIdx.x + s * (int)gridDim.x, tstep = NS * (int)gridDim.x;
    float va[RPW], vb[RPW];
    int n_smp = -1;
    RowData nd{-1, 0, 0.0f, 0.0f, 0.0f};
    if (ok && tile0 < n_tiles) {
        if (ts < 128)
            put_row_data(S, ts, row_data(p, a, advp, retp, mean, istd,
                                         tile0 * 128 + ts < p.mb_size ? perm[tile0 * 128 + ts] : -1));
        stream_sync(s);
        load_rows(p, S, sw, lane, va, vb);
    }
    for (int tile = tile0; tile < n_tiles && ok; tile += tstep) {
        const int next = tile + tstep;
        // ---- [X | 1] (scaled, bf16) from the rows loaded ahead; W1's column D
        // is zero, so the forward reads the same tile
        // features 2 lane and 2 lane + 1 of each of this warp's rows: one
        // 4-byte store of the bf16 pair (adjacent in the core-matrix row)
        {
            const int k0 = 2 * lane, k1 = 2 * lane + 1;
            const float s0 = k0 < D ? pol::obs_scale(k0, p.L) : 0.0f, s1 = k1 < D ? pol::obs_scale(k1, p.L) : 0.0f;
            const float c0 = k0 == D ? 1.0f : 0.0f, c1 = k1 == D ? 1.0f : 0.0f;   // the ones column
#pragma unroll
            for (int j = 0; j < RPW; j++) {
                const int i = sw + (SPT / 32) * j;
                if (k0 < Dp) {
                    const bool valid = S.orow[i] >= 0;
                    const float v0 = valid ? (k0 < D ? va[j] * s0 : c0) : 0.0f;
                    const float v1 = valid ? (k1 < D ? vb[j] * s1 : c1) : 0.0f;
                    const __nv_bfloat162 t2 = __floats2bfloat162_rn(v0, v1);
                    *reinterpret_cast<__nv_bfloat162 *>(S.x + cm_off(i, k0, Dp)) = t2;
                }
            }
        }
        to_async(s);
        // ---- U1 = X W1^T
        if (ts == 0) gemm(tmem + TA, S.x, Dp, false, sm.w1, Dp, false, Dp, H, false);
        if (ts < 128) n_smp = next < n_tiles && next * 128 + ts < p.mb_size ? perm[next * 128 + ts] : -1;
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
        // h1 = tanh(U1 + b1) -> [H1 | 1] (r2): this thread's row, 16-byte stores
        for (int c0 = cb; c0 < ce; c0 += 32) {
            float v[32];
            pol::tm_ld32(lrow + TA + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                unsigned w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float h0 = pol::tanh_approx(v[j + 2 * q] + sm.b1[c0 + j + 2 * q]);
                    const float h1 = pol::tanh_approx(v[j + 2 * q + 1] + sm.b1[c0 + j + 2 * q + 1]);
                    const __nv_bfloat162 t2 = __floats2bfloat162_rn(h0, h1);
                    w[q] = *reinterpret_cast<const unsigned *>(&t2);
                }
                *reinterpret_cast<uint4 *>(S.r2 + cm_off(row, c0 + j, H1W)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        if (part == NQ - 1) {   // the ones column (valid samples) and the zero padding of [H1 | 1]
            const bool valid = tile * 128 + row < p.mb_size;
            const __nv_bfloat162 one = __floats2bfloat162_rn(valid ? 1.0f : 0.0f, 0.0f);
            const unsigned o = *reinterpret_cast<const unsigned *>(&one);
            *reinterpret_cast<uint4 *>(S.r2 + cm_off(row, H, H1W)) = make_uint4(o, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(S.r2 + cm_off(row, H + 8, H1W)) = make_uint4(0u, 0u, 0u, 0u);
        }
        to_async(s);
        // ---- U2 = H1 W2^T
        if (ts == 0) gemm(tmem + TA, S.r2, H1W, false, sm.w2, H, false, H, H, false);
        if (ts < 128) nd = row_data(p, a, advp, retp, mean, istd, n_smp);   // the next tile's, in flight
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
        for (int c0 = cb; c0 < ce; c0 += 32) {
            float v[32];
            pol::tm_ld32(lrow + TA + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                unsigned w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float h0 = pol::tanh_approx(v[j + 2 * q] + sm.b2[c0 + j + 2 * q]);
                    const float h1 = pol::tanh_approx(v[j + 2 * q + 1] + sm.b2[c0 + j + 2 * q + 1]);
                    const __nv_bfloat162 t2 = __floats2bfloat162_rn(h0, h1);
                    w[q] = *reinterpret_cast<const unsigned *>(&t2);
                }
                *reinterpret_cast<uint4 *>(S.r1 + cm_off(row, c0 + j, H)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        to_async(s);
        // ---- Y = H2 W3^T, then the loss gradient dY per sample
        if (ts == 0) gemm(tmem + TY, S.r1, H, false, sm.w3, H, false, H, 16, false);
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
        if (part == 0) {
            float v[16];
            pol::tm_ld16(lrow + TY, v);
            const bool valid = tile * 128 + row < p.mb_size;
            float z[NA];
            float m = -INFINITY;
#pragma unroll
            for (int j = 0; j < NA; j++) {
                z[j] = v[j] + sm.b3[j];
                m = fmaxf(m, z[j]);
            }
            const float V = v[NA] + sm.b3[NA];
            float se = 0.0f;
#pragma unroll
            for (int j = 0; j < NA; j++) se += __expf(z[j] - m);
            const float lse = m + __logf(se);
            float pj[NA], lp[NA], Sent = 0.0f;
#pragma unroll
            for (int j = 0; j < NA; j++) {
                lp[j] = z[j] - lse;
                pj[j] = __expf(lp[j]);
                Sent -= pj[j] * lp[j];
            }
            const int act = S.act[row];
            float lpa = lp[0];
#pragma unroll
            for (int j = 1; j < NA; j++)
                if (j == act) lpa = lp[j];
            const float rho = __expf(lpa - S.lpo[row]);
            const float An = S.an[row];
            const float rc = fminf(fmaxf(rho, 1.0f - p.clip_eps), 1.0f + p.clip_eps);
            const float g_rho = (rho * An <= rc * An) ? -An : 0.0f;
            float dy[16];
#pragma unroll
            for (int j = 0; j < NA; j++) {
                const float pg = g_rho * rho * ((j == act ? 1.0f : 0.0f) - pj[j]);
                dy[j] = valid ? (pg + p.ent_coef * pj[j] * (lp[j] + Sent)) * inv_b : 0.0f;
            }
            dy[NA] = valid ? p.vf_coef * (V - S.rt[row]) * inv_b : 0.0f;
#pragma unroll
            for (int j = NA + 1; j < 16; j++) dy[j] = 0.0f;
            unsigned w[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const __nv_bfloat162 t2 = __floats2bfloat162_rn(dy[2 * q], dy[2 * q + 1]);
                w[q] = *reinterpret_cast<const unsigned *>(&t2);
            }
            *reinterpret_cast<uint4 *>(S.dy + cm_off(row, 0, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(S.dy + cm_off(row, 8, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
            // db3: the bf16-rounded dY the other products use, summed over the
            // tile by a reduce-scatter butterfly (each step halves the columns a
            // lane carries: 16 shuffles for the 16 columns), then one atomic
            // per column from the even lanes
            {
                float r16[16];
#pragma unroll
                for (int j = 0; j < 16; j++) r16[j] = __bfloat162float(__float2bfloat16_rn(dy[j]));
                float r8[8], r4[4], r2[2];
                const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0, b1 = (lane & 2) != 0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    r8[j] = (b4 ? r16[j + 8] : r16[j]) + __shfl_xor_sync(0xffffffffu, b4 ? r16[j] : r16[j + 8], 16);
#pragma unroll
                for (int j = 0; j < 4; j++)
                    r4[j] = (b3 ? r8[j + 4] : r8[j]) + __shfl_xor_sync(0xffffffffu, b3 ? r8[j] : r8[j + 4], 8);
#pragma unroll
                for (int j = 0; j < 2; j++)
                    r2[j] = (b2 ? r4[j + 2] : r4[j]) + __shfl_xor_sync(0xffffffffu, b2 ? r4[j] : r4[j + 2], 4);
                float r1 = (b1 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? r2[0] : r2[1], 2);
                r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
                const int col = (b4 ? 8 : 0) + (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
                if ((lane & 1) == 0) atomicAdd(&sm.db3[col], r1);
            }
        }
        to_async(s);
        // ---- dH2 = dY W3 and dW3^T += H2^T dY (this tile's per-row data is no
        // longer read: the next tile's takes its place)
        if (ts < 128) put_row_data(S, ts, nd);
        if (ts == 0) {
            gemm(tmem + TA, S.dy, 16, false, sm.w3, H, true, 16, H, false);        // W3^T: W3 read MN-major
            gemm(tmem + TC_DW3, S.r1, H, true, S.dy, 16, true, 128, 16, true);     // H2^T, dY^T: both MN-major
        }
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
        // dU2 = dH2 (1 - h2^2): dU2 into r1 in place of H2
        for (int c0 = cb; c0 < ce; c0 += 32) {
            float v[32];
            pol::tm_ld32(lrow + TA + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                const uint4 hv = *reinterpret_cast<const uint4 *>(S.r1 + cm_off(row, c0 + j, H));
                const unsigned hw[4] = {hv.x, hv.y, hv.z, hv.w};
                unsigned w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162 *>(&hw[q]);
                    const float ha = __low2float(h2), hb = __high2float(h2);
                    const float d0 = v[j + 2 * q] * (1.0f - ha * ha), d1 = v[j + 2 * q + 1] * (1.0f - hb * hb);
                    const __nv_bfloat162 t2 = __floats2bfloat162_rn(d0, d1);
                    w[q] = *reinterpret_cast<const unsigned *>(&t2);
                }
                *reinterpret_cast<uint4 *>(S.r1 + cm_off(row, c0 + j, H)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        to_async(s);
        // ---- dH1 = dU2 W2 and dW2 += dU2^T [H1 | 1]; the next tile's rows in flight
        load_rows(p, S, sw, lane, va, vb);
        if (ts == 0) {
            gemm(tmem + TA, S.r1, H, false, sm.w2, H, true, H, H, false);          // W2^T: W2 read MN-major
            gemm(tmem + TC_DW2, S.r1, H, true, S.r2, H1W, true, 128, H1W, true);   // dU2^T, [H1 | 1]^T
        }
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
        // dU1 = dH1 (1 - h1^2), h1 from [H1 | 1]: dU1 into r1 (this thread's row)
        for (int c0 = cb; c0 < ce; c0 += 32) {
            float v[32];
            pol::tm_ld32(lrow + TA + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                const uint4 hv = *reinterpret_cast<const uint4 *>(S.r2 + cm_off(row, c0 + j, H1W));
                const unsigned hw[4] = {hv.x, hv.y, hv.z, hv.w};
                unsigned w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const __nv_bfloat162 h1 = *reinterpret_cast<const __nv_bfloat162 *>(&hw[q]);
                    const float ha = __low2float(h1), hb = __high2float(h1);
                    const __nv_bfloat162 t2 = __floats2bfloat162_rn(v[j + 2 * q] * (1.0f - ha * ha),
                                                                    v[j + 2 * q + 1] * (1.0f - hb * hb));
                    w[q] = *reinterpret_cast<const unsigned *>(&t2);
                }
                *reinterpret_cast<uint4 *>(S.r1 + cm_off(row, c0 + j, H)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        to_async(s);
        // ---- dW1 += dU1^T [X | 1]
        if (ts == 0) gemm(tmem + TC_DW1, S.r1, H, true, S.x, Dp, true, 128, Dp, true);   // both MN-major
        if (!(ok = mma_round(S, s, phase, p, ts))) break;
    }
    // ---- both streams done: the CTA's weight gradients, plain stores into its
    // own slice of the partial buffer (k_ppo_reduce sums the slices); all 16
    // warps, four per TMEM lane quarter, 32-column parts
    pol::tc_fence_before();
    __syncthreads();
    pol::tc_fence_after();
    {
        const int fp = warp >> 2;                    // flush part 0..3
        float *g = p.gpart + ((long long)a * p.gpart_ct + blockIdx.x) * p.wf32_stride;
        float *gW1 = g, *gb1 = g + H * D, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + NOUT * H;
        // dW1 (row = u1 unit): columns < D, column D = db1
        for (int c0 = 32 * fp; c0 < Dp; c0 += PPT / 4) {
            float v[32];
            pol::tm_ld32(lrow + TC_DW1 + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int k = c0 + j;
                if (k < D) gW1[row * D + k] = v[j];
                else if (k == D) gb1[row] = v[j];
            }
        }
        // dW2 (row = u2 unit): columns < 128, column 128 = db2
        for (int c0 = 32 * fp; c0 < H1W; c0 += PPT / 4) {
            float v[32];
            pol::tm_ld32(lrow + TC_DW2 + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int k = c0 + j;
                if (k < H) gW2[row * H + k] = v[j];
                else if (k == H) gb2[row] = v[j];
            }
        }
        // dW3^T (row = h2 unit, column = output)
        if (fp == 0) {
            float v[16];
            pol::tm_ld16(lrow + TC_DW3, v);
#pragma unroll
            for (int o = 0; o < NOUT; o++) gW3[o * H + row] = v[o];
        }
        if (tid < NOUT) gb3[tid] = sm.db3[tid];
    }
    pol::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        pol::tc_fence_after();
        pol::tm_dealloc(tmem, 512);
    }
}

// Advantages and value targets (GAE) over the rollout, backwards in t:
// delta = r + gamma (1 - d) V' - V, A = delta + gamma lambda (1 - d) A'.  A
// block takes GAE_PAIRS (agent, env) pairs, each split into GAE_CH chunks of
// steps, one warp per chunk (lane = pair): every chunk composes its steps
// into one affine map A_lo = P + Q A_hi, one warp chains the maps from
// A_T = 0 to get each chunk's boundary value, and every chunk then runs the
// recurrence over its own steps from that value (the rollout reads hit L2 the
// second time).  Launch: ceil(n A / GAE_PAIRS) blocks of GAE_PAIRS * GAE_CH threads.
constexpr int GAE_PAIRS = 32, GAE_CH = 16;
__global__ void __launch_bounds__(GAE_PAIRS * GAE_CH) k_ppo_gae(const long long *rewards, const float *values,
                                                                const unsigned char *done, int T, int n, int A,
                                                                float gamma, float lam, float reward_scale,
                                                                float *adv, float *ret) {
    __shared__ float sP[GAE_CH][GAE_PAIRS], sQ[GAE_CH][GAE_PAIRS], sE[GAE_CH][GAE_PAIRS];
    const int li = threadIdx.x % GAE_PAIRS, c = threadIdx.x / GAE_PAIRS;
    const int i = blockIdx.x * GAE_PAIRS + li;
    const bool on = i < n * A;
    const int e = on ? i / A : 0, a = on ? i - e * A : 0;
    const long long ns = (long long)T * n;
    const int CH = (T + GAE_CH - 1) / GAE_CH;
    const int t_lo = min(T, c * CH), t_hi = min(T, t_lo + CH);
    float P = 0.0f, Q = 1.0f;
    if (on) {
        float vn = values[((long long)t_hi * n + e) * A + a];
#pragma unroll 4
        for (int t = t_hi - 1; t >= t_lo; t--) {
            const long long ra = ((long long)t * n + e) * A + a;
            const float live = done[(long long)t * n + e] ? 0.0f : 1.0f;
            const float v = values[ra];
            const float delta = reward_scale * (float)rewards[ra] + gamma * live * vn - v;
            const float ct = gamma * lam * live;
            P = delta + ct * P;
            Q = ct * Q;
            vn = v;
        }
    }
    sP[c][li] = P;
    sQ[c][li] = Q;
    __syncthreads();
    if (c == 0) {
        float A_end = 0.0f;   // A_T
        for (int k = GAE_CH - 1; k >= 0; k--) {
            sE[k][li] = A_end;
            A_end = sP[k][li] + sQ[k][li] * A_end;
        }
    }
    __syncthreads();
    if (on) {
        float nxt = sE[c][li];
        float vn = values[((long long)t_hi * n + e) * A + a];
#pragma unroll 4
        for (int t = t_hi - 1; t >= t_lo; t--) {
            const long long ra = ((long long)t * n + e) * A + a;
            const float live = done[(long long)t * n + e] ? 0.0f : 1.0f;
            const float v = values[ra];
            const float delta = reward_scale * (float)rewards[ra] + gamma * live * vn - v;
            nxt = delta + gamma * lam * live * nxt;
            adv[(long long)a * ns + (long long)t * n + e] = nxt;
            ret[(long long)a * ns + (long long)t * n + e] = nxt + v;
            vn = v;
        }
    }
}

// Sum over a block of 256 threads (FP64), valid in thread 0.
__device__ __forceinline__ double block_sum256(double v, double *red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; w++) t += red[w];
    __syncthreads();
    return t;
}

// Sum and sum of squares (FP64) of every minibatch's advantages per agent
// (blockIdx.z = minibatch, of mb_size consecutive positions of the sample
// order; one atomic pair per block), then, in the last block of a minibatch
// to finish, their mean and 1 / (std + 1e-8) (population std) per agent.
// acc: [n_mb][A][2] sums, zeroed before the launch; ctr: [n_mb] block counters,
// zeroed before the launch; stats: [n_mb][A][2].  Launch: blocks of 256
// threads, grid (x, A, n_mb), once per epoch after GAE.
__global__ void __launch_bounds__(256) k_ppo_stats(const float *adv, const int *perm, long long ns, int mb_size, int A,
                                                   double *acc, unsigned *ctr, float *stats) {
    __shared__ double red[8];
    __shared__ bool last;
    const int a = blockIdx.y, k = blockIdx.z;
    const long long mb_begin = (long long)k * mb_size;
    double *acc_k = acc + (long long)k * 2 * A;
    double s = 0.0, s2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < mb_size; i += (long long)gridDim.x * blockDim.x) {
        const double v = adv[(long long)a * ns + perm[(long long)a * ns + mb_begin + i]];
        s += v;
        s2 += v * v;
    }
    s = block_sum256(s, red);
    s2 = block_sum256(s2, red);
    if (threadIdx.x == 0) {
        atomicAdd(&acc_k[2 * a], s);
        atomicAdd(&acc_k[2 * a + 1], s2);
        __threadfence();
        last = atomicAdd(ctr + k, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < A) {
        const int b = threadIdx.x;
        const volatile double *va = acc_k;
        const double mean = va[2 * b] / mb_size;
        double var = va[2 * b + 1] / mb_size - mean * mean;
        var = var > 0.0 ? var : 0.0;
        stats[((long long)k * A + b) * 2] = (float)mean;
        stats[((long long)k * A + b) * 2 + 1] = (float)(1.0 / (sqrt(var) + 1e-8));
    }
}

// Each agent's gradient: the sum over the n_ct gradient CTAs' slices of the
// partial buffer ([A][stride_ct][P]), and its squared L2 norm (FP64 sums, one
// atomic per block into sqnorm[a]).  Launch: blocks of 256 threads, grid (x, A).
__global__ void __launch_bounds__(256) k_ppo_reduce(const float *gpart, int n_ct, int stride_ct, long long P,
                                                    float *grad, double *sqnorm) {
    __shared__ double red[8];
    const int a = blockIdx.y;
    const float *src = gpart + (long long)a * stride_ct * P;
    double sq = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        // 16 slices' loads in flight at a time
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int c = 0;
        for (; c + 16 <= n_ct; c += 16) {
            float t[16];
#pragma unroll
            for (int u = 0; u < 16; u++) t[u] = src[(long long)(c + u) * P + i];
#pragma unroll
            for (int u = 0; u < 16; u++) acc[u & 3] += t[u];
        }
        for (; c < n_ct; c++) acc[0] += src[(long long)c * P + i];
        const float gsum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        grad[(long long)a * P + i] = gsum;
        sq += (double)gsum * gsum;
    }
    sq = block_sum256(sq, red);
    if (threadIdx.x == 0) atomicAdd(&sqnorm[a], sq);
}

struct AdamParams {
    int A, D, Dp, Dpf;               // Dp: the update's padded width, Dpf: the rollout forward's
    long long P;
    float *w;                        // [A][P] master FP32 parameters
    float *m, *v;                    // [A][P] Adam moments
    const float *grad;               // [A][P]
    const double *sqnorm;            // [A]
    float lr, beta1, beta2, eps, max_norm;
    float bc1, bc2;                  // 1 - beta^t for this step
    unsigned char *wpk;              // the update's packed bf16 weights
    long long wpk_stride;
    unsigned char *wfwd;             // the rollout forward's packed bf16 weights (W1 [128 x Dpf], W2, W3)
    long long wfwd_stride;
};

// Weight i of an agent's block (a weight matrix entry; biases are skipped)
// into both packed bf16 layouts: the update's (W1 with its zero bias column, W2, W3) and the
// rollout forward's (W1, W2, W3).
__device__ __forceinline__ void repack_one(const AdamParams &p, int a, long long i, float w) {
    const int D = p.D;
    unsigned char *u = p.wpk + (long long)a * p.wpk_stride;
    unsigned char *f = p.wfwd + (long long)a * p.wfwd_stride;
    const unsigned n1 = (unsigned)(H * p.Dp * 2), n1f = (unsigned)(H * p.Dpf * 2), n2 = H * H * 2;
    long long o = i;
    if (o < (long long)H * D) {
        const int r = (int)(o / D), c = (int)(o % D);
        st_bf16(u, cm_off(r, c, p.Dp), w);
        st_bf16(f, cm_off(r, c, p.Dpf), w);
        return;
    }
    o -= (long long)H * D + H;
    if (o >= 0 && o < (long long)H * H) {
        const int r = (int)(o / H), c = (int)(o % H);
        st_bf16(u + n1, cm_off(r, c, H), w);                      // W2 [out x in]
        st_bf16(f + n1f, cm_off(r, c, H), w);
        return;
    }
    o -= (long long)H * H + H;
    if (o >= 0 && o < (long long)NOUT * H) {
        const int r = (int)(o / H), c = (int)(o % H);
        st_bf16(u + n1 + n2, cm_off(r, c, H), w);                 // W3 [16 x 128]
        st_bf16(f + n1f + n2, cm_off(r, c, H), w);
    }
}

// The packed layouts from the FP32 weights (before the first update; the
// padding of the update's layout is zeroed by the host).
__global__ void k_ppo_pack(const AdamParams p) {
    const int a = blockIdx.y;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += (long long)gridDim.x * blockDim.x)
        repack_one(p, a, i, p.w[(long long)a * p.P + i]);
}

// Clip to the global norm, one Adam step, and the bf16 repack of every
// changed weight into both packed layouts.
__global__ void k_ppo_adam(const AdamParams p) {
    const int a = blockIdx.y;
    const double n2 = p.sqnorm[a];
    const float nrm = (float)sqrt(n2);
    const float sc = (nrm > p.max_norm && nrm > 0.0f) ? p.max_norm / nrm : 1.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += (long long)gridDim.x * blockDim.x) {
        const long long k = (long long)a * p.P + i;
        const float g = p.grad[k] * sc;
        const float m = p.beta1 * p.m[k] + (1.0f - p.beta1) * g;
        const float v = p.beta2 * p.v[k] + (1.0f - p.beta2) * g * g;
        p.m[k] = m;
        p.v[k] = v;
        const float w = p.w[k] - p.lr * (m / p.bc1) / (sqrtf(v / p.bc2) + p.eps);
        p.w[k] = w;
        repack_one(p, a, i, w);   // the weight matrices (biases stay FP32)
    }
}

}  // namespace ppo
