// policy_api.cu -- host side of the actor-critic policy entry points of
// include/lob.h: weight packing (FP32 -> BF16 core-matrix layout), device
// buffers, the two forward launches of policy.cuh and the IPPO update of
// ppo.cuh (optimiser state and work buffers live in the policy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lob.h"
#include "policy.cuh"
#include "policy_internal.h"
#include "ppo.cuh"
#include "fused.cuh"

using namespace pol;

struct lob_policy {
    int A = 0, D = 0, Dp = 0, L = 0;
    unsigned char *d_wpack = nullptr;
    long long wpack_stride = 0;
    float *d_wf32 = nullptr;
    long long wf32_stride = 0;
    int *d_status = nullptr;
    long long launches = 0;
    // IPPO update (allocated by the first lob_ppo_update)
    int upd_Dp = 0;                       // padded (D + 1)
    unsigned char *d_wpk = nullptr;       // the update's packed weights (W1 with a zero bias column, W2, W3)
    long long wpk_stride = 0;
    float *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    float *d_gpart = nullptr;             // [A][gpart_ctas][P]: each gradient CTA's own weight gradients
    int gpart_ctas = 0;
    float *d_adv = nullptr, *d_ret = nullptr;
    long long adv_cap = 0;                // samples per agent the advantage buffers hold
    int mb_cap = 0;                       // minibatches the statistics buffers hold
    float *d_stats = nullptr;             // [mb][A][2]: mean, 1 / (std + 1e-8) of each minibatch's advantages
    double *d_acc = nullptr;              // [mb][A][2] sums, [mb][A] squared norms, [mb] block counters; zeroed per update
    long long adam_t = 0;
};

static unsigned short f2bf(float f) {
    // round to nearest even, as __float2bfloat16_rn does for finite values
    unsigned u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (unsigned short)((u >> 16) | ((u & 0xFFFF) ? 0x40 : 0));
    const unsigned r = 0x7FFFu + ((u >> 16) & 1u);
    return (unsigned short)((u + r) >> 16);
}

extern "C" int64_t lob_policy_param_count(int32_t obs_dim) {
    if (obs_dim < 1 || obs_dim > DMAX) return 0;
    return (int64_t)H * obs_dim + H + (int64_t)H * H + H + (int64_t)NOUT * H + NOUT;
}

extern "C" int lob_policy_create(int32_t n_agents, int32_t obs_dim, const float *h_params, lob_policy **out) {
    if (!out) return LOB_EINVAL;
    *out = nullptr;
    if (n_agents < 1 || n_agents > 2 * LOB_MAX_PER_TYPE || !h_params || obs_dim < 5 || (obs_dim - 5) % 4 != 0)
        return LOB_EINVAL;
    if (obs_dim > DMAX) return LOB_ECAPACITY;
    // opt both forward kernels into their shared memory (per device, at creation)
    if (cudaFuncSetAttribute(k_policy_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Bf16Smem)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_policy_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(F32Smem)) !=
            cudaSuccess)
        return LOB_ECUDA;
    lob_policy *p = new (std::nothrow) lob_policy();
    if (!p) return LOB_ENOMEM;
    p->A = n_agents;
    p->D = obs_dim;
    p->Dp = (obs_dim + 15) / 16 * 16;
    p->L = (obs_dim - 5) / 4;
    p->wf32_stride = lob_policy_param_count(obs_dim);
    p->wpack_stride = ((long long)H * p->Dp + (long long)H * H + 16LL * H) * 2;
    std::vector<unsigned char> pack((size_t)(p->wpack_stride * n_agents), 0);
    for (int a = 0; a < n_agents; a++) {
        const float *w = h_params + (size_t)a * p->wf32_stride;
        const float *w1 = w, *w2 = w + H * obs_dim + H, *w3 = w2 + H * H + H;
        unsigned char *dst = pack.data() + (size_t)a * p->wpack_stride;
        unsigned char *d1 = dst, *d2 = dst + (size_t)H * p->Dp * 2, *d3 = d2 + (size_t)H * H * 2;
        for (int r = 0; r < H; r++)
            for (int k = 0; k < p->Dp; k++) {
                const unsigned short v = k < obs_dim ? f2bf(w1[r * obs_dim + k]) : 0;
                std::memcpy(d1 + cm_off(r, k, p->Dp), &v, 2);
            }
        for (int r = 0; r < H; r++)
            for (int k = 0; k < H; k++) {
                const unsigned short v = f2bf(w2[r * H + k]);
                std::memcpy(d2 + cm_off(r, k, H), &v, 2);
            }
        for (int r = 0; r < 16; r++)
            for (int k = 0; k < H; k++) {
                const unsigned short v = r < NOUT ? f2bf(w3[r * H + k]) : 0;
                std::memcpy(d3 + cm_off(r, k, H), &v, 2);
            }
    }
    bool fail = cudaMalloc(&p->d_wpack, pack.size()) != cudaSuccess;
    fail = fail || cudaMalloc(&p->d_wf32, sizeof(float) * (size_t)(p->wf32_stride * n_agents)) != cudaSuccess;
    fail = fail || cudaMalloc(&p->d_status, 4) != cudaSuccess;
    if (fail) {
        cudaGetLastError();
        if (p->d_wpack) cudaFree(p->d_wpack);
        if (p->d_wf32) cudaFree(p->d_wf32);
        if (p->d_status) cudaFree(p->d_status);
        delete p;
        return LOB_ENOMEM;
    }
    int rc = cudaMemcpy(p->d_wpack, pack.data(), pack.size(), cudaMemcpyHostToDevice) == cudaSuccess ? 0 : 1;
    rc |= cudaMemcpy(p->d_wf32, h_params, sizeof(float) * (size_t)(p->wf32_stride * n_agents),
                     cudaMemcpyHostToDevice) == cudaSuccess ? 0 : 1;
    rc |= cudaMemset(p->d_status, 0, 4) == cudaSuccess ? 0 : 1;
    if (rc) {
        lob_policy_destroy(p);
        return LOB_ECUDA;
    }
    *out = p;
    return LOB_OK;
}

extern "C" int lob_policy_destroy(lob_policy *p) {
    if (!p) return LOB_EINVAL;
    cudaDeviceSynchronize();
    void *bufs[] = {p->d_wpack, p->d_wf32, p->d_status, p->d_wpk, p->d_m, p->d_v, p->d_grad, p->d_gpart,
                    p->d_adv, p->d_ret, p->d_stats, p->d_acc};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
    return LOB_OK;
}

extern "C" int lob_policy_get_params(lob_policy *pol, float *d_out, void *stream) {
    if (!pol || !d_out) return LOB_EINVAL;
    return cudaMemcpyAsync(d_out, pol->d_wf32, sizeof(float) * (size_t)(pol->wf32_stride * pol->A),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

// ---------------------------------------------------------------- IPPO update
static ppo::AdamParams adam_params(lob_policy *p) {
    ppo::AdamParams a;
    std::memset(&a, 0, sizeof(a));
    a.A = p->A; a.D = p->D; a.Dp = p->upd_Dp; a.Dpf = p->Dp;
    a.P = p->wf32_stride;
    a.w = p->d_wf32; a.m = p->d_m; a.v = p->d_v; a.grad = p->d_grad;
    a.sqnorm = nullptr;   // per minibatch, set by the update
    a.wpk = p->d_wpk; a.wpk_stride = p->wpk_stride;
    a.wfwd = p->d_wpack; a.wfwd_stride = p->wpack_stride;
    return a;
}

// First update: optimiser state, gradient buffer, the update's packed weights.
static int ppo_setup(lob_policy *p, cudaStream_t s) {
    if (p->d_wpk) return LOB_OK;
    if (cudaFuncSetAttribute(ppo::k_ppo_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ppo::GradSmem)) != cudaSuccess)
        return LOB_ECUDA;
    p->upd_Dp = (p->D + 1 + 15) / 16 * 16;
    p->wpk_stride = ((long long)H * p->upd_Dp + (long long)H * H + 16LL * H) * 2;
    const size_t P = (size_t)(p->wf32_stride * p->A);
    bool fail = cudaMalloc(&p->d_wpk, (size_t)(p->wpk_stride * p->A)) != cudaSuccess;
    fail = fail || cudaMalloc(&p->d_m, P * 4) != cudaSuccess;
    fail = fail || cudaMalloc(&p->d_v, P * 4) != cudaSuccess;
    fail = fail || cudaMalloc(&p->d_grad, P * 4) != cudaSuccess;
    {
        int n_sm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        p->gpart_ctas = std::max(1, n_sm / p->A);
        fail = fail || cudaMalloc(&p->d_gpart, P * (size_t)p->gpart_ctas * 4) != cudaSuccess;
    }

    if (fail) {
        cudaGetLastError();
        return LOB_ENOMEM;
    }
    if (cudaMemsetAsync(p->d_wpk, 0, (size_t)(p->wpk_stride * p->A), s) != cudaSuccess ||
        cudaMemsetAsync(p->d_m, 0, P * 4, s) != cudaSuccess || cudaMemsetAsync(p->d_v, 0, P * 4, s) != cudaSuccess)
        return LOB_ECUDA;
    const ppo::AdamParams a = adam_params(p);
    ppo::k_ppo_pack<<<dim3(64, p->A), 256, 0, s>>>(a);
    p->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

extern "C" int lob_ppo_update(lob_policy *p, const lob_ppo_batch *b, const lob_ppo_hparams *hp, void *stream) {
    if (!p || !b || !hp) return LOB_EINVAL;
    if (b->T < 1 || b->n_envs < 1 || hp->n_minibatches < 1 || !b->d_obs || !b->d_actions || !b->d_logp_old ||
        !b->d_values || !b->d_rewards || !b->d_done || !b->d_perm)
        return LOB_EINVAL;
    const long long N = (long long)b->T * b->n_envs;
    if (N % hp->n_minibatches != 0 || N / hp->n_minibatches > 0x7fffffffLL) return LOB_EINVAL;
    if (p->D + 1 > ppo::DPMAX) return LOB_ECAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ppo_setup(p, s);
    if (rc != LOB_OK) return rc;
    const int nmb = hp->n_minibatches;
    if (p->mb_cap < nmb) {
        if (p->d_stats) cudaFree(p->d_stats);
        if (p->d_acc) cudaFree(p->d_acc);
        p->d_stats = nullptr;
        p->d_acc = nullptr;
        p->mb_cap = 0;
        if (cudaMalloc(&p->d_stats, (size_t)nmb * p->A * 2 * 4) != cudaSuccess ||
            cudaMalloc(&p->d_acc, (size_t)nmb * (p->A * 3 + 1) * 8) != cudaSuccess) {
            cudaGetLastError();
            return LOB_ENOMEM;
        }
        p->mb_cap = nmb;
    }
    if (p->adv_cap < N) {
        if (p->d_adv) cudaFree(p->d_adv);
        if (p->d_ret) cudaFree(p->d_ret);
        p->d_adv = p->d_ret = nullptr;
        p->adv_cap = 0;
        if (cudaMalloc(&p->d_adv, (size_t)(N * p->A) * 4) != cudaSuccess ||
            cudaMalloc(&p->d_ret, (size_t)(N * p->A) * 4) != cudaSuccess) {
            cudaGetLastError();
            return LOB_ENOMEM;
        }
        p->adv_cap = N;
    }
    const int A = p->A;
    const long long P = p->wf32_stride;
    const int nenv_a = b->n_envs * A;
    ppo::k_ppo_gae<<<(nenv_a + ppo::GAE_PAIRS - 1) / ppo::GAE_PAIRS, ppo::GAE_PAIRS * ppo::GAE_CH, 0, s>>>(
        reinterpret_cast<const long long *>(b->d_rewards), b->d_values, b->d_done, b->T, b->n_envs, A, hp->gamma,
        hp->gae_lambda, hp->reward_scale, p->d_adv, p->d_ret);
    p->launches++;
    const int mb = (int)(N / hp->n_minibatches);
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (mb + 127) / 128;
    // each CTA runs ppo::NS tile streams and owns one slice of the partial-gradient buffer
    const int ctas = std::max(1, std::min((tiles + ppo::NS - 1) / ppo::NS, std::min(p->gpart_ctas, n_sm / A > 0 ? n_sm / A : 1)));
    ppo::GradParams g;
    std::memset(&g, 0, sizeof(g));
    g.A = A; g.D = p->D; g.Dp = p->upd_Dp; g.L = p->L; g.n_envs = b->n_envs; g.n_samples = N;
    g.obs = b->d_obs; g.actions = b->d_actions; g.logp_old = b->d_logp_old; g.adv = p->d_adv; g.ret = p->d_ret;
    g.perm = b->d_perm; g.mb_size = mb; g.stats = p->d_stats;
    g.wpk = p->d_wpk; g.wpk_stride = p->wpk_stride; g.wf32 = p->d_wf32; g.wf32_stride = P;
    g.gpart = p->d_gpart; g.gpart_ct = p->gpart_ctas; g.clip_eps = hp->clip_eps; g.vf_coef = hp->vf_coef; g.ent_coef = hp->ent_coef;
    g.status = p->d_status; g.wait_budget = 2000000000LL;
    ppo::AdamParams ad = adam_params(p);
    ad.lr = hp->lr; ad.beta1 = hp->beta1; ad.beta2 = hp->beta2; ad.eps = hp->adam_eps; ad.max_norm = hp->max_grad_norm;
    // every minibatch's statistics in one launch after GAE; the sums, squared
    // norms and block counters of all minibatches start at zero
    double *d_sums = p->d_acc, *d_sq = p->d_acc + (size_t)nmb * 2 * A;
    unsigned *d_ctr = reinterpret_cast<unsigned *>(p->d_acc + (size_t)nmb * 3 * A);
    if (cudaMemsetAsync(p->d_acc, 0, (size_t)nmb * (A * 3 + 1) * 8, s) != cudaSuccess) return LOB_ECUDA;
    ppo::k_ppo_stats<<<dim3(std::max(1, std::min(64, (mb + 255) / 256)), A, nmb), 256, 0, s>>>(
        p->d_adv, b->d_perm, N, mb, A, d_sums, d_ctr, p->d_stats);
    p->launches++;
    const int red_blocks = (int)std::min<long long>(128, (P + 255) / 256);
    for (int k = 0; k < nmb; k++) {
        g.mb_begin = (long long)k * mb;
        g.stats = p->d_stats + (size_t)k * 2 * A;
        ppo::k_ppo_grad<<<dim3(ctas, A), ppo::PPT, sizeof(ppo::GradSmem), s>>>(g);
        ppo::k_ppo_reduce<<<dim3(red_blocks, A), 256, 0, s>>>(p->d_gpart, ctas, p->gpart_ctas, P, p->d_grad,
                                                               d_sq + (size_t)k * A);
        if (b->d_grad_out &&
            cudaMemcpyAsync(b->d_grad_out + (size_t)k * A * P, p->d_grad, (size_t)(P * A) * 4, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return LOB_ECUDA;
        p->adam_t++;
        ad.bc1 = (float)(1.0 - std::pow((double)hp->beta1, (double)p->adam_t));
        ad.bc2 = (float)(1.0 - std::pow((double)hp->beta2, (double)p->adam_t));
        ad.sqnorm = d_sq + (size_t)k * A;
        ppo::k_ppo_adam<<<dim3(64, A), 256, 0, s>>>(ad);
        p->launches += 3;
    }
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int policy_forward_internal(lob_policy *pol, const float *d_obs, int32_t n_envs, int32_t precision, float *d_logits,
                            float *d_values, int32_t *d_actions, cudaStream_t s) {
    if (!pol || !d_obs || n_envs < 1) return LOB_EINVAL;
    if (precision != LOB_PREC_FP32 && precision != LOB_PREC_BF16) return LOB_EINVAL;
    PolicyParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.obs = d_obs;
    pp.n_envs = n_envs;
    pp.A = pol->A; pp.D = pol->D; pp.Dp = pol->Dp; pp.L = pol->L;
    pp.wpack = pol->d_wpack; pp.wpack_stride = pol->wpack_stride;
    pp.wf32 = pol->d_wf32; pp.wf32_stride = pol->wf32_stride;
    pp.logits = d_logits; pp.values = d_values; pp.actions = d_actions;
    pp.status = pol->d_status;
    pp.wait_budget = 2000000000LL;
    if (precision == LOB_PREC_BF16) {
        dim3 grid((n_envs + 127) / 128, pol->A);
        k_policy_bf16<<<grid, PT, sizeof(Bf16Smem), s>>>(pp);
    } else {
        dim3 grid((n_envs + 127) / 128, pol->A);
        k_policy_fp32<<<grid, FT, sizeof(F32Smem), s>>>(pp);
    }
    pol->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int policy_n_agents(const lob_policy *pol) { return pol ? pol->A : 0; }
void policy_fused_params(const lob_policy *pol, lobk::FusedParams *f) {
    f->wpack = pol->d_wpack;
    f->wpack_stride = pol->wpack_stride;
    f->wf32 = pol->d_wf32;
    f->wf32_stride = pol->wf32_stride;
    f->D = pol->D;
    f->Dp = pol->Dp;
    f->L = pol->L;
    f->status = pol->d_status;
    f->wait_budget = 2000000000LL;
}
void policy_count_launch(lob_policy *pol) { pol->launches++; }
int policy_obs_dim(const lob_policy *pol) { return pol ? pol->D : 0; }
long long policy_launches(const lob_policy *pol) { return pol ? pol->launches : 0; }

extern "C" int lob_policy_forward(lob_policy *pol, const float *d_obs, int32_t n_envs, int32_t precision,
                                  float *d_logits, float *d_values, int32_t *d_actions, void *stream) {
    return policy_forward_internal(pol, d_obs, n_envs, precision, d_logits, d_values, d_actions, (cudaStream_t)stream);
}

extern "C" int lob_policy_sync(lob_policy *pol, void *stream) {
    if (!pol) return LOB_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LOB_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, pol->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LOB_ECUDA;
    if (st) cudaMemset(pol->d_status, 0, 4);
    return st ? LOB_ETIMEOUT : LOB_OK;
}
