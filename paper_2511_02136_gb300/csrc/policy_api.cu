// policy_api.cu -- host side of the actor-critic policy entry points of
// include/lob.h: weight packing (FP32 -> BF16 core-matrix layout), device
// buffers and the two forward launches of policy.cuh.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "lob.h"
#include "policy.cuh"
#include "policy_internal.h"

using namespace pol;

struct lob_policy {
    int A = 0, D = 0, Dp = 0, L = 0;
    unsigned char *d_wpack = nullptr;
    long long wpack_stride = 0;
    float *d_wf32 = nullptr;
    long long wf32_stride = 0;
    int *d_status = nullptr;
    long long launches = 0;
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
    if (p->d_wpack) cudaFree(p->d_wpack);
    if (p->d_wf32) cudaFree(p->d_wf32);
    if (p->d_status) cudaFree(p->d_status);
    delete p;
    return LOB_OK;
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
        dim3 grid((n_envs + 63) / 64, pol->A);
        k_policy_fp32<<<grid, 64, sizeof(F32Smem), s>>>(pp);
    }
    pol->launches++;
    return cudaGetLastError() == cudaSuccess ? LOB_OK : LOB_ECUDA;
}

int policy_n_agents(const lob_policy *pol) { return pol ? pol->A : 0; }
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
