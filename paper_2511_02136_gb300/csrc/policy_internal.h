// policy_internal.h -- what lob_api.cu needs from policy_api.cu (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include "lob.h"
#include "fused.cuh"

int policy_forward_internal(lob_policy *pol, const float *d_obs, int32_t n_envs, int32_t precision, float *d_logits,
                            float *d_values, int32_t *d_actions, cudaStream_t s);
int policy_n_agents(const lob_policy *pol);
int policy_obs_dim(const lob_policy *pol);
long long policy_launches(const lob_policy *pol);
// Weights and shapes of the fused rollout's forward.
void policy_fused_params(const lob_policy *pol, lobk::FusedParams *f);
void policy_count_launch(lob_policy *pol);
