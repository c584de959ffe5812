// rollout_fused_k8.cu -- fused BF16 rollout kernel of capacity class K = 8.
#define LOB_K 8
#include "rollout_fused.cuh"
