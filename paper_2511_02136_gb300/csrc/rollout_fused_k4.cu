// rollout_fused_k4.cu -- fused BF16 rollout kernel of capacity class K = 4.
#define LOB_K 4
#include "rollout_fused.cuh"
