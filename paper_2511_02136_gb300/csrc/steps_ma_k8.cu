// steps_ma_k8.cu -- several-agents step kernels of capacity class K = 8 (256 slots per side).
#define LOB_K 8
#include "steps_ma_inst.cuh"
