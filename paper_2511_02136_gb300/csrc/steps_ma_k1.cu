// steps_ma_k1.cu -- several-agents step kernels of capacity class K = 1 (32 slots per side).
#define LOB_K 1
#include "steps_ma_inst.cuh"
