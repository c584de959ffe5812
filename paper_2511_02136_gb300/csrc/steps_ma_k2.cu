// steps_ma_k2.cu -- several-agents step kernels of capacity class K = 2 (64 slots per side).
#define LOB_K 2
#include "steps_ma_inst.cuh"
