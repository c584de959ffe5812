// steps_ma_k4.cu -- several-agents step kernels of capacity class K = 4 (128 slots per side).
#define LOB_K 4
#include "steps_ma_inst.cuh"
