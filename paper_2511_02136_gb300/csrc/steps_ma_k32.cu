// steps_ma_k32.cu -- several-agents step kernels of capacity class K = 32 (1024 slots per side).
#define LOB_K 32
#include "steps_ma_inst.cuh"
