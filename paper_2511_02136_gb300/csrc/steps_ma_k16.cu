// steps_ma_k16.cu -- several-agents step kernels of capacity class K = 16 (512 slots per side).
#define LOB_K 16
#include "steps_ma_inst.cuh"
