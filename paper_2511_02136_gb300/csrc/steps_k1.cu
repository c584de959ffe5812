// steps_k1.cu -- step kernels of capacity class K = 1 (32 slots per side).
#define LOB_K 1
#include "steps_inst.cuh"
