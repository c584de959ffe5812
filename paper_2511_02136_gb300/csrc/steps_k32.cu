// steps_k32.cu -- step kernels of capacity class K = 32 (1024 slots per side).
#define LOB_K 32
#include "steps_inst.cuh"
