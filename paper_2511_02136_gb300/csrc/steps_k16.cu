// steps_k16.cu -- step kernels of capacity class K = 16 (512 slots per side).
#define LOB_K 16
#include "steps_inst.cuh"
