// steps_k8.cu -- step kernels of capacity class K = 8 (256 slots per side).
#define LOB_K 8
#include "steps_inst.cuh"
