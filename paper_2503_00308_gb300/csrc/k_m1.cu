// Kernels for M = 1 pose variables.
#define AR_M 1
#include "k_inst.cuh"
