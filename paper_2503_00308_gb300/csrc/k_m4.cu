// Kernels for M = 4 pose variables.
#define AR_M 4
#include "k_inst.cuh"
