// Kernels for M = 6 pose variables.
#define AR_M 6
#include "k_inst.cuh"
