// Kernel set for p = 7.
#define BFLY_P 7
#include "kernels_inst.cuh"
