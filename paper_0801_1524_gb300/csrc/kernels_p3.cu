// Kernel set for p = 3.
#define BFLY_P 3
#include "kernels_inst.cuh"
