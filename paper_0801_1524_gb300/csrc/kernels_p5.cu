// Kernel set for p = 5.
#define BFLY_P 5
#include "kernels_inst.cuh"
