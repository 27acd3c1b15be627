// Kernel set for p = 9.
#define BFLY_P 9
#include "kernels_inst.cuh"
