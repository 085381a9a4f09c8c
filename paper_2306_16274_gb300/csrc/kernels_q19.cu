// D3Q19 instantiation of the step kernels.
#define LBM_Q 19
#include "kernels_impl.cuh"
