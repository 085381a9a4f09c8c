// D3Q27 instantiation of the step kernels.
#define LBM_Q 27
#include "kernels_impl.cuh"
