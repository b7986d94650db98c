// FP32 instantiation of the launchers.
#define VLBM_T float
#include "kernels_impl.cuh"
