// FP64 instantiation of the launchers.
#define VLBM_T double
#include "kernels_impl.cuh"
