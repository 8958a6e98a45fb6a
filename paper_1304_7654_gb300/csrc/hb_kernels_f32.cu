// FP32 instantiation of the tile, halo, init and force kernels.
#include "hb_kernels.cuh"
#define HB_T float
#include "hb_launch.inc"
