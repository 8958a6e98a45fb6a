// F32 instantiation of the 3D tile, halo and init kernels.
#include "hb_kernels3d.cuh"
#define HB_T float
#include "hb_launch3d.inc"
