// F32 instantiation of the persistent batched RK driver.
#include "hb_persist.cuh"
#define HB_T float
#define HB_PERSIST_ALL_SHAPES 1
#include "hb_launch_persist.inc"
