// F64 instantiation of the persistent batched RK driver.
#include "hb_persist.cuh"
#define HB_T double
#define HB_PERSIST_ALL_SHAPES 0
#include "hb_launch_persist.inc"
