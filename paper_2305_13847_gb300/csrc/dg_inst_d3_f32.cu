// Kernel instantiations for dimension 3, storage type float, orders 1..5.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS(launchers_d3_f32, 3, float)
