// Kernel instantiations for dimension 2, storage type float, orders 1..5.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS(launchers_d2_f32, 2, float)
