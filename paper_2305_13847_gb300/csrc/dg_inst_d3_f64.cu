// Kernel instantiations for dimension 3, storage type double, orders 1..5.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS(launchers_d3_f64, 3, double)
