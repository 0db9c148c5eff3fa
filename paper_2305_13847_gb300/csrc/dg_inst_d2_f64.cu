// Kernel instantiations for dimension 2, storage type double, orders 1..5.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS(launchers_d2_f64, 2, double)
