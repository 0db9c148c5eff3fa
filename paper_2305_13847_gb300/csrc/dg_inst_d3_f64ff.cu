// Kernel instantiations for dimension 3, storage type double, orders 1..5,
// with the float-float contractions of DG_FP64_FFC.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS_FF(launchers_d3_f64ff, 3)
