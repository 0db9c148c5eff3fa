// Kernel instantiations for dimension 2, storage type double, orders 1..5,
// with the float-float contractions of DG_FP64_FFC.
#include "dg_launch.cuh"
DGM_DEFINE_LAUNCHERS_FF(launchers_d2_f64ff, 2)
