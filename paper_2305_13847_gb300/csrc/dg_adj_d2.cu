// Adjoint kernel instantiations for dimension 2, float64, orders 1..5.
#include "dg_launch.cuh"
DGM_DEFINE_ADJ_LAUNCHERS(adj_launchers_d2, 2)
