// Kernel instantiations for lattice D1Q3 (all three precisions).
#include "lbm_launch.cuh"
LBM_DEFINE_LATTICE_LAUNCHERS(1)
