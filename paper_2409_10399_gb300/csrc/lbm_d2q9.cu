// Kernel instantiations for lattice D2Q9 (all three precisions).
#include "lbm_launch.cuh"
LBM_DEFINE_LATTICE_LAUNCHERS(2)
