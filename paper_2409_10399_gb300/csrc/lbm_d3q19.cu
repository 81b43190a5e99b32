// Kernel instantiations for lattice D3Q19 (all three precisions).
#include "lbm_launch.cuh"
LBM_DEFINE_LATTICE_LAUNCHERS(3)
