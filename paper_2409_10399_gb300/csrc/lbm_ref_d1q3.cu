// FP64 reference-path kernels for lattice D1Q3 (compiled with -fmad=false).
#include "lbm_ref_launch.cuh"
LBM_DEFINE_REF_LAUNCHERS(1)
