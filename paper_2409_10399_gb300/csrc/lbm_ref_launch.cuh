// Launchers of the FP64 reference path of one lattice.  Included by exactly
// one translation unit per lattice (lbm_ref_d1q3.cu, ...), which the build
// compiles with -fmad=false.
#pragma once
#include <cuda_runtime.h>

#include "lbm_ref.cuh"

#define LBM_DEFINE_REF_LAUNCHERS(LAT)                                                                          \
  namespace lbm {                                                                                            \
  cudaError_t launch_ref_step_##LAT(const StepArgs &a, dim3 g, dim3 b, size_t sm, cudaStream_t st) {          \
    k_step_ref<Lattice<LAT>><<<g, b, sm, st>>>(a);                                                           \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  cudaError_t launch_ref_moments_##LAT(const MomArgs &ma, int mode, unsigned n, cudaStream_t st) {            \
    k_moments_ref<Lattice<LAT>><<<n, 256, 0, st>>>(ma, mode);                                                \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  cudaError_t launch_ref_init_##LAT(const MomArgs &ma, const double *a, const double *ug, const double *ul,   \
                                    const double *pk, unsigned n, cudaStream_t st) {                         \
    k_init_ref<Lattice<LAT>><<<n, 256, 0, st>>>(ma, a, ug, ul, pk);                                          \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  }
