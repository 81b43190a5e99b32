// Launchers of one lattice for the three storage/arithmetic precisions.
// Included by exactly one translation unit per lattice (lbm_d1q3.cu, ...).
#pragma once
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbm {

template <int LAT>
struct Launch {
  using L = Lattice<LAT>;
  // prec: 1 = FP32, 2 = FP16 store, 3 = FP64 deviations, 4 = FP16AB (0, the FP64
  // reference path, has its own launchers in lbm_ref_*.cu)
  // bs: the beta-stencil form (StepArgs::cfield); every kernel below comes
  // in both forms
  // one launch of a step kernel; blocks that need more than the default
  // 48 KB of dynamic shared memory (the beta-stencil form's c halo with large
  // FP64-deviation tiles) get the kernel's limit raised first
  template <class K>
  static void go(K kern, const StepArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, st>>>(a);
  }
  template <bool BS, class OffT>
  static void step_form(int prec, const StepArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    // the fast six-scheme forms also come without the inlet/outlet rules,
    // for lattices with walls and periodic axes only (a smaller kernel)
    constexpr bool WO = !BS && std::is_same<OffT, unsigned>::value;
    const bool io = a.has_inlet || a.has_outlet;
    if (prec == 3) go(k_step<L, double, double, BS, OffT>, a, grid, block, smem, st);
    else if (prec == 4 && WO && !io) go(k_step<L, MixAB, float, BS, OffT, false>, a, grid, block, smem, st);
    else if (prec == 4) go(k_step<L, MixAB, float, BS, OffT>, a, grid, block, smem, st);
    else if (prec == 1 && WO && !io) go(k_step<L, float, float, BS, OffT, false>, a, grid, block, smem, st);
    else if (prec == 1) go(k_step<L, float, float, BS, OffT>, a, grid, block, smem, st);
    else if (WO && !io) go(k_step<L, __half, float, BS, OffT, false>, a, grid, block, smem, st);
    else go(k_step<L, __half, float, BS, OffT>, a, grid, block, smem, st);
  }
  // 32-bit population offsets where they fit
  static cudaError_t step(int prec, const StepArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    if (a.cfield && a.off32) step_form<true, unsigned>(prec, a, grid, block, smem, st);
    else if (a.cfield) step_form<true, long long>(prec, a, grid, block, smem, st);
    else if (a.off32) step_form<false, unsigned>(prec, a, grid, block, smem, st);
    else step_form<false, long long>(prec, a, grid, block, smem, st);
    return cudaGetLastError();
  }
  template <class OffT>
  static void batch_form(int prec, const StepArgs *args, const WorkItem *work, unsigned nwork, dim3 block,
                         int parity, int latch, cudaStream_t st) {
    if (prec == 3) k_batch_step<L, double, double, OffT><<<nwork, block, 0, st>>>(args, work, parity, latch);
    else if (prec == 1) k_batch_step<L, float, float, OffT><<<nwork, block, 0, st>>>(args, work, parity, latch);
    else if (prec == 4) k_batch_step<L, MixAB, float, OffT><<<nwork, block, 0, st>>>(args, work, parity, latch);
    else k_batch_step<L, __half, float, OffT><<<nwork, block, 0, st>>>(args, work, parity, latch);
  }
  // off32: every instance has Q*plane < 2^32
  static cudaError_t batch_step(int prec, const StepArgs *args, const WorkItem *work, unsigned nwork, dim3 block,
                                int parity, int latch, int off32, cudaStream_t st) {
    if (off32) batch_form<unsigned>(prec, args, work, nwork, block, parity, latch, st);
    else batch_form<long long>(prec, args, work, nwork, block, parity, latch, st);
    return cudaGetLastError();
  }
  template <bool BS> static void moments_form(int prec, const MomArgs &ma, int mode, unsigned nblk, cudaStream_t st) {
    if (prec == 3) k_moments<L, double, double, BS><<<nblk, 256, 0, st>>>(ma, mode);
    else if (prec == 1) k_moments<L, float, float, BS><<<nblk, 256, 0, st>>>(ma, mode);
    else if (prec == 4) k_moments<L, MixAB, float, BS><<<nblk, 256, 0, st>>>(ma, mode);
    else k_moments<L, __half, float, BS><<<nblk, 256, 0, st>>>(ma, mode);
  }
  static cudaError_t moments(int prec, const MomArgs &ma, int mode, unsigned nblk, cudaStream_t st) {
    if (ma.s.cfield) moments_form<true>(prec, ma, mode, nblk, st);
    else moments_form<false>(prec, ma, mode, nblk, st);
    return cudaGetLastError();
  }
  template <bool BS> static void pops_form(int prec, const MomArgs &ma, int s, unsigned nblk, cudaStream_t st) {
    if (prec == 0 || prec == 3) k_pops<L, double, double, BS><<<nblk, 256, 0, st>>>(ma, s);
    else if (prec == 1) k_pops<L, float, float, BS><<<nblk, 256, 0, st>>>(ma, s);
    else if (prec == 4) k_pops<L, MixAB, float, BS><<<nblk, 256, 0, st>>>(ma, s);
    else k_pops<L, __half, float, BS><<<nblk, 256, 0, st>>>(ma, s);
  }
  static cudaError_t pops(int prec, const MomArgs &ma, int s, unsigned nblk, cudaStream_t st) {
    if (ma.s.cfield) pops_form<true>(prec, ma, s, nblk, st);
    else pops_form<false>(prec, ma, s, nblk, st);
    return cudaGetLastError();
  }
  template <bool BS>
  static void init_form(int prec, const MomArgs &ma, const double *a, const double *ug, const double *ul,
                        const double *pk, unsigned nblk, cudaStream_t st) {
    if (prec == 3) k_init<L, double, BS><<<nblk, 256, 0, st>>>(ma, a, ug, ul, pk);
    else if (prec == 1) k_init<L, float, BS><<<nblk, 256, 0, st>>>(ma, a, ug, ul, pk);
    else if (prec == 4) k_init<L, MixAB, BS><<<nblk, 256, 0, st>>>(ma, a, ug, ul, pk);
    else k_init<L, __half, BS><<<nblk, 256, 0, st>>>(ma, a, ug, ul, pk);
  }
  static cudaError_t init(int prec, const MomArgs &ma, const double *a, const double *ug, const double *ul,
                          const double *pk, unsigned nblk, cudaStream_t st) {
    if (ma.s.cfield) init_form<true>(prec, ma, a, ug, ul, pk, nblk, st);
    else init_form<false>(prec, ma, a, ug, ul, pk, nblk, st);
    return cudaGetLastError();
  }
};

// Entry points exported by the per-lattice translation units.
cudaError_t launch_step(int lat, int prec, const StepArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st);
cudaError_t launch_moments(int lat, int prec, const MomArgs &ma, int mode, unsigned nblk, cudaStream_t st);
cudaError_t launch_pops(int lat, int prec, const MomArgs &ma, int s, unsigned nblk, cudaStream_t st);
cudaError_t launch_init(int lat, int prec, const MomArgs &ma, const double *a, const double *ug, const double *ul,
                        const double *pk, unsigned nblk, cudaStream_t st);

}  // namespace lbm

#define LBM_DEFINE_LATTICE_LAUNCHERS(LAT)                                                                      \
  namespace lbm {                                                                                            \
  cudaError_t launch_step_##LAT(int prec, const StepArgs &a, dim3 g, dim3 b, size_t sm, cudaStream_t st) {    \
    return Launch<LAT>::step(prec, a, g, b, sm, st);                                                         \
  }                                                                                                          \
  cudaError_t launch_batch_step_##LAT(int prec, const StepArgs *args, const WorkItem *work, unsigned nwork,     \
                                     dim3 block, int parity, int latch, int off32, cudaStream_t st) {         \
    return Launch<LAT>::batch_step(prec, args, work, nwork, block, parity, latch, off32, st);                 \
  }                                                                                                          \
  cudaError_t launch_moments_##LAT(int prec, const MomArgs &ma, int mode, unsigned n, cudaStream_t st) {      \
    return Launch<LAT>::moments(prec, ma, mode, n, st);                                                      \
  }                                                                                                          \
  cudaError_t launch_pops_##LAT(int prec, const MomArgs &ma, int s, unsigned n, cudaStream_t st) {            \
    return Launch<LAT>::pops(prec, ma, s, n, st);                                                            \
  }                                                                                                          \
  cudaError_t launch_init_##LAT(int prec, const MomArgs &ma, const double *a, const double *ug,               \
                                const double *ul, const double *pk, unsigned n, cudaStream_t st) {            \
    return Launch<LAT>::init(prec, ma, a, ug, ul, pk, n, st);                                                \
  }                                                                                                          \
  }
