// Internal state shared by the library's host translation units (not part of
// the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

struct lbm_ctx {
  int lattice, D, Q, prec;
  int n[3];
  long long N, plane;
  lbm_params p;
  void *pop = nullptr, *held = nullptr;
  void *cfield = nullptr;    // beta-stencil form: 2 x 2*D planes of c
  double *partials = nullptr, *diag_dev = nullptr;
  double *h_diag = nullptr;  // pinned, 8 doubles
  cudaEvent_t diag_ev = nullptr;
  int diag_pending = 0;
  unsigned nblk_flat = 0;
  void *stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t stream = 0;
  long long t = 0;
  // the next step is the first since an initialisation (lbm_init, or the
  // surrogate window's re-initialisation at a later clock): it latches S''
  // and Lambda' and, in the beta-stencil form, takes every q from the node's
  // own c, whatever t is
  int first_step = 0;
  int initialised = 0, sticky = 0;
  double r_ag = 0.5, r_al = 0.5;
  double mass0 = 0.0;
  int T[3] = {1, 1, 1}, shift[3] = {0, 0, 0}, grid[3] = {1, 1, 1};
  size_t smem = 0;
  int halo_off = 0;  // beta-stencil form: byte offset of the c halo in the step kernel's shared memory
  long long launches = 0;
  // steps replayed from a CUDA graph of one period of the step arguments
  // (lbm_step; lattices whose arguments repeat: no inlet ramp)
  int use_graph = 1;
  cudaGraphExec_t graph = nullptr;
  int graph_period = 0;
  long long graph_launches = 0;   // kernels in one replay
  cudaStream_t cap_stream = nullptr;  // capture stream of the lattice's own
  char err[512] = {0};
};


namespace lbm {
// helpers of lbm_capi.cu used by the batched form (lbm_batch.cu)
StepArgs ctx_step_args(const lbm_ctx *c, long long t);
// largest block of the fused step kernel of this lattice and precision
int step_max_threads(int lattice, int prec);
cudaError_t launch_batch_step(int lattice, int prec, const StepArgs *args, const WorkItem *work, unsigned nwork,
                              dim3 block, int parity, int latch, int off32, cudaStream_t st);
}  // namespace lbm
