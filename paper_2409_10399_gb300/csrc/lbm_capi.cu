// Host side of the C ABI declared in include/lbm.h: context lifetime,
// argument validation, tile selection, the stepping loop (per-step scalars of
// the lag latch and the inlet ramp of Eq. (transient)) and the FP64
// diagnostics pipeline.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_ref.cuh"

namespace lbm {
cudaError_t launch_step_1(int, const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_step_2(int, const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_step_3(int, const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_moments_1(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_moments_2(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_moments_3(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_pops_1(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_pops_2(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_pops_3(int, const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_init_1(int, const MomArgs &, const double *, const double *, const double *, const double *,
                          unsigned, cudaStream_t);
cudaError_t launch_init_2(int, const MomArgs &, const double *, const double *, const double *, const double *,
                          unsigned, cudaStream_t);
cudaError_t launch_init_3(int, const MomArgs &, const double *, const double *, const double *, const double *,
                          unsigned, cudaStream_t);
cudaError_t launch_batch_step_1(int, const StepArgs *, const WorkItem *, unsigned, dim3, int, int, int,
                               cudaStream_t);
cudaError_t launch_batch_step_2(int, const StepArgs *, const WorkItem *, unsigned, dim3, int, int, int,
                               cudaStream_t);
cudaError_t launch_batch_step_3(int, const StepArgs *, const WorkItem *, unsigned, dim3, int, int, int,
                               cudaStream_t);
cudaError_t launch_ref_step_1(const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_ref_step_2(const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_ref_step_3(const StepArgs &, dim3, dim3, size_t, cudaStream_t);
cudaError_t launch_ref_moments_1(const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_ref_moments_2(const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_ref_moments_3(const MomArgs &, int, unsigned, cudaStream_t);
cudaError_t launch_ref_init_1(const MomArgs &, const double *, const double *, const double *, const double *,
                              unsigned, cudaStream_t);
cudaError_t launch_ref_init_2(const MomArgs &, const double *, const double *, const double *, const double *,
                              unsigned, cudaStream_t);
cudaError_t launch_ref_init_3(const MomArgs &, const double *, const double *, const double *, const double *,
                              unsigned, cudaStream_t);

__global__ void k_diag_final(const double *partials, int nblocks, double *out) {
  // One warp per diagnostic, each lane sums a fixed strided subset, then a
  // fixed-order shuffle tree: the result does not depend on scheduling.
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= 8) return;
  double acc = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    double v = partials[(long long)b * 8 + k];
    acc = (k == 4) ? fmax(acc, v) : acc + v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, acc, o);
    acc = (k == 4) ? fmax(acc, v) : acc + v;
  }
  if (lane == 0) out[k] = acc;
}
}  // namespace lbm

using namespace lbm;

#include "lbm_ctx_access.h"
#include "lbm_internal.h"

static int set_err(lbm_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CUDA_TRY(c, call)                                                                              \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return set_err((c), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Bytes of one direction of one node of the whole population store (nsch
// schemes): FP16AB keeps f_g, f_l in float and the other schemes in half.
static size_t store_bytes_per_dir(int prec, int nsch) {
  if (prec == LBM_FP16AB) return 2 * 4 + (size_t)(nsch - 2) * 2;
  return (size_t)nsch * ((prec == LBM_FP64 || prec == LBM_FP64DEV) ? 8 : (prec == LBM_FP32 ? 4 : 2));
}
static size_t held_size(int prec) { return (prec == LBM_FP64 || prec == LBM_FP64DEV) ? 8 : 4; }

static cudaError_t dispatch_step(lbm_ctx *c, const StepArgs &a) {
  dim3 g(c->grid[0], c->grid[1], c->grid[2]), b(c->T[0], c->T[1], c->T[2]);
  c->launches++;
  if (c->prec == LBM_FP64) {
    if (c->lattice == 1) return launch_ref_step_1(a, g, b, c->smem, c->stream);
    if (c->lattice == 2) return launch_ref_step_2(a, g, b, c->smem, c->stream);
    return launch_ref_step_3(a, g, b, c->smem, c->stream);
  }
  if (c->lattice == 1) return launch_step_1(c->prec, a, g, b, c->smem, c->stream);
  if (c->lattice == 2) return launch_step_2(c->prec, a, g, b, c->smem, c->stream);
  return launch_step_3(c->prec, a, g, b, c->smem, c->stream);
}
static cudaError_t dispatch_moments(lbm_ctx *c, const MomArgs &ma, int mode) {
  c->launches++;
  if (c->prec == LBM_FP64) {
    if (c->lattice == 1) return launch_ref_moments_1(ma, mode, c->nblk_flat, c->stream);
    if (c->lattice == 2) return launch_ref_moments_2(ma, mode, c->nblk_flat, c->stream);
    return launch_ref_moments_3(ma, mode, c->nblk_flat, c->stream);
  }
  if (c->lattice == 1) return launch_moments_1(c->prec, ma, mode, c->nblk_flat, c->stream);
  if (c->lattice == 2) return launch_moments_2(c->prec, ma, mode, c->nblk_flat, c->stream);
  return launch_moments_3(c->prec, ma, mode, c->nblk_flat, c->stream);
}
static cudaError_t dispatch_pops(lbm_ctx *c, const MomArgs &ma, int s) {
  c->launches++;
  if (c->lattice == 1) return launch_pops_1(c->prec, ma, s, c->nblk_flat, c->stream);
  if (c->lattice == 2) return launch_pops_2(c->prec, ma, s, c->nblk_flat, c->stream);
  return launch_pops_3(c->prec, ma, s, c->nblk_flat, c->stream);
}
static cudaError_t dispatch_init(lbm_ctx *c, const MomArgs &ma, const double *a, const double *ug, const double *ul,
                                 const double *pk) {
  c->launches++;
  if (c->prec == LBM_FP64) {
    if (c->lattice == 1) return launch_ref_init_1(ma, a, ug, ul, pk, c->nblk_flat, c->stream);
    if (c->lattice == 2) return launch_ref_init_2(ma, a, ug, ul, pk, c->nblk_flat, c->stream);
    return launch_ref_init_3(ma, a, ug, ul, pk, c->nblk_flat, c->stream);
  }
  if (c->lattice == 1) return launch_init_1(c->prec, ma, a, ug, ul, pk, c->nblk_flat, c->stream);
  if (c->lattice == 2) return launch_init_2(c->prec, ma, a, ug, ul, pk, c->nblk_flat, c->stream);
  return launch_init_3(c->prec, ma, a, ug, ul, pk, c->nblk_flat, c->stream);
}

static double ramp(const double mm[2], long long t, int nt) {
  if (nt <= 0) return mm[1];
  return (mm[1] - mm[0]) * tanh((double)t / (double)nt) + mm[0];
}

// Per-step arguments: everything constant plus parity, latch and inlet values.
static StepArgs make_args(const lbm_ctx *c, long long t) {
  const lbm_params &p = c->p;
  StepArgs a;
  memset(&a, 0, sizeof a);
  a.pop = c->pop;
  a.held = c->held;
  a.plane = c->plane;
  for (int d = 0; d < 3; d++) {
    a.n[d] = c->n[d];
    a.shift[d] = c->shift[d];
    a.T[d] = c->T[d];
    a.bc_lo[d] = d < c->D ? p.bc_lo[d] : BC_PERIODIC;
    a.bc_hi[d] = d < c->D ? p.bc_hi[d] : BC_PERIODIC;
  }
  a.parity = (int)(t & 1);
  a.latch = (t % p.n_gamma) == 0 || c->first_step;
  a.g_axis = p.g_axis;
  a.tr_axis = -1;
  for (int d = 0; d < c->D; d++)
    if (d != p.g_axis) { a.tr_axis = d; break; }
  a.inlet_lo = p.inlet_lo;
  a.inlet_hi = p.inlet_hi;
  a.has_inlet = p.bc_lo[p.g_axis] == BC_INLET;
  a.has_outlet = p.bc_hi[p.g_axis] == BC_OUTLET;
  a.R = p.R;
  a.invR = 1.0 / p.R;
  a.omega_g = p.omega_g;
  a.omega_l = p.omega_l;
  a.omega_a = p.omega_alpha;
  a.kgrad = p.omega_alpha / CS2;
  const double w0 = c->lattice == 1 ? 2.0 / 3.0 : (c->lattice == 2 ? 4.0 / 9.0 : 1.0 / 3.0);
  a.k0 = (1.0 - w0) / w0;
  if (c->D == 1) {
    // Eq. (taylor-second31Db): sigma = nu_ef [omega (Pi^eq - Pi) + psi cs2 S]
    double nug = (1.0 / p.omega_g - 0.5) - CS2 * p.psi_g / p.omega_g;
    double nul = (1.0 / p.omega_l - 0.5) - CS2 * p.psi_l / p.omega_l;
    a.A_g = nug * p.omega_g;
    a.B_g = nug * p.psi_g * CS2;
    a.A_l = nul * p.omega_l;
    a.B_l = nul * p.psi_l * CS2;
  } else {
    // Eq. (lbm-sigma3): sigma = (1 - omega/2)(Pi^eq - Pi) - cs2 psi/2 S I
    a.A_g = 1.0 - 0.5 * p.omega_g;
    a.B_g = -0.5 * CS2 * p.psi_g;
    a.A_l = 1.0 - 0.5 * p.omega_l;
    a.B_l = -0.5 * CS2 * p.psi_l;
  }
  a.psi_g = p.psi_g;
  a.psi_l = p.psi_l;
  a.eta0_g = 1.0 + a.k0 * (1.0 - p.psi_g);
  a.eta0_l = 1.0 + a.k0 * (1.0 - p.psi_l);
  a.kappa_I = p.kappa_I;
  a.kappa_W = p.kappa_W;
  a.cgw = p.drag_model == LBM_DRAG_CGW;
  a.buoy = (p.R - 1.0) * p.g_hat;
  a.gamma = p.gamma;
  a.afloor = p.alpha_floor;
  a.spalding = p.spalding_mode;
  a.r_ag = c->r_ag;
  a.r_al = c->r_al;
  a.aIN = ramp(p.in_alpha, t, p.ramp_nt);
  a.ugIN = ramp(p.in_ug, t, p.ramp_nt);
  a.ulIN = p.inlet_ul_mode == 1 ? -a.aIN * a.ugIN / (1.0 - a.aIN) : ramp(p.in_ul, t, p.ramp_nt);
  a.plain = c->prec == LBM_FP64;
  a.cfield = c->cfield;
  a.beta_own = c->cfield && c->first_step;
  a.halo_off = c->halo_off;
  a.off32 = (long long)c->Q * c->plane < (1LL << 32);
  // the same constants in the kernels' arithmetic types
  PhysT<double> &d = a.pd;
  d.R_ = a.R; d.invR = a.invR; d.omega_g = a.omega_g; d.omega_l = a.omega_l; d.omega_a = a.omega_a;
  d.kgrad = a.kgrad; d.A_g = a.A_g; d.B_g = a.B_g; d.A_l = a.A_l; d.B_l = a.B_l; d.eta0_g = a.eta0_g;
  d.eta0_l = a.eta0_l; d.psi_g = a.psi_g; d.psi_l = a.psi_l; d.k0 = a.k0; d.kappa_I = a.kappa_I;
  d.kappa_W = a.kappa_W; d.buoy = a.buoy; d.gamma = a.gamma; d.afloor = a.afloor; d.r_ag = a.r_ag;
  d.r_al = a.r_al; d.aIN = a.aIN; d.ugIN = a.ugIN; d.ulIN = a.ulIN;
  {
    // r_ag + r_al - 1 exactly (two-sum of the double references)
    const double sm = d.r_ag + d.r_al, bb = sm - d.r_ag;
    const double er = (d.r_ag - (sm - bb)) + (d.r_al - bb);
    d.rsum1 = (sm - 1.0) + er;
  }
  PhysT<float> &f = a.pf;
  f.R_ = (float)d.R_; f.invR = (float)d.invR; f.omega_g = (float)d.omega_g; f.omega_l = (float)d.omega_l;
  f.omega_a = (float)d.omega_a; f.kgrad = (float)d.kgrad; f.A_g = (float)d.A_g; f.B_g = (float)d.B_g;
  f.A_l = (float)d.A_l; f.B_l = (float)d.B_l; f.eta0_g = (float)d.eta0_g; f.eta0_l = (float)d.eta0_l;
  f.psi_g = (float)d.psi_g; f.psi_l = (float)d.psi_l; f.k0 = (float)d.k0; f.kappa_I = (float)d.kappa_I;
  f.kappa_W = (float)d.kappa_W; f.buoy = (float)d.buoy; f.gamma = (float)d.gamma; f.afloor = (float)d.afloor;
  f.r_ag = (float)d.r_ag; f.r_al = (float)d.r_al; f.aIN = (float)d.aIN; f.ugIN = (float)d.ugIN;
  // float references sum exactly in double
  f.rsum1 = (float)(((double)f.r_ag + (double)f.r_al) - 1.0);
  f.ulIN = (float)d.ulIN;
  a.cs2 = CS2;
  a.two_cs4 = 2.0 * CS2 * CS2;
  a.nuef_g = (1.0 / p.omega_g - 0.5) - CS2 * p.psi_g / p.omega_g;
  a.nuef_l = (1.0 / p.omega_l - 0.5) - CS2 * p.psi_l / p.omega_l;
  return a;
}

static MomArgs make_mom(const lbm_ctx *c, double *out) {
  MomArgs ma;
  ma.s = make_args(c, c->t);
  ma.out = out;
  ma.N = c->N;
  ma.partials = c->partials;
  return ma;
}

static int ensure_stage(lbm_ctx *c, size_t bytes) {
  if (c->stage_bytes >= bytes) return LBM_OK;
  if (c->stage) cudaFree(c->stage);
  c->stage = nullptr;
  c->stage_bytes = 0;
  if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, LBM_ENOMEM, "staging allocation of %zu bytes failed", bytes);
  }
  c->stage_bytes = bytes;
  return LBM_OK;
}

// Tile of the fused kernel: x fastest; the axis of the inlet/outlet faces
// gets a tile of at least 2 and a shift so that each edge node and its inward
// neighbour share a block (their values are exchanged in shared memory).
// Largest block the fused step kernel of this lattice and precision was
// compiled for (its launch bounds); the FP64 reference kernels take 256.
template <int LAT> static int bound_threads(int prec) {
  if (prec == LBM_FP32) return StepBounds<Lattice<LAT>, float>::threads;
  if (prec == LBM_FP16DEV) return StepBounds<Lattice<LAT>, __half>::threads;
  if (prec == LBM_FP64DEV) return StepBounds<Lattice<LAT>, double>::threads;
  if (prec == LBM_FP16AB) return StepBounds<Lattice<LAT>, MixAB>::threads;
  return 256;
}

namespace lbm {
int step_max_threads(int lattice, int prec) {
  return lattice == 1 ? bound_threads<1>(prec) : (lattice == 2 ? bound_threads<2>(prec) : bound_threads<3>(prec));
}
}  // namespace lbm

static int max_tile_threads(const lbm_ctx *c) { return step_max_threads(c->lattice, c->prec); }

// Default tile: the kernel's full block size (the shapes measured fastest on
// the workloads: 64 x 2 for D2Q9, 16 x 8 for D3Q19 at 128 threads).
static void default_tile(lbm_ctx *c) {
  const lbm_params &p = c->p;
  const int mt = max_tile_threads(c);
  if (c->D == 1) { c->T[0] = 32; c->T[1] = 1; c->T[2] = 1; }  // small 1D domains: spread over SMs
  else if (c->D == 2) { c->T[0] = 64; c->T[1] = mt >= 128 ? mt / 64 : 1; c->T[2] = 1; }
  else if (mt == 128) { c->T[0] = 16; c->T[1] = 8; c->T[2] = 1; }
  else { c->T[0] = 32; c->T[1] = mt >= 128 ? 4 : 2; c->T[2] = mt >= 128 ? mt / 128 : 1; }
  const int ga = p.g_axis;
  const int io = (p.bc_lo[ga] == LBM_BC_INLET) || (p.bc_hi[ga] == LBM_BC_OUTLET);
  if (io && c->D == 3 && ga == 2) { c->T[0] = 32; c->T[1] = 2; c->T[2] = mt / 64; }  // >= 2 along z
  if (io && c->D == 2 && ga == 1 && c->T[1] < 2) { c->T[0] = mt / 2; c->T[1] = 2; }
}

static int choose_tiles(lbm_ctx *c) {
  const lbm_params &p = c->p;
  const int ga = p.g_axis;
  const int io = (p.bc_lo[ga] == LBM_BC_INLET) || (p.bc_hi[ga] == LBM_BC_OUTLET);
  if (io && c->T[ga] < 2) return set_err(c, LBM_EINVAL, "tile along g_axis must be >= 2 with an inlet/outlet");
  for (int d = 0; d < 3; d++) c->shift[d] = 0;
  if (io) {
    const int T = c->T[ga], n = c->n[ga];
    int s = -1;
    for (int cand = 0; cand <= T - 2; cand++) {
      if (p.bc_hi[ga] == LBM_BC_OUTLET && ((n - 1 + cand) % T) == 0) continue;
      s = cand;
      break;
    }
    if (s < 0) return set_err(c, LBM_EINVAL, "no tile shift keeps the outlet pair in one block");
    c->shift[ga] = s;
    const size_t per = c->prec == LBM_FP64 ? RXCH * 8 : (c->prec == LBM_FP64DEV ? XCH * 8 : XCH * 4);
    c->smem = (size_t)c->T[0] * c->T[1] * c->T[2] * per;
  } else {
    c->smem = 0;
  }
  // beta-stencil form: the block's c tile plus a one-node halo, 2*D values
  // per node padded to a multiple of 4 in the held type, after the exchange
  // area (16-byte aligned)
  c->halo_off = 0;
  if (c->cfield || c->p.beta_stencil) {
    const size_t box = (size_t)(c->T[0] + 2) * (c->D > 1 ? c->T[1] + 2 : 1) * (c->D > 2 ? c->T[2] + 2 : 1);
    c->halo_off = (int)((c->smem + 15) / 16 * 16);
    c->smem = (size_t)c->halo_off + box * (size_t)((2 * c->D + 3) / 4 * 4) * held_size(c->prec);
  }
  if (c->smem > 227 * 1024) return set_err(c, LBM_EINVAL, "tile needs %zu bytes of shared memory (> 227 KB)", c->smem);
  for (int d = 0; d < 3; d++) c->grid[d] = (c->n[d] + c->shift[d] + c->T[d] - 1) / c->T[d];
  return LBM_OK;
}

namespace lbm {
StepArgs ctx_step_args(const lbm_ctx *c, long long t) { return make_args(c, t); }
cudaError_t launch_batch_step(int lattice, int prec, const StepArgs *args, const WorkItem *work, unsigned nwork,
                              dim3 block, int parity, int latch, int off32, cudaStream_t st) {
  if (lattice == 1) return launch_batch_step_1(prec, args, work, nwork, block, parity, latch, off32, st);
  if (lattice == 2) return launch_batch_step_2(prec, args, work, nwork, block, parity, latch, off32, st);
  return launch_batch_step_3(prec, args, work, nwork, block, parity, latch, off32, st);
}
}  // namespace lbm

static void drop_graph(lbm_ctx *c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_period = 0;
}

// Equilibrium populations from device fields whose alpha_g (all in [0, 1])
// sums to alpha_sum: the deviation reference is its mean; clock at 0.
static int init_fields(lbm_ctx *c, const double *da, const double *dug, const double *dul, const double *dpk,
                       double alpha_sum) {
  c->r_ag = alpha_sum / (double)c->N;
  c->r_al = 1.0 - c->r_ag;
  c->t = 0;
  drop_graph(c);  // the deviation references are step arguments
  MomArgs ma = make_mom(c, nullptr);
  CUDA_TRY(c, dispatch_init(c, ma, da, dug, dul, dpk));
  c->mass0 = alpha_sum;
  c->first_step = 1;
  c->initialised = 1;
  c->sticky = 0;
  c->diag_pending = 0;
  c->err[0] = 0;
  return LBM_OK;
}

namespace lbm {
void ctx_window_info(const lbm_ctx *c, int *lattice, int n[3], long long *t, int *ready) {
  *lattice = c->lattice;
  for (int d = 0; d < 3; d++) n[d] = c->n[d];
  *t = c->t;
  *ready = c->initialised && !c->sticky;
}
void ctx_set_time(lbm_ctx *c, long long t) { c->t = t; }
int ctx_init_device(lbm_ctx *c, const double *alpha_g, const double *u_g, const double *u_l, const double *p_k,
                    double alpha_sum) {
  return init_fields(c, alpha_g, u_g, u_l, p_k, alpha_sum);
}
int ctx_error(lbm_ctx *c, int code, const char *msg) { return set_err(c, code, "%s", msg); }
}  // namespace lbm

extern "C" {

void lbm_default_params(lbm_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->R = 2.0;
  p->omega_g = p->omega_l = 1.0;
  p->omega_alpha = 1.5;
  p->n_gamma = 1;
  p->spalding_mode = 2;
  p->alpha_floor = 1e-8;
  p->precision = LBM_FP32;
}

int lbm_lattice(int lattice, int *Q, int *v, double *w) {
  if (lattice < 1 || lattice > 3 || !Q) return LBM_EINVAL;
  int q_ = lattice == 1 ? 3 : (lattice == 2 ? 9 : 19);
  *Q = q_;
  for (int q = 0; q < q_; q++)
    for (int a = 0; a < 3; a++) {
      int val = lattice == 1 ? Lattice<1>::v(q, a) : (lattice == 2 ? Lattice<2>::v(q, a) : Lattice<3>::v(q, a));
      if (v) v[3 * q + a] = val;
      if (w && a == 0) w[q] = lattice == 1 ? Lattice<1>::w(q) : (lattice == 2 ? Lattice<2>::w(q) : Lattice<3>::w(q));
    }
  return LBM_OK;
}

int lbm_create(int dim, int lattice, int nx, int ny, int nz, const lbm_params *p, lbm_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!p) return LBM_EINVAL;
  if (lattice < 1 || lattice > 3 || dim != lattice) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || (dim < 2 && ny != 1) || (dim < 3 && nz != 1)) return LBM_EINVAL;
  if ((long long)nx * ny * nz >= (1LL << 31)) return LBM_EINVAL;  // 32-bit node indices
  const lbm_params &q = *p;
  if (!(q.R >= 1.0) || !(q.omega_g > 0 && q.omega_g < 2) || !(q.omega_l > 0 && q.omega_l < 2) ||
      !(q.omega_alpha > 0 && q.omega_alpha < 2) || q.n_gamma < 1 || q.spalding_mode < 0 || q.spalding_mode > 2 ||
      !(q.alpha_floor > 0) || q.g_axis < 0 || q.g_axis >= dim || q.precision < 0 || q.precision > 4 ||
      (q.drag_model != LBM_DRAG_CONST && q.drag_model != LBM_DRAG_CGW) || q.diag_every < 0 ||
      (q.beta_stencil != 0 && q.beta_stencil != 1) || (q.beta_stencil && q.precision == LBM_FP64))
    return LBM_EINVAL;
  int dims[3] = {nx, ny, nz};
  for (int d = 0; d < dim; d++) {
    for (int side = 0; side < 2; side++) {
      int bc = side ? q.bc_hi[d] : q.bc_lo[d];
      if (bc < 0 || bc > 3) return LBM_EINVAL;
      if (bc == LBM_BC_INLET && !(side == 0 && d == q.g_axis)) return LBM_EINVAL;
      if (bc == LBM_BC_OUTLET && !(side == 1 && d == q.g_axis)) return LBM_EINVAL;
    }
    if ((q.bc_lo[d] == LBM_BC_PERIODIC) != (q.bc_hi[d] == LBM_BC_PERIODIC)) return LBM_EINVAL;
  }
  if ((q.bc_lo[q.g_axis] == LBM_BC_INLET || q.bc_hi[q.g_axis] == LBM_BC_OUTLET) && dims[q.g_axis] < 2)
    return LBM_EINVAL;
  if (q.bc_lo[q.g_axis] == LBM_BC_INLET && q.inlet_ul_mode == 1 && !(q.in_alpha[0] < 1 && q.in_alpha[1] < 1))
    return LBM_EINVAL;

  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  c->lattice = lattice;
  c->D = dim;
  c->Q = lattice == 1 ? 3 : (lattice == 2 ? 9 : 19);
  c->prec = q.precision;
  c->n[0] = nx; c->n[1] = ny; c->n[2] = nz;
  c->N = (long long)nx * ny * nz;
  c->plane = (c->N + 63) / 64 * 64;  // 256-byte aligned planes for every store type
  c->p = q;
  c->nblk_flat = (unsigned)((c->N + 255) / 256);
  default_tile(c);
  int rc = choose_tiles(c);
  if (rc) { int e = rc; delete c; return e; }
  const int nsch = q.beta_stencil ? 4 : 6;
  size_t pop_bytes = store_bytes_per_dir(c->prec, nsch) * c->Q * c->plane;
  size_t held_bytes = (size_t)3 * c->plane * held_size(c->prec);
  size_t c_bytes = (size_t)4 * dim * c->plane * held_size(c->prec);
  if (cudaMalloc(&c->pop, pop_bytes) != cudaSuccess || cudaMalloc(&c->held, held_bytes) != cudaSuccess ||
      (q.beta_stencil && cudaMalloc(&c->cfield, c_bytes) != cudaSuccess) ||
      cudaMalloc((void **)&c->partials, (size_t)c->nblk_flat * 8 * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&c->diag_dev, 8 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void **)&c->h_diag, 8 * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->diag_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(c);
    return LBM_ENOMEM;
  }
  *out = c;
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx *c, void *s) {
  if (!c) return LBM_EINVAL;
  c->stream = (cudaStream_t)s;
  return LBM_OK;
}

int lbm_init(lbm_ctx *c, const double *alpha_g, const double *u_g, const double *u_l, const double *p_k,
             int on_device) {
  if (!c) return LBM_EINVAL;
  if (!alpha_g || !u_g || !u_l || !p_k) return set_err(c, LBM_EINVAL, "lbm_init: NULL field");
  const long long N = c->N;
  const int D = c->D;
  // deviation reference of the alpha schemes: mean of the initial alpha_g
  std::vector<double> ha;
  const double *ah = alpha_g;
  if (on_device) {
    ha.resize(N);
    CUDA_TRY(c, cudaMemcpyAsync(ha.data(), alpha_g, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ah = ha.data();
  }
  double sum = 0.0;
  for (long long i = 0; i < N; i++) {
    if (!(ah[i] >= 0.0 && ah[i] <= 1.0)) return set_err(c, LBM_EINVAL, "lbm_init: alpha_g[%lld] outside [0,1]", i);
    sum += ah[i];
  }
  const double *da = alpha_g, *dug = u_g, *dul = u_l, *dpk = p_k;
  if (!on_device) {
    int rc = ensure_stage(c, (size_t)(2 + 2 * D) * N * sizeof(double));
    if (rc) return rc;
    double *s = (double *)c->stage;
    CUDA_TRY(c, cudaMemcpyAsync(s, alpha_g, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + N, u_g, D * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + (1 + D) * N, u_l, D * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(s + (1 + 2 * D) * N, p_k, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    da = s;
    dug = s + N;
    dul = s + (1 + D) * N;
    dpk = s + (1 + 2 * D) * N;
  }
  return init_fields(c, da, dug, dul, dpk, sum);
}

// Check the diagnostics a previous lbm_step enqueued, if they have arrived.
static int check_diag(lbm_ctx *c, int wait) {
  if (!c->diag_pending) return LBM_OK;
  if (wait) {
    CUDA_TRY(c, cudaEventSynchronize(c->diag_ev));
  } else {
    cudaError_t q = cudaEventQuery(c->diag_ev);
    if (q == cudaErrorNotReady) return LBM_OK;
    if (q != cudaSuccess) return set_err(c, LBM_ECUDA, "diagnostics event: %s", cudaGetErrorString(q));
  }
  c->diag_pending = 0;
  const double *d = c->h_diag;
  if (d[5] != 0.0 || !isfinite(d[0]) || !isfinite(d[1])) {
    c->sticky = LBM_ENAN;
    return set_err(c, LBM_ENAN, "non-finite populations at %.0f nodes", d[5]);
  }
  const int closed = c->p.bc_lo[c->p.g_axis] != LBM_BC_INLET && c->p.bc_hi[c->p.g_axis] != LBM_BC_OUTLET;
  if (closed && c->p.drift_limit > 0 && c->mass0 > 0 && fabs(d[0] - c->mass0) > c->p.drift_limit * c->mass0) {
    c->sticky = LBM_EDRIFT;
    return set_err(c, LBM_EDRIFT, "sum(a_g) drifted from %.17g to %.17g", c->mass0, d[0]);
  }
  return LBM_OK;
}

static int enqueue_diag(lbm_ctx *c, double *dev_out) {
  MomArgs ma = make_mom(c, nullptr);
  CUDA_TRY(c, dispatch_moments(c, ma, 2));
  c->launches++;
  k_diag_final<<<1, 256, 0, c->stream>>>(c->partials, (int)c->nblk_flat, dev_out);
  CUDA_TRY(c, cudaGetLastError());
  return LBM_OK;
}

// One step: the launch, and the diagnostics every diag_every steps.
static int one_step(lbm_ctx *c) {
  StepArgs a = make_args(c, c->t);
  CUDA_TRY(c, dispatch_step(c, a));
  c->first_step = 0;
  c->t++;
  if (c->p.diag_every > 0 && (c->t % c->p.diag_every) == 0) {
    if (c->diag_pending) {
      int rc = check_diag(c, 1);
      if (rc) return rc;
    }
    int rc = enqueue_diag(c, c->diag_dev);
    if (rc) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_diag, c->diag_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaEventRecord(c->diag_ev, c->stream));
    c->diag_pending = 1;
  }
  return LBM_OK;
}

static long long gcd_ll(long long a, long long b) { return b ? gcd_ll(b, a % b) : a; }

// Period after which the step arguments (parity, lag latch, diagnostics)
// repeat exactly, or 0 when they do not (an inlet ramp still changing them,
// the first step after an initialisation) or the period would be long.
static int graph_period(const lbm_ctx *c) {
  if (!c->use_graph) return 0;
  if (c->p.bc_lo[c->p.g_axis] == LBM_BC_INLET && c->p.ramp_nt > 0) return 0;
  if (c->first_step) return 0;
  long long per = c->p.n_gamma % 2 == 0 ? c->p.n_gamma : 2LL * c->p.n_gamma;
  if (c->p.diag_every > 0) per = per / gcd_ll(per, c->p.diag_every) * c->p.diag_every;
  return per <= 4096 ? (int)per : 0;
}

// One period from the graph, captured at its first use on a stream of the
// lattice's own (the legacy default stream cannot be captured) and replayed on
// the lattice's stream.  The diagnostics are taken once per period, after its
// last step (the period is a multiple of diag_every): one reduction, one copy
// to the host and one event record per replay, so the host's wait on the
// event is a wait on that copy.
static int replay_period(lbm_ctx *c, int period) {
  if (c->diag_pending) {
    int rc = check_diag(c, 1);
    if (rc) return rc;
  }
  if (!c->graph || c->graph_period != period) {
    drop_graph(c);
    if (!c->cap_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t user = c->stream;
    const long long t0 = c->t, l0 = c->launches;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->stream = c->cap_stream;
    int rc = LBM_OK;
    for (int k = 0; k < period && !rc; k++) {
      StepArgs a = make_args(c, t0 + k);
      cudaError_t e = dispatch_step(c, a);
      if (e != cudaSuccess) rc = set_err(c, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
      if (!rc && c->p.diag_every > 0 && k == period - 1) {
        rc = enqueue_diag(c, c->diag_dev);
        // an event record node the host can wait on (a plain record inside a
        // capture only orders work within the graph)
        if (!rc && (cudaMemcpyAsync(c->h_diag, c->diag_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream) != cudaSuccess ||
                    cudaEventRecordWithFlags(c->diag_ev, c->stream, cudaEventRecordExternal) != cudaSuccess))
          rc = set_err(c, LBM_ECUDA, "graph capture of the diagnostics");
      }
    }
    c->stream = user;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    if (!rc && e != cudaSuccess) rc = set_err(c, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    if (!rc) {
      e = cudaGraphInstantiate(&c->graph, g, 0);
      if (e != cudaSuccess) rc = set_err(c, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    if (g) cudaGraphDestroy(g);
    if (rc) {
      cudaGetLastError();
      drop_graph(c);
      return rc;
    }
    c->graph_period = period;
  }
  CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
  c->launches += c->graph_launches;
  c->t += period;
  if (c->p.diag_every > 0) c->diag_pending = 1;
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n) {
  if (!c || n < 0) return LBM_EINVAL;
  if (!c->initialised) return set_err(c, LBM_ESTATE, "lbm_step before lbm_init");
  if (c->sticky) return set_err(c, LBM_ESTATE, "sticky error %d; call lbm_init", c->sticky);
  int rc = check_diag(c, 0);
  if (rc) return rc;
  long long left = n;
  while (left > 0) {
    const int period = graph_period(c);
    if (period > 0 && c->t % period == 0 && left >= period) {
      rc = replay_period(c, period);
      left -= period;
    } else {
      rc = one_step(c);
      left--;
    }
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_set_graph(lbm_ctx *c, int enable) {
  if (!c) return LBM_EINVAL;
  c->use_graph = enable ? 1 : 0;
  drop_graph(c);
  return LBM_OK;
}

int lbm_get_moments(lbm_ctx *c, double *alpha_g, double *u_g, double *u_l, double *p_k, double *S_g, double *S_l,
                    int on_device) {
  if (!c) return LBM_EINVAL;
  if (!c->initialised) return set_err(c, LBM_ESTATE, "lbm_get_moments before lbm_init");
  const long long N = c->N;
  const int D = c->D;
  int rc = ensure_stage(c, (size_t)(4 + 2 * D) * N * sizeof(double));
  if (rc) return rc;
  double *s = (double *)c->stage;
  MomArgs ma = make_mom(c, s);
  CUDA_TRY(c, dispatch_moments(c, ma, 1));
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double *dst[6] = {alpha_g, u_g, u_l, p_k, S_g, S_l};
  long long off[6] = {0, N, (1 + D) * N, (1 + 2 * D) * N, (2 + 2 * D) * N, (3 + 2 * D) * N};
  long long len[6] = {N, D * N, D * N, N, N, N};
  for (int k = 0; k < 6; k++)
    if (dst[k]) CUDA_TRY(c, cudaMemcpyAsync(dst[k], s + off[k], len[k] * sizeof(double), kind, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx *c, int sch, double *out, int on_device) {
  if (!c || !out || sch < 0 || sch > 5) return LBM_EINVAL;
  if (!c->initialised) return set_err(c, LBM_ESTATE, "lbm_get_populations before lbm_init");
  size_t bytes = (size_t)c->Q * c->N * sizeof(double);
  double *dst = out;
  if (!on_device) {
    int rc = ensure_stage(c, bytes);
    if (rc) return rc;
    dst = (double *)c->stage;
  }
  MomArgs ma = make_mom(c, dst);
  CUDA_TRY(c, dispatch_pops(c, ma, sch));
  if (!on_device) CUDA_TRY(c, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_get_diag(lbm_ctx *c, double out[8]) {
  if (!c || !out) return LBM_EINVAL;
  if (!c->initialised) return set_err(c, LBM_ESTATE, "lbm_get_diag before lbm_init");
  int rc = check_diag(c, 1);
  if (rc && rc != LBM_ENAN && rc != LBM_EDRIFT) return rc;
  rc = enqueue_diag(c, c->diag_dev);
  if (rc) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(out, c->diag_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_tile_limit(int lattice, int precision, int *max_threads) {
  if (lattice < 1 || lattice > 3 || precision < 0 || precision > 4 || !max_threads) return LBM_EINVAL;
  *max_threads = step_max_threads(lattice, precision);
  return LBM_OK;
}

int lbm_set_tile(lbm_ctx *c, int tx, int ty, int tz) {
  if (!c) return LBM_EINVAL;
  const int n = tx * ty * tz;
  if (tx < 1 || ty < 1 || tz < 1 || n > max_tile_threads(c) || n % 32 != 0 || (c->D < 2 && ty != 1) ||
      (c->D < 3 && tz != 1))
    return set_err(c, LBM_EINVAL, "invalid tile %dx%dx%d (at most %d threads, a multiple of 32)", tx, ty, tz,
                   max_tile_threads(c));
  int old[3] = {c->T[0], c->T[1], c->T[2]};
  drop_graph(c);  // the launch shape is part of the captured launches
  c->T[0] = tx;
  c->T[1] = ty;
  c->T[2] = tz;
  int rc = choose_tiles(c);
  if (rc) {
    for (int d = 0; d < 3; d++) c->T[d] = old[d];
    choose_tiles(c);
    return rc;
  }
  return LBM_OK;
}

int lbm_get_tile(const lbm_ctx *c, int tile[3]) {
  if (!c || !tile) return LBM_EINVAL;
  for (int d = 0; d < 3; d++) tile[d] = c->T[d];
  return LBM_OK;
}

int lbm_time(const lbm_ctx *c, long long *t) {
  if (!c || !t) return LBM_EINVAL;
  *t = c->t;
  return LBM_OK;
}

int lbm_launch_count(const lbm_ctx *c, long long *n) {
  if (!c || !n) return LBM_EINVAL;
  *n = c->launches;
  return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err : ""; }

int lbm_destroy(lbm_ctx *c) {
  if (!c) return LBM_OK;
  if (c->stream || c->pop) cudaStreamSynchronize(c->stream);
  if (c->pop) cudaFree(c->pop);
  if (c->held) cudaFree(c->held);
  if (c->cfield) cudaFree(c->cfield);
  if (c->partials) cudaFree(c->partials);
  if (c->diag_dev) cudaFree(c->diag_dev);
  if (c->h_diag) cudaFreeHost(c->h_diag);
  if (c->diag_ev) cudaEventDestroy(c->diag_ev);
  if (c->stage) cudaFree(c->stage);
  drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return LBM_OK;
}

}  // extern "C"
