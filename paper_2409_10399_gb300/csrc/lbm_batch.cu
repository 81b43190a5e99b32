// Batched form: many independent lattices of one lattice type and precision
// advanced together -- one kernel launch per step over a device work list of
// (instance, tile) items, and the launches of one period of the step pattern
// captured once into a CUDA graph and replayed.
//
// Every instance is an ordinary lbm_ctx (its own store, held fields and
// scratch), so initialisation, moments and diagnostics reuse the single-
// lattice code; the batch owns the per-instance argument table, the work list
// and the graph.  Parity (t & 1) and the lag latch (t % n_gamma == 0) are
// common to all instances, which advance in lockstep; they repeat with period
// lcm(2, n_gamma), so that many launches form a replayable graph (instances
// have no time-dependent inlet values: inlet and outlet faces are rejected).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "lbm_internal.h"

using namespace lbm;

struct lbm_batch {
  int lattice = 0, prec = 0, n = 0, n_gamma = 1;
  std::vector<lbm_ctx *> inst;
  StepArgs *d_args = nullptr;
  WorkItem *d_work = nullptr;
  unsigned nwork = 0;
  int T[3] = {64, 2, 1};
  cudaStream_t user_stream = 0, own_stream = nullptr;
  int use_graph = 1;
  cudaGraphExec_t graph = nullptr;
  int graph_period = 0;
  long long t = 0, launches = 0;
  int off32 = 1;  // every instance has Q*plane < 2^32 (32-bit population offsets)
  char err[512] = {0};
};

static int berr(lbm_batch *b, int code, const char *fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof b->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

#define BTRY(b, call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return berr((b), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static int max_threads(const lbm_batch *b) { return step_max_threads(b->lattice, b->prec); }

static cudaStream_t launch_stream(lbm_batch *b) {
  // graphs cannot be captured on the legacy default stream: use an own
  // blocking stream then, which stays ordered with the legacy stream
  return b->user_stream ? b->user_stream : b->own_stream;
}

static void drop_graph(lbm_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_period = 0;
}

// Work list: the tiles of every instance, instance by instance.
static int build_work(lbm_batch *b) {
  std::vector<WorkItem> w;
  for (int i = 0; i < b->n; i++) {
    const lbm_ctx *c = b->inst[i];
    for (int z = 0; z < c->n[2]; z += b->T[2])
      for (int y = 0; y < c->n[1]; y += b->T[1])
        for (int x = 0; x < c->n[0]; x += b->T[0]) w.push_back(WorkItem{i, x, y, z});
  }
  if (w.size() >= (1ULL << 31)) return berr(b, LBM_EINVAL, "work list too long");
  if (b->d_work) cudaFree(b->d_work);
  b->d_work = nullptr;
  BTRY(b, cudaMalloc((void **)&b->d_work, w.size() * sizeof(WorkItem)));
  BTRY(b, cudaMemcpy(b->d_work, w.data(), w.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  b->nwork = (unsigned)w.size();
  drop_graph(b);
  return LBM_OK;
}

static int upload_args(lbm_batch *b) {
  std::vector<StepArgs> a(b->n);
  for (int i = 0; i < b->n; i++) a[i] = ctx_step_args(b->inst[i], b->t);
  BTRY(b, cudaMemcpy(b->d_args, a.data(), b->n * sizeof(StepArgs), cudaMemcpyHostToDevice));
  return LBM_OK;
}

static int launch_one(lbm_batch *b, long long t, cudaStream_t st) {
  dim3 block(b->T[0], b->T[1], b->T[2]);
  const int parity = (int)(t & 1), latch = (t % b->n_gamma) == 0;
  b->launches++;
  BTRY(b, launch_batch_step(b->lattice, b->prec, b->d_args, b->d_work, b->nwork, block, parity, latch, b->off32, st));
  return LBM_OK;
}

extern "C" {

int lbm_batch_create(int lattice, int n, const int *dims, const lbm_params *params, lbm_batch **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (lattice < 1 || lattice > 3 || n < 1 || !dims || !params) return LBM_EINVAL;
  const int prec = params[0].precision, ng = params[0].n_gamma;
  if (prec == LBM_FP64) return LBM_EINVAL;  // the batched kernel runs the deviation forms
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->lattice = lattice;
  b->prec = prec;
  b->n = n;
  b->n_gamma = ng;
  if (lattice == 3) { b->T[0] = 32; b->T[1] = 4; b->T[2] = max_threads(b) / 128; }
  if (lattice == 1) { b->T[0] = 128; b->T[1] = 1; b->T[2] = 1; }
  for (int i = 0; i < n; i++) {
    const lbm_params &p = params[i];
    if (p.precision != prec || p.n_gamma != ng || p.bc_lo[p.g_axis] == LBM_BC_INLET ||
        p.bc_hi[p.g_axis] == LBM_BC_OUTLET || p.beta_stencil) {
      lbm_batch_destroy(b);
      return LBM_EINVAL;
    }
    lbm_ctx *c = nullptr;
    int rc = lbm_create(lattice, lattice, dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], &p, &c);
    if (rc) {
      lbm_batch_destroy(b);
      return rc;
    }
    b->inst.push_back(c);
    if ((long long)c->Q * c->plane >= (1LL << 32)) b->off32 = 0;
  }
  if (cudaMalloc((void **)&b->d_args, n * sizeof(StepArgs)) != cudaSuccess ||
      cudaStreamCreate(&b->own_stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ENOMEM;
  }
  if (build_work(b) || upload_args(b)) {
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_size(const lbm_batch *b, int *n) {
  if (!b || !n) return LBM_EINVAL;
  *n = b->n;
  return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch *b, void *stream) {
  if (!b) return LBM_EINVAL;
  b->user_stream = (cudaStream_t)stream;
  for (auto *c : b->inst) lbm_set_stream(c, stream ? stream : (void *)b->own_stream);
  drop_graph(b);
  return LBM_OK;
}

int lbm_batch_set_graph(lbm_batch *b, int enable) {
  if (!b) return LBM_EINVAL;
  b->use_graph = enable ? 1 : 0;
  drop_graph(b);
  return LBM_OK;
}

int lbm_batch_set_tile(lbm_batch *b, int tx, int ty, int tz) {
  if (!b) return LBM_EINVAL;
  const int nt = tx * ty * tz;
  if (tx < 1 || ty < 1 || tz < 1 || nt % 32 || nt > max_threads(b) || (b->lattice < 2 && ty != 1) ||
      (b->lattice < 3 && tz != 1))
    return berr(b, LBM_EINVAL, "invalid tile %dx%dx%d (at most %d threads, a multiple of 32)", tx, ty, tz,
                max_threads(b));
  b->T[0] = tx;
  b->T[1] = ty;
  b->T[2] = tz;
  return build_work(b);
}

int lbm_batch_get_tile(const lbm_batch *b, int tile[3]) {
  if (!b || !tile) return LBM_EINVAL;
  for (int d = 0; d < 3; d++) tile[d] = b->T[d];
  return LBM_OK;
}

int lbm_batch_init(lbm_batch *b, int i, const double *alpha_g, const double *u_g, const double *u_l,
                   const double *p_k, int on_device) {
  if (!b || i < 0 || i >= b->n) return LBM_EINVAL;
  int rc = lbm_init(b->inst[i], alpha_g, u_g, u_l, p_k, on_device);
  if (rc) return berr(b, rc, "instance %d: %s", i, lbm_last_error(b->inst[i]));
  // all instances restart together: t = 0, and the init changed the
  // instance's deviation reference, which lives in the argument table
  for (auto *c : b->inst) c->t = 0;
  b->t = 0;
  drop_graph(b);
  return upload_args(b);
}

int lbm_batch_step(lbm_batch *b, int nsteps) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  for (auto *c : b->inst)
    if (!c->initialised) return berr(b, LBM_ESTATE, "lbm_batch_step before every instance is initialised");
  cudaStream_t st = launch_stream(b);
  // 2 and n_gamma divide the period, so parity and latch repeat with it
  int period = b->n_gamma % 2 == 0 ? b->n_gamma : 2 * b->n_gamma;
  long long left = nsteps;
  while (left > 0) {
    if (b->use_graph && b->t % period == 0 && left >= period) {
      if (!b->graph || b->graph_period != period) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        BTRY(b, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = 0;
        for (int k = 0; k < period && !rc; k++) rc = launch_one(b, b->t + k, st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return berr(b, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return berr(b, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        b->graph_period = period;
        b->launches -= period;  // counted again on each replay
      }
      BTRY(b, cudaGraphLaunch(b->graph, st));
      b->launches += period;
      b->t += period;
      left -= period;
    } else {
      int rc = launch_one(b, b->t, st);
      if (rc) return rc;
      b->t++;
      left--;
    }
  }
  for (auto *c : b->inst) c->t = b->t;
  return LBM_OK;
}

int lbm_batch_get_moments(lbm_batch *b, int i, double *alpha_g, double *u_g, double *u_l, double *p_k, double *S_g,
                          double *S_l, int on_device) {
  if (!b || i < 0 || i >= b->n) return LBM_EINVAL;
  if (!b->user_stream) BTRY(b, cudaStreamSynchronize(b->own_stream));
  int rc = lbm_get_moments(b->inst[i], alpha_g, u_g, u_l, p_k, S_g, S_l, on_device);
  return rc ? berr(b, rc, "instance %d: %s", i, lbm_last_error(b->inst[i])) : LBM_OK;
}

int lbm_batch_get_diag(lbm_batch *b, int i, double out[8]) {
  if (!b || i < 0 || i >= b->n) return LBM_EINVAL;
  if (!b->user_stream) BTRY(b, cudaStreamSynchronize(b->own_stream));
  int rc = lbm_get_diag(b->inst[i], out);
  return rc ? berr(b, rc, "instance %d: %s", i, lbm_last_error(b->inst[i])) : LBM_OK;
}

int lbm_batch_time(const lbm_batch *b, long long *t) {
  if (!b || !t) return LBM_EINVAL;
  *t = b->t;
  return LBM_OK;
}

int lbm_batch_launch_count(const lbm_batch *b, long long *n) {
  if (!b || !n) return LBM_EINVAL;
  *n = b->launches;
  return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err : ""; }

int lbm_batch_destroy(lbm_batch *b) {
  if (!b) return LBM_OK;
  cudaStream_t st = launch_stream(b);
  if (st) cudaStreamSynchronize(st);
  drop_graph(b);
  for (auto *c : b->inst) lbm_destroy(c);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_work) cudaFree(b->d_work);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
  return LBM_OK;
}

}  // extern "C"
