/*
 * lbm.h -- C ABI of the GB300 library for the six coupled lattice Boltzmann
 * schemes of the Eulerian-Eulerian multiphase framework of Piredda & Asinari
 * (arXiv 2409.10399): f_g, f_l (artificially compressible phase momenta,
 * Sec. 2.1.1), f_alpha_g, f_alpha_l (volume fractions, Sec. 2.2) and f_beta_g,
 * f_beta_l (continuity sources, Sec. 2.3), on one D1Q3, D2Q9 or D3Q19 lattice.
 *
 * Conventions (all entry points):
 *  - Every function returns an int status: LBM_OK (0) or a negative LBM_E*
 *    code.  Nothing aborts or exits.  lbm_last_error() gives a one-line text.
 *  - Lattice units (hatted quantities of the paper).  Node index
 *    i = x + nx*(y + ny*z); a vector field is D consecutive planes of N nodes
 *    (SoA), D = 1, 2, 3 for D1Q3, D2Q9, D3Q19.
 *  - Buffers passed in are owned by the caller; the library copies from/to
 *    them during the call (or on the context's stream for on_device = 1) and
 *    never keeps a pointer.  `on_device` = 1 means the pointers are CUDA
 *    device pointers of the current device, 0 means host memory.
 *  - The library owns the population store (6*Q planes in HBM) and all
 *    scratch.  Work is enqueued on the context's stream (default: the legacy
 *    default stream; see lbm_set_stream).
 *  - Errors are sticky: after LBM_ENAN or LBM_EDRIFT, lbm_step returns
 *    LBM_ESTATE until the next lbm_init.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,   /* bad argument: sizes, rates, boundary codes, NULL */
  LBM_ENOMEM = -2,   /* device allocation failed */
  LBM_ECUDA = -3,    /* a CUDA call failed (text in lbm_last_error) */
  LBM_ENAN = -4,     /* diagnostics found a non-finite population */
  LBM_EDRIFT = -5,   /* per-phase volume drifted beyond drift_limit */
  LBM_ETIMEOUT = -6, /* a bounded wait ran out */
  LBM_ESTATE = -7    /* call out of order (not initialised, sticky error) */
};

enum { LBM_D1Q3 = 1, LBM_D2Q9 = 2, LBM_D3Q19 = 3 };

/* Storage/arithmetic of the populations.
 * FP64: the reference path -- full populations in double, every formula of
 *   the paper evaluated literally in the order it is written, without
 *   floating-point contraction (bitwise reproducible against any other such
 *   evaluation, e.g. a CPU one).
 * FP32: float store of the deviations f - w_q*r_s (r = 1, or the mean alpha
 *   for the alpha schemes) and float arithmetic written in those deviations.
 * FP16DEV: half store of the same deviations, float arithmetic.
 * FP64DEV: the FP32 kernel's deviation arithmetic in double (validation of
 *   the fast path's algebra at double precision).
 * FP16AB: f_g and f_l (the phase momenta and pressure, Sec. 2.1.1) in the
 *   float store, f_alpha and f_beta (Secs. 2.2, 2.3) in the half store;
 *   float arithmetic.  The liquid velocity is the first moment of f_l, which
 *   in half storage keeps 11 significant bits per population per step; this
 *   form carries it at FP32 resolution for 16 instead of 24 bytes per
 *   direction and node. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16DEV = 2, LBM_FP64DEV = 3, LBM_FP16AB = 4 };

/* Face conditions.  WALL: half-way bounce-back for all six schemes (Eq.
 * (BCINLET), BB rule with zero wall velocity).  INLET: Table 1, only on the
 * low face of g_axis, inside the strip [inlet_lo, inlet_hi) of the first
 * transverse axis (a wall elsewhere on that face; the whole face in 1D).
 * OUTLET: Table 2, only on the high face of g_axis. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_INLET = 2, LBM_BC_OUTLET = 3 };

/* K_I = kappa_I (CONST) or K_I = kappa_I * Lambda' with Lambda of Eq. (Lambda)
 * (Clift-Grace-Weber, Eq. (CliftGraceWeber)); the liquid wall friction of
 * Eq. (wallmomentum1D) uses kappa_W the same way and is active when
 * kappa_W != 0. */
enum { LBM_DRAG_CONST = 0, LBM_DRAG_CGW = 1 };

typedef struct {
  double R;                  /* rho_l / rho_g >= 1, Eq. (lbm-phi-l) */
  double omega_g, omega_l;   /* BGK rates of f_g, f_l in (0,2), Eq. (colloperator) */
  double omega_alpha;        /* rate of f_alpha in (0,2), Eq. (lbmalpha) */
  double psi_g, psi_l;       /* forcing knob of Eq. (forcingoperator); 0 = the
                                paper's choice xi = 5/3 nu (Sec. 3.5) */
  int drag_model;            /* LBM_DRAG_* */
  double kappa_I, kappa_W;
  double g_hat;              /* buoyancy (R-1)*g_hat on the gas along +g_axis,
                                kinematic-pressure form, Eq. (Gg1D) */
  int g_axis;                /* 0, 1, 2 < D */
  double gamma;              /* Ohwada dashpot, Eqs. (lbm-cont-g1Dhat), (lbm-cont-l1Dhat) */
  int n_gamma;               /* >= 1: S'' and Lambda' latched when t % n_gamma == 0,
                                Eqs. (lbm-cont-1D-update), (Lambda-update) */
  int spalding_mode;         /* 0 off; 1 alpha^B in couplings only; 2 alpha^B also
                                in the f_alpha equilibrium (Eq. (spalding)) */
  double alpha_floor;        /* floor of alpha in the 1/alpha factors (> 0) */
  int bc_lo[3], bc_hi[3];    /* LBM_BC_* per axis face; unused axes ignored */
  int inlet_lo, inlet_hi;    /* inlet strip on the first transverse axis */
  double in_alpha[2];        /* (min, max) of alpha_g^IN, ramp Eq. (transient) */
  double in_ug[2];           /* (min, max) of u_g^IN along +g_axis */
  double in_ul[2];           /* (min, max) of u_l^IN (inlet_ul_mode 0) */
  int ramp_nt;               /* n_t of Eq. (transient); <= 0: the max at once */
  int inlet_ul_mode;         /* 0: u_l^IN ramp; 1: u_l^IN = -a u_g^IN/(1-a)
                                (zero net volume flux through the strip) */
  int precision;             /* LBM_FP64 / LBM_FP32 / LBM_FP16DEV / LBM_FP64DEV / LBM_FP16AB */
  int diag_every;            /* > 0: FP64 diagnostics every that many steps
                                inside lbm_step, checked for NaN / drift */
  double drift_limit;        /* relative drift of sum(a_g) that raises
                                LBM_EDRIFT (closed domains only); <= 0: off */
  int beta_stencil;          /* 0: six-scheme store (6*Q population planes).
                                1: beta-stencil form -- the beta schemes are
                                reset to f^eq(1, c) every step (Eq. (lbmbeta)
                                with beta = 1), so the store keeps 4*Q planes
                                plus c_g, c_l (2*D planes, double-buffered, in
                                the held type) and re-evaluates the streamed
                                beta populations from c at x - v_q.  The same
                                method, equal to the six-scheme store to
                                rounding, not bit for bit: the two forms are
                                separate kernels whose multiply-adds the
                                compiler contracts differently (the initial
                                beta equilibria alone are bitwise equal).
                                FP16DEV holds c in FP32, more precise than its
                                FP16 beta planes.  Not with LBM_FP64. */
} lbm_params;

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

/* Fill `p` with the defaults (R = 2, omega = 1, omega_alpha = 1.5, psi = 0,
 * CONST drag 0, no gravity, gamma = 0, n_gamma = 1, Spalding mode 2,
 * alpha_floor = 1e-8, all faces periodic, FP32, no diagnostics). */
void lbm_default_params(lbm_params *p);

/* Allocate a simulation of one lattice.  dim must equal the lattice's D
 * (ny = nz = 1 for D1Q3, nz = 1 for D2Q9).  Validates rates, sizes and
 * boundary codes (LBM_EINVAL), allocates 6*Q*N populations (4*Q*N plus
 * 4*D*N values of c with beta_stencil) plus three held fields (S''_g,
 * S''_l, Lambda') and small scratch on the current CUDA device
 * (LBM_ENOMEM).  *out is NULL on failure. */
int lbm_create(int dim, int lattice, int nx, int ny, int nz, const lbm_params *p, lbm_ctx **out);

/* Set every scheme to its equilibrium from macroscopic fields and reset t = 0:
 * f_g = f_I^eq(1, eps_g, u_g) with eps_g = p_k/cs2 (Eq. (sigmag1D)),
 * f_l = f_I^eq(phi, 1, u_l) with phi of Eq. (lbm-phi-l), f_alpha = f^eq(alpha, u)
 * with alpha_l = 1 - alpha_g, f_beta = f^eq(1, c) with c of Eq. (velocitybeta);
 * S'' = 0, Lambda' = Lambda(alpha_g).  alpha_g, p_k: N doubles; u_g, u_l:
 * D*N doubles.  Clears sticky errors. */
int lbm_init(lbm_ctx *c, const double *alpha_g, const double *u_g, const double *u_l,
             const double *p_k, int on_device);

/* Enqueue n fused collide-and-stream steps (n >= 0) on the context stream:
 * moments, sources, Spalding, coupling, dashpot, lag, grad(alpha), stress,
 * drag, forces, the six BGK/LKS collisions and AA-pattern in-place streaming
 * with the face conditions (Sec. 2-3).  Returns after enqueueing; with
 * diag_every > 0 it also checks the diagnostics it has already received
 * (LBM_ENAN, LBM_EDRIFT).  LBM_ESTATE before lbm_init or after a sticky
 * error. */
int lbm_step(lbm_ctx *c, int n);

/* Macroscopic fields of the current state (as the next step sees them), in
 * FP64: alpha_g^B (Eq. (spalding)), u_g, u_l (D*N each), p_k = cs2*eps_g,
 * S_g, S_l = 1 - beta (Eq. (lbmbetataylorzeroth5)).  Any pointer may be NULL.
 * Synchronises the context stream before returning. */
int lbm_get_moments(lbm_ctx *c, double *alpha_g, double *u_g, double *u_l, double *p_k,
                    double *S_g, double *S_l, int on_device);

/* Populations of scheme s (0 g, 1 l, 2 alpha_g, 3 alpha_l, 4 beta_g, 5 beta_l)
 * as full values f (not deviations) in FP64, q-major: out[q*N + i], with the
 * velocity order of lbm_lattice().  Synchronises. */
int lbm_get_populations(lbm_ctx *c, int s, double *out, int on_device);

/* Velocity set of lattice LBM_D1Q3/D2Q9/D3Q19 in the library's order:
 * v[3*q + a] (a < 3, zero-padded), w[q]; returns Q through *Q.  Host
 * pointers of length >= 3*19 and 19 (v or w may be NULL).  Needs no GPU. */
int lbm_lattice(int lattice, int *Q, int *v, double *w);

/* FP64 diagnostics of the current state (warp/block/grid reduction on the
 * GPU): [0] sum a_g, [1] sum a_l, [2] sum alpha_g^B, [3] sum (a_g+a_l-1)^2,
 * [4] max |u| over both phases, [5] number of nodes with a non-finite
 * population, [6] sum (eps_g - 1), [7] sum (eps_l - 1).  Synchronises. */
int lbm_get_diag(lbm_ctx *c, double out[8]);
/* Graph replay of lbm_step (default on).  When the step arguments repeat
 * exactly (no inlet ramp in progress; after the beta-stencil form's first
 * step) with period lcm(2, n_gamma, diag_every) <= 4096, lbm_step replays
 * whole periods from a CUDA graph captured once on a stream of the library's
 * own, which removes the launch gaps between steps; the results are bitwise
 * those of plain launches.  Within a replayed period the diagnostics are
 * taken once, after its last step (the period is a multiple of diag_every),
 * so a non-finite state or a drift is reported at most one period after it
 * arises.  enable = 0 launches every step.  lbm_init and
 * lbm_set_tile drop the captured graph.  Not in the paper. */
int lbm_set_graph(lbm_ctx *c, int enable);

/* Use `cuda_stream` (a cudaStream_t of the current device, e.g. the value of
 * torch.cuda.current_stream().cuda_stream) for all later work; NULL selects
 * the legacy default stream.  The caller keeps the stream alive. */
int lbm_set_stream(lbm_ctx *c, void *cuda_stream);

/* Thread-block tile of the fused step kernel, tx*ty*tz threads over
 * (x, y, z), a multiple of 32 and at most 128 (D1Q3, D2Q9 in FP32/FP16DEV)
 * or 256 (the other lattices and precisions).  The default is chosen at
 * lbm_create; an autotuner may try others.  With an inlet or outlet face the
 * tile along g_axis must be >= 2 (LBM_EINVAL otherwise).  Takes effect at the
 * next lbm_step; results do not depend on the tile. */
int lbm_set_tile(lbm_ctx *c, int tx, int ty, int tz);

/* Current tile (tile[0..2]) of the fused step kernel. */
int lbm_get_tile(const lbm_ctx *c, int tile[3]);

/* Largest tile (threads per block) of the fused step kernel of lattice
 * LBM_D1Q3/D2Q9/D3Q19 in precision LBM_FP* (its launch bounds), through
 * *max_threads.  Host only, no GPU needed; LBM_EINVAL for unknown codes. */
int lbm_tile_limit(int lattice, int precision, int *max_threads);

/* Time step counter t (number of completed steps since lbm_init). */
int lbm_time(const lbm_ctx *c, long long *t);

/* Number of GPU kernel launches this context has issued since creation. */
int lbm_launch_count(const lbm_ctx *c, long long *n);

/* Text of the last error of this context ("" if none); NULL-safe. */
const char *lbm_last_error(const lbm_ctx *c);

/* Free the context and its device memory (synchronises); NULL-safe. */
int lbm_destroy(lbm_ctx *c);

/* ---- Batched form ---------------------------------------------------------
 * Many independent lattices ("instances") of one lattice type and precision,
 * each with its own sizes and lbm_params (density ratio, drag, ...), advanced
 * together: one kernel launch per step over a device work list of
 * (instance, tile) items, in lockstep (common t).  Parity and the lag latch
 * repeat with period lcm(2, n_gamma), so when enabled (default) the launches
 * of one period are captured once into a CUDA graph and replayed.  Every
 * instance must use the same precision (not LBM_FP64) and n_gamma and have
 * no inlet/outlet face (their values depend on t) and the six-scheme store
 * (beta_stencil = 0); LBM_EINVAL otherwise.
 * Instance i computes what a single lbm_ctx with the same arguments computes
 * (the same node arithmetic in a second kernel; equal up to rounding).
 * dims: 3 ints per instance (nx, ny, nz).  All other conventions as above. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(int lattice, int n, const int *dims, const lbm_params *params, lbm_batch **out);
int lbm_batch_size(const lbm_batch *b, int *n);
/* lbm_init of instance i; resets the common t to 0 for all instances. */
int lbm_batch_init(lbm_batch *b, int i, const double *alpha_g, const double *u_g, const double *u_l,
                   const double *p_k, int on_device);
/* Enqueue n steps of every instance. */
int lbm_batch_step(lbm_batch *b, int n);
int lbm_batch_get_moments(lbm_batch *b, int i, double *alpha_g, double *u_g, double *u_l, double *p_k,
                          double *S_g, double *S_l, int on_device);
int lbm_batch_get_diag(lbm_batch *b, int i, double out[8]);
/* Tile (work-item shape) of the batched kernel; same limits as lbm_set_tile. */
int lbm_batch_set_tile(lbm_batch *b, int tx, int ty, int tz);
int lbm_batch_get_tile(const lbm_batch *b, int tile[3]);
/* Replay the steps through a captured CUDA graph (1, default) or launch them
 * one by one (0). */
int lbm_batch_set_graph(lbm_batch *b, int enable);
/* Stream for all work (NULL: an internal blocking stream, ordered with the
 * legacy default stream). */
int lbm_batch_set_stream(lbm_batch *b, void *cuda_stream);
int lbm_batch_time(const lbm_batch *b, long long *t);
int lbm_batch_launch_count(const lbm_batch *b, long long *n);
const char *lbm_batch_last_error(const lbm_batch *b);
int lbm_batch_destroy(lbm_batch *b);

/* ---- Diagnostics that allocate nothing ------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that may not call cudaMalloc themselves or have the library do it: an
 * application that hands out device memory only from its own pool, or code
 * that runs where the CUDA allocator must not be touched.
 *
 * It computes the same eight FP64 diagnostics as lbm_get_diag ([0] sum a_g,
 * [1] sum a_l, [2] sum alpha_g^B, [3] sum (a_g + a_l - 1)^2, [4] max |u| over
 * both phases, [5] nodes with a non-finite population, [6] sum (eps_g - 1),
 * [7] sum (eps_l - 1)) of a population set the caller owns: `pops` is a
 * device pointer to 6*Q*n_nodes doubles, full values f (not deviations),
 * pops[(s*Q + q)*n_nodes + i] for scheme s (g, l, alpha_g, alpha_l, beta_g,
 * beta_l), velocity q in lbm_lattice() order -- e.g. six lbm_get_populations
 * calls with on_device = 1 into one buffer.  `spalding_mode` as in
 * lbm_params.  `out` receives 8 doubles: a device pointer if out_on_device,
 * else host memory (the call then synchronises `stream`).  Work is enqueued
 * on `stream` (a cudaStream_t of the current device; NULL = legacy default).
 *
 * No cudaMalloc, cudaFree or other allocation happens: the per-block partial
 * sums use one fixed scratch array of 65,600 bytes (1024 blocks x 8 doubles
 * plus 8 results) that is a file-scope __device__ variable, so every GPU that
 * loads the library holds it until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  The
 * address is cached together with the id of the CUDA context it was looked
 * up in: after a device reset, or under another context made current by the
 * caller, the next call looks it up again (and that call, too, belongs
 * outside a stream capture).
 * Every call uses the same array, which keeps the last call's contents (each
 * call overwrites the parts it reads), so calls that overlap on the GPU --
 * on different streams, or from different host threads -- race and must be
 * serialised by the caller.
 *
 * Returns LBM_EINVAL for a bad lattice or Spalding mode, a NULL pointer, or
 * n_nodes outside [1, LBM_NOALLOC_MAX_NODES]; LBM_ECUDA if a CUDA call fails.
 * A CUDA error already pending from the caller's earlier work
 * (cudaPeekAtLastError) makes it return LBM_ECUDA before launching anything,
 * and that error stays pending for the caller; errors of its own launches it
 * reads and clears. */
#define LBM_NOALLOC_MAX_NODES 2147483647LL
int lbm_diag_populations_noalloc(int lattice, int spalding_mode, const double *pops, long long n_nodes,
                                 double *out, int out_on_device, void *stream);

/* ---- Learned surrogate (not in the paper) ---------------------------------
 * A factorised Fourier neural operator that maps a 2D state to its change
 * over a fixed number of LBM steps (64 in the surrogate workload), trained on
 * trajectories the library's own LBM produces; the plain LBM step is its
 * reference and its fallback.  Model (channels C, K modes per axis, L layers;
 * state channels padded to 16):
 *   h_0 = W_in x + b_in;  h_l = GELU(W_l h + b_l + S^x_l h + S^y_l h);
 *   y = W_out h_L + b_out;  next = now + s_out * y.
 * S^x projects every row onto the truncated real Fourier basis of the x axis
 * (cos k x, sin k x, k < K), mixes the channels of each mode with complex
 * weights A_k + i B_k, and projects back; S^y likewise along y.  Every
 * contraction is a BF16 matrix product with FP32 accumulation; parameters,
 * gradients and Adam moments are FP32.  2,115,920 parameters at C = 64,
 * K = 32, L = 4.
 *
 * The state is six FP64 device planes of nx*ny values, [alpha_g][u_g,x]
 * [u_g,y][u_l,x][u_l,y][p_k], node x + nx*y (the layout of lbm_get_moments
 * for D2Q9).  Inputs are normalised with (mean, std_in) per channel and the
 * model's output is scaled by std_out (lbm_fno_set_norm).  All work runs on
 * the model's stream; the calls that return a number synchronise it. */
typedef struct lbm_fno lbm_fno;
/* nx, ny: multiples of 16; channels: a multiple of 16; modes: a multiple of 8
 * with 2*modes <= nx, ny; 1 <= layers <= 16.  Parameters start at zero
 * (lbm_fno_set_params sets them).  LBM_EINVAL / LBM_ENOMEM. */
int lbm_fno_create(int nx, int ny, int channels, int modes, int layers, lbm_fno **out);
int lbm_fno_num_params(const lbm_fno *f, long long *n);
/* Host FP32 arrays of lbm_fno_num_params values, in this order: W_in (C x 16),
 * b_in (C); per layer W (C x C), b (C), A_x, B_x, A_y, B_y (K x C x C each,
 * [k][c_out][c_in]); W_out (16 x C), b_out (16). */
int lbm_fno_set_params(lbm_fno *f, const float *host, long long n);
int lbm_fno_get_params(const lbm_fno *f, float *host, long long n);
int lbm_fno_get_grads(const lbm_fno *f, float *host, long long n);
int lbm_fno_zero_grads(lbm_fno *f);
int lbm_fno_set_norm(lbm_fno *f, const float mean[6], const float std_in[6], const float std_out[6]);
int lbm_fno_set_stream(lbm_fno *f, void *cuda_stream);
/* One training sample: forward from `now`, loss = mean over the six state
 * channels and the nodes of (y - (next - now)/std_out)^2 (returned in *loss),
 * and its gradient added to the accumulated gradients.  `now`, `next`: FP64
 * device states. */
int lbm_fno_accumulate(lbm_fno *f, const double *now, const double *next, double *loss);
/* Weight lambda >= 0 of the loss's conservation term (default 0): the loss
 * of lbm_fno_accumulate becomes the mean squared error plus
 * lambda * (mean over the nodes of y_0 - t_0)^2, channel 0 being alpha_g in
 * the model's units; it penalises the error of the window's change of
 * sum(alpha_g), the quantity the volume check of lbm_fno_advance tests.
 * LBM_EINVAL for a negative or non-finite weight. */
int lbm_fno_set_loss(lbm_fno *f, double cons_weight);
/* Expected change dV of sum(alpha_g) over one model call (default 0, a
 * closed box): the gas a lattice's inlet brings in during the window the
 * call stands for.  The volume check of lbm_fno_advance (and so of
 * lbm_surrogate_advance) then tests the change of each phase's volume
 * against it: |(sum alpha_g' - sum alpha_g) - dV| relative to sum alpha_g
 * and to sum (1 - alpha_g).  LBM_EINVAL for a non-finite dV.  Not in the
 * paper. */
int lbm_fno_set_inflow(lbm_fno *f, double dV);
/* Adam step (Kingma & Ba, bias-corrected) with the accumulated gradients
 * times grad_scale, then gradients zeroed and the BF16 weights refreshed. */
int lbm_fno_adam(lbm_fno *f, float lr, float beta1, float beta2, float eps, float grad_scale);
/* Surrogate step: next = now + std_out * model(now) (device states, distinct
 * buffers).  *drift = relative change of the per-phase volumes sum(alpha_g)
 * and sum(1 - alpha_g) beyond the expected inflow (lbm_fno_set_inflow; the
 * larger of the two; infinite if any value of the new state is not finite);
 * *ok = drift <= max_drift and every new alpha_g in [0, 1].  Synchronises the
 * stream (the host reads the FP64 sums).  A caller that gets ok = 0
 * advances the state with the LBM instead (the surrogate's fallback). */
int lbm_fno_advance(lbm_fno *f, const double *now, double *next, double max_drift, double *drift, int *ok);
/* One surrogate window on a live lattice: the surrogate's use with the LBM as
 * its fallback.  `ctx` must be a D2Q9 lattice of the model's nx x ny,
 * initialised, at an even time t (populations in their natural slots);
 * `window` (even) is the number of LBM steps one model call stands for (64
 * for the trained workload model).  The lattice's moments go through
 * lbm_fno_advance; when its check passes (*used = 1) the lattice is
 * re-initialised from the predicted fields exactly as lbm_init does
 * (equilibrium populations, held sources re-latched) and its clock set to
 * t + window; otherwise (*used = 0) the lattice advances `window` LBM steps
 * from its own populations (lbm_step).  *drift as for lbm_fno_advance.
 * LBM_EINVAL for a lattice of another type or size or an odd window,
 * LBM_ESTATE for an odd time or a lattice in error.  Uses the model's stream
 * for the model and the lattice's stream for the lattice; synchronises both.
 * Not in the paper. */
int lbm_surrogate_advance(lbm_ctx *ctx, lbm_fno *model, int window, double max_drift, double *drift, int *used);
int lbm_fno_launch_count(const lbm_fno *f, long long *n);
const char *lbm_fno_last_error(const lbm_fno *f);
int lbm_fno_destroy(lbm_fno *f);
/* The surrogate's matrix product alone (for tests and measurement):
 * C[b] = alpha op(A[b]) op(B[b]) + beta C[b], b < batch, BF16 A and B (device,
 * row-major; op(A) = A^T when ta, stored K x M), FP32 (out_f32) or BF16 C,
 * on the tcgen05 tensor cores (FP32 accumulation in tensor memory, operands
 * staged by TMA).  M, N, K multiples of 16, leading dimensions and batch
 * strides multiples of 8 elements, pointers 32-byte aligned; a batch stride
 * of 0 shares that operand across the batch (not for C when beta != 0).
 * ksplit > 1 splits K over blocks with FP32 atomics (needs out_f32 and
 * beta = 1).  Enqueued on `stream`; LBM_EINVAL for bad shapes (an operand
 * the TMA unit cannot describe included). */
int lbm_fno_gemm(int ta, int tb, int M, int N, int K, float alpha, const void *A, int lda, long long sA,
                 const void *B, int ldb, long long sB, float beta, void *C, int ldc, long long sC, int batch,
                 int out_f32, int ksplit, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
