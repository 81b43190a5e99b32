// Learned surrogate of the 2D step: a factorised Fourier neural operator
// (per-axis spectral convolutions with truncated real-DFT bases) that maps the
// state (alpha_g, u_g, u_l, p_k) to its increment over 64 LBM steps.  Not in
// the paper; the plain lattice Boltzmann step is its reference and fallback.
//
// Model, channels C, K modes per axis, L layers (state channels padded to 16):
//   h_0 = W_in x + b_in
//   h_l = GELU(W_l h_{l-1} + b_l + S^x_l(h_{l-1}) + S^y_l(h_{l-1})),  l = 1..L
//   y   = W_out h_L + b_out,   x_next = x + s_out * y   (s_out per channel)
// S^x: coefficients H = h B_x (B_x: n_x x 2K, columns cos k x, sin k x for
// k < K, interleaved), per mode the complex channel mixing
// [O_c; O_s] = [[A_k, -B_k], [B_k, A_k]] [H_c; H_s], back with the inverse
// basis (B_x scaled by 1/n_x for k = 0, 2/n_x otherwise).  S^y likewise
// along y.  Every contraction of the layers is a BF16 matrix product with
// FP32 accumulation (fno_kernels.cuh); the lifting and output projection are
// products too in training, and direct passes over the nodes with the same
// numerics in inference (lbm_fno_advance).  Activations of the backward pass
// are kept per layer (z in FP32, h and the spectral coefficients in BF16).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "fno_kernels.cuh"
#include "fno_umma.cuh"
#include "lbm_ctx_access.h"

using fno::bf16;

namespace {

struct Off {  // offsets of one model's parameters in the FP32 parameter buffer
  long long W_in, b_in, W_out, b_out;
  std::vector<long long> W, b, Ax, Bx, Ay, By;
  long long total;
};

Off layout(int C, int K, int L, int cin, int cout) {
  Off o;
  long long at = 0;
  o.W_in = at; at += (long long)C * cin;
  o.b_in = at; at += C;
  for (int l = 0; l < L; l++) {
    o.W.push_back(at); at += (long long)C * C;
    o.b.push_back(at); at += C;
    o.Ax.push_back(at); at += (long long)K * C * C;
    o.Bx.push_back(at); at += (long long)K * C * C;
    o.Ay.push_back(at); at += (long long)K * C * C;
    o.By.push_back(at); at += (long long)K * C * C;
  }
  o.W_out = at; at += (long long)cout * C;
  o.b_out = at; at += cout;
  o.total = at;
  return o;
}

}  // namespace

struct lbm_fno {
  int nx, ny, C, K, L, cin = 16, cout = 16, cv = 6;
  long long P;
  Off off;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  long long adam_t = 0;
  bf16 *W_in16 = nullptr, *W_out16 = nullptr, *W16 = nullptr, *Wfx16 = nullptr, *Wfy16 = nullptr;
  bf16 *Bx = nullptr, *Bxi = nullptr, *By = nullptr, *Byi = nullptr;
  bf16 *x16 = nullptr, *h16 = nullptr, *Hx16 = nullptr, *Hy16 = nullptr, *O16 = nullptr;
  float *z = nullptr, *y = nullptr, *tgt = nullptr;
  float *dy = nullptr, *dh = nullptr, *dz = nullptr, *dWf = nullptr;
  float *coef32 = nullptr;  // FP32 scratch of the split y-axis projections (2K x C x nx)
  bf16 *dy16 = nullptr, *dz16 = nullptr, *dO16 = nullptr, *dH16 = nullptr;
  double *part = nullptr, *h_part = nullptr, *red = nullptr, *h_red = nullptr;
  double *st = nullptr;  // FP64 states of lbm_surrogate_advance (now, next), allocated on first use
  double last_sums[4] = {0, 0, 0, 0};  // the check sums of the last lbm_fno_advance
  double cons = 0.0;                   // weight of the loss's conservation term
  double inflow = 0.0;                 // expected change of sum(alpha_g) over one call
  float norm_mean[6] = {0, 0, 0, 0, 0, 0}, norm_std[6] = {1, 1, 1, 1, 1, 1}, out_std[6] = {1, 1, 1, 1, 1, 1};
  cudaStream_t stream = 0;
  long long launches = 0;
  // the inference layers as a CUDA graph, captured at the first call (all
  // their buffers belong to the model) and replayed on the model's stream
  cudaGraphExec_t layers_exec = nullptr;
  long long layers_launches = 0;  // kernels in one replay
  bool layers_graph_off = false;  // capture failed: plain launches
  char err[512] = {0};
};

static int ferr(lbm_fno *f, int code, const char *fmt, ...) {
  if (f) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(f->err, sizeof f->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

#define FTRY(f, call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return ferr((f), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// After a synchronisation of the model's stream: a product whose pipeline
// stalled (an mbarrier wait in k_umma ran out; its results are not valid)
// is reported, and the flag cleared.
static int umma_status(lbm_fno *f) {
  int t = 0;
  FTRY(f, cudaMemcpyFromSymbol(&t, fno::umma_timeout, sizeof t));
  if (t) {
    const int zero = 0;
    FTRY(f, cudaMemcpyToSymbol(fno::umma_timeout, &zero, sizeof zero));
    return ferr(f, LBM_ECUDA, "tensor-core product: a pipeline wait ran out (results invalid)");
  }
  return LBM_OK;
}

// ------------------------------------------------------------------ GEMM

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], b < batch.  op(A) is M x K,
// op(B) is K x N.  Row-major storage: A is M x K (lda >= K), or K x M
// (lda >= M) when ta; B is K x N (ldb >= N), or N x K (ldb >= K) when tb;
// C is M x N (ldc >= N), float or bf16.  M, N, K multiples of 16, leading
// dimensions and batch strides multiples of 8, bases 32-byte aligned.
// ksplit > 1 splits K into chunks (multiples of 64) over blocks, each adding
// alpha times its partial product into a float C with atomics (C += alpha
// op(A) op(B); beta must be 1).
// With bias (float C, no split) the epilogue adds bias[b] (one value per
// batch entry) or, with bias_rows, bias[row].  With hout it stores act ?
// GELU(result) : result as bf16 at the same index of hout (the last product
// of a surrogate layer, the lifting); C may then be null (beta 0), and the
// float result is not stored; store_c = false keeps C as an input only.
// The second segment (A2, batch 1, no split) adds a second product to the
// same tile: C += A2_t B2_t over K2, where for output columns n (in rows of
// seg_nx columns, seg_nx a multiple of 128) A2_t = A2 + (n / seg_nx) a2_rs is
// K2 x M (lda2) and B2_t = B2 + (n % seg_nx) ldb2 is N x K2 (ldb2), both read
// transposed: the pointwise product of a layer fused with the reconstruction
// of its x spectrum, whose coefficients differ from row to row.
struct G {
  const bf16 *A, *B;
  void *C;
  int M, N, K, lda, ldb, ldc;
  long long sA = 0, sB = 0, sC = 0;
  int batch = 1;
  float alpha = 1.0f, beta = 0.0f;
  bool ta = false, tb = false, out_f32 = true;
  int ksplit = 1;  // > 1: K split over blocks, FP32 atomic accumulation (beta must be 1)
  const float *bias = nullptr;  // fused epilogue: + bias[batch] (bias[row] with bias_rows)
  bf16 *hout = nullptr;         // ... and (act ? GELU : identity) of the result as bf16; C may be null
  bool bias_rows = false, act = true, store_c = true;
  // second product of the same tile: pointwise + x reconstruction
  const bf16 *A2 = nullptr, *B2 = nullptr;
  int K2 = 0, lda2 = 0, ldb2 = 0, seg_nx = 0;
  long long a2_rs = 0;
};

// ---- tensor maps (cuTensorMapEncodeTiled, from the driver through the runtime's entry-point query)

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
  // looked up once (a function-local static: thread-safe initialisation)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

// One operand as a 3D tensor (contiguous dimension `inner`, `rows` at
// row_stride elements, `batch` at batch_stride elements), boxes of
// box0 x box1; *bat says where the kernel puts the batch index (UmmaArgs).
// A batch stride below the row stride is encoded with the outer dimensions
// swapped, so that the map's strides grow outward.
static cudaError_t operand_map(CUtensorMap *m, int *bat, const void *base, bool f32, long long inner, long long rows,
                               int batch, long long row_stride, long long batch_stride, int box0, int box1, bool swz) {
  EncodeTiledFn enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const long long es = f32 ? 4 : 2;
  cuuint64_t dims[3];
  cuuint64_t strides[2];
  cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1}, estr[3] = {1, 1, 1};
  if (batch <= 1 || batch_stride == 0) {
    *bat = 0;
    dims[0] = inner; dims[1] = rows; dims[2] = 1;
    strides[0] = row_stride * es; strides[1] = rows * row_stride * es;
  } else if (batch_stride >= row_stride) {
    *bat = 1;
    dims[0] = inner; dims[1] = rows; dims[2] = batch;
    strides[0] = row_stride * es; strides[1] = batch_stride * es;
  } else {
    *bat = 2;
    dims[0] = inner; dims[1] = batch; dims[2] = rows;
    strides[0] = batch_stride * es; strides[1] = row_stride * es;
    box[1] = 1; box[2] = (cuuint32_t)box1;
  }
  const CUresult r = enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                         const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// SMs of the current device
static int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n < 1)
    return 1;
  return n;
}

// Buffers of one launch: three accumulators (with their old-C and staging
// tiles) where shared memory allows, else two; a ring of two tiles' stages
// (2 to 6); outputs through TMA stores when their staging tiles fit, else
// stored directly.
template <int NT, class OutT, bool OLDC>
static int pick_smem(fno::UmmaArgs &a, int nk, bool want_c, bool want_h) {
  typedef fno::UmmaSmem<NT, OutT, OLDC> SM;
  const int limit = 227 * 1024;
  const int stages = 2 * nk < 2 ? 2 : (2 * nk > 6 ? 6 : 2 * nk);
  for (int st_out = 1; st_out >= 0; st_out--)
    for (a.nacc = fno::UMMA_MAX_ACC; a.nacc >= 2; a.nacc--) {
      a.st_c = st_out && want_c;
      a.st_h = st_out && want_h;
      for (a.stages = stages; a.stages >= 2; a.stages--) {
        const int b = SM::bytes(a.stages, a.nacc, a.st_c, a.st_h);
        if (b <= limit) {
          a.tmem_cols = 32;
          while (a.tmem_cols < a.nacc * NT) a.tmem_cols *= 2;
          return b;
        }
      }
    }
  return -1;
}

template <bool AK, bool BKM, int NT, class OutT, bool SEG2, bool OLDC>
static cudaError_t launch_umma(fno::UmmaArgs &a, int nk, bool want_c, bool want_h, cudaStream_t st) {
  auto kern = fno::k_umma<AK, BKM, NT, OutT, SEG2, OLDC>;
  const int smem = pick_smem<NT, OutT, OLDC>(a, nk, want_c, want_h);
  if (smem < 0) return cudaErrorInvalidValue;
  // the kernel's dynamic shared-memory limit, raised per device to the largest asked
  static std::atomic<int> raised[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  std::atomic<int> &lim = raised[dev & 63];
  if (smem > 48 * 1024 && smem > lim.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    lim.store(smem);
  }
  // persistent: as many blocks as fit on the GPU at once (and whose
  // accumulators fit the 512 columns of an SM's tensor memory)
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, fno::UMMA_THREADS, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  if (per_sm > 512 / a.tmem_cols) per_sm = 512 / a.tmem_cols;
  const long long cap = (long long)per_sm * num_sms();
  const int grid = (int)(a.tiles < cap ? a.tiles : cap);
  kern<<<grid, fno::UMMA_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool AK, bool BKM>
static cudaError_t launch_umma_nt(fno::UmmaArgs &a, int nt, bool f32, bool oldc, int nk, bool want_c, bool want_h,
                                  cudaStream_t st) {
  if (oldc) return launch_umma<AK, BKM, 64, float, false, true>(a, nk, want_c, want_h, st);
  if (f32) return nt == 64 ? launch_umma<AK, BKM, 64, float, false, false>(a, nk, want_c, want_h, st)
                           : launch_umma<AK, BKM, 128, float, false, false>(a, nk, want_c, want_h, st);
  return nt == 64 ? launch_umma<AK, BKM, 64, bf16, false, false>(a, nk, want_c, want_h, st)
                  : launch_umma<AK, BKM, 128, bf16, false, false>(a, nk, want_c, want_h, st);
}

static cudaError_t gemm(const G &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.M % 16 || g.N % 16 || g.K % 16 || g.lda % 8 || g.ldb % 8 || g.ldc % 8 || g.batch < 1 || g.sA % 8 ||
      g.sB % 8 || g.sC % 8)
    return cudaErrorInvalidValue;
  if ((g.bias || g.hout) && (!g.out_f32 || g.ksplit > 1 || ((uintptr_t)g.hout & 31))) return cudaErrorInvalidValue;
  if (!g.C && (!g.hout || g.beta != 0.0f)) return cudaErrorInvalidValue;
  if (!g.store_c && (!g.hout || !g.C)) return cudaErrorInvalidValue;
  if (g.A2 && (!g.B2 || g.ta || g.tb || !g.out_f32 || g.batch != 1 || g.ksplit > 1 || g.K2 < 16 || g.K2 % 16 ||
               g.lda2 % 8 || g.ldb2 % 8 || g.a2_rs % 8 || g.seg_nx < fno::UMMA_M || g.seg_nx % fno::UMMA_M ||
               g.N % g.seg_nx || g.lda2 < g.M || g.ldb2 < g.K2 || (((uintptr_t)g.A2 | (uintptr_t)g.B2) & 31)))
    return cudaErrorInvalidValue;
  if (((uintptr_t)g.A | (uintptr_t)g.B | (uintptr_t)g.C) & 31) return cudaErrorMisalignedAddress;
  if (g.ksplit > 1 && !g.out_f32) return cudaErrorInvalidValue;
  int ks = g.ksplit < 1 ? 1 : g.ksplit;
  int kchunk = ((g.K + ks - 1) / ks + fno::UMMA_BK - 1) / fno::UMMA_BK * fno::UMMA_BK;
  ks = (g.K + kchunk - 1) / kchunk;
  if ((long long)g.batch * ks > 65535) return cudaErrorInvalidValue;
  const bool oldc = g.out_f32 && g.beta != 0.0f && ks == 1;
  if (oldc && g.batch > 1 && g.sC == 0) return cudaErrorInvalidValue;
  const int nt = (oldc || g.M <= 64) ? 64 : 128;
  fno::UmmaArgs a;
  memset(&a, 0, sizeof a);
  cudaError_t e;
  // MMA A operand = op(B)^T: K-major when B is stored N x K (tb)
  if (g.tb) e = operand_map(&a.ma, &a.a_bat, g.B, false, g.K, g.N, g.batch, g.ldb, g.sB, 64, fno::UMMA_M, true);
  else e = operand_map(&a.ma, &a.a_bat, g.B, false, g.N, g.K, g.batch, g.ldb, g.sB, 64, 64, true);
  if (e != cudaSuccess) return e;
  // MMA B operand = op(A)^T: K-major when A is stored M x K (not ta)
  if (!g.ta) e = operand_map(&a.mb, &a.b_bat, g.A, false, g.K, g.M, g.batch, g.lda, g.sA, 64, nt, true);
  else e = operand_map(&a.mb, &a.b_bat, g.A, false, g.M, g.K, g.batch, g.lda, g.sA, 64, 64, true);
  if (e != cudaSuccess) return e;
  int unused;
  if (g.A2) {
    // second segment: B2 (seg_nx rows of K2, K-major) and the per-row tiles
    // A2 + y a2_rs (K2 x M, MN-major), y over the N / seg_nx lattice rows
    e = operand_map(&a.ma2, &unused, g.B2, false, g.K2, g.seg_nx, 1, g.ldb2, 0, 64, fno::UMMA_M, true);
    if (e != cudaSuccess) return e;
    if (g.a2_rs < (long long)g.K2 * g.lda2) return cudaErrorInvalidValue;
    e = operand_map(&a.mb2, &unused, g.A2, false, g.M, g.K2, g.N / g.seg_nx, g.lda2, g.a2_rs, 64, 64, true);
    if (e != cudaSuccess) return e;
  }
  // C's and hout's tiles (same layout): the old C tile is loaded through the
  // map of C, and the output tiles leave through them when staged
  const bool want_c = g.C && g.store_c && ks == 1, want_h = g.hout != nullptr;
  if (g.C && (oldc || want_c)) {
    e = operand_map(&a.mc, &a.c_bat, g.C, g.out_f32, g.N, g.M, g.batch, g.ldc, g.sC, fno::UMMA_M, nt, false);
    if (e != cudaSuccess) return e;
  }
  if (want_h) {
    e = operand_map(&a.mh, &a.c_bat, g.hout, false, g.N, g.M, g.batch, g.ldc, g.sC, fno::UMMA_M, nt, false);
    if (e != cudaSuccess) return e;
  }
  a.C = g.C; a.M = g.M; a.N = g.N; a.K = g.K; a.ldc = g.ldc; a.sC = g.sC;
  a.alpha = g.alpha; a.beta = g.beta; a.ksplit = ks; a.kchunk = kchunk;
  a.bias = g.bias; a.hout = g.hout; a.bias_rows = g.bias_rows ? 1 : 0; a.act = g.act ? 1 : 0;
  a.store_c = g.store_c ? 1 : 0; a.K2 = g.A2 ? g.K2 : 0; a.seg_nx = g.seg_nx;
  a.tiles_n = (g.N + fno::UMMA_M - 1) / fno::UMMA_M;
  a.tiles_m = (g.M + nt - 1) / nt;
  const long long tiles = (long long)a.tiles_n * a.tiles_m * g.batch * ks;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  a.tiles = (int)tiles;
  const int nk = (kchunk + fno::UMMA_BK - 1) / fno::UMMA_BK + (g.A2 ? (g.K2 + fno::UMMA_BK - 1) / fno::UMMA_BK : 0);
  if (g.A2) return launch_umma<false, true, 64, float, true, false>(a, nk, want_c, want_h, st);
  if (g.tb && !g.ta) return launch_umma_nt<true, true>(a, nt, g.out_f32, oldc, nk, want_c, want_h, st);
  if (g.tb && g.ta) return launch_umma_nt<true, false>(a, nt, g.out_f32, oldc, nk, want_c, want_h, st);
  if (!g.tb && !g.ta) return launch_umma_nt<false, true>(a, nt, g.out_f32, oldc, nk, want_c, want_h, st);
  return launch_umma_nt<false, false>(a, nt, g.out_f32, oldc, nk, want_c, want_h, st);
}

// ------------------------------------------------------------------ kernels of the state interface

// per-channel scales of the state interface
struct Norm {
  float mean[6], inv_in[6], std_out[6], inv_out[6];
};

// The state kernels run on grids (blocks over P, 6 state channels); the
// padding channels of x16 and of the target stay zero from creation on.

// x16[c][p] = (state[c][p] - mean[c]) / std_in[c]
__global__ void k_pack_state(const double *state, bf16 *x16, long long P, Norm nm) {
  const int c = blockIdx.y;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  x16[c * P + p] = __float2bfloat16((float)(state[c * P + p] - (double)nm.mean[c]) * nm.inv_in[c]);
}

// target increment in the model's units: t[c][p] = (next - now) / std_out[c]
__global__ void k_pack_target(const double *now, const double *next, float *t, long long P, Norm nm) {
  const int c = blockIdx.y;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const long long i = c * P + p;
  t[i] = (float)(next[i] - now[i]) * nm.inv_out[c];
}


// Inference ends of the model, each one pass over the nodes (two per thread)
// instead of a tensor-core product on mostly padded tiles.  Their numerics
// are the products': BF16 inputs and weights, FP32 sums, bias added last.

// h_0[c][p] = sum_j W_in[c][j] x_j[p] + b_in[c] from the FP64 state, with
// x_j the standardised state channel j rounded to BF16 (as k_pack_state)
// and only the 6 state columns of W_in (the padding inputs are zero)
__global__ void k_lift(const double *state, const bf16 *W16, int cin, const float *bias, bf16 *h, int C, long long P,
                       Norm nm) {
  extern __shared__ float sw[];  // [C][6] weights, then [C] biases
  for (int i = threadIdx.x; i < C * 6; i += blockDim.x) sw[i] = __bfloat162float(W16[(i / 6) * cin + i % 6]);
  for (int i = threadIdx.x; i < C; i += blockDim.x) sw[C * 6 + i] = bias[i];
  __syncthreads();
  const long long p = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= P) return;
  float x0[6], x1[6];
#pragma unroll
  for (int j = 0; j < 6; j++) {
    const double m = (double)nm.mean[j];
    x0[j] = __bfloat162float(__float2bfloat16((float)(state[j * P + p] - m) * nm.inv_in[j]));
    x1[j] = __bfloat162float(__float2bfloat16((float)(state[j * P + p + 1] - m) * nm.inv_in[j]));
  }
  for (int c = 0; c < C; c++) {
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      a0 = fmaf(sw[c * 6 + j], x0[j], a0);
      a1 = fmaf(sw[c * 6 + j], x1[j], a1);
    }
    const float b = sw[C * 6 + c];
    *reinterpret_cast<__nv_bfloat162 *>(h + c * P + p) = __floats2bfloat162_rn(a0 + b, a1 + b);
  }
}

// next[c][p] = now[c][p] + std_out[c] (sum_k W_out[c][k] h_L[k][p] + b_out[c])
// for the 6 state channels (the padding outputs are not needed)
__global__ void k_project_out(const bf16 *hL, const bf16 *W16, const float *bias, const double *now, double *next,
                              int C, long long P, Norm nm) {
  extern __shared__ float sw[];  // [6][C] weights, then [6] biases
  for (int i = threadIdx.x; i < 6 * C; i += blockDim.x) sw[i] = __bfloat162float(W16[i]);
  if (threadIdx.x < 6) sw[6 * C + threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const long long p = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= P) return;
  float a0[6], a1[6];
#pragma unroll
  for (int c = 0; c < 6; c++) a0[c] = a1[c] = 0.0f;
  for (int k = 0; k < C; k++) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(hL + k * P + p));
#pragma unroll
    for (int c = 0; c < 6; c++) {
      a0[c] = fmaf(sw[c * C + k], v.x, a0[c]);
      a1[c] = fmaf(sw[c * C + k], v.y, a1[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 6; c++) {
    const double s = (double)nm.std_out[c];
    const float b = sw[6 * C + c];
    next[c * P + p] = now[c * P + p] + s * (double)(a0[c] + b);
    next[c * P + p + 1] = now[c * P + p + 1] + s * (double)(a1[c] + b);
  }
}

// FP64 sums for the checks of a call, block partials in
// part[y * gridDim.x + x]: alpha_g before (blockIdx.y = 0) and after (1) the
// call, all six channels after it (2; finite only if every value is), and
// the number of new alpha_g values outside [0, 1] (3)
__global__ void k_checks(const double *a0, const double *a1, long long n, double *part) {
  __shared__ double s[8];
  const double *a = blockIdx.y == 0 ? a0 : a1;
  const long long m = blockIdx.y == 2 ? 6 * n : n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const double v = a[i];
    acc += blockIdx.y == 3 ? (v >= 0.0 && v <= 1.0 ? 0.0 : 1.0) : v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s[w];
    part[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------ model pieces

static int refresh_weights(lbm_fno *f) {
  const int C = f->C, K = f->K, L = f->L;
  cudaStream_t st = f->stream;
  fno::k_to_bf16<<<nblk((long long)C * f->cin), 256, 0, st>>>(f->p + f->off.W_in, f->W_in16, (long long)C * f->cin);
  fno::k_to_bf16<<<nblk((long long)f->cout * C), 256, 0, st>>>(f->p + f->off.W_out, f->W_out16, (long long)f->cout * C);
  f->launches += 2;
  for (int l = 0; l < L; l++) {
    fno::k_to_bf16<<<nblk((long long)C * C), 256, 0, st>>>(f->p + f->off.W[l], f->W16 + (long long)l * C * C,
                                                          (long long)C * C);
    const long long wf = (long long)K * 4 * C * C;
    fno::k_assemble_complex<<<nblk(wf), 256, 0, st>>>(f->p + f->off.Ax[l], f->p + f->off.Bx[l], f->Wfx16 + l * wf, C, K);
    fno::k_assemble_complex<<<nblk(wf), 256, 0, st>>>(f->p + f->off.Ay[l], f->p + f->off.By[l], f->Wfy16 + l * wf, C, K);
    f->launches += 3;
  }
  FTRY(f, cudaGetLastError());
  return LBM_OK;
}

#define GTRY(f, gg)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = gemm((gg), (f)->stream);                                            \
    (f)->launches++;                                                                     \
    if (e_ != cudaSuccess) return ferr((f), LBM_ECUDA, "gemm %s (line %d): %s", #gg, __LINE__, cudaGetErrorString(e_)); \
  } while (0)

// z = W_l h + S^x(h): h is C x (ny x nx) bf16, z is C x (ny x nx) float.
// The mixed x coefficients are laid out [ny][2K][C], so that for one row y
// they form the (2K x C) left factor of that row's reconstruction; when nx is
// a multiple of the 64-column tile the pointwise product and the
// reconstruction run as one two-segment product and z is written once.
static int pointwise_and_spec_x(lbm_fno *f, const bf16 *W, const bf16 *h, bf16 *Hx, const bf16 *Wf, float *z) {
  const int C = f->C, K2 = 2 * f->K, nx = f->nx, ny = f->ny;
  const long long P = f->P;
  G a;  // Hx (2K x C ny) = B_x^T h^T
  a.A = f->Bx; a.ta = true; a.lda = K2;
  a.B = h; a.tb = true; a.ldb = nx;
  a.C = Hx; a.out_f32 = false; a.ldc = C * ny;
  a.M = K2; a.N = C * ny; a.K = nx;
  GTRY(f, a);
  G b;  // per mode k: O[:, k, :] (ny x 2C) = H_k^T Wf_k^T
  b.A = Hx; b.ta = true; b.lda = ny; b.sA = 2LL * C * ny;
  b.B = Wf; b.tb = true; b.ldb = 2 * C; b.sB = 4LL * C * C;
  b.C = f->O16; b.out_f32 = false; b.ldc = K2 * C; b.sC = 2LL * C;
  b.M = ny; b.N = 2 * C; b.K = 2 * C; b.batch = f->K;
  GTRY(f, b);
  G w;  // z = W h (C x P)
  w.A = W; w.lda = C; w.B = h; w.ldb = (int)P; w.C = z; w.ldc = (int)P;
  w.M = C; w.N = (int)P; w.K = C;
  if (nx % fno::UMMA_M == 0) {
    // ... + for the tile of row y: O[y]^T (C x 2K) B_xi^T (2K x columns)
    w.A2 = f->O16; w.lda2 = C; w.a2_rs = (long long)K2 * C;
    w.B2 = f->Bxi; w.ldb2 = K2; w.K2 = K2; w.seg_nx = nx;
    GTRY(f, w);
    return LBM_OK;
  }
  GTRY(f, w);
  G c;  // per row y: z[:, y, :] (C x nx) += O[y]^T B_xi^T
  c.A = f->O16; c.ta = true; c.lda = C; c.sA = (long long)K2 * C;
  c.B = f->Bxi; c.tb = true; c.ldb = K2;
  c.C = z; c.ldc = (int)P; c.sC = nx; c.beta = 1.0f;
  c.M = C; c.N = nx; c.K = K2; c.batch = ny;
  GTRY(f, c);
  return LBM_OK;
}

// out[:, c, :] (2K x nx, layout [2K][C][nx], bf16) = basis^T x[c] for every
// channel: a contraction over the ny nodes of a column, split over blocks
// into the FP32 scratch (few output tiles, long K) and rounded once.
static int project_y(lbm_fno *f, const bf16 *basis, const bf16 *x, bf16 *out) {
  const int C = f->C, K2 = 2 * f->K, nx = f->nx, ny = f->ny;
  const long long n = (long long)K2 * C * nx;
  FTRY(f, cudaMemsetAsync(f->coef32, 0, n * sizeof(float), f->stream));
  G a;
  a.A = basis; a.ta = true; a.lda = K2;
  a.B = x; a.ldb = nx; a.sB = f->P;
  a.C = f->coef32; a.ldc = C * nx; a.sC = nx; a.beta = 1.0f;
  a.M = K2; a.N = nx; a.K = ny; a.batch = C;
  a.ksplit = ny >= 512 ? ny / 256 : 1;
  GTRY(f, a);
  fno::k_to_bf16<<<nblk(n), 256, 0, f->stream>>>(f->coef32, out, n);
  f->launches++;
  return LBM_OK;
}

// z += S^y(h); Hy is [2K][C][nx].  The last product of the layer: it also adds
// the bias and writes GELU(z) into hnext (fused epilogue).
static int spec_y(lbm_fno *f, const bf16 *h, bf16 *Hy, const bf16 *Wf, float *z, const float *bias, bf16 *hnext,
                  bool keep_z) {
  const int C = f->C, K2 = 2 * f->K, nx = f->nx, ny = f->ny;
  const long long P = f->P;
  int rc = project_y(f, f->By, h, Hy);  // Hy[:, c, :] (2K x nx) = B_y^T h[c]
  if (rc) return rc;
  G b;  // per mode: O_k (2C x nx) = Wf_k H_k, rows (j C + c)
  b.A = Wf; b.lda = 2 * C; b.sA = 4LL * C * C;
  b.B = Hy; b.ldb = nx; b.sB = 2LL * C * nx;
  b.C = f->O16; b.out_f32 = false; b.ldc = nx; b.sC = 2LL * C * nx;
  b.M = 2 * C; b.N = nx; b.K = 2 * C; b.batch = f->K;
  GTRY(f, b);
  G c;  // per channel: z[c] (ny x nx) += Byi O[:, c, :]
  c.A = f->Byi; c.lda = K2;
  c.B = f->O16; c.ldb = C * nx; c.sB = nx;
  c.C = z; c.ldc = nx; c.sC = P; c.beta = 1.0f;
  c.M = ny; c.N = nx; c.K = K2; c.batch = C;
  c.bias = bias; c.hout = hnext; c.store_c = keep_z;
  GTRY(f, c);
  return LBM_OK;
}

// the L layers, from h_0 to h_L; keeps Hx_l, Hy_l, and the pre-activations
// z_l when `train` (the backward pass needs GELU'(z_l))
static int layers(lbm_fno *f, bool train) {
  const int C = f->C, L = f->L;
  const long long P = f->P, CP = (long long)C * P;
  const long long hx = 2LL * f->K * C * f->ny, hy = 2LL * f->K * C * f->nx, wf = (long long)f->K * 4 * C * C;
  for (int l = 0; l < L; l++) {
    const bf16 *h = f->h16 + l * CP;
    float *z = f->z + l * CP;
    int rc = pointwise_and_spec_x(f, f->W16 + (long long)l * C * C, h, f->Hx16 + l * hx, f->Wfx16 + l * wf, z);
    if (rc) return rc;
    rc = spec_y(f, h, f->Hy16 + l * hy, f->Wfy16 + l * wf, z, f->p + f->off.b[l], f->h16 + (l + 1) * CP, train);
    if (rc) return rc;
  }
  return LBM_OK;
}

// training forward from f->x16 to f->y (cout x P float): lifting product,
// layers, output product
static int forward_train(lbm_fno *f) {
  const int C = f->C, L = f->L;
  const long long P = f->P, CP = (long long)C * P;
  G a;  // lifting: h_0 = W_in x + b_in, stored as bf16 only
  a.A = f->W_in16; a.lda = f->cin; a.B = f->x16; a.ldb = (int)P; a.C = nullptr; a.ldc = (int)P;
  a.M = C; a.N = (int)P; a.K = f->cin;
  a.bias = f->p + f->off.b_in; a.bias_rows = true; a.act = false; a.hout = f->h16;
  GTRY(f, a);
  int rc = layers(f, true);
  if (rc) return rc;
  G o;  // y = W_out h_L + b_out
  o.A = f->W_out16; o.lda = C; o.B = f->h16 + L * CP; o.ldb = (int)P; o.C = f->y; o.ldc = (int)P;
  o.M = f->cout; o.N = (int)P; o.K = C;
  o.bias = f->p + f->off.b_out; o.bias_rows = true;
  GTRY(f, o);
  FTRY(f, cudaGetLastError());
  return LBM_OK;
}

// dh_prev += (S^x)^T dz; gradients of A_x, B_x into the parameter gradient
static int spec_x_back(lbm_fno *f, const bf16 *dz16, const bf16 *Hx, const bf16 *Wf, float *dh, float *gA,
                       float *gB) {
  const int C = f->C, K2 = 2 * f->K, nx = f->nx, ny = f->ny;
  G a;  // dO (2K x C ny) = Bxi^T dz^T
  a.A = f->Bxi; a.ta = true; a.lda = K2;
  a.B = dz16; a.tb = true; a.ldb = nx;
  a.C = f->dO16; a.out_f32 = false; a.ldc = C * ny;
  a.M = K2; a.N = C * ny; a.K = nx;
  GTRY(f, a);
  G w;  // dWf_k (2C x 2C) = dO_k H_k^T
  w.A = f->dO16; w.lda = ny; w.sA = 2LL * C * ny;
  w.B = Hx; w.tb = true; w.ldb = ny; w.sB = 2LL * C * ny;
  w.C = f->dWf; w.ldc = 2 * C; w.sC = 4LL * C * C;
  w.M = 2 * C; w.N = 2 * C; w.K = ny; w.batch = f->K;
  GTRY(f, w);
  fno::k_fold_complex<<<nblk((long long)f->K * C * C), 256, 0, f->stream>>>(f->dWf, gA, gB, C, f->K);
  f->launches++;
  G b;  // dH_k = Wf_k^T dO_k
  b.A = Wf; b.ta = true; b.lda = 2 * C; b.sA = 4LL * C * C;
  b.B = f->dO16; b.ldb = ny; b.sB = 2LL * C * ny;
  b.C = f->dH16; b.out_f32 = false; b.ldc = ny; b.sC = 2LL * C * ny;
  b.M = 2 * C; b.N = ny; b.K = 2 * C; b.batch = f->K;
  GTRY(f, b);
  G c;  // dh (C ny x nx) += dH^T B_x^T
  c.A = f->dH16; c.ta = true; c.lda = C * ny;
  c.B = f->Bx; c.tb = true; c.ldb = K2;
  c.C = dh; c.ldc = nx; c.beta = 1.0f;
  c.M = C * ny; c.N = nx; c.K = K2;
  GTRY(f, c);
  return LBM_OK;
}

static int spec_y_back(lbm_fno *f, const bf16 *dz16, const bf16 *Hy, const bf16 *Wf, float *dh, float *gA,
                       float *gB) {
  const int C = f->C, K2 = 2 * f->K, nx = f->nx, ny = f->ny;
  const long long P = f->P;
  int rc = project_y(f, f->Byi, dz16, f->dO16);  // dO[:, c, :] = Byi^T dz[c]
  if (rc) return rc;
  G w;  // dWf_k = dO_k H_k^T
  w.A = f->dO16; w.lda = nx; w.sA = 2LL * C * nx;
  w.B = Hy; w.tb = true; w.ldb = nx; w.sB = 2LL * C * nx;
  w.C = f->dWf; w.ldc = 2 * C; w.sC = 4LL * C * C;
  w.M = 2 * C; w.N = 2 * C; w.K = nx; w.batch = f->K;
  GTRY(f, w);
  fno::k_fold_complex<<<nblk((long long)f->K * C * C), 256, 0, f->stream>>>(f->dWf, gA, gB, C, f->K);
  f->launches++;
  G b;  // dH_k = Wf_k^T dO_k
  b.A = Wf; b.ta = true; b.lda = 2 * C; b.sA = 4LL * C * C;
  b.B = f->dO16; b.ldb = nx; b.sB = 2LL * C * nx;
  b.C = f->dH16; b.out_f32 = false; b.ldc = nx; b.sC = 2LL * C * nx;
  b.M = 2 * C; b.N = nx; b.K = 2 * C; b.batch = f->K;
  GTRY(f, b);
  G c;  // per channel: dh[c] += B_y dH[:, c, :]
  c.A = f->By; c.lda = K2;
  c.B = f->dH16; c.ldb = C * nx; c.sB = nx;
  c.C = dh; c.ldc = nx; c.sC = P; c.beta = 1.0f;
  c.M = ny; c.N = nx; c.K = K2; c.batch = C;
  GTRY(f, c);
  return LBM_OK;
}

// split of the long contractions over pixels (weight gradients)
static int ksplit_for(long long K) {
  const long long chunk = 512;
  long long s = (K + chunk - 1) / chunk;
  return (int)(s < 1 ? 1 : (s > 512 ? 512 : s));
}

// loss of f->y against f->tgt; gradients accumulated into f->g
static int backward(lbm_fno *f, double *loss) {
  const int C = f->C, L = f->L;
  const long long P = f->P, CP = (long long)C * P;
  const long long hx = 2LL * f->K * C * f->ny, hy = 2LL * f->K * C * f->nx, wf = (long long)f->K * 4 * C * C;
  const unsigned nb = nblk(P) * f->cv, nb0 = nblk(P);
  fno::k_mse<<<dim3(nb0, f->cv), 256, 0, f->stream>>>(f->y, f->tgt, f->dy, f->dy16, P,
                                                      (float)(2.0 / ((double)f->cv * P)), f->part);
  f->launches++;
  if (f->cons > 0.0) {
    fno::k_cons_grad<<<nb0, 256, 0, f->stream>>>(f->part + nb, (int)nb0, f->dy, f->dy16, P, f->cons);
    f->launches++;
  }
  FTRY(f, cudaMemcpyAsync(f->h_part, f->part, (nb + nb0) * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  G go;  // dW_out += dy h_L^T
  go.A = f->dy16; go.lda = (int)P; go.B = f->h16 + L * CP; go.tb = true; go.ldb = (int)P;
  go.C = f->g + f->off.W_out; go.ldc = C; go.beta = 1.0f; go.ksplit = ksplit_for(P);
  go.M = f->cout; go.N = C; go.K = (int)P;
  GTRY(f, go);
  fno::k_bias_grad<<<dim3(64, f->cout), 256, 0, f->stream>>>(f->dy, f->g + f->off.b_out, P);
  f->launches++;
  G gh;  // dh = W_out^T dy
  gh.A = f->W_out16; gh.ta = true; gh.lda = C; gh.B = f->dy16; gh.ldb = (int)P; gh.C = f->dh; gh.ldc = (int)P;
  gh.M = C; gh.N = (int)P; gh.K = f->cout;
  GTRY(f, gh);
  for (int l = L - 1; l >= 0; l--) {
    fno::k_act_back<<<nblk(CP), 256, 0, f->stream>>>(f->dh, f->z + l * CP, f->dz, f->dz16, CP, 1);
    fno::k_bias_grad<<<dim3(64, C), 256, 0, f->stream>>>(f->dz, f->g + f->off.b[l], P);
    f->launches += 2;
    const bf16 *h = f->h16 + l * CP;
    G gw;  // dW_l += dz h^T
    gw.A = f->dz16; gw.lda = (int)P; gw.B = h; gw.tb = true; gw.ldb = (int)P;
    gw.C = f->g + f->off.W[l]; gw.ldc = C; gw.beta = 1.0f; gw.ksplit = ksplit_for(P);
    gw.M = C; gw.N = C; gw.K = (int)P;
    GTRY(f, gw);
    G gd;  // dh = W_l^T dz (the previous dh is consumed)
    gd.A = f->W16 + (long long)l * C * C; gd.ta = true; gd.lda = C; gd.B = f->dz16; gd.ldb = (int)P;
    gd.C = f->dh; gd.ldc = (int)P; gd.M = C; gd.N = (int)P; gd.K = C;
    GTRY(f, gd);
    int rc = spec_x_back(f, f->dz16, f->Hx16 + l * hx, f->Wfx16 + l * wf, f->dh, f->g + f->off.Ax[l],
                         f->g + f->off.Bx[l]);
    if (rc) return rc;
    rc = spec_y_back(f, f->dz16, f->Hy16 + l * hy, f->Wfy16 + l * wf, f->dh, f->g + f->off.Ay[l],
                     f->g + f->off.By[l]);
    if (rc) return rc;
  }
  // lifting (no activation)
  fno::k_act_back<<<nblk(CP), 256, 0, f->stream>>>(f->dh, nullptr, f->dz, f->dz16, CP, 0);
  fno::k_bias_grad<<<dim3(64, C), 256, 0, f->stream>>>(f->dz, f->g + f->off.b_in, P);
  f->launches += 2;
  G gi;  // dW_in += dz x^T
  gi.A = f->dz16; gi.lda = (int)P; gi.B = f->x16; gi.tb = true; gi.ldb = (int)P;
  gi.C = f->g + f->off.W_in; gi.ldc = f->cin; gi.beta = 1.0f; gi.ksplit = ksplit_for(P);
  gi.M = C; gi.N = f->cin; gi.K = (int)P;
  GTRY(f, gi);
  FTRY(f, cudaStreamSynchronize(f->stream));
  if (int rc = umma_status(f)) return rc;
  double s = 0.0;
  for (unsigned i = 0; i < nb; i++) s += f->h_part[i];
  double e0 = 0.0;
  for (unsigned i = 0; i < nb0; i++) e0 += f->h_part[nb + i];
  const double mean_e0 = e0 / (double)P;
  if (loss) *loss = s / ((double)f->cv * P) + f->cons * mean_e0 * mean_e0;
  FTRY(f, cudaGetLastError());
  return LBM_OK;
}

// ------------------------------------------------------------------ set-up

// Truncated real-DFT bases of an axis of n points and K modes, columns
// (cos 0, sin 0, cos 1, sin 1, ...): forward b[x][2k+j], inverse scaled so
// that a signal with modes < K is reproduced (1/n for k = 0, 2/n otherwise).
static void basis(int n, int K, std::vector<float> &fw, std::vector<float> &inv) {
  fw.assign((size_t)n * 2 * K, 0.0f);
  inv.assign((size_t)n * 2 * K, 0.0f);
  const double two_pi = 6.283185307179586476925286766559;
  for (int x = 0; x < n; x++)
    for (int k = 0; k < K; k++) {
      const double ph = two_pi * (double)k * (double)x / (double)n;
      const double c = cos(ph), s = sin(ph), sc = (k == 0 ? 1.0 : 2.0) / (double)n;
      fw[(size_t)x * 2 * K + 2 * k] = (float)c;
      fw[(size_t)x * 2 * K + 2 * k + 1] = (float)s;
      inv[(size_t)x * 2 * K + 2 * k] = (float)(c * sc);
      inv[(size_t)x * 2 * K + 2 * k + 1] = (float)(s * sc);
    }
}

static int upload_bf16(lbm_fno *f, const std::vector<float> &h, bf16 *dst) {
  float *tmp = nullptr;
  FTRY(f, cudaMalloc((void **)&tmp, h.size() * sizeof(float)));
  cudaError_t e = cudaMemcpy(tmp, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fno::k_to_bf16<<<nblk((long long)h.size()), 256>>>(tmp, dst, (long long)h.size());
    e = cudaDeviceSynchronize();
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return ferr(f, LBM_ECUDA, "upload: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" {

int lbm_fno_destroy(lbm_fno *f) {
  if (!f) return LBM_OK;
  cudaStreamSynchronize(f->stream);
  void *bufs[] = {f->p, f->g, f->m, f->v, f->W_in16, f->W_out16, f->W16, f->Wfx16, f->Wfy16, f->Bx, f->Bxi, f->By,
                  f->Byi, f->x16, f->h16, f->Hx16, f->Hy16, f->O16, f->z, f->y, f->tgt, f->dy, f->dh,
                  f->dz, f->dWf, f->dy16, f->dz16, f->dO16, f->dH16, f->part, f->red, f->coef32, f->st};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (f->h_part) cudaFreeHost(f->h_part);
  if (f->h_red) cudaFreeHost(f->h_red);
  if (f->layers_exec) cudaGraphExecDestroy(f->layers_exec);
  delete f;
  return LBM_OK;
}

int lbm_fno_create(int nx, int ny, int channels, int modes, int layers, lbm_fno **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (nx < 16 || ny < 16 || nx % 16 || ny % 16 || channels < 16 || channels % 16 || modes < 8 || modes % 8 ||
      2 * modes > nx || 2 * modes > ny || layers < 1 || layers > 16 || (long long)nx * ny >= (1LL << 31) / 64)
    return LBM_EINVAL;
  lbm_fno *f = new (std::nothrow) lbm_fno();
  if (!f) return LBM_ENOMEM;
  f->nx = nx; f->ny = ny; f->C = channels; f->K = modes; f->L = layers;
  f->P = (long long)nx * ny;
  f->off = layout(channels, modes, layers, f->cin, f->cout);
  const long long P = f->P, C = channels, CP = C * P, K2 = 2LL * modes;
  const long long hmax = K2 * C * (nx > ny ? nx : ny), wf = (long long)modes * 4 * C * C;
  const long long np = f->off.total;
  struct A { void **p; long long bytes; } al[] = {
      {(void **)&f->p, np * 4}, {(void **)&f->g, np * 4}, {(void **)&f->m, np * 4}, {(void **)&f->v, np * 4},
      {(void **)&f->W_in16, C * f->cin * 2}, {(void **)&f->W_out16, f->cout * C * 2},
      {(void **)&f->W16, layers * C * C * 2}, {(void **)&f->Wfx16, layers * wf * 2},
      {(void **)&f->Wfy16, layers * wf * 2}, {(void **)&f->Bx, nx * K2 * 2},
      {(void **)&f->Bxi, nx * K2 * 2}, {(void **)&f->By, ny * K2 * 2},
      {(void **)&f->Byi, ny * K2 * 2}, {(void **)&f->x16, f->cin * P * 2},
      {(void **)&f->h16, (layers + 1) * CP * 2}, {(void **)&f->Hx16, layers * K2 * C * ny * 2},
      {(void **)&f->Hy16, layers * K2 * C * nx * 2}, {(void **)&f->O16, hmax * 2},
      {(void **)&f->z, layers * CP * 4}, {(void **)&f->y, f->cout * P * 4},
      {(void **)&f->tgt, f->cout * P * 4}, {(void **)&f->dy, f->cout * P * 4},
      {(void **)&f->dh, CP * 4}, {(void **)&f->dz, CP * 4}, {(void **)&f->dWf, wf * 4},
      {(void **)&f->dy16, f->cout * P * 2}, {(void **)&f->dz16, CP * 2},
      {(void **)&f->dO16, hmax * 2}, {(void **)&f->dH16, hmax * 2},
      {(void **)&f->part, (long long)nblk((long long)f->cout * P) * 8}, {(void **)&f->red, 4 * 640 * 8},
      {(void **)&f->coef32, K2 * C * nx * 4}};
  for (auto &a : al) {
    if (cudaMalloc(a.p, (size_t)a.bytes) != cudaSuccess) {
      cudaGetLastError();
      lbm_fno_destroy(f);
      return LBM_ENOMEM;
    }
  }
  if (cudaMallocHost((void **)&f->h_part, (size_t)nblk((long long)f->cout * P) * 8) != cudaSuccess ||
      cudaMallocHost((void **)&f->h_red, 4 * 640 * 8) != cudaSuccess) {
    cudaGetLastError();
    lbm_fno_destroy(f);
    return LBM_ENOMEM;
  }
  cudaMemset(f->p, 0, np * 4);
  cudaMemset(f->g, 0, np * 4);
  cudaMemset(f->m, 0, np * 4);
  cudaMemset(f->v, 0, np * 4);
  // padding channels of the input, target and output gradient stay zero
  cudaMemset(f->x16, 0, f->cin * P * 2);
  cudaMemset(f->tgt, 0, f->cout * P * 4);
  cudaMemset(f->dy, 0, f->cout * P * 4);
  cudaMemset(f->dy16, 0, f->cout * P * 2);
  std::vector<float> fw, inv;
  basis(nx, modes, fw, inv);
  int rc = upload_bf16(f, fw, f->Bx);
  if (!rc) rc = upload_bf16(f, inv, f->Bxi);
  if (!rc) {
    basis(ny, modes, fw, inv);
    rc = upload_bf16(f, fw, f->By);
  }
  if (!rc) rc = upload_bf16(f, inv, f->Byi);
  if (!rc) rc = refresh_weights(f);
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = LBM_ECUDA;
  if (rc) {
    lbm_fno_destroy(f);
    return rc;
  }
  *out = f;
  return LBM_OK;
}

int lbm_fno_num_params(const lbm_fno *f, long long *n) {
  if (!f || !n) return LBM_EINVAL;
  *n = f->off.total;
  return LBM_OK;
}

int lbm_fno_set_stream(lbm_fno *f, void *stream) {
  if (!f) return LBM_EINVAL;
  f->stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_fno_set_params(lbm_fno *f, const float *host, long long n) {
  if (!f || !host || n != f->off.total) return LBM_EINVAL;
  FTRY(f, cudaMemcpyAsync(f->p, host, n * 4, cudaMemcpyHostToDevice, f->stream));
  int rc = refresh_weights(f);
  if (rc) return rc;
  FTRY(f, cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

int lbm_fno_get_params(const lbm_fno *f, float *host, long long n) {
  if (!f || !host || n != f->off.total) return LBM_EINVAL;
  if (cudaMemcpyAsync(host, f->p, n * 4, cudaMemcpyDeviceToHost, f->stream) != cudaSuccess ||
      cudaStreamSynchronize(f->stream) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}

int lbm_fno_get_grads(const lbm_fno *f, float *host, long long n) {
  if (!f || !host || n != f->off.total) return LBM_EINVAL;
  if (cudaMemcpyAsync(host, f->g, n * 4, cudaMemcpyDeviceToHost, f->stream) != cudaSuccess ||
      cudaStreamSynchronize(f->stream) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}

int lbm_fno_zero_grads(lbm_fno *f) {
  if (!f) return LBM_EINVAL;
  FTRY(f, cudaMemsetAsync(f->g, 0, f->off.total * 4, f->stream));
  return LBM_OK;
}

int lbm_fno_set_norm(lbm_fno *f, const float mean[6], const float std_in[6], const float std_out[6]) {
  if (!f || !mean || !std_in || !std_out) return LBM_EINVAL;
  for (int c = 0; c < 6; c++) {
    if (!(std_in[c] > 0.0f) || !(std_out[c] > 0.0f)) return ferr(f, LBM_EINVAL, "non-positive scale");
    f->norm_mean[c] = mean[c];
    f->norm_std[c] = std_in[c];
    f->out_std[c] = std_out[c];
  }
  return LBM_OK;
}

static Norm norm_of(const lbm_fno *f) {
  Norm nm;
  for (int c = 0; c < 6; c++) {
    nm.mean[c] = f->norm_mean[c];
    nm.inv_in[c] = 1.0f / f->norm_std[c];
    nm.std_out[c] = f->out_std[c];
    nm.inv_out[c] = 1.0f / f->out_std[c];
  }
  return nm;
}

int lbm_fno_set_inflow(lbm_fno *f, double dV) {
  if (!f || !isfinite(dV)) return LBM_EINVAL;
  f->inflow = dV;
  return LBM_OK;
}

int lbm_fno_set_loss(lbm_fno *f, double cons_weight) {
  if (!f || !(cons_weight >= 0.0) || !isfinite(cons_weight)) return LBM_EINVAL;
  f->cons = cons_weight;
  return LBM_OK;
}

int lbm_fno_accumulate(lbm_fno *f, const double *now, const double *next, double *loss) {
  if (!f || !now || !next) return LBM_EINVAL;
  const long long P = f->P;
  const Norm nm = norm_of(f);
  k_pack_state<<<dim3(nblk(P), 6), 256, 0, f->stream>>>(now, f->x16, P, nm);
  k_pack_target<<<dim3(nblk(P), 6), 256, 0, f->stream>>>(now, next, f->tgt, P, nm);
  f->launches += 2;
  int rc = forward_train(f);
  if (rc) return rc;
  return backward(f, loss);
}

int lbm_fno_adam(lbm_fno *f, float lr, float beta1, float beta2, float eps, float grad_scale) {
  if (!f || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return LBM_EINVAL;
  f->adam_t++;
  const double t = (double)f->adam_t;
  const float lr_t = (float)(lr * sqrt(1.0 - pow((double)beta2, t)) / (1.0 - pow((double)beta1, t)));
  fno::k_adam<<<nblk(f->off.total), 256, 0, f->stream>>>(f->p, f->g, f->m, f->v, f->off.total, lr_t, beta1, beta2, eps,
                                                         grad_scale);
  f->launches++;
  FTRY(f, cudaGetLastError());
  FTRY(f, cudaMemsetAsync(f->g, 0, f->off.total * 4, f->stream));
  return refresh_weights(f);
}

// The four sums of k_checks (fixed-order reductions) with one
// synchronisation: s[0] = sum alpha_g of now, s[1] of next, s[2] = sum of
// every value of next, s[3] = number of new alpha_g outside [0, 1]
static int check_sums(lbm_fno *f, const double *now, const double *next, double s[4]) {
  const int blocks = 640;
  k_checks<<<dim3(blocks, 4), 256, 0, f->stream>>>(now, next, f->P, f->red);
  f->launches++;
  FTRY(f, cudaMemcpyAsync(f->h_red, f->red, 4 * blocks * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  FTRY(f, cudaStreamSynchronize(f->stream));
  if (int rc = umma_status(f)) return rc;
  for (int k = 0; k < 4; k++) {
    double t = 0.0;
    for (int i = 0; i < blocks; i++) t += f->h_red[k * blocks + i];
    s[k] = t;
  }
  return LBM_OK;
}

// The inference layers: replayed from a graph captured on a stream of the
// model's own (the legacy default stream cannot be captured), else launched.
static int run_layers_inference(lbm_fno *f) {
  if (!f->layers_exec && !f->layers_graph_off) {
    cudaStream_t user = f->stream, cap = nullptr;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
      // the capture must not start before earlier work on the user's stream
      cudaEvent_t ev = nullptr;
      ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventRecord(ev, user) == cudaSuccess && cudaStreamWaitEvent(cap, ev, 0) == cudaSuccess;
      if (ev) cudaEventDestroy(ev);
    }
    const long long l0 = f->launches;
    if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = LBM_OK;
    if (ok) {
      f->stream = cap;
      rc = layers(f, false);
      f->stream = user;
      ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess && rc == LBM_OK;
    }
    if (ok) ok = cudaGraphInstantiate(&f->layers_exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    f->layers_launches = f->launches - l0;
    f->launches = l0;
    if (!ok) {
      cudaGetLastError();
      if (f->layers_exec) cudaGraphExecDestroy(f->layers_exec);
      f->layers_exec = nullptr;
      f->layers_graph_off = true;
      f->err[0] = 0;
    }
  }
  if (f->layers_exec) {
    FTRY(f, cudaGraphLaunch(f->layers_exec, f->stream));
    f->launches += f->layers_launches;
    return LBM_OK;
  }
  return layers(f, false);
}

int lbm_fno_advance(lbm_fno *f, const double *now, double *next, double max_drift, double *drift, int *ok) {
  if (!f || !now || !next || now == next) return LBM_EINVAL;
  const long long P = f->P;
  const Norm nm = norm_of(f);
  const int C = f->C;
  k_lift<<<nblk(P / 2), 256, (size_t)C * 7 * sizeof(float), f->stream>>>(now, f->W_in16, f->cin,
                                                                         f->p + f->off.b_in, f->h16, C, P, nm);
  f->launches++;
  int rc = run_layers_inference(f);
  if (rc) return rc;
  k_project_out<<<nblk(P / 2), 256, (size_t)(6 * C + 6) * sizeof(float), f->stream>>>(
      f->h16 + (long long)f->L * C * P, f->W_out16, f->p + f->off.b_out, now, next, C, P, nm);
  f->launches++;
  FTRY(f, cudaGetLastError());
  // per-phase volume: sum alpha_g and sum (1 - alpha_g) = P - sum alpha_g,
  // each changed by the expected inflow (the liquid's by minus it); a
  // non-finite value anywhere in the new state, or a volume fraction outside
  // [0, 1], fails the check too
  double sm[4];
  rc = check_sums(f, now, next, sm);
  if (rc) return rc;
  for (int k = 0; k < 4; k++) f->last_sums[k] = sm[k];
  const double g0 = sm[0], g1 = sm[1];
  const double ex = fabs((g1 - g0) - f->inflow);
  const double dg = ex / fmax(g0, 1e-300), dl = ex / fmax((double)P - g0, 1e-300);
  const double d = isfinite(sm[2]) ? fmax(dg, dl) : INFINITY;
  if (drift) *drift = d;
  if (ok) *ok = d <= max_drift && sm[3] == 0.0;
  return LBM_OK;
}

int lbm_surrogate_advance(lbm_ctx *ctx, lbm_fno *f, int window, double max_drift, double *drift, int *used) {
  if (!ctx || !f) return LBM_EINVAL;
  if (used) *used = 0;
  int lattice, n[3], ready;
  long long t0;
  lbm::ctx_window_info(ctx, &lattice, n, &t0, &ready);
  if (lattice != LBM_D2Q9 || n[0] != f->nx || n[1] != f->ny || n[2] != 1)
    return lbm::ctx_error(ctx, LBM_EINVAL, "lbm_surrogate_advance: the lattice is not a D2Q9 grid of the model's size");
  if (window < 2 || window % 2) return lbm::ctx_error(ctx, LBM_EINVAL, "lbm_surrogate_advance: window must be even");
  if (!ready) return lbm::ctx_error(ctx, LBM_ESTATE, "lbm_surrogate_advance: lattice not initialised or in error");
  if (t0 % 2) return lbm::ctx_error(ctx, LBM_ESTATE, "lbm_surrogate_advance: odd time (populations mid-swap)");
  const long long P = f->P;
  if (!f->st) FTRY(f, cudaMalloc((void **)&f->st, 12 * P * sizeof(double)));
  double *now = f->st, *next = f->st + 6 * P;
  int rc = lbm_get_moments(ctx, now, now + P, now + 3 * P, now + 5 * P, nullptr, nullptr, 1);
  if (rc) return rc;
  double d = 0.0;
  int ok = 0;
  rc = lbm_fno_advance(f, now, next, max_drift, &d, &ok);
  if (rc) return rc;
  if (drift) *drift = d;
  if (ok) {
    // the check verified every new alpha_g in [0, 1] and summed them on the device
    rc = lbm::ctx_init_device(ctx, next, next + P, next + 3 * P, next + 5 * P, f->last_sums[1]);
    if (rc) return rc;
    lbm::ctx_set_time(ctx, t0 + window);
    if (used) *used = 1;
    return LBM_OK;
  }
  return lbm_step(ctx, window);  // the fallback: the lattice's own populations
}

int lbm_fno_launch_count(const lbm_fno *f, long long *n) {
  if (!f || !n) return LBM_EINVAL;
  *n = f->launches;
  return LBM_OK;
}

const char *lbm_fno_last_error(const lbm_fno *f) { return f ? f->err : ""; }

int lbm_fno_gemm(int ta, int tb, int M, int N, int K, float alpha, const void *A, int lda, long long sA,
                 const void *B, int ldb, long long sB, float beta, void *C, int ldc, long long sC, int batch,
                 int out_f32, int ksplit, void *stream) {
  if (!A || !B || !C) return LBM_EINVAL;
  G g;
  g.A = (const bf16 *)A; g.B = (const bf16 *)B; g.C = C;
  g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb; g.ldc = ldc; g.sA = sA; g.sB = sB; g.sC = sC;
  g.batch = batch; g.alpha = alpha; g.beta = beta; g.ta = ta != 0; g.tb = tb != 0; g.out_f32 = out_f32 != 0;
  g.ksplit = ksplit;
  if (ksplit > 1 && beta != 1.0f) return LBM_EINVAL;
  cudaError_t e = gemm(g, (cudaStream_t)stream);
  return e == cudaSuccess ? LBM_OK : (e == cudaErrorInvalidValue || e == cudaErrorMisalignedAddress ? LBM_EINVAL : LBM_ECUDA);
}

}  // extern "C"
