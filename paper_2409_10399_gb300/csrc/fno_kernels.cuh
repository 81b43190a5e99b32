// Kernels of the learned surrogate (a factorised Fourier neural operator that
// advances the 2D state by 64 LBM steps): one batched, strided BF16 matrix
// product with FP32 accumulation (tensor-core fragments), and the FP32
// elementwise operations around it.  Not part of the paper's method: the
// surrogate is judged against, and falls back to, the lattice Boltzmann step.
#pragma once
#include <cuda_bf16.h>
#include <mma.h>
#include <stdint.h>

#include <type_traits>

namespace fno {

typedef __nv_bfloat16 bf16;

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], b < batch.  op(A) is M x K,
// op(B) is K x N.  Row-major storage: A is M x K (lda >= K), or K x M
// (lda >= M) when ta; B is K x N (ldb >= N), or N x K (ldb >= K) when tb;
// C is M x N (ldc >= N), float or bf16.  M, N, K multiples of 16, leading
// dimensions multiples of 8, bases 32-byte aligned (checked by the host).
// ksplit > 1 splits K into chunks of kchunk (a multiple of 32) over blocks,
// each adding alpha times its partial product into a float C with atomics
// (C += alpha op(A) op(B); beta is not applied).
// With bias != null (float C, ksplit 1) the epilogue also adds a bias to the
// result: bias[b] (one value per batch entry) or, with bias_rows, bias[row].
// With hout != null it stores act ? GELU(result) : result as bf16 at the same
// index of hout (the last product of a surrogate layer, the lifting); C may
// then be null (beta 0), and the float result is not stored; store_c = 0
// keeps C as an input only (beta 1: C is read, the result goes to hout).
// The SEG2 form (batch 1, ksplit 1) adds a second product to the same tile:
// C += A2_t B2_t over K2, where for the tile at output columns n0.. (all in
// one row of seg_nx columns) A2_t = A2 + (n0 / seg_nx) a2_rs is K2 x M
// (lda2) and B2_t = B2 + (n0 % seg_nx) ldb2 is N x K2 (ldb2), both read
// transposed: the pointwise product of a layer fused with the reconstruction
// of its x spectrum, whose coefficients differ from row to row.
struct GemmArgs {
  const bf16 *A, *B;
  void *C;
  int M, N, K, lda, ldb, ldc;
  long long sA, sB, sC;  // batch strides (elements)
  float alpha, beta;
  int ksplit, kchunk;
  const float *bias;
  bf16 *hout;
  int bias_rows, act, store_c;
  const bf16 *A2, *B2;
  int K2, lda2, ldb2, seg_nx;
  long long a2_rs;
};

__device__ __forceinline__ float gelu(float z);

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8, GSTAGES = 3;

// 16-byte asynchronous global -> shared copy; with pred false nothing is
// read (source size 0) and the 16 bytes are zero-filled
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool TA, bool TB>
struct GemmSmem {
  // A tile: [GBM][GBK] (TA: [GBK][GBM]); B tile: [GBK][GBN] (TB: [GBN][GBK])
  static constexpr int A_ROWS = TA ? GBK : GBM, A_COLS = TA ? GBM : GBK;
  static constexpr int B_ROWS = TB ? GBN : GBK, B_COLS = TB ? GBK : GBN;
  static constexpr int A_LD = A_COLS + GPAD, B_LD = B_COLS + GPAD;
  static constexpr int A_BYTES = A_ROWS * A_LD * 2, B_BYTES = B_ROWS * B_LD * 2;
  // second segment's tiles (both transposed): [GBK][GBM] and [GBN][GBK]
  static constexpr int A2_LD = GBM + GPAD, B2_LD = GBK + GPAD, A2_BYTES = GBK * A2_LD * 2;
  static constexpr int SEG2_BYTES = A2_BYTES + GBN * B2_LD * 2;
  static constexpr int S1 = A_BYTES + B_BYTES;
  static constexpr int STAGE = ((S1 > SEG2_BYTES ? S1 : SEG2_BYTES) + 127) / 128 * 128;
  static constexpr int PIPE = GSTAGES * STAGE;
  static constexpr int C_BYTES = GBM * (GBN + 4) * 4;
  static constexpr int BYTES = PIPE > C_BYTES ? PIPE : C_BYTES;
};

// PRE (float C, beta != 0, ksplit 1): the old C tile is loaded into
// registers before the product, so that its read from memory overlaps the
// operand loads and the tensor-core work instead of following them.
template <bool TA, bool TB, class OutT, bool SEG2 = false, bool PRE = false>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
  using namespace nvcuda;
  typedef GemmSmem<TA, TB> SM;
  constexpr int A_ROWS = SM::A_ROWS, A_COLS = SM::A_COLS, B_ROWS = SM::B_ROWS, B_COLS = SM::B_COLS;
  constexpr int A_LD = SM::A_LD, B_LD = SM::B_LD;
  // one buffer: a ring of GSTAGES (A, B) tiles for the main product, reused
  // after it by the second segment's tiles and then by the FP32 output tile
  __shared__ __align__(128) unsigned char smem[SM::BYTES];
  float(*sC)[GBN + 4] = reinterpret_cast<float(*)[GBN + 4]>(smem);

  const int b = blockIdx.z / g.ksplit, split = blockIdx.z % g.ksplit;
  const int kbeg = split * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  const bf16 *A = g.A + (long long)b * g.sA;
  const bf16 *B = g.B + (long long)b * g.sB;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // 2 x 2 warps of 32 x 32
  // epilogue: groups of 4 columns (N and ldc are multiples of 8), PER per thread
  constexpr int PER = GBM * GBN / 4 / 128;
  float4 pre[PRE ? PER : 1];
  if constexpr (PRE) {
    const float *Cb = reinterpret_cast<const float *>(g.C) + (long long)b * g.sC;
#pragma unroll
    for (int j = 0; j < PER; j++) {
      const int v = tid + j * 128, r = v / (GBN / 4), c = (v % (GBN / 4)) * 4, gr = m0 + r, gc = n0 + c;
      pre[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < g.M && gc < g.N) pre[j] = *reinterpret_cast<const float4 *>(Cb + (long long)gr * g.ldc + gc);
    }
  }

  typedef wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16,
                         typename std::conditional<TA, wmma::col_major, wmma::row_major>::type> FragA;
  typedef wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16,
                         typename std::conditional<TB, wmma::col_major, wmma::row_major>::type> FragB;
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++) wmma::fill_fragment(acc[i][j], 0.0f);

  // stage the k-slice starting at k0 into ring slot st, zero outside the matrix
  auto load_stage = [&](int st, int k0) {
    bf16 *sA = reinterpret_cast<bf16 *>(smem + st * SM::STAGE);
    bf16 *sB = reinterpret_cast<bf16 *>(smem + st * SM::STAGE + SM::A_BYTES);
#pragma unroll
    for (int v = tid; v < A_ROWS * A_COLS / 8; v += 128) {
      const int r = v / (A_COLS / 8), c = (v % (A_COLS / 8)) * 8;
      const int gr = (TA ? k0 : m0) + r, gc = (TA ? m0 : k0) + c;
      const int mi = TA ? gc : gr, ki = TA ? gr : gc;
      const bool ok = mi < g.M && ki < kend;
      cp_async16(sA + r * A_LD + c, ok ? A + (long long)gr * g.lda + gc : A, ok);
    }
#pragma unroll
    for (int v = tid; v < B_ROWS * B_COLS / 8; v += 128) {
      const int r = v / (B_COLS / 8), c = (v % (B_COLS / 8)) * 8;
      const int gr = (TB ? n0 : k0) + r, gc = (TB ? k0 : n0) + c;
      const int ni = TB ? gr : gc, ki = TB ? gc : gr;
      const bool ok = ni < g.N && ki < kend;
      cp_async16(sB + r * B_LD + c, ok ? B + (long long)gr * g.ldb + gc : B, ok);
    }
  };

  // the second segment's k-slices follow the first's through the same ring
  const bf16 *A2 = nullptr, *B2 = nullptr;
  if constexpr (SEG2) {
    A2 = g.A2 + (long long)(n0 / g.seg_nx) * g.a2_rs;
    B2 = g.B2 + (long long)(n0 % g.seg_nx) * g.ldb2;
  }
  auto load_stage2 = [&](int st, int k0) {
    bf16 *sA2 = reinterpret_cast<bf16 *>(smem + st * SM::STAGE);
    bf16 *sB2 = reinterpret_cast<bf16 *>(smem + st * SM::STAGE + SM::A2_BYTES);
#pragma unroll
    for (int v = tid; v < GBK * GBM / 8; v += 128) {
      const int r = v / (GBM / 8), c = (v % (GBM / 8)) * 8, ki = k0 + r, mi = m0 + c;
      const bool ok = mi < g.M && ki < g.K2;
      cp_async16(sA2 + r * SM::A2_LD + c, ok ? A2 + (long long)ki * g.lda2 + mi : A2, ok);
    }
#pragma unroll
    for (int v = tid; v < GBN * GBK / 8; v += 128) {
      const int r = v / (GBK / 8), c = (v % (GBK / 8)) * 8, ni = n0 + r, ki = k0 + c;
      const bool ok = ni < g.N && ki < g.K2;
      cp_async16(sB2 + r * SM::B2_LD + c, ok ? B2 + (long long)r * g.ldb2 + ki : B2, ok);
    }
  };
  const int nk1 = kend > kbeg ? (kend - kbeg + GBK - 1) / GBK : 0;
  const int nk = nk1 + (SEG2 ? (g.K2 + GBK - 1) / GBK : 0);
  auto load_slice = [&](int st, int it) {
    if (!SEG2 || it < nk1) load_stage(st, kbeg + it * GBK);
    else load_stage2(st, (it - nk1) * GBK);
  };
#pragma unroll
  for (int st = 0; st < GSTAGES - 1; st++) {
    if (st < nk) load_slice(st, st);
    cp_async_commit();
  }
  for (int it = 0; it < nk; it++) {
    cp_async_wait<GSTAGES - 2>();  // slice `it` has landed (this thread's copies)
    __syncthreads();               // ... everyone's; and slot (it - 1) % GSTAGES is free
    if (it + GSTAGES - 1 < nk) load_slice((it + GSTAGES - 1) % GSTAGES, it + GSTAGES - 1);
    cp_async_commit();
    const unsigned char *slot = smem + (it % GSTAGES) * SM::STAGE;
    if (!SEG2 || it < nk1) {
      const bf16 *sA = reinterpret_cast<const bf16 *>(slot);
      const bf16 *sB = reinterpret_cast<const bf16 *>(slot + SM::A_BYTES);
#pragma unroll
      for (int kk = 0; kk < GBK; kk += 16) {
        FragA fa[2];
        FragB fb[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
          const bf16 *pa = TA ? sA + kk * A_LD + wm + 16 * i : sA + (wm + 16 * i) * A_LD + kk;
          wmma::load_matrix_sync(fa[i], pa, A_LD);
          const bf16 *pb = TB ? sB + (wn + 16 * i) * B_LD + kk : sB + kk * B_LD + wn + 16 * i;
          wmma::load_matrix_sync(fb[i], pb, B_LD);
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
          for (int j = 0; j < 2; j++) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
      }
    } else if constexpr (SEG2) {
      typedef wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> FragA2;
      typedef wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> FragB2;
      const bf16 *sA2 = reinterpret_cast<const bf16 *>(slot);
      const bf16 *sB2 = reinterpret_cast<const bf16 *>(slot + SM::A2_BYTES);
#pragma unroll
      for (int kk = 0; kk < GBK; kk += 16) {
        FragA2 fa[2];
        FragB2 fb[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
          wmma::load_matrix_sync(fa[i], sA2 + kk * SM::A2_LD + wm + 16 * i, SM::A2_LD);
          wmma::load_matrix_sync(fb[i], sB2 + (wn + 16 * i) * SM::B2_LD + kk, SM::B2_LD);
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
          for (int j = 0; j < 2; j++) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // the ring is free for the output tile
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++)
      wmma::store_matrix_sync(&sC[wm + 16 * i][wn + 16 * j], acc[i][j], GBN + 4, wmma::mem_row_major);
  __syncthreads();
  OutT *C = reinterpret_cast<OutT *>(g.C) + (long long)b * g.sC;
  // epilogue in groups of 4 columns (N and ldc are multiples of 8): every read
  // of the old C is issued before any write, so the reads overlap
  if constexpr (std::is_same<OutT, float>::value) {
    if (g.ksplit > 1) {
      for (int v = tid; v < GBM * GBN; v += 128) {
        const int r = v / GBN, c = v % GBN, gr = m0 + r, gc = n0 + c;
        if (gr < g.M && gc < g.N) atomicAdd(C + (long long)gr * g.ldc + gc, g.alpha * sC[r][c]);
      }
      return;
    }
  }
  float4 old[PER];
#pragma unroll
  for (int j = 0; j < PER; j++) {
    const int v = tid + j * 128, r = v / (GBN / 4), c = (v % (GBN / 4)) * 4, gr = m0 + r, gc = n0 + c;
    old[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (PRE) {
      old[j] = pre[j];
    } else if (g.beta != 0.0f && gr < g.M && gc < g.N) {
      const OutT *p = C + (long long)gr * g.ldc + gc;
      if constexpr (std::is_same<OutT, float>::value) {
        old[j] = *reinterpret_cast<const float4 *>(p);
      } else {
        const uint2 raw = *reinterpret_cast<const uint2 *>(p);
        const bf16 *hb = reinterpret_cast<const bf16 *>(&raw);
        old[j] = make_float4((float)hb[0], (float)hb[1], (float)hb[2], (float)hb[3]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PER; j++) {
    const int v = tid + j * 128, r = v / (GBN / 4), c = (v % (GBN / 4)) * 4, gr = m0 + r, gc = n0 + c;
    if (gr >= g.M || gc >= g.N) continue;
    float o[4] = {g.alpha * sC[r][c] + g.beta * old[j].x, g.alpha * sC[r][c + 1] + g.beta * old[j].y,
                  g.alpha * sC[r][c + 2] + g.beta * old[j].z, g.alpha * sC[r][c + 3] + g.beta * old[j].w};
    OutT *p = C + (long long)gr * g.ldc + gc;
    if constexpr (std::is_same<OutT, float>::value) {
      if (g.bias) {
        const float bb = g.bias_rows ? g.bias[gr] : g.bias[b];
#pragma unroll
        for (int e = 0; e < 4; e++) o[e] += bb;
      }
      if (g.hout) {
        bf16 hv[4];
#pragma unroll
        for (int e = 0; e < 4; e++) hv[e] = __float2bfloat16(g.act ? gelu(o[e]) : o[e]);
        *reinterpret_cast<uint2 *>(g.hout + (long long)b * g.sC + (long long)gr * g.ldc + gc) =
            *reinterpret_cast<const uint2 *>(hv);
      }
      if (g.C && g.store_c) *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
      bf16 hv[4] = {__float2bfloat16(o[0]), __float2bfloat16(o[1]), __float2bfloat16(o[2]), __float2bfloat16(o[3])};
      *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(hv);
    }
  }
}

// ---------------------------------------------------------------- elementwise

// hardware tanh (PTX tanh.approx.f32, relative error ~2^-11): below the
// 2^-9 of the BF16 activations it feeds
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu(float z) {
  // tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
  const float k = 0.7978845608028654f;
  return 0.5f * z * (1.0f + tanh_fast(k * (z + 0.044715f * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float k = 0.7978845608028654f;
  const float u = k * (z + 0.044715f * z * z * z);
  const float t = tanh_fast(u);
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * z * z);
}

// dz = act ? dh * gelu'(z) : dh  (float and bf16 copies)
__global__ void k_act_back(const float *dh, const float *z, float *dz, bf16 *dz16, long long n, int act) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = act ? dh[i] * gelu_grad(z[i]) : dh[i];
  dz[i] = v;
  dz16[i] = __float2bfloat16(v);
}

// db[c] += sum_p dz[c][p]: blocks (chunk, c), each reducing its chunk of the
// channel in a tree and adding it atomically
__global__ void k_bias_grad(const float *dz, float *db, long long P) {
  __shared__ float s[256];
  const int c = blockIdx.y;
  const long long chunk = (P + gridDim.x - 1) / gridDim.x, p0 = blockIdx.x * chunk;
  const long long p1 = p0 + chunk < P ? p0 + chunk : P;
  float acc = 0.0f;
  for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) acc += dz[(long long)c * P + p];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(db + c, s[0]);
}

// sum over a block of 256 threads (8 warps), result in thread 0
__device__ __forceinline__ double block_sum(double v, double *s8) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s8[threadIdx.x >> 5] = v;
  __syncthreads();
  double a = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) a += s8[w];
  return a;
}

// squared error of the first cv channels: d = scale (y - t) with scale =
// 2 / (cv P) (the padding channels of d stay zero); grid (blocks over P, cv),
// one FP64 partial sum of (y - t)^2 per block in part[y * gridDim.x + x], and
// for channel 0 (alpha_g) the partial sums of (y - t) in
// part[cv * gridDim.x + x]
__global__ void k_mse(const float *y, const float *t, float *d, bf16 *d16, long long P, float scale,
                      double *part) {
  __shared__ double s[8];
  const long long i = (long long)blockIdx.y * P + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e1 = 0.0, e2 = 0.0;
  if ((long long)blockIdx.x * blockDim.x + threadIdx.x < P) {
    const float e = y[i] - t[i];
    e1 = e;
    e2 = (double)e * e;
    const float g = scale * e;
    d[i] = g;
    d16[i] = __float2bfloat16(g);
  }
  const double a2 = block_sum(e2, s);
  if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = a2;
  if (blockIdx.y == 0) {
    __syncthreads();
    const double a1 = block_sum(e1, s);
    if (threadIdx.x == 0) part[(long long)gridDim.y * gridDim.x + blockIdx.x] = a1;
  }
}

// conservation term of the loss, lambda (mean_p e_0)^2 with e_0 = y_0 - t_0
// (the alpha_g channel): its gradient 2 lambda mean(e_0) / P is added to
// every node of channel 0 of d (and d16).  esum: the nb partial sums of e_0
// from k_mse, reduced in the same order by every block.
__global__ void k_cons_grad(const double *esum, int nb, float *d, bf16 *d16, long long P, double lambda) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < nb; i++) a += esum[i];
    tot = a;
  }
  __syncthreads();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float g = d[p] + (float)(2.0 * lambda * (tot / (double)P) / (double)P);
  d[p] = g;
  d16[p] = __float2bfloat16(g);
}

// Adam (Kingma & Ba) on FP32 master parameters, bias-corrected step size lr_t
// (gradient scaled by gscale, e.g. 1 / samples accumulated)
__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr_t, float b1, float b2,
                       float eps, float gscale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] * gscale;
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr_t * mi / (sqrtf(vi) + eps);
}

__global__ void k_to_bf16(const float *x, bf16 *y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// Complex channel mixing of mode k as a real 2C x 2C matrix:
// W[k] = [[A_k, -B_k], [B_k, A_k]] (rows: cosine block, then sine block)
__global__ void k_assemble_complex(const float *A, const float *B, bf16 *W, int C, int K) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = 4LL * C * C;
  if (i >= per * K) return;
  const int k = (int)(i / per);
  const int r = (int)((i % per) / (2 * C)), c = (int)(i % (2 * C));
  const int ri = r % C, ci = c % C;
  const float a = A[(long long)k * C * C + (long long)ri * C + ci], bb = B[(long long)k * C * C + (long long)ri * C + ci];
  float val;
  if (r < C) val = c < C ? a : -bb;
  else val = c < C ? bb : a;
  W[i] = __float2bfloat16(val);
}

// gradient of the real 2C x 2C matrices back onto A_k, B_k:
// dA = dW11 + dW22, dB = dW21 - dW12
__global__ void k_fold_complex(const float *dW, float *dA, float *dB, int C, int K) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)K * C * C) return;
  const int k = (int)(i / ((long long)C * C));
  const int r = (int)((i / C) % C), c = (int)(i % C);
  const float *W = dW + (long long)k * 4 * C * C;
  const int L = 2 * C;
  dA[i] += W[r * L + c] + W[(r + C) * L + c + C];
  dB[i] += W[(r + C) * L + c] - W[r * L + c + C];
}

}  // namespace fno
