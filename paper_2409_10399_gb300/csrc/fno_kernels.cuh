// Kernels of the learned surrogate (a factorised Fourier neural operator that
// advances the 2D state by 64 LBM steps): the FP32 elementwise operations
// around its matrix products (the products themselves: fno_umma.cuh).  Not part of the paper's method: the
// surrogate is judged against, and falls back to, the lattice Boltzmann step.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace fno {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float gelu(float z);

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
