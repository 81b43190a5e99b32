// Diagnostics of a caller-owned population set without any allocation.
//
// Same eight FP64 quantities as lbm_get_diag (a warp/block/grid reduction),
// for callers that may not call cudaMalloc -- an application with its own
// device memory pool, or code running where the CUDA allocator must not be
// touched.  The per-block partial sums live in one file-scope __device__ array
// of fixed size instead of allocated scratch; the caller passes the input
// populations and the output.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_lattice.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_BLOCKS = 1024;  // grid of the partial pass (it strides over all nodes)
constexpr int NA_DEVICES = 64;

// Scratch shared by every call on a device: NA_BLOCKS x 8 partials followed
// by the 8 final values, 65,600 bytes, held by every GPU that loads the
// library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NA_BLOCKS * 8 + 8];

std::mutex g_mu;
// Cached device address of the scratch array, per device, together with the
// id of the CUDA context it was looked up in: a device reset, or a caller
// that makes another context current, gets a fresh lookup.
struct ScratchSlot {
  unsigned long long ctx_id;
  double *addr;
};
ScratchSlot g_slot[NA_DEVICES] = {};

__device__ __forceinline__ double na_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double na_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int LAT>
__global__ void __launch_bounds__(NA_THREADS) k_diag_pops_noalloc(const double *pops, long long n, int spalding,
                                                                  double *partials) {
  using L = lbm::Lattice<LAT>;
  constexpr int Q = L::Q, D = L::D;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double eg = 0, el = 0, ag = 0, al = 0, ug[3] = {0, 0, 0}, ul[3] = {0, 0, 0};
    bool bad = false;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      double f[6];
#pragma unroll
      for (int s = 0; s < 6; s++) {
        f[s] = pops[(long long)(s * Q + q) * n + i];
        bad = bad || !isfinite(f[s]);
      }
      eg += f[0];
      el += f[1];
      ag += f[2];
      al += f[3];
#pragma unroll
      for (int d = 0; d < D; d++) {
        ug[d] += L::v(q, d) * f[0];
        ul[d] += L::v(q, d) * f[1];
      }
    }
    double alg = ag;
    if (spalding != 0) {  // Eq. (spalding), B = clamp to [0, 1]
      const double Bg = ag <= 0.0 ? 0.0 : (ag >= 1.0 ? 1.0 : ag);
      const double Bl = al <= 0.0 ? 0.0 : (al >= 1.0 ? 1.0 : al);
      alg = (Bg + Bl > 0.0) ? Bg / (Bg + Bl) : 0.5;
    }
    const double sum = ag + al - 1.0;
    double ug2 = 0, ul2 = 0;
#pragma unroll
    for (int d = 0; d < D; d++) {
      ug2 += ug[d] * ug[d];
      ul2 += ul[d] * ul[d];
    }
    v[0] += ag;
    v[1] += al;
    v[2] += alg;
    v[3] += sum * sum;
    v[4] = fmax(v[4], sqrt(fmax(ug2, ul2)));
    v[5] += bad ? 1.0 : 0.0;
    v[6] += eg - 1.0;
    v[7] += el - 1.0;
  }
  __shared__ double red[8][NA_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = k == 4 ? na_max(v[k]) : na_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 8; k++) red[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      double x = lane < NA_THREADS / 32 ? red[k][lane] : 0.0;
      x = k == 4 ? na_max(x) : na_sum(x);
      if (lane == 0) partials[blockIdx.x * 8 + k] = x;  // every slot used is overwritten
    }
  }
}

__global__ void k_diag_pops_noalloc_final(const double *partials, int nblocks, double *out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= 8) return;
  double acc = 0.0;
  for (int b = lane; b < nblocks; b += 32) acc = k == 4 ? fmax(acc, partials[b * 8 + k]) : acc + partials[b * 8 + k];
  acc = k == 4 ? na_max(acc) : na_sum(acc);
  if (lane == 0) out[k] = acc;
}

// Id of the CUDA context current on this thread (cuCtxGetId, reached through
// the runtime's driver entry points so that the library needs no link to the
// driver library); false when there is none or the driver lacks the calls.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
bool current_ctx_id(unsigned long long *id) {
  static std::once_flag once;
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
    if (!get_cur || !get_id) cudaGetLastError();  // no error left pending by the queries
  });
  if (!get_cur || !get_id) return false;
  void *ctx = nullptr;
  if (get_cur(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's current
// context, looked up (cudaGetSymbolAddress, with that device current) at the
// first call in each context and cached with the context's id.  In host code
// the array's name is only a stand-in and must never be handed to a kernel.
// A failed lookup leaves no error pending for the caller.
int scratch_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  if (dev < 0 || dev >= NA_DEVICES) return LBM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (current_ctx_id(&id) && g_slot[dev].addr && g_slot[dev].ctx_id == id) {
    *out = g_slot[dev].addr;
    return LBM_OK;
  }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  // the lookup made the device's context current if it was not yet
  if (current_ctx_id(&id)) {
    g_slot[dev].ctx_id = id;
    g_slot[dev].addr = (double *)p;
  } else {
    g_slot[dev].addr = nullptr;  // no context id: look the address up at every call
  }
  *out = (double *)p;
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_diag_populations_noalloc(int lattice, int spalding_mode, const double *pops, long long n_nodes,
                                            double *out, int out_on_device, void *stream) {
  if (lattice < LBM_D1Q3 || lattice > LBM_D3Q19 || !pops || !out || spalding_mode < 0 || spalding_mode > 2)
    return LBM_EINVAL;
  if (n_nodes < 1 || n_nodes > LBM_NOALLOC_MAX_NODES) return LBM_EINVAL;
  // an error left pending by earlier work of the caller stays pending (and is
  // not mistaken for this call's): nothing is launched
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long want = (n_nodes + NA_THREADS - 1) / NA_THREADS;
  const int nblk = (int)(want < NA_BLOCKS ? want : NA_BLOCKS);
  if (lattice == LBM_D1Q3)
    k_diag_pops_noalloc<1><<<nblk, NA_THREADS, 0, st>>>(pops, n_nodes, spalding_mode, scratch);
  else if (lattice == LBM_D2Q9)
    k_diag_pops_noalloc<2><<<nblk, NA_THREADS, 0, st>>>(pops, n_nodes, spalding_mode, scratch);
  else
    k_diag_pops_noalloc<3><<<nblk, NA_THREADS, 0, st>>>(pops, n_nodes, spalding_mode, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  double *final_dev = out_on_device ? out : scratch + NA_BLOCKS * 8;
  k_diag_pops_noalloc_final<<<1, 256, 0, st>>>(scratch, nblk, final_dev);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (!out_on_device) {
    if (cudaMemcpyAsync(out, final_dev, 8 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return LBM_ECUDA;
    }
  }
  return LBM_OK;
}
