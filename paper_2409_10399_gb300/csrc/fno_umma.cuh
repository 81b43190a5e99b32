// The surrogate's matrix products on the fifth-generation tensor cores:
// tcgen05.mma (BF16 operands from shared memory, FP32 accumulator in tensor
// memory), operands staged by TMA (cp.async.bulk.tensor) through a ring of
// mbarrier-tracked stages, the accumulator read back with tcgen05.ld for a
// fused epilogue.  Not part of the paper's method (the surrogate is judged
// against, and falls back to, the lattice Boltzmann step).
//
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b] (the conventions of lbm_fno.cu's G) is
// computed as its transpose, D = C^T (N x M) = op(B)^T op(A)^T: the long
// dimension of every product here (nodes, rows, columns of the lattice) is
// N, and as D's row index it runs along the 128 lanes of tensor memory, one
// thread per output column n, so that the epilogue's stores of one output
// row m are coalesced across a warp without a transposing pass.
//   MMA A operand (128 x 64 per stage) = op(B)^T: B stored N x K (tb) is
//     K-major, stored K x N is MN-major;
//   MMA B operand (NT x 64 per stage)  = op(A)^T: A stored M x K is K-major,
//     stored K x M (ta) is MN-major.
// Both are loaded as 128-byte-swizzled boxes of 64 BF16 along the contiguous
// dimension (one box of 64 K x rows for K-major; boxes of 64 MN x 64 K rows
// for MN-major), the canonical layouts of the shared-memory matrix
// descriptor.  Out-of-range rows and columns of a box read as zero, so
// ragged M, N and K need no masking in the main loop.
//
// Persistent, warp-specialised blocks of 320 threads (k_umma): a TMA
// producer, an MMA issuer that owns two or three accumulators in tensor
// memory, and eight epilogue warps, so that a block's loads, products and
// output of consecutive tiles overlap.  Every mbarrier wait is bounded; one
// that runs out sets fno::umma_timeout and the block skips the rest of its
// work and frees its tensor memory.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace fno {

typedef __nv_bfloat16 bf16;

// set by a block whose wait on an mbarrier ran out (a stalled pipeline);
// read and cleared by the host after the product's stream has synchronised
__device__ int umma_timeout;

struct UmmaArgs {
  CUtensorMap ma;   // MMA A operand: op(B)^T
  CUtensorMap mb;   // MMA B operand: op(A)^T
  CUtensorMap ma2;  // second segment's A operand (SEG2): B2 rows, K-major
  CUtensorMap mb2;  // second segment's B operand (SEG2): A2 tiles, MN-major
  CUtensorMap mc;   // C's tiles: the old FP32 tile (OLDC) and the staged output tile (st_c)
  CUtensorMap mh;   // hout's tiles (st_h), C's layout in BF16
  void *C;
  int M, N, K, ldc;
  long long sC;
  float alpha, beta;
  int ksplit, kchunk, stages;
  const float *bias;
  bf16 *hout;
  int bias_rows, act, store_c;
  int K2, seg_nx;
  // where a block's batch index goes in the operand maps' coordinates: 0 the
  // operand is shared by the batch (coordinate 0), 1 the map's third
  // dimension, 2 its second (a map whose batch stride is below its row
  // stride is encoded with the two outer dimensions swapped)
  int a_bat, b_bat, c_bat;
  int tiles_n, tiles_m, tiles;  // tiles along N, along M, in all (x batch x K split)
  int st_c, st_h;               // C / hout tiles staged in shared memory and stored by TMA
  int nacc, tmem_cols;          // accumulators (and old-C and staging tiles) in flight; columns allocated
};

constexpr int UMMA_M = 128, UMMA_BK = 64, UMMA_MAX_ACC = 3;
constexpr long long UMMA_WAIT_CYCLES = 2000000000LL;  // about a second at the SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of `parity` to complete (try_wait suspends the thread
// in hardware until it does, or for a system-dependent time); false, and the
// timeout flag set, when it has not within UMMA_WAIT_CYCLES
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < UMMA_WAIT_CYCLES)
    if (mbar_try(bar, parity)) return true;
  atomicExch(&umma_timeout, 1);
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// one box of an operand: c0 along the contiguous dimension, row along the
// other, the batch index where the operand's map keeps it
__device__ __forceinline__ void tma_op(uint32_t dst, const CUtensorMap *map, int bat, int c0, int row, int zb,
                                       uint32_t bar) {
  if (bat == 2) tma_load_3d(dst, map, c0, zb, row, bar);
  else tma_load_3d(dst, map, c0, row, bat ? zb : 0, bar);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets, descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}
// the kk-th K = 16 slice of a 64-wide stage.  K-major (rows of 128 bytes, 8-row
// atoms 1024 bytes apart): the slice starts 32 bytes further along the row.
// MN-major (per 64-wide MN chunk 64 K-rows of 128 bytes; chunks 8 KB apart):
// the slice starts 16 K-rows (2 KB) further down.
template <bool KMAJOR>
__device__ __forceinline__ uint64_t slice_desc(uint32_t base, int kk) {
  return KMAJOR ? smem_desc(base + 32u * kk, 16u, 1024u) : smem_desc(base + 2048u * kk, 8192u, 1024u);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// operand majors (0 K-major, 1 MN-major), N >> 3, M >> 4
__device__ __forceinline__ uint32_t instr_desc(bool a_kmajor, bool b_kmajor, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_kmajor ? 0u : 1u) << 15) | ((b_kmajor ? 0u : 1u) << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UMMA_M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on `bar` once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z);

// Dynamic shared memory of one block: the operand ring (`stages` stages),
// `nacc` old-C tiles (OLDC) and staging tiles of the C and of the hout
// output (when they leave by TMA stores), the mbarriers, the tensor-memory
// slot.
template <int NT, class OutT, bool OLDC>
struct UmmaSmem {
  static constexpr int A_BYTES = UMMA_M * UMMA_BK * 2, B_BYTES = NT * UMMA_BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;  // a multiple of 1024 (swizzle atoms stay aligned)
  static constexpr int OLD_TILE = OLDC ? NT * UMMA_M * 4 : 0;
  static constexpr int C_TILE = NT * UMMA_M * (int)sizeof(OutT), H_TILE = NT * UMMA_M * 2;
  static __host__ __device__ constexpr int bytes(int stages, int nacc, int st_c, int st_h) {
    return 1024 + stages * STAGE + nacc * OLD_TILE + (st_c ? nacc * C_TILE : 0) + (st_h ? nacc * H_TILE : 0) +
           (2 * stages + 4 * UMMA_MAX_ACC) * 8 + 16;
  }
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// TMA store of a staged tile (box of the map) at c0 (contiguous), row, batch
__device__ __forceinline__ void tma_store_op(const CUtensorMap *map, int bat, uint32_t src, int c0, int row, int zb) {
  const int c1 = bat == 2 ? zb : row, c2 = bat == 2 ? row : (bat ? zb : 0);
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
constexpr int UMMA_EPI_WARPS = 8, UMMA_THREADS = 64 + 32 * UMMA_EPI_WARPS;
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * UMMA_EPI_WARPS) : "memory"); }

// AK: the MMA A operand (op(B)^T) is K-major (B stored N x K); BKM: the MMA B
// operand (op(A)^T) is K-major (A stored M x K).  NT: output rows m per tile
// (the MMA's N).  OLDC: the old FP32 C tile is loaded by TMA (beta != 0, no
// split).  SEG2: a second product over K2 is accumulated into the same tile
// (the pointwise product fused with the x reconstruction).
//
// Persistent: block i takes tiles i, i + gridDim.x, ... (n fastest, then m,
// then batch and K split).  Warp 0 (one lane) streams every tile's stages
// through the ring (and its old C tile), running ahead into the next tiles;
// warp 1 owns the tensor memory (nacc accumulators of NT columns) and one of
// its lanes issues the MMAs, tile j into accumulator j % nacc once the
// epilogue has emptied it; warps 2-9 run the epilogue of tile j while the
// MMAs of the next tiles proceed, and hand their output tiles to TMA stores (or store
// directly, or add with atomics for a split K).
template <bool AK, bool BKM, int NT, class OutT, bool SEG2, bool OLDC>
__global__ void __launch_bounds__(UMMA_THREADS) k_umma(const __grid_constant__ UmmaArgs g) {
  typedef UmmaSmem<NT, OutT, OLDC> SM;
  extern __shared__ unsigned char umma_smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(umma_smem_raw) + 1023) &
                                                        ~(uintptr_t)1023);
  const int S = g.stages, NA = g.nacc;
  unsigned char *p = sm + S * SM::STAGE;
  float *oldc = reinterpret_cast<float *>(p);
  p += NA * SM::OLD_TILE;
  OutT *stc = reinterpret_cast<OutT *>(p);
  p += g.st_c ? NA * SM::C_TILE : 0;
  bf16 *sth = reinterpret_cast<bf16 *>(p);
  p += g.st_h ? NA * SM::H_TILE : 0;
  const uint32_t bars = smem_u32(p);
  constexpr int MA = UMMA_MAX_ACC;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(p + (2 * S + 4 * MA) * 8);
  volatile int *flag = reinterpret_cast<volatile int *>(p + (2 * S + 4 * MA) * 8 + 8);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (S + s); };
  auto accf = [&](int b) { return bars + 8u * (2 * S + b); };
  auto acce = [&](int b) { return bars + 8u * (2 * S + MA + b); };
  auto oldf = [&](int b) { return bars + 8u * (2 * S + 2 * MA + b); };
  auto olde = [&](int b) { return bars + 8u * (2 * S + 3 * MA + b); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < 2 * S; i++) mbar_init(bars + 8u * i, 1);
    for (int b = 0; b < MA; b++) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), UMMA_EPI_WARPS);
      mbar_init(oldf(b), 1);
      mbar_init(olde(b), UMMA_EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // tile t: output columns n0.., rows m0.., batch entry zb, K range [kbeg, kend)
  auto decode = [&](int t, int &n0, int &m0, int &zb, int &kbeg, int &kend) {
    const int nt = t % g.tiles_n, r = t / g.tiles_n, mt = r % g.tiles_m, z = r / g.tiles_m;
    n0 = nt * UMMA_M;
    m0 = mt * NT;
    zb = z / g.ksplit;
    kbeg = (z % g.ksplit) * g.kchunk;
    kend = min(g.K, kbeg + g.kchunk);
  };
  auto iters1 = [&](int kbeg, int kend) { return kend > kbeg ? (kend - kbeg + UMMA_BK - 1) / UMMA_BK : 0; };
  const int nk2 = SEG2 ? (g.K2 + UMMA_BK - 1) / UMMA_BK : 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      int it = 0, j = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < g.tiles && ok; t += gridDim.x, j++) {
        int n0, m0, zb, kbeg, kend;
        decode(t, n0, m0, zb, kbeg, kend);
        const int b = j % NA, u = j / NA;
        if constexpr (OLDC) {
          if (u >= 1 && !mbar_wait(olde(b), (u - 1) & 1)) break;
          mbar_expect_tx(oldf(b), SM::OLD_TILE);
          tma_op(smem_u32(oldc + b * (SM::OLD_TILE / 4)), &g.mc, g.c_bat, n0, m0, zb, oldf(b));
        }
        const int nk1 = iters1(kbeg, kend), nk = nk1 + nk2;
        const int seg_y = SEG2 ? n0 / g.seg_nx : 0, seg_x = SEG2 ? n0 % g.seg_nx : 0;
        for (int i = 0; i < nk; i++, it++) {
          const int s = it % S;
          if (it >= S && !mbar_wait(empty(s), ((it / S) - 1) & 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full(s), SM::STAGE);
          const uint32_t sa = smem_u32(sm + s * SM::STAGE), sb = sa + SM::A_BYTES;
          if (!SEG2 || i < nk1) {
            const int k0 = kbeg + i * UMMA_BK;
            if (AK) tma_op(sa, &g.ma, g.a_bat, k0, n0, zb, full(s));
            else {
              tma_op(sa, &g.ma, g.a_bat, n0, k0, zb, full(s));
              tma_op(sa + 8192u, &g.ma, g.a_bat, n0 + 64, k0, zb, full(s));
            }
            if (BKM) tma_op(sb, &g.mb, g.b_bat, k0, m0, zb, full(s));
            else {
#pragma unroll
              for (int q = 0; q < NT / 64; q++) tma_op(sb + 8192u * q, &g.mb, g.b_bat, m0 + 64 * q, k0, zb, full(s));
            }
          } else if constexpr (SEG2) {
            const int k0 = (i - nk1) * UMMA_BK;
            tma_load_3d(sa, &g.ma2, k0, seg_x, 0, full(s));
#pragma unroll
            for (int q = 0; q < NT / 64; q++) tma_load_3d(sb + 8192u * q, &g.mb2, m0 + 64 * q, k0, seg_y, full(s));
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issue: four K = 16 slices per stage; a stage is released
      //      (empty) when its MMAs complete, an accumulator (accf) after its
      //      tile's last stage
      const uint32_t id1 = instr_desc(AK, BKM, NT), id2 = instr_desc(true, false, NT);
      int it = 0, j = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < g.tiles && ok; t += gridDim.x, j++) {
        int n0, m0, zb, kbeg, kend;
        decode(t, n0, m0, zb, kbeg, kend);
        const int b = j % NA, u = j / NA;
        if (u >= 1 && !mbar_wait(acce(b), (u - 1) & 1)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * NT);
        const int nk1 = iters1(kbeg, kend), nk = nk1 + nk2;
        for (int i = 0; i < nk; i++, it++) {
          const int s = it % S;
          if (!mbar_wait(full(s), (it / S) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(sm + s * SM::STAGE), sb = sa + SM::A_BYTES;
          const bool seg1 = !SEG2 || i < nk1;
#pragma unroll
          for (int kk = 0; kk < UMMA_BK / 16; kk++) {
            const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
            if (seg1) umma_bf16(d, slice_desc<AK>(sa, kk), slice_desc<BKM>(sb, kk), id1, acc);
            else umma_bf16(d, slice_desc<true>(sa, kk), slice_desc<false>(sb, kk), id2, acc);
          }
          umma_commit(empty(s));
        }
        umma_commit(accf(b));
      }
    }
  } else {
    // ---- epilogue (warps 2 .. 1 + UMMA_EPI_WARPS; warp w reads tensor-memory
    //      lanes 32 (w % 4) .., the warps of a lane quadrant take the tile's
    //      16-column chunks in turn)
    constexpr int PER_Q = UMMA_EPI_WARPS / 4;
    const int e = tid - 64, q = warp & 3, sub = (warp - 2) >> 2, row = 32 * q + lane;
    const bool staged = g.st_c || g.st_h;
    const bool split = g.ksplit > 1, with_c = g.C && g.store_c, with_h = g.hout != nullptr;
    const bool bias_r = g.bias && g.bias_rows, bias_z = g.bias && !g.bias_rows;
    const float alpha = g.alpha, beta = g.beta;
    OutT *C = reinterpret_cast<OutT *>(g.C);
    int j = 0;
    for (int t = blockIdx.x; t < g.tiles; t += gridDim.x, j++) {
      int n0, m0, zb, kbeg, kend;
      decode(t, n0, m0, zb, kbeg, kend);
      const int b = j % NA, u = j / NA;
      if (e == 0) {
        bool ok = mbar_wait(accf(b), u & 1);
        if (OLDC) ok = mbar_wait(oldf(b), u & 1) && ok;
        // the TMA store that last read staging buffer b (tile j - nacc) is done
        if (staged && j >= NA) {
          if (NA == 3) bulk_wait_read<2>();
          else bulk_wait_read<1>();
        }
        flag[j & 1] = ok ? 1 : 0;  // two slots: a thread may still read the last tile's
      }
      epi_sync();
      if (!flag[j & 1]) break;
      tc_fence_after();
      const bool has = iters1(kbeg, kend) + nk2 > 0;
      const int n = n0 + row;
      const bool n_in = n < g.N;
      const float bz = bias_z ? __ldg(g.bias + zb) : 0.0f;
      // row m of the output at element offset mrow(m) + n
      const long long cb = (long long)zb * g.sC + n;
      const float *old = oldc + b * (SM::OLD_TILE / 4) + row;  // nacc tiles of NT x 128
      OutT *tc = stc + b * (SM::C_TILE / (int)sizeof(OutT)) + row;
      bf16 *th = sth + b * (SM::H_TILE / 2) + row;
#pragma unroll 1
      for (int c0 = 16 * sub; c0 < NT; c0 += 16 * PER_Q) {
        float o[16];
        tmem_ld16(tmem + (uint32_t)(b * NT) + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, o);
        const int mc = m0 + c0;  // first output row of the chunk
        if (!has) {
#pragma unroll
          for (int jj = 0; jj < 16; jj++) o[jj] = 0.0f;
        }
        if (split) {
          // split K: this block's partial product is added into C
          if constexpr (std::is_same<OutT, float>::value) {
            if (has && n_in)
#pragma unroll
              for (int jj = 0; jj < 16; jj++)
                if (mc + jj < g.M) atomicAdd(C + cb + (long long)(mc + jj) * g.ldc, alpha * o[jj]);
          }
          continue;
        }
#pragma unroll
        for (int jj = 0; jj < 16; jj++) o[jj] *= alpha;
        if constexpr (OLDC) {
#pragma unroll
          for (int jj = 0; jj < 16; jj++) o[jj] = fmaf(beta, old[(c0 + jj) * UMMA_M], o[jj]);
        }
        if constexpr (!std::is_same<OutT, float>::value) {
          if (beta != 0.0f && n_in)
#pragma unroll
            for (int jj = 0; jj < 16; jj++)
              if (mc + jj < g.M) o[jj] = fmaf(beta, __bfloat162float(C[cb + (long long)(mc + jj) * g.ldc]), o[jj]);
        }
        if (bias_r) {
#pragma unroll
          for (int jj = 0; jj < 16; jj++) o[jj] += mc + jj < g.M ? __ldg(g.bias + mc + jj) : 0.0f;
        } else if (bias_z) {
#pragma unroll
          for (int jj = 0; jj < 16; jj++) o[jj] += bz;
        }
        if (with_h) {
          bf16 hv[16];
          if (g.act) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++) hv[jj] = __float2bfloat16(gelu(o[jj]));
          } else {
#pragma unroll
            for (int jj = 0; jj < 16; jj++) hv[jj] = __float2bfloat16(o[jj]);
          }
          if (g.st_h) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++) th[(c0 + jj) * UMMA_M] = hv[jj];
          } else if (n_in) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++)
              if (mc + jj < g.M) g.hout[cb + (long long)(mc + jj) * g.ldc] = hv[jj];
          }
        }
        if (with_c) {
          if (g.st_c) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++) tc[(c0 + jj) * UMMA_M] = (OutT)o[jj];
          } else if (n_in) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++)
              if (mc + jj < g.M) C[cb + (long long)(mc + jj) * g.ldc] = (OutT)o[jj];
          }
        }
      }
      // accumulator b and old-C buffer b are free for tile j + nacc
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(acce(b));
        if (OLDC) mbar_arrive(olde(b));
      }
      if (staged) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_sync();
        if (e == 0) {
          if (g.st_c) tma_store_op(&g.mc, g.c_bat, smem_u32(stc + b * (SM::C_TILE / (int)sizeof(OutT))), n0, m0, zb);
          if (g.st_h) tma_store_op(&g.mh, g.c_bat, smem_u32(sth + b * (SM::H_TILE / 2)), n0, m0, zb);
          bulk_commit();
        }
      }
    }
    if (e == 0 && staged) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
}

}  // namespace fno
