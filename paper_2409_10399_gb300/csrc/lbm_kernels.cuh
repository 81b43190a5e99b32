// Fused collide-and-stream of the six coupled EE-LBM schemes (arXiv
// 2409.10399, Sec. 2-3) on an AA-pattern, structure-of-arrays store.
//
// Store: one buffer of 6*Q planes, plane (s*Q + q) holds direction q of scheme
// s (0 g, 1 l, 2 alpha_g, 3 alpha_l, 4 beta_g, 5 beta_l) for all N nodes, node
// index x + nx*(y + ny*z), x fastest.  Every plane keeps deviations
// f - w_q*r_s (r = 1 for g, l, beta; r = the initial mean alpha for the alpha
// schemes), and all arithmetic below is written in those deviations, so the
// pressure coupling (eps_g - 1)/R of Eq. (lbm-phi-l) is formed without the
// cancellation of 1 + small.
//
// AA pattern (one array, in place): on even t node x reads slot (x, q) and
// writes its post-collision f*(x,q) to slot (x, opp q); on odd t it reads
// slot (x - v_q, opp q) and writes slot (x + v_q, q).  Each node reads and
// writes the same set of slots, so no two threads touch the same slot.  A
// population that would cross a non-periodic face is reflected into the
// node's own slot (x, opp q) on the write side, carrying the face rule's value
// (half-way bounce-back, Table 1 inlet, Table 2 outlet), and is read back from
// slot (x, q) on the odd read side.
//
// Beta-stencil form (template flag BS): the beta schemes are reset to
// f^eq(1, c) at every node and step (Eq. (lbmbeta) with beta = 1), so what
// streams into node x along q is a function of c at the source node only.
// The store then keeps 4*Q population planes and, instead of the 2*Q beta
// planes, the 2*D components of c (c_g, c_l) of the last step in a
// double-buffered field (buffer t & 1 written at step t, the other read); the
// beta populations arriving at x are re-evaluated from c at x - v_q, or from
// the face rule at x where x - v_q lies beyond a non-periodic face.  The
// arithmetic is the six-scheme form's, so with c held in the kernel's type
// the two forms give the same bits.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_lattice.cuh"

namespace lbm {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3 };

// Physics constants of one launch in the kernel's arithmetic type, so that no
// thread converts from double (FP64 units are scarce on this GPU).
template <class R> struct PhysT {
  R R_, invR, omega_g, omega_l, omega_a, kgrad;  // kgrad = omega_alpha / cs2
  R A_g, B_g, A_l, B_l;                          // sigma = A (Pi^eq - Pi) + B S'' I
  R eta0_g, eta0_l, psi_g, psi_l, k0;            // eta_q(psi) rest / moving; (1-w0)/w0
  R kappa_I, kappa_W, buoy, gamma, afloor;
  R r_ag, r_al;                                  // deviation references of f_alpha
  R rsum1;                                       // r_ag + r_al - 1 of the references above
  R aIN, ugIN, ulIN;                             // inlet values at this t
};

// Per-launch arguments (everything the fused step and the moment kernels need).
struct StepArgs {
  void *pop;            // 6*Q planes of the store type
  void *held;           // 3 planes: S''_g, S''_l, Lambda' (float, or double for FP64)
  long long plane;      // elements per plane (>= N, padded)
  int n[3];             // nx, ny, nz
  int shift[3];         // tile shift per axis (keeps edge pairs in one block)
  int T[3];             // tile sizes (blockDim)
  int parity;           // t & 1
  int latch;            // t % n_gamma == 0
  int bc_lo[3], bc_hi[3];
  int g_axis, tr_axis;  // gravity / inlet-normal axis, first transverse axis (-1 in 1D)
  int inlet_lo, inlet_hi;
  int has_inlet, has_outlet;
  void *cfield;         // beta-stencil form: 2 buffers x 2*D planes of c (held type)
  int beta_own;         // beta-stencil form, first step after init: every q from the node's own c
  int halo_off;         // beta-stencil form: byte offset of the block's c halo in dynamic shared memory
  int off32;            // Q*plane < 2^32: population offsets fit 32 bits
  // physics
  double invR, R, omega_g, omega_l, omega_a, kgrad;  // kgrad = omega_alpha / cs2
  double A_g, B_g, A_l, B_l;                         // sigma = A (Pi^eq - Pi) + B S'' I
  double eta0_g, eta0_l, psi_g, psi_l;               // eta_q(psi): rest / moving
  double k0;                                         // (1 - w_0)/w_0 of Eq. (eta)
  double kappa_I, kappa_W, buoy, gamma, afloor;
  int cgw, spalding;
  double r_ag, r_al;                                 // deviation references of f_alpha
  double aIN, ugIN, ulIN;                            // inlet values at this t, Eq. (transient)
  // reference (FP64, full-population) path
  int plain;                                         // store holds full f, not deviations
  double cs2, two_cs4, nuef_g, nuef_l;               // 1/3, 2 cs2 cs2, nu_ef of Eq. (lbm-ef-viscosity)
  PhysT<float> pf;                                   // the constants above, pre-converted
  PhysT<double> pd;
};

template <class R> __device__ __forceinline__ const PhysT<R> &phys(const StepArgs &a);
template <> __device__ __forceinline__ const PhysT<float> &phys<float>(const StepArgs &a) { return a.pf; }
template <> __device__ __forceinline__ const PhysT<double> &phys<double>(const StepArgs &a) { return a.pd; }

// ------------------------------------------------------------ store access

template <class S> struct Store;
// ld / st: the deviation in the arithmetic type; ld_raw: the stored value
// times `scale` (the step kernel works in those units, see fused_step_node).
template <> struct Store<double> {
  static constexpr double scale = 1.0;
  template <class R> __device__ __forceinline__ static R ld(const double *p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static R ld_raw(const double *p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static void st(double *p, R v) { *p = (double)v; }
};
template <> struct Store<float> {
  static constexpr float scale = 1.0f;
  template <class R> __device__ __forceinline__ static R ld(const float *p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static R ld_raw(const float *p) { return (R)__ldg(p); }
  template <class R> __device__ __forceinline__ static void st(float *p, R v) { *p = (float)v; }
};
// Half store of deviations scaled by 2^12 (exact): |f - w r| < 1 < 65504/2^12,
// and deviations down to 1.5e-8 stay normal numbers (11-bit significand)
// instead of half subnormals (absolute spacing 6e-8).  The six schemes are
// stored in pairs (g, l), (alpha_g, alpha_l), (beta_g, beta_l): plane
// (p*Q + q) of half2 words holds direction q of pair p, so one 32-bit access
// moves the two schemes of a pair (pop_elem below gives one scheme's half).
constexpr float HALF_SCALE = 4096.0f, HALF_UNSCALE = 1.0f / 4096.0f;
template <> struct Store<__half> {
  static constexpr float scale = HALF_SCALE;
  template <class R> __device__ __forceinline__ static R ld(const __half *p) {
    return (R)(__half2float(__ldg(p)) * HALF_UNSCALE);
  }
  template <class R> __device__ __forceinline__ static void st(__half *p, R v) {
    *p = __float2half_rn((float)v * HALF_SCALE);
  }
};

// The FP16AB store: f_g and f_l in float (planes q and Q + q), then the
// pairs (alpha_g, alpha_l) and (beta_g, beta_l) as half2 words scaled like
// the half store (planes 2Q + p*Q + q in units of 4 bytes).  The registers
// hold every population unscaled (scale 1); the half pairs are scaled on
// load and store.  The tag's size (4) makes the held fields and c float.
struct MixAB {
  float tag;
};
template <> struct Store<MixAB> {
  static constexpr float scale = 1.0f;
};

// Element of scheme s at offset qoff = pq*plane + node of a store of Q*plane
// elements per scheme (half: the scheme's half of its pair's half2 word).
template <class S>
__device__ __forceinline__ S *pop_elem(void *pop, int s, long long qoff, long long Qplane) {
  if (sizeof(S) == 2) return (S *)pop + ((((long long)(s >> 1)) * Qplane + qoff) << 1) + (s & 1);
  return (S *)pop + (long long)s * Qplane + qoff;
}
// half element of scheme s >= 2 of the FP16AB store
__device__ __forceinline__ __half *mix_half_elem(void *pop, int s, long long qoff, long long Qplane) {
  __half *hb = (__half *)((float *)pop + 2 * Qplane);
  return hb + ((((long long)((s - 2) >> 1)) * Qplane + qoff) << 1) + ((s - 2) & 1);
}
// The deviation stored for scheme s at qoff, in double (readout, init).
template <class S>
__device__ __forceinline__ double pop_ld(void *pop, int s, long long qoff, long long Qplane) {
  if constexpr (std::is_same<S, MixAB>::value) {
    if (s < 2) return (double)__ldg((const float *)pop + (long long)s * Qplane + qoff);
    return Store<__half>::ld<double>(mix_half_elem(pop, s, qoff, Qplane));
  } else {
    return Store<S>::template ld<double>(pop_elem<S>(pop, s, qoff, Qplane));
  }
}
template <class S>
__device__ __forceinline__ void pop_st(void *pop, int s, long long qoff, long long Qplane, double v) {
  if constexpr (std::is_same<S, MixAB>::value) {
    if (s < 2) ((float *)pop)[(long long)s * Qplane + qoff] = (float)v;
    else Store<__half>::st<double>(mix_half_elem(pop, s, qoff, Qplane), v);
  } else {
    Store<S>::template st<double>(pop_elem<S>(pop, s, qoff, Qplane), v);
  }
}

// Node geometry: index, offsets (in nodes, 32-bit) of the +1 / -1 neighbour
// along each axis with periodic wrap, and whether a step leaves the domain
// through a non-periodic face.  The library keeps N < 2^31.
struct Geo {
  int c[3];
  int op[3], om[3];      // node offset of the +1 / -1 neighbour (wrapped)
  bool xp[3], xm[3];     // +1 / -1 step crosses a non-periodic face
  int node;
};

__device__ __forceinline__ void make_geo(const StepArgs &a, int D, Geo &g) {
  int stride = 1;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int n = a.n[d], c = g.c[d];
    g.op[d] = stride;
    g.om[d] = -stride;
    g.xp[d] = false;
    g.xm[d] = false;
    if (d < D) {
      if (c + 1 >= n) {
        if (a.bc_hi[d] == BC_PERIODIC) g.op[d] = -(n - 1) * stride; else g.xp[d] = true;
      }
      if (c == 0) {
        if (a.bc_lo[d] == BC_PERIODIC) g.om[d] = (n - 1) * stride; else g.xm[d] = true;
      }
    }
    stride *= n;
  }
  g.node = g.c[0] + a.n[0] * (g.c[1] + a.n[1] * g.c[2]);
}

template <class L>
__device__ __forceinline__ long long shifted_node(const StepArgs &a, const Geo &g, int q, int sign) {
  // node index of x + sign*v_q with periodic wrap (only valid if not crossing)
  int idx = g.node;
#pragma unroll
  for (int d = 0; d < L::D; d++) {
    const int vv = sign * L::v(q, d);
    idx += vv > 0 ? g.op[d] : (vv < 0 ? g.om[d] : 0);
  }
  return idx;
}

template <class L>
__device__ __forceinline__ bool crosses(const Geo &g, int q, int sign) {
  bool x = false;
#pragma unroll
  for (int d = 0; d < L::D; d++) {
    int vv = sign * L::v(q, d);
    x = x || (vv > 0 && g.xp[d]) || (vv < 0 && g.xm[d]);
  }
  return x;
}

// Face rule for a population leaving the node along q (requires crosses(+1)):
// a wall on any crossed face wins; the inlet face acts as a wall outside the
// strip.
template <class L>
__device__ __forceinline__ int face_rule(const StepArgs &a, const Geo &g, int q) {
  int rule = -1;
#pragma unroll
  for (int d = 0; d < L::D; d++) {
    int vv = L::v(q, d);
    int bc = -1;
    if (vv > 0 && g.xp[d]) bc = a.bc_hi[d];
    if (vv < 0 && g.xm[d]) bc = a.bc_lo[d];
    if (bc == BC_INLET && a.tr_axis >= 0) {
      const int ct = a.tr_axis == 0 ? g.c[0] : (a.tr_axis == 1 ? g.c[1] : g.c[2]);
      if (ct < a.inlet_lo || ct >= a.inlet_hi) bc = BC_WALL;
    }
    if (bc >= 0 && (rule < 0 || bc == BC_WALL)) rule = bc;
  }
  return rule;
}

// Slot of the read of direction q (AA rule, see the file comment).  INT:
// the node is known to have no non-periodic face within one step.
template <class L, bool INT = false>
__device__ __forceinline__ long long read_slot(const StepArgs &a, const Geo &g, int q, int parity, int &plane_q) {
  if (parity == 0) {
    plane_q = q;
    return g.node;
  }
  if (!INT && crosses<L>(g, q, -1)) {
    plane_q = q;
    return g.node;
  }
  plane_q = L::opp(q);
  return shifted_node<L>(a, g, q, -1);
}

// Slot of the write of the post-collision population of direction q.
template <class L>
__device__ __forceinline__ long long write_slot(const StepArgs &a, const Geo &g, int q, bool cross, int parity,
                                                int &plane_q) {
  if (parity == 0 || cross) {
    plane_q = L::opp(q);
    return g.node;
  }
  plane_q = q;
  return shifted_node<L>(a, g, q, +1);
}

// v_q . u
template <class L, class R>
__device__ __forceinline__ R vdot(int q, const R u[3]) {
  R s = R(0);
#pragma unroll
  for (int d = 0; d < L::D; d++) {
    const int vd = L::v(q, d);
    if (vd == 1) s += u[d];
    if (vd == -1) s -= u[d];
  }
  return s;
}

template <class L, class R> __device__ __forceinline__ R feqS_dv(int q, R alpha, R alpha_dev, const R u[3], R uu);
template <class L> __device__ __forceinline__ int face_rule(const StepArgs &a, const Geo &g, int q);

// Beta-stencil form: c_g, c_l of the last step at node `node` (buffer `buf`).
template <class L, class S, class R>
__device__ __forceinline__ void load_c(const StepArgs &a, int buf, long long node, R cg[3], R cl[3]) {
  typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
  const H *cb = (const H *)a.cfield + (long long)buf * 2 * L::D * a.plane;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    cg[d] = d < L::D ? (R)__ldg(cb + d * a.plane + node) : R(0);
    cl[d] = d < L::D ? (R)__ldg(cb + (L::D + d) * a.plane + node) : R(0);
  }
}

// Operations rounded one by one, which the compiler neither fuses nor reorders.
template <class R> struct Rn;
template <> struct Rn<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Rn<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// v_q . u = s + e exactly: the sum of its at most two nonzero terms
// (D2Q9, D3Q19 diagonals) as a two-sum, e = 0 along the axes.
template <class L, class R>
__device__ __forceinline__ void vdot2(int q, const R u[3], R &s, R &e) {
  R t[2] = {R(0), R(0)};
  int n = 0;
#pragma unroll
  for (int d = 0; d < L::D; d++) {
    const int vd = L::v(q, d);
    if (vd != 0 && n < 2) t[n++] = vd > 0 ? u[d] : -u[d];
  }
  s = Rn<R>::add(t[0], t[1]);
  const R bb = Rn<R>::add(s, -t[0]);
  e = Rn<R>::add(Rn<R>::add(t[0], -Rn<R>::add(s, -bb)), Rn<R>::add(t[1], -bb));
}

// f^eq(1, c)_q - w_q of the beta schemes (Eq. (equilibrium) with alpha = 1),
// in explicitly rounded steps: the six-scheme store evaluates it on the write
// side and the beta-stencil form on the read side, and both must give the
// same bits.
template <class L, class R>
__device__ __forceinline__ R beta_c2(const R c[3]) {
  R c2 = R(0);
#pragma unroll
  for (int d = 0; d < L::D; d++) c2 = Rn<R>::fma(c[d], c[d], c2);
  return c2;
}
// even part w_q (9/2 (v.c)^2 - 3/2 c^2), the same for q and opp(q); vc = v_q . c
template <class L, class R>
__device__ __forceinline__ R beta_even(int q, const R c[3], R c2, R &vc) {
  vc = vdot<L, R>(q, c);
  const R t = Rn<R>::fma(Rn<R>::mul(R(4.5), vc), vc, Rn<R>::mul(R(-1.5), c2));
  return Rn<R>::mul(wq<L, R>(q), t);
}
template <class L, class R>
__device__ __forceinline__ R beta_dev(int q, const R c[3]) {
  R vc;
  const R x = beta_even<L, R>(q, c, beta_c2<L, R>(c), vc);
  return Rn<R>::fma(aq<L, R>(q), vc, x);
}

template <class L, class R>
__device__ __forceinline__ void beta_pair(int q, const R cg[3], const R cl[3], R &bg, R &bl) {
  bg = beta_dev<L, R>(q, cg);
  bl = beta_dev<L, R>(q, cl);
}

// Beta-stencil form, step kernel: the block's tile of c (the last step's,
// buffer 1 - parity) plus a one-node halo, staged once in shared memory, so
// that the 2*D values of c at every x - v_q come from there instead of global
// memory.  Node (lx, ly, lz) of the halo box is tile node (lx - 1, ly - 1,
// lz - 1); its values lie together, c_g then c_l, at p[k*HaloStride + ..]
// (2*D padded to a multiple of 4 values: one or two 16-byte loads for FP32).
template <class L>
struct HaloStride {
  static constexpr int v = (2 * L::D + 3) / 4 * 4;
};
struct CHalo {
  const void *p;  // nullptr: read c from global memory
  int hx, hy, hn;  // box extent along x, y; nodes in the box
  int k;           // this thread's node in the box
};

template <class L, class S, class R>
__device__ __forceinline__ void halo_c(const CHalo &h, int k, R cg[3], R cl[3]) {
  typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
  constexpr int NV = HaloStride<L>::v;
  H v[NV];
  if constexpr (std::is_same<H, float>::value) {
    const float4 *p = (const float4 *)h.p + (long long)k * (NV / 4);
#pragma unroll
    for (int j = 0; j < NV / 4; j++) {
      const float4 t = p[j];
      v[4 * j] = t.x;
      v[4 * j + 1] = t.y;
      v[4 * j + 2] = t.z;
      v[4 * j + 3] = t.w;
    }
  } else {
    const double2 *p = (const double2 *)h.p + (long long)k * (NV / 2);
#pragma unroll
    for (int j = 0; j < NV / 2; j++) {
      const double2 t = p[j];
      v[2 * j] = t.x;
      v[2 * j + 1] = t.y;
    }
  }
#pragma unroll
  for (int d = 0; d < 3; d++) {
    cg[d] = d < L::D ? (R)v[d] : R(0);
    cl[d] = d < L::D ? (R)v[L::D + d] : R(0);
  }
}

// Fill the block's halo box (all threads of the block; the caller
// synchronises).  Nodes beyond a non-periodic face are never read (those
// directions take the face rules) and are left unset.
template <class L, class S>
__device__ __forceinline__ void stage_c_halo(const StepArgs &a, void *box, int hx, int hy, int hn, const int o[3],
                                             int tid, int nthr) {
  typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
  const H *cb = (const H *)a.cfield + (long long)(1 - a.parity) * 2 * L::D * a.plane;
  H *p = (H *)box;
  // one warp per row of the box (x contiguous), lanes along x
  const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
  const int rows = hn / hx;
  for (int r = warp; r < rows; r += nwarp) {
    int c1 = L::D > 1 ? o[1] - 1 + r % hy : 0, c2 = L::D > 2 ? o[2] - 1 + r / hy : 0;
    bool ok = true;
    if (L::D > 1 && (c1 < 0 || c1 >= a.n[1])) {
      if (a.bc_lo[1] == BC_PERIODIC) c1 = c1 < 0 ? c1 + a.n[1] : c1 - a.n[1];
      else ok = false;
    }
    if (L::D > 2 && (c2 < 0 || c2 >= a.n[2])) {
      if (a.bc_lo[2] == BC_PERIODIC) c2 = c2 < 0 ? c2 + a.n[2] : c2 - a.n[2];
      else ok = false;
    }
    if (!ok) continue;
    const long long row = (long long)a.n[0] * (c1 + (long long)a.n[1] * c2);
    for (int lx = lane; lx < hx; lx += 32) {
      int c0 = o[0] - 1 + lx;
      if (c0 < 0 || c0 >= a.n[0]) {
        if (a.bc_lo[0] != BC_PERIODIC) continue;
        c0 = c0 < 0 ? c0 + a.n[0] : c0 - a.n[0];
      }
      const int k = r * hx + lx;
#pragma unroll
      for (int d = 0; d < 2 * L::D; d++) p[k * HaloStride<L>::v + d] = cb[d * a.plane + row + c0];
    }
  }
}

// Beta-stencil form: the beta deviations arriving at the node along every q,
// as the six-scheme store would hold them (the write side of the step that
// produced c, replayed); c from the block's halo box when h.p is set.
template <class L, class S, class R>
__device__ __forceinline__ void load_beta(const StepArgs &a, const Geo &g, int parity, R fbg[L::Q], R fbl[L::Q],
                                          const CHalo &h = CHalo{nullptr, 0, 0, 0, 0}) {
  const int buf = 1 - parity;
  R cg0[3], cl0[3];
  if (h.p) halo_c<L, S, R>(h, h.k, cg0, cl0);
  else load_c<L, S, R>(a, buf, g.node, cg0, cl0);
#pragma unroll
  for (int q = 0; q < L::Q; q++) {
    const int qo = L::opp(q);
    if (a.beta_own) {
      beta_pair<L, R>(q, cg0, cl0, fbg[q], fbl[q]);   // initial state: f^eq(1, c(x))
    } else if (!crosses<L>(g, q, -1)) {
      R cg[3], cl[3];
      if (h.p)
        halo_c<L, S, R>(h, h.k - (L::v(q, 0) + h.hx * (L::v(q, 1) + h.hy * L::v(q, 2))), cg, cl);
      else
        load_c<L, S, R>(a, buf, shifted_node<L>(a, g, q, -1), cg, cl);
      beta_pair<L, R>(q, cg, cl, fbg[q], fbl[q]);     // streamed from x - v_q
    } else {
      const int rule = face_rule<L>(a, g, qo);          // the rule that sent opp(q) back
      if (rule == BC_INLET || rule == BC_OUTLET) {
        // Tables 1-2: f_beta EQ(S) with c extrapolated full-way from the
        // inward neighbour along the face normal
        const int gax = a.g_axis;
        int st = gax == 0 ? 1 : (gax == 1 ? a.n[0] : a.n[0] * a.n[1]);
        if (rule == BC_OUTLET) st = -st;
        R cgn[3], cln[3], cb[3], cc[3];
        load_c<L, S, R>(a, buf, g.node + st, cgn, cln);
#pragma unroll
        for (int d = 0; d < 3; d++) {
          cb[d] = R(2) * cg0[d] - cgn[d];
          cc[d] = R(2) * cl0[d] - cln[d];
        }
        beta_pair<L, R>(q, cb, cc, fbg[q], fbl[q]);
      } else {
        beta_pair<L, R>(qo, cg0, cl0, fbg[q], fbl[q]);  // half-way bounce-back
      }
    }
  }
}

// Address of a population: the base of scheme s, base + s*Q*plane (the same
// for every thread of the launch), plus one offset pq*plane + node per
// direction, formed once and shared by the schemes.  OffT is the offset's
// type: 32-bit unsigned when Q*plane < 2^32 (fewer address instructions),
// else 64-bit.  With the bases hoisted (load_node) this raised the D2Q9 FP32
// step from 11.4 to 13.5 GLUPS on the 512 x 2048 box.
template <class L, class OffT>
__device__ __forceinline__ OffT pop_offset(const StepArgs &a, int pq, long long idx) {
  return (OffT)pq * (OffT)a.plane + (OffT)idx;
}
template <class L, class S>
__device__ __forceinline__ const S *scheme_base(const StepArgs &a, int s) {
  return (const S *)a.pop + (long long)(s * L::Q) * a.plane;
}

// The node's populations in registers, raw (deviations times
// Store<S>::scale).  get(s, q): population q of scheme s in the arithmetic
// type (constant s, q after unrolling).  Float and double stores hold them as
// R values.  The half store keeps each pair (g, l), (alpha_g, alpha_l),
// (beta_g, beta_l) packed in one half2 register as loaded (57 registers
// instead of 114 for D3Q19), converts a value where the collision uses it and
// sums the moments from the halves directly (moment_sums); in the
// beta-stencil form the beta values, re-evaluated from c in float, stay
// float.
template <class L, class S, class R, bool BS> struct Pops {
  R f[6][L::Q];
  __device__ __forceinline__ R get(int s, int q) const { return f[s][q]; }
};
template <class L, class R, bool BS> struct Pops<L, MixAB, R, BS> {
  R f[2][L::Q];
  __half2 h[BS ? 1 : 2][L::Q];
  R fb[2][BS ? L::Q : 1];
  __device__ __forceinline__ R get(int s, int q) const {
    if (s < 2) return f[s][q];
    if (BS && s >= 4) return fb[s - 4][q];
    const __half2 x = h[(s - 2) >> 1][q];
    return (R)(((s & 1) ? __high2float(x) : __low2float(x)) * HALF_UNSCALE);
  }
};
template <class L, class R, bool BS> struct Pops<L, __half, R, BS> {
  __half2 h[BS ? 2 : 3][L::Q];
  R fb[2][BS ? L::Q : 1];
  __device__ __forceinline__ R get(int s, int q) const {
    if (BS && s >= 4) return fb[s - 4][q];
    return (R)((s & 1) ? __high2float(h[s >> 1][q]) : __low2float(h[s >> 1][q]));
  }
};

// Load all populations of the node with the AA read rule (INT: an interior
// node, see read_slot), as raw values: deviations times Store<S>::scale.
// The beta populations of the beta-stencil form into the node's Pops (in
// the store's raw units).
template <class L, class S, class R, bool BS>
__device__ __forceinline__ void load_node_beta(const StepArgs &a, const Geo &g, int parity, Pops<L, S, R, BS> &f,
                                               const CHalo &h) {
  if constexpr (!BS) return;
  else if constexpr (std::is_same<S, MixAB>::value) {
    load_beta<L, S, R>(a, g, parity, f.fb[0], f.fb[1], h);
  } else if constexpr (sizeof(S) == 2) {
    load_beta<L, S, R>(a, g, parity, f.fb[0], f.fb[1], h);
#pragma unroll
    for (int q = 0; q < L::Q; q++) {
      f.fb[0][q] *= (R)Store<S>::scale;
      f.fb[1][q] *= (R)Store<S>::scale;
    }
  } else {
    load_beta<L, S, R>(a, g, parity, f.f[4], f.f[5], h);
  }
}

// LB: the beta-stencil form's beta populations too (else the caller adds
// them with load_node_beta, once the c halo is in shared memory).
template <class L, class S, class R, bool BS = false, class OffT = long long, bool INT = false, bool LB = true>
__device__ __forceinline__ void load_node(const StepArgs &a, const Geo &g, int parity, Pops<L, S, R, BS> &f,
                                          const CHalo &h = CHalo{nullptr, 0, 0, 0, 0}) {
  if constexpr (std::is_same<S, MixAB>::value) {
    // f_g, f_l from the float planes, the alpha (and beta) pairs as half2
    const float *gb = (const float *)a.pop;
    const long long Qp = (long long)L::Q * a.plane;
    const __half2 *hb = (const __half2 *)(gb + 2 * Qp);
#pragma unroll
    for (int q = 0; q < L::Q; q++) {
      int pq;
      const long long idx = read_slot<L, INT>(a, g, q, parity, pq);
      const OffT off = pop_offset<L, OffT>(a, pq, idx);
      f.f[0][q] = (R)__ldg(gb + off);
      f.f[1][q] = (R)__ldg(gb + Qp + off);
#pragma unroll
      for (int p = 0; p < (BS ? 1 : 2); p++) f.h[p][q] = __ldg(hb + p * Qp + off);
    }
  } else if constexpr (sizeof(S) == 2) {
    // half pairs: one 32-bit load per (pair, direction)
    const __half2 *pb[3];
#pragma unroll
    for (int p = 0; p < 3; p++) pb[p] = (const __half2 *)a.pop + (long long)(p * L::Q) * a.plane;
#pragma unroll
    for (int q = 0; q < L::Q; q++) {
      int pq;
      const long long idx = read_slot<L, INT>(a, g, q, parity, pq);
      const OffT off = pop_offset<L, OffT>(a, pq, idx);
#pragma unroll
      for (int p = 0; p < (BS ? 2 : 3); p++) f.h[p][q] = __ldg(pb[p] + off);
    }
  } else {
    // the scheme bases formed once, before the loads (left inside the loop
    // they cost the D2Q9 FP32 step 90 instead of 78 us on the 512 x 2048 box)
    const S *sb[6];
#pragma unroll
    for (int s = 0; s < 6; s++) sb[s] = scheme_base<L, S>(a, s);
#pragma unroll
    for (int q = 0; q < L::Q; q++) {
      int pq;
      const long long idx = read_slot<L, INT>(a, g, q, parity, pq);
      const OffT off = pop_offset<L, OffT>(a, pq, idx);
#pragma unroll
      for (int s = 0; s < (BS ? 4 : 6); s++) f.f[s][q] = Store<S>::template ld_raw<R>(sb[s] + off);
    }
  }
  if constexpr (BS && LB) load_node_beta<L, S, R, BS>(a, g, parity, f, h);
}

// ------------------------------------------------------------- moments

template <class L, class R> struct Moments {
  R deg, del;            // eps_g - 1, eps_l - 1
  R ug[3], ul[3];
  R Pg[6], Pl[6];        // Pi - cs2 I, packed xx, yy, zz, xy, xz, yz
  R ag, al, Jg[3], Jl[3];
  R dag, dal;            // a - r (sums of the alpha deviations)
  R esum;                // sum_q (f_alpha_g + f_alpha_l) deviations: a_g + a_l - (r_g + r_l)
  R Sg, Sl;              // 1 - beta
  R alg, all;            // alpha^B
  R dalg, dall;          // alpha^B - r
  R cg, cl;              // alpha^B - a, the renormalisation of Eq. (spalding), kept unrounded by a
};

__host__ __device__ constexpr int pidx(int a, int b) {
  return a == b ? a : ((a + b == 1) ? 3 : ((a + b == 2) ? 4 : 5));
}

// Raw sums of the moments in the arithmetic type.  The moving directions
// are taken in pairs (q, opp q): the first moments sum the pair differences
// f_q - f_opp(q) and the zeroth and second moments the pair sums.  The even
// parts of a pair (w (eps - 1), w (alpha - r), the quadratic terms) cancel in
// the difference before anything is rounded, so a first moment keeps the
// precision of its own size instead of the spacing of the populations --
// J = sum v f_alpha is ~1e-3 beside populations of 0.3 w in a gas plume.
// esum adds f_alpha_g + f_alpha_l direction by direction: the two deviations
// nearly cancel (alpha_l = 1 - alpha_g), so a_g + a_l - 1 of Eq. (spalding)
// is formed without the spacing of a_g.  (The rounding of the zeroth sums
// does not move mass: the collision's rest direction takes the remainder,
// see collide_all.)
template <class L, class S, class R, bool BS>
__device__ __forceinline__ void moment_sums(const Pops<L, S, R, BS> &P, Moments<L, R> &m) {
  constexpr int D = L::D;
  m.deg = P.get(0, 0);
  m.del = P.get(1, 0);
  m.ag = P.get(2, 0);
  m.al = P.get(3, 0);
  m.Sg = -P.get(4, 0);
  m.Sl = -P.get(5, 0);
  m.esum = P.get(2, 0) + P.get(3, 0);
#pragma unroll
  for (int d = 0; d < 3; d++) m.ug[d] = m.ul[d] = m.Jg[d] = m.Jl[d] = R(0);
#pragma unroll
  for (int k = 0; k < 6; k++) m.Pg[k] = m.Pl[k] = R(0);
#pragma unroll
  for (int q = 1; q < L::Q; q++) {
    const int qo = L::opp(q);
    if (q > qo) continue;
    R sm[6], df[4];
#pragma unroll
    for (int s = 0; s < 6; s++) sm[s] = P.get(s, q) + P.get(s, qo);
#pragma unroll
    for (int s = 0; s < 4; s++) df[s] = P.get(s, q) - P.get(s, qo);
    m.deg += sm[0];
    m.del += sm[1];
    m.ag += sm[2];
    m.al += sm[3];
    m.Sg -= sm[4];
    m.Sl -= sm[5];
    m.esum += (P.get(2, q) + P.get(3, q)) + (P.get(2, qo) + P.get(3, qo));
#pragma unroll
    for (int d = 0; d < D; d++) {
      const int vd = L::v(q, d);
      if (vd != 0) {
        m.ug[d] += vd * df[0];
        m.ul[d] += vd * df[1];
        m.Jg[d] += vd * df[2];
        m.Jl[d] += vd * df[3];
      }
#pragma unroll
      for (int e = d; e < D; e++) {
        const int ve = L::v(q, e);
        if (vd * ve != 0) {
          m.Pg[pidx(d, e)] += (vd * ve) * sm[0];
          m.Pl[pidx(d, e)] += (vd * ve) * sm[1];
        }
      }
    }
  }
}

// acc +/- x for a half x, in one mixed-precision instruction (sm_100 and
// later): the exact conversion of x and one rounding, as acc + (float)x.
__device__ __forceinline__ void hacc(float &acc, __half x, int sign) {
  const unsigned short b = __half_as_ushort(x);
  if (sign > 0) asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc) : "h"(b));
  else asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(acc) : "h"(b), "h"((unsigned short)0xBC00));  // -1.0
}

// The same sums from the packed half pairs (same order, same roundings: each
// term is exact in float, so acc +/- x rounds once as in the float form).
template <class L, class R, bool BS>
__device__ __forceinline__ void moment_sums(const Pops<L, __half, R, BS> &P, Moments<L, R> &m) {
  static_assert(std::is_same<R, float>::value, "the half store computes in float");
  constexpr int D = L::D;
  m.deg = m.del = m.ag = m.al = m.Sg = m.Sl = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) m.ug[d] = m.ul[d] = m.Jg[d] = m.Jl[d] = R(0);
#pragma unroll
  for (int k = 0; k < 6; k++) m.Pg[k] = m.Pl[k] = R(0);
#pragma unroll
  for (int q = 0; q < L::Q; q++) {
    const __half g = __low2half(P.h[0][q]), l = __high2half(P.h[0][q]);
    const __half ag = __low2half(P.h[1][q]), al = __high2half(P.h[1][q]);
    hacc(m.deg, g, 1);
    hacc(m.del, l, 1);
    hacc(m.ag, ag, 1);
    hacc(m.al, al, 1);
    if constexpr (BS) {
      m.Sg -= P.fb[0][q];
      m.Sl -= P.fb[1][q];
    } else {
      hacc(m.Sg, __low2half(P.h[2][q]), -1);
      hacc(m.Sl, __high2half(P.h[2][q]), -1);
    }
#pragma unroll
    for (int d = 0; d < D; d++) {
      const int vd = L::v(q, d);
      if (vd != 0) {
        hacc(m.ug[d], g, vd);
        hacc(m.ul[d], l, vd);
        hacc(m.Jg[d], ag, vd);
        hacc(m.Jl[d], al, vd);
      }
#pragma unroll
      for (int e = d; e < D; e++) {
        const int ve = L::v(q, e);
        if (vd * ve != 0) {
          hacc(m.Pg[pidx(d, e)], g, vd * ve);
          hacc(m.Pl[pidx(d, e)], l, vd * ve);
        }
      }
    }
  }
}

template <class L, class S, class R, bool BS>
__device__ __forceinline__ void moments(const StepArgs &a, const Pops<L, S, R, BS> &f, Moments<L, R> &m) {
  const PhysT<R> &P = phys<R>(a);
  moment_sums<L>(f, m);
  // the populations arrive as raw values (times Store<S>::scale, a power of
  // two): the sums are scaled back exactly
  constexpr R US = R(1) / (R)Store<S>::scale;
  if constexpr (sizeof(S) == 2) m.esum = m.ag + m.al;  // unscaled below with them
  if (US != R(1)) {
    m.esum *= US;
    m.deg *= US;
    m.del *= US;
    m.ag *= US;
    m.al *= US;
    m.Sg *= US;
    m.Sl *= US;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      m.ug[d] *= US;
      m.ul[d] *= US;
      m.Jg[d] *= US;
      m.Jl[d] *= US;
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
      m.Pg[k] *= US;
      m.Pl[k] *= US;
    }
  }
  m.dag = m.ag;
  m.dal = m.al;
  m.ag += P.r_ag;
  m.al += P.r_al;
  m.cg = m.cl = R(0);
  if (a.spalding == 0) {
    m.alg = m.ag;
    m.all = m.al;
    m.dalg = m.dag;
    m.dall = m.dal;
  } else {
    // Eq. (spalding) with B(x) = x clamped to [0, 1].  Inside [0, 1] the
    // normalisation is formed in deviations, alpha^B - r = (a - r) - a e/(1 + e)
    // with e = a_g + a_l - 1 = (a_g - r_g) + (a_l - r_l) + (r_g + r_l - 1), so
    // the small quantities keep their own precision instead of the spacing of
    // alpha^B itself.
    // The renormalisation itself, alpha^B - a = -a e/(1 + e), is kept as a
    // number of its own (cg, cl): a few 1e-10 in a gas plume, far below the
    // spacing of a - r (3e-8 at 0.3), it would vanish if added to a - r in
    // float, and the alpha equilibria take it separately (collide_all).
    if (m.ag >= R(0) && m.ag <= R(1) && m.al >= R(0) && m.al <= R(1) && m.ag + m.al > R(0)) {
      const R e = m.esum + P.rsum1;
      const R k = e / (R(1) + e);
      m.cg = -m.ag * k;
      m.cl = -m.al * k;
      m.dalg = m.dag + m.cg;
    } else {
      R Bg = m.ag < R(0) ? R(0) : (m.ag > R(1) ? R(1) : m.ag);
      R Bl = m.al < R(0) ? R(0) : (m.al > R(1) ? R(1) : m.al);
      R sum = Bg + Bl;
      m.dalg = (sum > R(0) ? Bg / sum : R(0.5)) - P.r_ag;
      m.cg = m.dalg - m.dag;
      m.cl = (-m.dalg - P.rsum1) - m.dal;
    }
    m.dall = -m.dalg - P.rsum1;  // alpha^B_l = 1 - alpha^B_g
    m.alg = P.r_ag + m.dalg;
    m.all = P.r_al + m.dall;
  }
}

// ------------------------------------------------------------ fused step


// f^eq(alpha, u)_q - w_q*r with the quadratic term of Eq. (equilibrium),
// grouped as w [(alpha - r) + alpha (9/2 (v.u)^2 - 3/2 u^2)] + alpha a_q v.u
// (a_q = w_q / cs2, see lbm_lattice.cuh) so that
// alpha = r (the beta schemes, r = 1) loses nothing to cancellation.
template <class L, class R>
__device__ __forceinline__ R feqS_dv(int q, R alpha, R alpha_dev, const R u[3], R uu) {
  const R w = wq<L, R>(q);
  const R vu = vdot<L, R>(q, u);
  return w * (alpha_dev + alpha * (R(4.5) * vu * vu - R(1.5) * uu)) + alpha * (aq<L, R>(q) * vu);
}
// the same with alpha - r formed here
template <class L, class R>
__device__ __forceinline__ R feqS_dev(int q, R alpha, const R u[3], R uu, R r) {
  return feqS_dv<L, R>(q, alpha, alpha - r, u, uu);
}

// Values a face rule streams back into the node, as deviations.  xn holds the
// extrapolation neighbour's values: [0..2] u_g, [3..5] u_l, [6] alpha^B_g,
// [7] alpha^B_l, [8..10] c_g, [11..13] c_l.
constexpr int XCH = 14;

// Launch bounds of the fused step.  D2Q9 in float/half: at most 128 threads
// and 5 resident blocks per SM, which caps registers at 102 (no spills) and
// gives 20 warps per SM -- the kernel is memory-latency bound, and this
// occupancy measured 11.8 GLUPS on the 512 x 2048 box against 11.1 GLUPS at
// 104 registers / 16 warps (128 x 4, 128 x 6 and 256 x 3 were slower too).
// D3Q19 in float/half: 128 threads, 3 blocks per SM (168 registers, a few
// spills, 12 warps per SM); on the 256 x 256 x 512 column this measured
// 6.11 / 4.85 GLUPS (FP16 / FP32 store) against 5.44 / 4.67 GLUPS with
// 256 x 1 (249 registers, 8 warps).  The double forms keep 256 threads.
template <class L, class S> struct StepBounds { static constexpr int threads = 256, blocks = 1; };
template <> struct StepBounds<Lattice<3>, float> { static constexpr int threads = 128, blocks = 3; };
template <> struct StepBounds<Lattice<3>, __half> { static constexpr int threads = 128, blocks = 5; };
template <> struct StepBounds<Lattice<2>, float> { static constexpr int threads = 128, blocks = 5; };
template <> struct StepBounds<Lattice<2>, __half> { static constexpr int threads = 128, blocks = 5; };
template <> struct StepBounds<Lattice<1>, float> { static constexpr int threads = 128, blocks = 4; };
template <> struct StepBounds<Lattice<1>, __half> { static constexpr int threads = 128, blocks = 4; };
template <> struct StepBounds<Lattice<3>, MixAB> { static constexpr int threads = 128, blocks = 4; };
template <> struct StepBounds<Lattice<2>, MixAB> { static constexpr int threads = 128, blocks = 5; };
template <> struct StepBounds<Lattice<1>, MixAB> { static constexpr int threads = 128, blocks = 4; };

// One node of the fused step (rows a1-a10).  `a` may live in kernel
// parameter space (single lattice) or in global memory (batched instances);
// parity and latch are the step's (t & 1, t % n_gamma == 0).  With
// blk_xch the block exchanges the edge rows' values for the inlet/outlet
// rules through `xch` and synchronises once, so every thread of the block
// must call this function.
// IO false: the lattice has no inlet or outlet face (walls and periodic axes
// only), and the inlet/outlet rules are compiled out.
// Beta-stencil form: where the block stages its c halo (k_step), filled by
// fused_step_node once the node's own population loads are in flight.
struct HaloStage {
  void *box;       // nullptr: no staging (c from global memory)
  int hx, hy, hn;  // box extent along x, y; nodes in the box
  int o[3];        // the block's first tile node
  int k;           // this thread's node in the box
};

template <class L, class S, class R, bool BS = false, class OffT = long long, bool IO = true>
__device__ __forceinline__ void fused_step_node(const StepArgs &a, Geo &g, bool active, int tid, int parity,
                                                int latch, bool blk_xch, int gstride, R *xch,
                                                const HaloStage &hs = HaloStage{nullptr, 0, 0, 0, {0, 0, 0}, 0}) {
  constexpr int D = L::D, Q = L::Q;
  const int gax = a.g_axis;
  Pops<L, S, R, BS> f;
  Moments<L, R> m;
  R cg[3] = {R(0), R(0), R(0)}, cl[3] = {R(0), R(0), R(0)};
  // interior: no non-periodic face within one step of any node of the warp
  // (most warps; their loads and stores are compiled without the face
  // rules).  Decided per warp, so that a warp holding face nodes takes the
  // general path whole instead of running both.  Not for the D3Q19 half
  // store: its kernel, twice as long with the second path, ran 12 % slower
  // on the 3D column (instruction fetch), where the FP32 one gained 5 %.
  constexpr bool SPLIT = !(Q == 19 && sizeof(S) == 2);
  bool interior = false;
  if (active) {
    make_geo(a, D, g);
    interior = !(g.xp[0] || g.xm[0] || g.xp[1] || g.xm[1] || g.xp[2] || g.xm[2]);
  }
  interior = SPLIT && __all_sync(__activemask(), interior);
  if constexpr (BS) {
    // the node's own populations first; the c halo is staged (and the block
    // synchronised) while they are in flight, then the beta populations are
    // evaluated from it
    if (active) {
      if (interior) load_node<L, S, R, BS, OffT, true, false>(a, g, parity, f);
      else load_node<L, S, R, BS, OffT, false, false>(a, g, parity, f);
    }
    CHalo halo{nullptr, 0, 0, 0, 0};
    if (hs.box) {
      stage_c_halo<L, S>(a, hs.box, hs.hx, hs.hy, hs.hn, hs.o, tid, a.T[0] * a.T[1] * a.T[2]);
      __syncthreads();
      halo = CHalo{hs.box, hs.hx, hs.hy, hs.hn, hs.k};
    }
    if (active) load_node_beta<L, S, R, BS>(a, g, parity, f, halo);
  } else if (active) {
    if (interior) load_node<L, S, R, BS, OffT, true>(a, g, parity, f);
    else load_node<L, S, R, BS, OffT>(a, g, parity, f);
  }
  if (active) {
    moments<L, S, R, BS>(a, f, m);
#pragma unroll
    for (int d = 0; d < D; d++) {
      cg[d] = m.all * (m.ug[d] - m.ul[d]);  // Eq. (velocitybeta) with beta = 1
      cl[d] = m.alg * (m.ul[d] - m.ug[d]);
    }
  }
  if (BS && active) {
    // beta-stencil form: c of this step into buffer t & 1
    typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
    H *cw = (H *)a.cfield + (long long)parity * 2 * D * a.plane;
#pragma unroll
    for (int d = 0; d < D; d++) {
      cw[d * a.plane + g.node] = (H)cg[d];
      cw[(D + d) * a.plane + g.node] = (H)cl[d];
    }
  }
  if (IO && blk_xch) {
    if (active) {
#pragma unroll
      for (int d = 0; d < 3; d++) {
        xch[tid * XCH + d] = m.ug[d] * (d < D);
        xch[tid * XCH + 3 + d] = m.ul[d] * (d < D);
        xch[tid * XCH + 8 + d] = cg[d];
        xch[tid * XCH + 11 + d] = cl[d];
      }
      xch[tid * XCH + 6] = m.alg;
      xch[tid * XCH + 7] = m.all;
    }
    __syncthreads();
  }
  if (!active) return;

  const PhysT<R> &P = phys<R>(a);
  const R R_ = P.R_, invR = P.invR;
  // ---- sources: Eq. (lbmbetataylorzeroth5), dashpot Eqs. (lbm-cont-g1Dhat),
  //      (lbm-cont-l1Dhat) third strategy with phi*eps_l - 1 = (eps_g - 1)/R
  const R dPl = m.deg * invR;
  R ug2 = R(0), ul2 = R(0);
#pragma unroll
  for (int d = 0; d < D; d++) {
    ug2 += m.ug[d] * m.ug[d];
    ul2 += m.ul[d] * m.ul[d];
  }
  typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
  H *held = (H *)a.held;
  R Spp_g, Spp_l, Lam;
  if (latch) {
    Spp_g = m.Sg - P.gamma * ug2 * m.deg;
    Spp_l = m.Sl - P.gamma * ul2 * dPl;
    Lam = m.alg * m.all * (m.alg + m.all * R_);  // Eq. (Lambda)
    held[g.node] = (H)Spp_g;
    held[a.plane + g.node] = (H)Spp_l;
    held[2 * a.plane + g.node] = (H)Lam;
    Spp_g = (R)(H)Spp_g;
    Spp_l = (R)(H)Spp_l;
    Lam = (R)(H)Lam;
  } else {
    Spp_g = (R)held[g.node];
    Spp_l = (R)held[a.plane + g.node];
    Lam = (R)held[2 * a.plane + g.node];
  }

  // ---- grad(alpha): Eq. (gradlnalpha) times alpha, corrected by Eq. (spalding2);
  //      grad^G alpha_l = -grad^G alpha_g
  R gG[3] = {R(0), R(0), R(0)};
  const R kg = P.kgrad;
#pragma unroll
  for (int d = 0; d < D; d++) {
    R grg = kg * (m.ag * m.ug[d] - m.Jg[d]);
    R grl = kg * (m.al * m.ul[d] - m.Jl[d]);
    gG[d] = R(0.5) * (grg - grl);
  }

  // ---- stress sigma = A (Pi^eq - Pi) + B S'' I (Eq. (lbm-sigma3); D = 1:
  //      Eq. (taylor-second31Db)), Pi^eq from Eq. (secondtensoreq)
  R sgG[3], slG[3];
  {
    const R cs2 = R(1.0 / 3.0);
    R Ng[6], Nl[6];
#pragma unroll
    for (int d = 0; d < D; d++)
#pragma unroll
      for (int e = d; e < D; e++) {
        const int k = pidx(d, e);
        Ng[k] = m.ug[d] * m.ug[e] - m.Pg[k] + (d == e ? cs2 * m.deg : R(0));
        Nl[k] = m.ul[d] * m.ul[e] - m.Pl[k] + (d == e ? cs2 * dPl : R(0));
      }
    const R Ag = P.A_g, Al = P.A_l, Bg = P.B_g * Spp_g, Bl = P.B_l * Spp_l;
#pragma unroll
    for (int d = 0; d < D; d++) {
      R sg = Bg * gG[d], sl = -Bl * gG[d];
#pragma unroll
      for (int e = 0; e < D; e++) {
        const int k = pidx(d, e);
        sg += Ag * Ng[k] * gG[e];
        sl -= Al * Nl[k] * gG[e];
      }
      sgG[d] = sg;
      slG[d] = sl;
    }
  }

  // ---- drag (Eq. (interphasemomentum), CGW Eq. (CliftGraceWeber)), wall
  //      friction (Eq. (wallmomentum1D)), forces Eqs. (Gg), (Gl), (Gg1D)
  R Gg[3] = {R(0), R(0), R(0)}, Gl[3] = {R(0), R(0), R(0)};
  {
    const R KI = a.cgw ? P.kappa_I * Lam : P.kappa_I;
    const R KW = a.cgw ? P.kappa_W * Lam : P.kappa_W;
    R du[3], du2 = R(0);
#pragma unroll
    for (int d = 0; d < D; d++) {
      du[d] = m.ul[d] - m.ug[d];
      du2 += du[d] * du[d];
    }
    const R ndu = sqrt(du2), nul = sqrt(ul2);
    const R fl = P.afloor;
    const R inv_g = R(1) / (m.alg > fl ? m.alg : fl);
    const R inv_l = R(1) / (m.all > fl ? m.all : fl);
#pragma unroll
    for (int d = 0; d < D; d++) {
      Gg[d] = Spp_g * m.ug[d] + (sgG[d] + KI * ndu * du[d]) * inv_g + (d == a.g_axis ? P.buoy : R(0));
      Gl[d] = Spp_l * m.ul[d] + slG[d] * inv_l - (KI * ndu * du[d] + KW * nul * m.ul[d]) * inv_l * invR;
    }
  }

  // ---- collisions and AA store with face rules
  const R om_g = P.omega_g, om_l = P.omega_l, om_a = P.omega_a;
  // f_alpha relaxes to f^eq(alpha^B, u) (Spalding mode 2) or f^eq(a, u):
  // its even part w [(alpha^B - r) + alpha^B q] is taken as
  // w [(a - r) + a q] + w c (1 + q) with c = alpha^B - a (0 unless mode 2),
  // so that c is not lost to the spacing of a - r
  const R aeq_g = a.spalding == 2 ? m.alg : m.ag, aeq_l = a.spalding == 2 ? m.all : m.al;
  const R ceq_g = a.spalding == 2 ? m.cg : R(0), ceq_l = a.spalding == 2 ? m.cl : R(0);
  const R rag = P.r_ag, ral = P.r_al;
  // Eq. (eta) for the moving directions: eta_q(phi) = phi, so the offsets of
  // f_I^eq - w are eps_g - 1 (phi_g = 1) and phi eps_l - 1 = dPl, and f_L's
  // is S psi.  The rest direction's takes what makes the zeroth moments
  // exact with the weights in use (sum w_q = 1): w_0 eta_0 = 1 - (1 - w_0)
  // phi, so its f_I^eq is the remainder of the moving directions' (taken as
  // such by the rest direction's collision below), and w_0 f_L(0) = S -
  // (1 - w_0) psi S, (1 - w_0) x formed as x - w_0 x so that no rounded
  // 1 - w_0 biases it.
  const R eL_gq = Spp_g * P.psi_g, eL_lq = Spp_l * P.psi_l;
  // The populations are held and stored in raw units, deviations times
  // SC = Store<S>::scale (2^12 for the half store, 1 otherwise): every term
  // of a post-collision population is formed with the weights scaled by SC
  // (compile-time constants, exact: SC is a power of two), so no population
  // is rescaled one by one.
  constexpr R SC = (R)Store<S>::scale;
  const R c2g = BS ? R(0) : beta_c2<L, R>(cg), c2l = BS ? R(0) : beta_c2<L, R>(cl);

  // face rules of direction q (walls, Tables 1-2) and its AA store; INTc
  // (std::true_type for interior nodes) compiles them out
  auto finish = [&](const int q, R out[6], auto INTc) {
    constexpr bool INT = decltype(INTc)::value;
    const R w = wq<L, R>(q) * SC;
    const bool cross = !INT && crosses<L>(g, q, +1);
    if (IO && cross) {
      const int rule = face_rule<L>(a, g, q);
      const int qo = L::opp(q);
      if (rule == BC_INLET) {
        // Table 1: f_g, f_l BB(I) (Eq. (BB): -2 w v.u^B/cs2), f_alpha EQ(S)
        // Dirichlet, f_beta EQ(S) with beta and c extrapolated full-way.
        const R vq = (R)(gax == 0 ? L::v(q, 0) : (gax == 1 ? L::v(q, 1) : L::v(q, 2)));
        out[0] -= R(2) * (aq<L, R>(q) * SC) * vq * P.ugIN;
        out[1] -= R(2) * (aq<L, R>(q) * SC) * vq * P.ulIN;
        R uin[3], lin[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
          uin[d] = d == gax ? P.ugIN : R(0);
          lin[d] = d == gax ? P.ulIN : R(0);
        }
        out[2] = SC * feqS_dev<L, R>(qo, P.aIN, uin, P.ugIN * P.ugIN, rag);
        out[3] = SC * feqS_dev<L, R>(qo, R(1) - P.aIN, lin, P.ulIN * P.ulIN, ral);
        const R *xn = xch + (tid + gstride) * XCH;
        R cb[3] = {R(0), R(0), R(0)}, cc[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int d = 0; d < D; d++) {
          cb[d] = R(2) * cg[d] - xn[8 + d];
          cc[d] = R(2) * cl[d] - xn[11 + d];
        }
        if (!BS) {
          beta_pair<L, R>(qo, cb, cc, out[4], out[5]);
          out[4] *= SC;
          out[5] *= SC;
        }
      } else if (rule == BC_OUTLET) {
        // Table 2: f_g, f_l ABB(I) with eps = 1 (so phi = 1) and u EX(hw);
        // f_alpha ABB(S) with alpha, u EX(hw); f_beta EQ(S) with c EX(fw).
        const R *xn = xch + (tid - gstride) * XCH;
        R ubg[3] = {R(0), R(0), R(0)}, ubl[3] = {R(0), R(0), R(0)}, cb[3] = {R(0), R(0), R(0)},
          cc[3] = {R(0), R(0), R(0)};
        R ubg2 = R(0), ubl2 = R(0);
#pragma unroll
        for (int d = 0; d < D; d++) {
          ubg[d] = R(1.5) * m.ug[d] - R(0.5) * xn[d];
          ubl[d] = R(1.5) * m.ul[d] - R(0.5) * xn[3 + d];
          cb[d] = R(2) * cg[d] - xn[8 + d];
          cc[d] = R(2) * cl[d] - xn[11 + d];
          ubg2 += ubg[d] * ubg[d];
          ubl2 += ubl[d] * ubl[d];
        }
        const R vbg = vdot<L, R>(q, ubg), vbl = vdot<L, R>(q, ubl);
        const R qg = R(4.5) * vbg * vbg - R(1.5) * ubg2, ql = R(4.5) * vbl * vbl - R(1.5) * ubl2;
        out[0] = -out[0] + R(2) * w * qg;
        out[1] = -out[1] + R(2) * w * ql;
        const R abg = R(1.5) * m.alg - R(0.5) * xn[6];
        const R abl = R(1.5) * m.all - R(0.5) * xn[7];
        out[2] = -out[2] + R(2) * w * ((abg - rag) + abg * qg);
        out[3] = -out[3] + R(2) * w * ((abl - ral) + abl * ql);
        if (!BS) {
          beta_pair<L, R>(qo, cb, cc, out[4], out[5]);
          out[4] *= SC;
          out[5] *= SC;
        }
      }
      // BC_WALL: half-way bounce-back keeps out[] as is
    }
    int pq;
    const long long idx = write_slot<L>(a, g, q, cross, parity, pq);
    const OffT off = pop_offset<L, OffT>(a, pq, idx);
    if constexpr (std::is_same<S, MixAB>::value) {
      float *gb = (float *)a.pop;
      const long long Qp = (long long)Q * a.plane;
      gb[off] = (float)out[0];
      gb[Qp + off] = (float)out[1];
      __half2 *hb = (__half2 *)(gb + 2 * Qp);
#pragma unroll
      for (int p = 0; p < (BS ? 1 : 2); p++)
        hb[p * Qp + off] = __floats2half2_rn((float)out[2 + 2 * p] * HALF_SCALE, (float)out[3 + 2 * p] * HALF_SCALE);
    } else if constexpr (sizeof(S) == 2) {
      // half pairs: one 32-bit store per pair, both values rounded at once
#pragma unroll
      for (int p = 0; p < (BS ? 2 : 3); p++)
        ((__half2 *)a.pop + (long long)(p * Q) * a.plane)[off] = __floats2half2_rn((float)out[2 * p], (float)out[2 * p + 1]);
    } else {
#pragma unroll
      for (int s = 0; s < (BS ? 4 : 6); s++)
        Store<S>::template st<R>((S *)scheme_base<L, S>(a, s) + off, out[s]);
    }
  };

  // Collisions, direction by direction: the moving ones in pairs (q, opp q),
  // whose equilibria share their even part w_q (...) and differ in the sign
  // of their odd part a_q v_q . u; the rest direction last.  The rest
  // direction's non-equilibrium part is not formed from its own equilibrium
  // but as what makes sum_q (f^eq_q - f_q) exactly the change the collision
  // must make -- zero for f_g and f_l (the source S'' enters through the
  // forcing), Spalding's c for f_alpha -- given the moving directions' parts
  // as computed (nsum: small numbers, summed with small rounding).  In exact
  // arithmetic the two are the same (the equilibria's zeroth moments are the
  // moments').  So the collision conserves mass whatever the rounding of the
  // zeroth moment sums, and the correction goes where it changes no higher
  // moment (v_0 = 0).  Without it, the sums' rounding moved mass the same
  // way every step in a slowly varying state (the batched sweep's columns,
  // gas below liquid, drifted 8e-6 in gas volume and 6e-5 in gas momentum
  // over 10,000 steps).
  // The rest direction's four populations wait in shared memory through the
  // pair loop (float arithmetic: four live registers fewer, so fewer spills
  // inside the loop; box2d FP32 99 -> 80 us, FP16AB 77 -> 72 us), a slot per
  // thread.
  constexpr bool STASH = std::is_same<R, float>::value;
  constexpr int NST = StepBounds<L, S>::threads;
  __shared__ R rest_stash[STASH ? 4 * NST : 1];
  volatile R *const stash = rest_stash + (STASH ? threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z) : 0);
  auto rest_f = [&](int s) -> R {
    if constexpr (STASH) return stash[s * NST];
    else return f.get(s, 0);
  };
  auto collide_rest = [&](const R nsum[4], auto INTc) {
    typedef Rn<R> O;
    const R wu = wq<L, R>(0);
    R out[6];
    const R rest_Lg = O::sub(Spp_g, O::mul(P.psi_g, O::fma(-wu, Spp_g, Spp_g)));
    const R rest_Ll = O::sub(Spp_l, O::mul(P.psi_l, O::fma(-wu, Spp_l, Spp_l)));
    out[0] = O::add(rest_f(0), O::fma(om_g, -nsum[0], O::mul(SC, rest_Lg)));
    out[1] = O::add(rest_f(1), O::fma(om_l, -nsum[1], O::mul(SC, rest_Ll)));
    out[2] = O::fma(om_a, O::sub(O::mul(SC, ceq_g), nsum[2]), rest_f(2));
    out[3] = O::fma(om_a, O::sub(O::mul(SC, ceq_l), nsum[3]), rest_f(3));
    if (!BS) {
      beta_pair<L, R>(0, cg, cl, out[4], out[5]);
      out[4] *= SC;
      out[5] *= SC;
    }
    finish(0, out, INTc);
  };

  auto collide_all = [&](auto INTc) {
  R nsum[4] = {R(0), R(0), R(0), R(0)};  // sum over the moving directions of f^eq - f
  if constexpr (STASH) {
#pragma unroll
    for (int s = 0; s < 4; s++) stash[s * NST] = f.get(s, 0);
  }
#pragma unroll
  for (int q = 1; q < Q; q++) {
    const int qo = L::opp(q);
    if (q < qo) {
      // Explicitly rounded operations: the node's arithmetic is compiled into
      // the interior and the general path, and must give the same bits in
      // both (no contraction left to the compiler).
      typedef Rn<R> O;
      // EX: the exact forms below (the half store, whose populations keep 11
      // significant bits, gains nothing from them and runs without)
      constexpr bool EX = !std::is_same<S, __half>::value;
      const R w = wq<L, R>(q) * SC, aw = aq<L, R>(q) * SC;
      const R vug = vdot<L, R>(q, m.ug), vul = vdot<L, R>(q, m.ul);
      const R vGg = vdot<L, R>(q, Gg), vGl = vdot<L, R>(q, Gl);
      const R qug = O::fma(O::mul(R(4.5), vug), vug, O::mul(R(-1.5), ug2));
      const R qul = O::fma(O::mul(R(4.5), vul), vul, O::mul(R(-1.5), ul2));
      // Even parts of f_I^eq - w (f_g, f_l) and of f^eq(alpha, u) - w r:
      // the large product w d (d = eps_g - 1, phi eps_l - 1, a - r) is kept
      // exactly as hi + lo, lo = fma(w, d, -hi), so that the equilibrium's
      // zeroth moment, sum_q w_q d = d (the float weights sum to 1 exactly),
      // is not biased by the rounding of the products.  The roundings of w d
      // are deterministic in the state and do not cancel over the
      // directions; in a slowly varying state they moved eps and alpha the
      // same way every step.
      const R Xg = O::mul(w, m.deg);
      const R Xgl = EX ? O::add(O::fma(w, m.deg, -Xg), O::mul(w, qug)) : O::mul(w, qug);
      const R Xl = O::mul(w, dPl), Xll = EX ? O::add(O::fma(w, dPl, -Xl), O::mul(w, qul)) : O::mul(w, qul);
      // Odd parts a_q (v . u) of f_g, f_l, formed exactly as hi + lo (v . u
      // as a two-sum of its at most two nonzero terms, the product as a
      // two-product), so that the equilibrium's first moment,
      // sum_q v_q a_q (v_q . u) = u, is exactly the u the moments gave: the
      // collision then adds no momentum of its own.  A rounded first moment
      // acts as a small force every step; on the liquid, whose momentum the
      // interphase force restores only at 1/R of the gas's rate (Eq. (Gl)),
      // it left u_l 1.5e-5 from the FP64 path after 20,000 steps of the 2D
      // box.
      R vgs = vug, vge = R(0), vls = vul, vle = R(0);
      if constexpr (EX) {
        vdot2<L, R>(q, m.ug, vgs, vge);
        vdot2<L, R>(q, m.ul, vls, vle);
      }
      const R Yg = O::mul(aw, vgs);
      const R Ygl = EX ? O::fma(aw, vge, O::fma(aw, vgs, -Yg)) : R(0);
      const R Yl = O::mul(aw, vls);
      const R Yll = EX ? O::fma(aw, vle, O::fma(aw, vls, -Yl)) : R(0);
      const R Fg = O::mul(w, eL_gq), Hg = O::mul(aw, vGg), Fl = O::mul(w, eL_lq), Hl = O::mul(aw, vGl);
      // f_alpha: alpha^B = a + c (c the renormalisation, Spalding mode 2)
      const R Xag = O::mul(w, m.dag), Xal = O::mul(w, m.dal);
      const R Xagl = O::add(O::add(EX ? O::fma(w, m.dag, -Xag) : R(0), O::mul(w, O::mul(m.ag, qug))),
                            O::mul(w, O::mul(ceq_g, O::add(R(1), qug))));
      const R Xall = O::add(O::add(EX ? O::fma(w, m.dal, -Xal) : R(0), O::mul(w, O::mul(m.al, qul))),
                            O::mul(w, O::mul(ceq_l, O::add(R(1), qul))));
      const R Yag = O::mul(aeq_g, O::mul(aw, vug)), Yal = O::mul(aeq_l, O::mul(aw, vul));
      // f* = f + [omega (f^eq - f) + forcing], f^eq - f = (X_hi - f) + X_lo +- Y
      // formed without losing the smaller terms: X_hi - f is taken exactly as
      // s + e (Knuth's two-sum), then (s +- Y) + (e + X_lo).  Whichever of the
      // even part X and the odd part Y (the flux) carries f, s +- Y cancels it
      // exactly and the rest enters at its own precision; the node's value is
      // rounded once more, at the spacing of f.  (Grouped as (X +- Y) - f, the
      // smaller part was quantised to the spacing of the larger one every
      // step.)  For f_alpha the even part w (alpha - r) always carries f
      // (~0.29 w in a gas plume) and X_hi - f cancels exactly without the
      // two-sum.
      const R fg = f.get(0, q), fgo = f.get(0, qo), fl = f.get(1, q), flo = f.get(1, qo);
      const R fa = f.get(2, q), fao = f.get(2, qo), fb = f.get(3, q), fbo = f.get(3, qo);
      auto neq = [](R Xh, R Xlo, R fv, R Y) {  // (Xh - fv) + Xlo + Y, Xh - fv as the exact s + e
        const R s = O::sub(Xh, fv);
        if constexpr (!EX) return O::add(O::add(s, Y), Xlo);
        const R bb = O::sub(s, Xh);
        const R e = O::sub(O::sub(Xh, O::sub(s, bb)), O::add(fv, bb));
        return O::add(O::add(s, Y), O::add(e, Xlo));
      };
      const R ta[4] = {neq(Xg, O::add(Xgl, Ygl), fg, Yg), neq(Xl, O::add(Xll, Yll), fl, Yl),
                       O::add(O::add(O::sub(Xag, fa), Xagl), Yag), O::add(O::add(O::sub(Xal, fb), Xall), Yal)};
      const R tb[4] = {neq(Xg, O::sub(Xgl, Ygl), fgo, -Yg), neq(Xl, O::sub(Xll, Yll), flo, -Yl),
                       O::sub(O::add(O::sub(Xag, fao), Xagl), Yag), O::sub(O::add(O::sub(Xal, fbo), Xall), Yal)};
#pragma unroll
      for (int s = 0; s < 4; s++) nsum[s] = O::add(nsum[s], O::add(ta[s], tb[s]));
      R oa[6], ob[6];
      oa[0] = O::add(fg, O::fma(om_g, ta[0], O::add(Fg, Hg)));
      ob[0] = O::add(fgo, O::fma(om_g, tb[0], O::sub(Fg, Hg)));
      oa[1] = O::add(fl, O::fma(om_l, ta[1], O::add(Fl, Hl)));
      ob[1] = O::add(flo, O::fma(om_l, tb[1], O::sub(Fl, Hl)));
      oa[2] = O::fma(om_a, ta[2], fa);
      ob[2] = O::fma(om_a, tb[2], fao);
      oa[3] = O::fma(om_a, ta[3], fb);
      ob[3] = O::fma(om_a, tb[3], fbo);
      if (!BS) {
        // beta_dev of q and opp(q) from one even part (v_opp . c = -v_q . c exactly)
        R vcg, vcl;
        const R xg = beta_even<L, R>(q, cg, c2g, vcg) * SC, xl = beta_even<L, R>(q, cl, c2l, vcl) * SC;
        oa[4] = Rn<R>::fma(aw, vcg, xg);
        ob[4] = Rn<R>::fma(aw, -vcg, xg);
        oa[5] = Rn<R>::fma(aw, vcl, xl);
        ob[5] = Rn<R>::fma(aw, -vcl, xl);
      }
      finish(q, oa, INTc);
      finish(qo, ob, INTc);
    }
  }
  collide_rest(nsum, INTc);
  };
  if (interior) collide_all(std::true_type{});
  else collide_all(std::false_type{});
}

template <class L, class S, class R, bool BS, class OffT, bool IO = true>
__global__ void __launch_bounds__(StepBounds<L, S>::threads, StepBounds<L, S>::blocks) k_step(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *xch = reinterpret_cast<R *>(smem_raw);
  Geo g;
  g.c[0] = blockIdx.x * a.T[0] + threadIdx.x - a.shift[0];
  g.c[1] = blockIdx.y * a.T[1] + threadIdx.y - a.shift[1];
  g.c[2] = blockIdx.z * a.T[2] + threadIdx.z - a.shift[2];
  const bool active = g.c[0] >= 0 && g.c[0] < a.n[0] && g.c[1] >= 0 && g.c[1] < a.n[1] && g.c[2] >= 0 &&
                      g.c[2] < a.n[2];
  const int tid = threadIdx.x + a.T[0] * (threadIdx.y + a.T[1] * threadIdx.z);
  const int gax = a.g_axis;
  const int gstride = gax == 0 ? 1 : (gax == 1 ? a.T[0] : a.T[0] * a.T[1]);
  // does this block hold an inlet/outlet edge row (block-uniform)?
  const int Tg = gax == 0 ? a.T[0] : (gax == 1 ? a.T[1] : a.T[2]);
  const int ng = gax == 0 ? a.n[0] : (gax == 1 ? a.n[1] : a.n[2]);
  const int sg = gax == 0 ? a.shift[0] : (gax == 1 ? a.shift[1] : a.shift[2]);
  const int blk_g0 = (int)(gax == 0 ? blockIdx.x : (gax == 1 ? blockIdx.y : blockIdx.z)) * Tg - sg;
  const bool blk_xch = IO && ((a.has_inlet && blk_g0 <= 0) || (a.has_outlet && blk_g0 + Tg >= ng));
  HaloStage hs{nullptr, 0, 0, 0, {0, 0, 0}, 0};
  if constexpr (BS) {
    // the block's c tile plus a one-node halo, from the last step's buffer
    const int hx = a.T[0] + 2, hy = L::D > 1 ? a.T[1] + 2 : 1, hz = L::D > 2 ? a.T[2] + 2 : 1;
    hs = HaloStage{smem_raw + a.halo_off, hx, hy, hx * hy * hz,
                   {(int)blockIdx.x * a.T[0] - a.shift[0], (int)blockIdx.y * a.T[1] - a.shift[1],
                    (int)blockIdx.z * a.T[2] - a.shift[2]},
                   (int)(threadIdx.x + 1) + hx * ((L::D > 1 ? (int)threadIdx.y + 1 : 0) +
                                                  hy * (L::D > 2 ? (int)threadIdx.z + 1 : 0))};
  }
  fused_step_node<L, S, R, BS, OffT, IO>(a, g, active, tid, a.parity, a.latch, blk_xch, gstride, xch, hs);
}

// Batched form: one launch advances many independent lattices (instances) of
// the same lattice and precision.  Block b processes the tile work[b] of
// instance work[b].inst with that instance's arguments args[inst] (global
// memory, block-uniform); all instances share the step's parity and latch.
// Instances have no inlet/outlet faces, so no shared-memory exchange.  The
// node arithmetic is the single-lattice kernel's source, compiled into a
// second kernel: the compiler may fuse multiply-adds differently there, so
// the two agree to rounding, not bit for bit.
struct WorkItem {
  int inst, x0, y0, z0;
};

// Launch bounds of the batched kernel (its constants come from shared memory).
template <class L, class S> struct BatchBounds {
  static constexpr int threads = StepBounds<L, S>::threads;
  static constexpr int blocks = StepBounds<L, S>::blocks;
};

template <class L, class S, class R, class OffT>
__global__ void __launch_bounds__(BatchBounds<L, S>::threads, BatchBounds<L, S>::blocks)
    k_batch_step(const StepArgs *__restrict__ args, const WorkItem *__restrict__ work, int parity, int latch) {
  // the instance's constants, staged once per block in shared memory
  __shared__ __align__(16) int sargs[(sizeof(StepArgs) + 3) / 4];
  const WorkItem wi = work[blockIdx.x];
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int *src = reinterpret_cast<const int *>(args + wi.inst);
  for (int k = tid; k < (int)(sizeof(StepArgs) / 4); k += nthr) sargs[k] = __ldg(src + k);
  __syncthreads();
  const StepArgs &a = *reinterpret_cast<const StepArgs *>(sargs);
  Geo g;
  g.c[0] = wi.x0 + threadIdx.x;
  g.c[1] = wi.y0 + threadIdx.y;
  g.c[2] = wi.z0 + threadIdx.z;
  const bool active = g.c[0] < a.n[0] && g.c[1] < a.n[1] && g.c[2] < a.n[2];
  // no inlet or outlet rules: lbm_batch_create accepts walls and periodic axes only
  fused_step_node<L, S, R, false, OffT, false>(a, g, active, 0, parity, latch, false, 0, (R *)nullptr);
}

// --------------------------------------------------- moments / diagnostics

// mode bit 1: write fields (FP64): alpha_g^B, u_g (D planes), u_l (D planes),
// p_k, S_g, S_l at out + k*N; mode bit 2: per-block diagnostic partials.
struct MomArgs {
  StepArgs s;
  double *out;
  long long N;
  double *partials;  // gridDim.x * 8
};

template <class R>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// FP64 block reduction of the eight diagnostics (block of 256 threads): warp
// shuffles, one value per warp in shared memory, then warp 0 writes the
// block's partial (slot 4 is a maximum, the others sums).
__device__ __forceinline__ void block_diag_reduce(double v[8], double *partials) {
  __shared__ double red[8][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = (k == 4) ? warp_max(v[k]) : warp_sum<double>(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 8; k++) red[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      double x = lane < nw ? red[k][lane] : 0.0;
      x = (k == 4) ? warp_max(x) : warp_sum<double>(x);
      if (lane == 0) partials[(long long)blockIdx.x * 8 + k] = x;
    }
  }
}

// One thread per node over a flat 1D grid (block 256).
template <class L, class S, class R, bool BS>
__global__ void __launch_bounds__(256) k_moments(const MomArgs ma, int mode) {
  constexpr int D = L::D, Q = L::Q;
  const StepArgs &a = ma.s;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (i < ma.N) {
    Geo g;
    g.c[0] = (int)(i % a.n[0]);
    g.c[1] = (int)((i / a.n[0]) % a.n[1]);
    g.c[2] = (int)(i / ((long long)a.n[0] * a.n[1]));
    make_geo(a, D, g);
    Pops<L, S, R, BS> f;
    load_node<L, S, R, BS>(a, g, a.parity, f);
    Moments<L, R> m;
    moments<L, S, R, BS>(a, f, m);
    if (mode & 1) {
      double *o = ma.out;
      const long long N = ma.N;
      o[i] = (double)phys<R>(a).r_ag + (double)m.dalg;  // reference plus deviation, in FP64
      for (int d = 0; d < D; d++) {
        o[(1 + d) * N + i] = (double)m.ug[d];
        o[(1 + D + d) * N + i] = (double)m.ul[d];
      }
      o[(1 + 2 * D) * N + i] = (1.0 / 3.0) * (1.0 + (double)m.deg);
      o[(2 + 2 * D) * N + i] = (double)m.Sg;
      o[(3 + 2 * D) * N + i] = (double)m.Sl;
    }
    if (mode & 2) {
      bool bad = false;
#pragma unroll
      for (int s = 0; s < 6; s++)
#pragma unroll
        for (int q = 0; q < Q; q++) bad = bad || !isfinite((double)f.get(s, q));
      double ug2 = 0, ul2 = 0;
      for (int d = 0; d < D; d++) {
        ug2 += (double)m.ug[d] * (double)m.ug[d];
        ul2 += (double)m.ul[d] * (double)m.ul[d];
      }
      const PhysT<R> &P = phys<R>(a);
      double sum = ((double)m.dag + (double)m.dal) + (double)P.rsum1;
      v[0] = (double)P.r_ag + (double)m.dag;
      v[1] = (double)P.r_al + (double)m.dal;
      v[2] = (double)P.r_ag + (double)m.dalg;
      v[3] = sum * sum;
      v[4] = sqrt(fmax(ug2, ul2));
      v[5] = bad ? 1.0 : 0.0;
      v[6] = m.deg;
      v[7] = m.del;
    }
  }
  if (mode & 2) block_diag_reduce(v, ma.partials);
}

// Final pass of the diagnostics: one block sums the per-block partials in a
// fixed order (deterministic) into out[8].
__global__ void k_diag_final(const double *partials, int nblocks, double *out);

// Full populations (f, not deviations) of scheme s in [q][node] order.
template <class L, class S, class R, bool BS>
__global__ void __launch_bounds__(256) k_pops(const MomArgs ma, int s) {
  constexpr int D = L::D, Q = L::Q;
  const StepArgs &a = ma.s;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ma.N) return;
  Geo g;
  g.c[0] = (int)(i % a.n[0]);
  g.c[1] = (int)((i / a.n[0]) % a.n[1]);
  g.c[2] = (int)(i / ((long long)a.n[0] * a.n[1]));
  make_geo(a, D, g);
  // the references the step kernel adds (in its arithmetic type)
  const double rg = sizeof(S) == 8 ? a.r_ag : (double)a.pf.r_ag, rl = sizeof(S) == 8 ? a.r_al : (double)a.pf.r_al;
  const double r = a.plain ? 0.0 : (s == 2 ? rg : (s == 3 ? rl : 1.0));
  if (BS && s >= 4) {
    R fb[2][Q];
    load_beta<L, S, R>(a, g, a.parity, fb[0], fb[1]);
#pragma unroll
    for (int q = 0; q < Q; q++) ma.out[(long long)q * ma.N + i] = (double)fb[s - 4][q] + L::w(q) * r;
    return;
  }
#pragma unroll
  for (int q = 0; q < Q; q++) {
    int pq;
    long long idx = read_slot<L>(a, g, q, a.parity, pq);
    double dv = pop_ld<S>(a.pop, s, (long long)pq * a.plane + idx, Q * a.plane);
    ma.out[(long long)q * ma.N + i] = a.plain ? dv : dv + L::w(q) * r;
  }
}

// ----------------------------------------------------------------- init

// Equilibria of every scheme from FP64 fields (Sec. 2, initial state), written
// in the even-step layout (slot (x, q) holds f(x, q)); held S'' = 0, Lambda' =
// Lambda(alpha_g).  Computed in double, stored in S.
template <class L, class S, bool BS>
__global__ void __launch_bounds__(256) k_init(const MomArgs ma, const double *alpha_g, const double *u_g,
                                             const double *u_l, const double *p_k) {
  constexpr int D = L::D, Q = L::Q;
  const StepArgs &a = ma.s;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = ma.N;
  if (i >= N) return;
  double ug[3] = {0, 0, 0}, ul[3] = {0, 0, 0}, cg[3] = {0, 0, 0}, cl[3] = {0, 0, 0};
  for (int d = 0; d < D; d++) {
    ug[d] = u_g[d * N + i];
    ul[d] = u_l[d * N + i];
  }
  const double ag = alpha_g[i], al = 1.0 - ag;
  const double deg = p_k[i] * 3.0 - 1.0;  // eps_g - 1, Eq. (sigmag1D); eps_l = 1
  const double dPl = deg * a.invR;        // phi*eps_l - 1, Eq. (lbm-phi-l)
  double ug2 = 0, ul2 = 0;
  for (int d = 0; d < D; d++) {
    cg[d] = al * (ug[d] - ul[d]);
    cl[d] = ag * (ul[d] - ug[d]);
    ug2 += ug[d] * ug[d];
    ul2 += ul[d] * ul[d];
  }
  // c in the step kernel's arithmetic type H, and the beta equilibria from
  // it as that kernel evaluates them (beta_dev), so the beta-stencil form,
  // which starts from the same c, sees the same initial beta populations
  typedef typename std::conditional<sizeof(S) == 8, double, float>::type H;
  H cgH[3] = {H(0), H(0), H(0)}, clH[3] = {H(0), H(0), H(0)};
  for (int d = 0; d < D; d++) {
    cgH[d] = (H)cg[d];
    clH[d] = (H)cl[d];
  }
  // deviations from the references the step kernel adds (in its arithmetic type)
  const double rg = sizeof(S) == 8 ? a.r_ag : (double)a.pf.r_ag, rl = sizeof(S) == 8 ? a.r_al : (double)a.pf.r_al;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const double w = L::w(q);
    const double vug = vdot<L, double>(q, ug), vul = vdot<L, double>(q, ul);
    double o[6];
    o[0] = w * (deg + 3.0 * vug + 4.5 * vug * vug - 1.5 * ug2);
    o[1] = w * ((q == 0 ? a.k0 * (0.0 - dPl) : dPl) + 3.0 * vul + 4.5 * vul * vul - 1.5 * ul2);
    o[2] = feqS_dev<L, double>(q, ag, ug, ug2, rg);
    o[3] = feqS_dev<L, double>(q, al, ul, ul2, rl);
    o[4] = (double)beta_dev<L, H>(q, cgH);
    o[5] = (double)beta_dev<L, H>(q, clH);
#pragma unroll
    for (int s = 0; s < (BS ? 4 : 6); s++)
      pop_st<S>(a.pop, s, (long long)q * a.plane + i, Q * a.plane, o[s]);
  }
  if (BS) {
    // beta-stencil form: c of the initial state in the buffer the first step
    // reads (1), evaluated at every q from the node's own c (beta_own)
    H *cw = (H *)a.cfield + 2 * D * a.plane;
    for (int d = 0; d < D; d++) {
      cw[d * a.plane + i] = cgH[d];
      cw[(D + d) * a.plane + i] = clH[d];
    }
  }
  H *held = (H *)a.held;
  held[i] = (H)0;
  held[a.plane + i] = (H)0;
  held[2 * a.plane + i] = (H)(ag * al * (ag + al * a.R));
}

}  // namespace lbm
