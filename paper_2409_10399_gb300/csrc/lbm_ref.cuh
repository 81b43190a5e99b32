// FP64 reference path of the fused six-scheme step.
//
// Populations are stored as full values f (not deviations) and every formula
// is evaluated literally, in the order in which the paper writes it:
//   f_I^eq = w [eps eta(phi) + v.u/cs2 + ((v.u)^2 - cs2 u.u)/(2 cs2 cs2)],
//   f^eq   = w alpha [1 + v.u/cs2 + ((v.u)^2 - cs2 u.u)/(2 cs2 cs2)],
//   f_L^eq = w [S eta(psi) + v.G/cs2],
// moments are summed over q in lexicographic velocity order, divisions by
// cs2 are divisions, and the translation units that include this header are
// compiled without floating-point contraction (-fmad=false).  With IEEE-754
// double, correctly rounded division and square root, the result is the
// same, bit for bit, as any other implementation of the method that evaluates
// the same expressions in the same order without contraction; the tests use
// this to compare against the CPU oracle exactly.
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

template <class L>
__device__ __forceinline__ double rdotv(int q, const double u[3]) {
  // v.u as v_x u_x + v_y u_y + v_z u_z, left to right; products with a zero
  // component contribute an exact (signed) zero and are skipped
  double s = 0.0;
  bool first = true;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int vd = L::v(q, d);
    if (vd != 0) {
      const double t = vd > 0 ? u[d] : -u[d];
      s = first ? t : s + t;
      first = false;
    }
  }
  return s;
}

__device__ __forceinline__ double rdot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <class L>
__device__ __forceinline__ double reta(int q, double phi, double k0) {
  return q == 0 ? 1.0 + k0 * (1.0 - phi) : phi;
}

struct RefConst {
  double cs2, two_cs4, k0;
};

template <class L>
__device__ __forceinline__ double rfeqI(int q, const RefConst &k, double phi, double eps, const double u[3]) {
  const double vu = rdotv<L>(q, u), uu = rdot3(u, u);
  return L::w(q) * (eps * reta<L>(q, phi, k.k0) + vu / k.cs2 + (vu * vu - k.cs2 * uu) / k.two_cs4);
}
template <class L>
__device__ __forceinline__ double rfeqS(int q, const RefConst &k, double alpha, const double u[3]) {
  const double vu = rdotv<L>(q, u), uu = rdot3(u, u);
  return L::w(q) * alpha * (1.0 + vu / k.cs2 + (vu * vu - k.cs2 * uu) / k.two_cs4);
}
template <class L>
__device__ __forceinline__ double rfeqL(int q, const RefConst &k, double psi, double S, const double G[3]) {
  return L::w(q) * (S * reta<L>(q, psi, k.k0) + rdotv<L>(q, G) / k.cs2);
}

__device__ __forceinline__ double spalB(double x) { return x <= 0.0 ? 0.0 : (x >= 1.0 ? 1.0 : x); }

// Per-node macroscopic state of the reference path.
struct RefMom {
  double eps_g, eps_l, a_g, a_l, b_g, b_l;
  double u_g[3], u_l[3], J_g[3], J_l[3];
  double Pi_g[3][3], Pi_l[3][3];
  double al_g, al_l;
};

template <class L>
__device__ __forceinline__ void ref_moments(const StepArgs &a, const double f[6][L::Q], RefMom &m) {
  constexpr int D = L::D;
  m.eps_g = m.eps_l = m.a_g = m.a_l = m.b_g = m.b_l = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    m.u_g[d] = m.u_l[d] = m.J_g[d] = m.J_l[d] = 0.0;
#pragma unroll
    for (int e = 0; e < 3; e++) m.Pi_g[d][e] = m.Pi_l[d][e] = 0.0;
  }
#pragma unroll
  for (int q = 0; q < L::Q; q++) {
    m.eps_g += f[0][q];
    m.eps_l += f[1][q];
    m.a_g += f[2][q];
    m.a_l += f[3][q];
    m.b_g += f[4][q];
    m.b_l += f[5][q];
#pragma unroll
    for (int d = 0; d < D; d++) {
      const int vd = L::v(q, d);
      if (vd != 0) {
        m.u_g[d] += vd > 0 ? f[0][q] : -f[0][q];
        m.u_l[d] += vd > 0 ? f[1][q] : -f[1][q];
        m.J_g[d] += vd > 0 ? f[2][q] : -f[2][q];
        m.J_l[d] += vd > 0 ? f[3][q] : -f[3][q];
      }
#pragma unroll
      for (int e = 0; e < D; e++) {
        const int ve = L::v(q, d) * L::v(q, e);
        if (ve != 0) {
          m.Pi_g[d][e] += ve > 0 ? f[0][q] : -f[0][q];
          m.Pi_l[d][e] += ve > 0 ? f[1][q] : -f[1][q];
        }
      }
    }
  }
  // Eq. (spalding), B = clamp to [0,1]; alpha_l^B = 1 - alpha_g^B
  if (a.spalding == 0) {
    m.al_g = m.a_g;
    m.al_l = m.a_l;
  } else {
    const double Bg = spalB(m.a_g), Bl = spalB(m.a_l);
    m.al_g = (Bg + Bl > 0.0) ? Bg / (Bg + Bl) : 0.5;
    m.al_l = 1.0 - m.al_g;
  }
}

// neighbour values exchanged for the inlet/outlet rules
constexpr int RXCH = 16;  // eps_g, eps_l, u_g[3], u_l[3], alpha^B_g, alpha^B_l, c_g[3], c_l[3]

template <class L>
__global__ void __launch_bounds__(256) k_step_ref(const StepArgs a) {
  constexpr int D = L::D, Q = L::Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *xch = reinterpret_cast<double *>(smem_raw);
  const RefConst K{a.cs2, a.two_cs4, a.k0};

  Geo g;
  g.c[0] = blockIdx.x * a.T[0] + threadIdx.x - a.shift[0];
  g.c[1] = blockIdx.y * a.T[1] + threadIdx.y - a.shift[1];
  g.c[2] = blockIdx.z * a.T[2] + threadIdx.z - a.shift[2];
  const bool active = g.c[0] >= 0 && g.c[0] < a.n[0] && g.c[1] >= 0 && g.c[1] < a.n[1] && g.c[2] >= 0 &&
                      g.c[2] < a.n[2];
  const int tid = threadIdx.x + a.T[0] * (threadIdx.y + a.T[1] * threadIdx.z);
  const int gax = a.g_axis;
  const int gstride = gax == 0 ? 1 : (gax == 1 ? a.T[0] : a.T[0] * a.T[1]);
  const int Tg = gax == 0 ? a.T[0] : (gax == 1 ? a.T[1] : a.T[2]);
  const int ng = gax == 0 ? a.n[0] : (gax == 1 ? a.n[1] : a.n[2]);
  const int sg = gax == 0 ? a.shift[0] : (gax == 1 ? a.shift[1] : a.shift[2]);
  const int blk_g0 = (int)(gax == 0 ? blockIdx.x : (gax == 1 ? blockIdx.y : blockIdx.z)) * Tg - sg;
  const bool blk_xch = (a.has_inlet && blk_g0 <= 0) || (a.has_outlet && blk_g0 + Tg >= ng);

  Pops<L, double, double, false> P;  // full FP64 populations (plain store)
  double (&f)[6][Q] = P.f;
  RefMom m;
  double c_g[3] = {0.0, 0.0, 0.0}, c_l[3] = {0.0, 0.0, 0.0};
  if (active) {
    make_geo(a, D, g);
    load_node<L, double, double>(a, g, a.parity, P);
    ref_moments<L>(a, f, m);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      c_g[d] = m.al_l * (m.u_g[d] - m.u_l[d]);  // Eq. (velocitybeta), beta = 1
      c_l[d] = m.al_g * (m.u_l[d] - m.u_g[d]);
    }
  }
  if (blk_xch) {
    if (active) {
      double *x = xch + tid * RXCH;
      x[0] = m.eps_g;
      x[1] = m.eps_l;
#pragma unroll
      for (int d = 0; d < 3; d++) {
        x[2 + d] = m.u_g[d];
        x[5 + d] = m.u_l[d];
        x[10 + d] = c_g[d];
        x[13 + d] = c_l[d];
      }
      x[8] = m.al_g;
      x[9] = m.al_l;
    }
    __syncthreads();
  }
  if (!active) return;

  // sources, Eq. (lbmbetataylorzeroth5); pressure coupling, Eq. (lbm-phi-l);
  // Ohwada dashpot, Eqs. (lbm-cont-g1Dhat), (lbm-cont-l1Dhat)
  const double S_g = 1.0 - m.b_g, S_l = 1.0 - m.b_l;
  const double phi = (1.0 + (m.eps_g - 1.0) / a.R) / m.eps_l;
  double *held = (double *)a.held;
  double Spp_g, Spp_l, Lam;
  if (a.latch) {
    Spp_g = S_g - a.gamma * rdot3(m.u_g, m.u_g) * (m.eps_g - 1.0);
    Spp_l = S_l - a.gamma * rdot3(m.u_l, m.u_l) * (phi * m.eps_l - 1.0);
    Lam = m.al_g * m.al_l * (m.al_g + m.al_l * a.R);  // Eq. (Lambda)
    held[g.node] = Spp_g;
    held[a.plane + g.node] = Spp_l;
    held[2 * a.plane + g.node] = Lam;
  } else {
    Spp_g = held[g.node];
    Spp_l = held[a.plane + g.node];
    Lam = held[2 * a.plane + g.node];
  }

  // Eq. (gradlnalpha) times alpha, then Eq. (spalding2)
  double gG_g[3] = {0.0, 0.0, 0.0}, gG_l[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const double gr_g = d < D ? a.kgrad * (m.a_g * m.u_g[d] - m.J_g[d]) : 0.0;
    const double gr_l = d < D ? a.kgrad * (m.a_l * m.u_l[d] - m.J_l[d]) : 0.0;
    const double dl = gr_g + gr_l;
    gG_g[d] = gr_g - 0.5 * dl;
    gG_l[d] = gr_l - 0.5 * dl;
  }

  // stress: Eq. (lbm-sigma3) (D >= 2), Eq. (taylor-second31Db) (D = 1),
  // Pi^eq of Eq. (secondtensoreq)
  double sgG[3] = {0.0, 0.0, 0.0}, slG[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < D; d++) {
    double sgg = 0.0, slg = 0.0;
#pragma unroll
    for (int e = 0; e < D; e++) {
      const double Peq_g = (d == e ? K.cs2 * m.eps_g : 0.0) + m.u_g[d] * m.u_g[e];
      const double Peq_l = (d == e ? K.cs2 * phi * m.eps_l : 0.0) + m.u_l[d] * m.u_l[e];
      double sg_, sl_;
      if (D == 1) {
        sg_ = a.nuef_g * (a.omega_g * (Peq_g - m.Pi_g[d][e]) + a.psi_g * K.cs2 * Spp_g);
        sl_ = a.nuef_l * (a.omega_l * (Peq_l - m.Pi_l[d][e]) + a.psi_l * K.cs2 * Spp_l);
      } else {
        sg_ = (1.0 - 0.5 * a.omega_g) * (Peq_g - m.Pi_g[d][e]) - (d == e ? 0.5 * K.cs2 * a.psi_g * Spp_g : 0.0);
        sl_ = (1.0 - 0.5 * a.omega_l) * (Peq_l - m.Pi_l[d][e]) - (d == e ? 0.5 * K.cs2 * a.psi_l * Spp_l : 0.0);
      }
      sgg += sg_ * gG_g[e];
      slg += sl_ * gG_l[e];
    }
    sgG[d] = sgg;
    slG[d] = slg;
  }

  // drag (Eqs. (interphasemomentum), (CliftGraceWeber)), wall friction
  // (Eq. (wallmomentum1D)), forces (Eqs. (Gg), (Gl), (Gg1D))
  const double KI = a.cgw ? a.kappa_I * Lam : a.kappa_I;
  const double KW = a.cgw ? a.kappa_W * Lam : a.kappa_W;
  double du[3];
#pragma unroll
  for (int d = 0; d < 3; d++) du[d] = m.u_l[d] - m.u_g[d];
  const double ag_d = m.al_g > a.afloor ? m.al_g : a.afloor;
  const double al_d = m.al_l > a.afloor ? m.al_l : a.afloor;
  const double ndu = sqrt(rdot3(du, du)), nul = sqrt(rdot3(m.u_l, m.u_l));
  double G_g[3] = {0.0, 0.0, 0.0}, G_l[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < D; d++) {
    double gg = Spp_g * m.u_g[d] + sgG[d] / ag_d;
    if (d == gax) gg = gg + a.buoy;
    G_g[d] = gg + KI * ndu * du[d] / ag_d;
    G_l[d] = Spp_l * m.u_l[d] + slG[d] / al_d - KI * ndu * du[d] / (a.R * al_d) - KW * nul * m.u_l[d] / (a.R * al_d);
  }

  const double aeq_g = a.spalding == 2 ? m.al_g : m.a_g;
  const double aeq_l = a.spalding == 2 ? m.al_l : m.a_l;
  double *base = (double *)a.pop;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    double out[6];
    out[0] = f[0][q] + a.omega_g * (rfeqI<L>(q, K, 1.0, m.eps_g, m.u_g) - f[0][q]) + rfeqL<L>(q, K, a.psi_g, Spp_g, G_g);
    out[1] = f[1][q] + a.omega_l * (rfeqI<L>(q, K, phi, m.eps_l, m.u_l) - f[1][q]) + rfeqL<L>(q, K, a.psi_l, Spp_l, G_l);
    out[2] = f[2][q] + a.omega_a * (rfeqS<L>(q, K, aeq_g, m.u_g) - f[2][q]);
    out[3] = f[3][q] + a.omega_a * (rfeqS<L>(q, K, aeq_l, m.u_l) - f[3][q]);
    out[4] = rfeqS<L>(q, K, 1.0, c_g);
    out[5] = rfeqS<L>(q, K, 1.0, c_l);

    const bool cross = crosses<L>(g, q, +1);
    if (cross) {
      const int rule = face_rule<L>(a, g, q);
      const int qo = L::opp(q);
      if (rule == BC_INLET) {
        // Table 1 with Eqs. (BCIN), (BB): f_g, f_l BB(I) with eps EX(hw);
        // f_alpha EQ(S) Dirichlet; f_beta EQ(S) with beta, c EX(fw)
        const double *xn = xch + (tid + gstride) * RXCH;
        double uB[3], muB[3], lB[3], mlB[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
          uB[d] = d == gax ? a.ugIN : 0.0;
          muB[d] = d == gax ? -a.ugIN : 0.0;
          lB[d] = d == gax ? a.ulIN : 0.0;
          mlB[d] = d == gax ? -a.ulIN : 0.0;
        }
        const double epsB_g = 1.5 * m.eps_g - 0.5 * xn[0];
        const double epsB_l = 1.5 * m.eps_l - 0.5 * xn[1];
        out[0] = out[0] + rfeqI<L>(q, K, 1.0, epsB_g, muB) - rfeqI<L>(q, K, 1.0, epsB_g, uB);
        const double phiB = (1.0 + (epsB_g - 1.0) / a.R) / epsB_l;
        out[1] = out[1] + rfeqI<L>(q, K, phiB, epsB_l, mlB) - rfeqI<L>(q, K, phiB, epsB_l, lB);
        out[2] = rfeqS<L>(qo, K, a.aIN, uB);
        out[3] = rfeqS<L>(qo, K, 1.0 - a.aIN, lB);
        double cBg[3], cBl[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
          cBg[d] = 2.0 * c_g[d] - xn[10 + d];
          cBl[d] = 2.0 * c_l[d] - xn[13 + d];
        }
        const double betaB = 2.0 * 1.0 - 1.0;
        out[4] = rfeqS<L>(qo, K, betaB, cBg);
        out[5] = rfeqS<L>(qo, K, betaB, cBl);
      } else if (rule == BC_OUTLET) {
        // Table 2 with Eqs. (BCOUT), (ABB): f_g, f_l ABB(I) with eps = 1
        // (phi = 1) and u EX(hw); f_alpha ABB(S) with alpha, u EX(hw);
        // f_beta EQ(S) with beta, c EX(fw)
        const double *xn = xch + (tid - gstride) * RXCH;
        double ubg[3], mubg[3], ubl[3], mubl[3], cBg[3], cBl[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
          ubg[d] = 1.5 * m.u_g[d] - 0.5 * xn[2 + d];
          ubl[d] = 1.5 * m.u_l[d] - 0.5 * xn[5 + d];
          mubg[d] = -ubg[d];
          mubl[d] = -ubl[d];
          cBg[d] = 2.0 * c_g[d] - xn[10 + d];
          cBl[d] = 2.0 * c_l[d] - xn[13 + d];
        }
        out[0] = -out[0] + rfeqI<L>(q, K, 1.0, 1.0, mubg) + rfeqI<L>(q, K, 1.0, 1.0, ubg);
        out[1] = -out[1] + rfeqI<L>(q, K, 1.0, 1.0, mubl) + rfeqI<L>(q, K, 1.0, 1.0, ubl);
        const double aBg = 1.5 * m.al_g - 0.5 * xn[8];
        const double aBl = 1.5 * m.al_l - 0.5 * xn[9];
        out[2] = -out[2] + rfeqS<L>(q, K, aBg, mubg) + rfeqS<L>(q, K, aBg, ubg);
        out[3] = -out[3] + rfeqS<L>(q, K, aBl, mubl) + rfeqS<L>(q, K, aBl, ubl);
        const double betaB = 2.0 * 1.0 - 1.0;
        out[4] = rfeqS<L>(qo, K, betaB, cBg);
        out[5] = rfeqS<L>(qo, K, betaB, cBl);
      }
    }
    int pq;
    const long long idx = write_slot<L>(a, g, q, cross, a.parity, pq);
#pragma unroll
    for (int s = 0; s < 6; s++) base[(long long)(s * Q + pq) * a.plane + idx] = out[s];
  }
}

// Initial equilibria (full values), Sec. 2 initial state: eps_g = p_k/cs2,
// eps_l = 1, phi of Eq. (lbm-phi-l), alpha_l = 1 - alpha_g, c of Eq.
// (velocitybeta); held S'' = 0, Lambda' = Lambda(alpha_g).
template <class L>
__global__ void __launch_bounds__(256) k_init_ref(const MomArgs ma, const double *alpha_g, const double *u_g,
                                                 const double *u_l, const double *p_k) {
  constexpr int D = L::D, Q = L::Q;
  const StepArgs &a = ma.s;
  const RefConst K{a.cs2, a.two_cs4, a.k0};
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = ma.N;
  if (i >= N) return;
  double ug[3] = {0.0, 0.0, 0.0}, ul[3] = {0.0, 0.0, 0.0}, cg[3], cl[3];
  for (int d = 0; d < D; d++) {
    ug[d] = u_g[d * N + i];
    ul[d] = u_l[d * N + i];
  }
  const double ag = alpha_g[i], al = 1.0 - ag;
  const double eps_g = p_k[i] / K.cs2, eps_l = 1.0;
  const double phi = (1.0 + (eps_g - 1.0) / a.R) / eps_l;
  for (int d = 0; d < 3; d++) {
    cg[d] = al * (ug[d] - ul[d]);
    cl[d] = ag * (ul[d] - ug[d]);
  }
  double *base = (double *)a.pop;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    double o[6];
    o[0] = rfeqI<L>(q, K, 1.0, eps_g, ug);
    o[1] = rfeqI<L>(q, K, phi, eps_l, ul);
    o[2] = rfeqS<L>(q, K, ag, ug);
    o[3] = rfeqS<L>(q, K, al, ul);
    o[4] = rfeqS<L>(q, K, 1.0, cg);
    o[5] = rfeqS<L>(q, K, 1.0, cl);
#pragma unroll
    for (int s = 0; s < 6; s++) base[(long long)(s * Q + q) * a.plane + i] = o[s];
  }
  double *held = (double *)a.held;
  held[i] = 0.0;
  held[a.plane + i] = 0.0;
  held[2 * a.plane + i] = ag * al * (ag + al * a.R);
}

// Moments (fields, mode bit 1) and diagnostic partials (mode bit 2) of the
// reference store: alpha_g^B, u_g, u_l, p_k = cs2 eps_g, S = 1 - beta.
template <class L>
__global__ void __launch_bounds__(256) k_moments_ref(const MomArgs ma, int mode) {
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
    Pops<L, double, double, false> P;  // full FP64 populations (plain store)
    double (&f)[6][Q] = P.f;
    load_node<L, double, double>(a, g, a.parity, P);
    RefMom m;
    ref_moments<L>(a, f, m);
    if (mode & 1) {
      double *o = ma.out;
      const long long N = ma.N;
      o[i] = m.al_g;
      for (int d = 0; d < D; d++) {
        o[(1 + d) * N + i] = m.u_g[d];
        o[(1 + D + d) * N + i] = m.u_l[d];
      }
      o[(1 + 2 * D) * N + i] = a.cs2 * m.eps_g;
      o[(2 + 2 * D) * N + i] = 1.0 - m.b_g;
      o[(3 + 2 * D) * N + i] = 1.0 - m.b_l;
    }
    if (mode & 2) {
      bool bad = false;
#pragma unroll
      for (int s = 0; s < 6; s++)
#pragma unroll
        for (int q = 0; q < Q; q++) bad = bad || !isfinite(f[s][q]);
      const double sum = m.a_g + m.a_l - 1.0;
      v[0] = m.a_g;
      v[1] = m.a_l;
      v[2] = m.al_g;
      v[3] = sum * sum;
      v[4] = fmax(sqrt(rdot3(m.u_g, m.u_g)), sqrt(rdot3(m.u_l, m.u_l)));
      v[5] = bad ? 1.0 : 0.0;
      v[6] = m.eps_g - 1.0;
      v[7] = m.eps_l - 1.0;
    }
  }
  if (mode & 2) block_diag_reduce(v, ma.partials);
}

}  // namespace lbm
