/*
 * lbm_oracle.c -- plain, slow FP64 CPU implementation of the six coupled
 * lattice Boltzmann schemes of Piredda & Asinari, "Lattice Boltzmann framework
 * for multiphase flows by Eulerian-Eulerian Navier-Stokes equations"
 * (arXiv 2409.10399).
 *
 * TEST INFRASTRUCTURE.  This is the oracle the GPU library is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant with the CUDA
 * library: lattice tables are built here from their definitions, the layout
 * is node-major (f[s][node*Q + q]) with two copies (post-streaming state and
 * post-collision), and streaming is a plain push over every (node, q).
 *
 * Every step follows the paper's order (Sec. 2, Sec. 3.2-3.3, Sec. 3.5):
 *   moments -> sources (beta schemes) -> Spalding renormalisation ->
 *   pressure coupling -> Ohwada dashpot -> lagged update -> grad(alpha) ->
 *   stress -> drag -> forces -> BGK collisions -> streaming with BCs.
 * Readings of points the paper leaves open are marked "reading:".
 *
 * Parity: pinned by tests/test_oracle_*.py (App. A equilibria, moment
 * identities, projection of D2Q9/D3Q19 onto D1Q3, uniform fixed point,
 * homogeneous ODE limit and closed-form steady state, conservation, mirror
 * symmetry, brute-force tiny lattices, TEST #1 outlet values of Sec. 3.6).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PERIODIC 0
#define ORC_WALL 1
#define ORC_INLET 2
#define ORC_OUTLET 3

#define S_G 0
#define S_L 1
#define S_AG 2
#define S_AL 3
#define S_BG 4
#define S_BL 5

static const double CS2 = 1.0 / 3.0; /* lattice sound speed squared */

typedef struct {
  double R;                  /* rho_l / rho_g */
  double omega_g, omega_l;   /* BGK rates of f_g, f_l, Eq. (colloperator) */
  double omega_alpha;        /* rate of f_alpha, Eq. (lbmalpha) */
  double psi_g, psi_l;       /* forcing-operator knob, Eq. (forcingoperator) */
  int drag_model;            /* 0: K_I = kappa_I ; 1: Clift-Grace-Weber K_I = kappa_I*Lambda' */
  double kappa_I, kappa_W;
  double g_hat;              /* buoyancy (R-1)*g_hat on the gas along +g_axis */
  int g_axis;
  double gamma;              /* Ohwada dashpot constant, Sec. 3.2 */
  int n_gamma;               /* lag period of Eqs. (lbm-cont-1D-update), (Lambda-update) */
  int spalding_mode;         /* 0 off, 1 couplings only, 2 couplings and alpha equilibrium */
  double alpha_floor;        /* floor of alpha in denominators */
  int bc_lo[3], bc_hi[3];
  int inlet_lo, inlet_hi;    /* inlet strip along the first transverse axis */
  double in_alpha[2], in_ug[2], in_ul[2]; /* (min, max) of Eq. (transient) */
  int ramp_nt;
  int inlet_ul_mode;         /* 0: u_l^IN from its own ramp; 1: zero net volume flux */
} orc_params;

typedef struct {
  int lattice, D, Q;
  int n[3];
  long N;
  int v[19][3];
  double w[19];
  int opp[19];
  orc_params p;
  long t;
  int nthreads;
  double *f[6], *fp[6];
  double *Spp_g, *Spp_l, *Lam;      /* held fields S''_g, S''_l, Lambda' */
  /* per-node values of the current step that the boundary rules extrapolate */
  double *eps_g, *eps_l, *alB_g, *alB_l, *ug, *ul, *cg, *cl;
} orc;

/* ---------------------------------------------------------------- lattice */

/* D1Q3, D2Q9, D3Q19 built from their definitions: the velocities are the
 * vectors of {-1,0,1}^D (D3Q19: those with |v|^2 <= 2), the weights depend on
 * |v|^2 only (D1Q3: App. A, Eq. (D1Q3lattice); D2Q9/D3Q19: standard weights).
 * Index 0 is the rest velocity, as the delta_q of Eq. (delta) requires. */
static int lattice_build(orc *o, int lattice) {
  int D = lattice; /* 1 -> D1Q3, 2 -> D2Q9, 3 -> D3Q19 */
  double wt[3];
  if (lattice == 1) { wt[0] = 2.0 / 3.0; wt[1] = 1.0 / 6.0; wt[2] = 0.0; }
  else if (lattice == 2) { wt[0] = 4.0 / 9.0; wt[1] = 1.0 / 9.0; wt[2] = 1.0 / 36.0; }
  else if (lattice == 3) { wt[0] = 1.0 / 3.0; wt[1] = 1.0 / 18.0; wt[2] = 1.0 / 36.0; }
  else return -1;
  int Q = 0;
  o->v[0][0] = o->v[0][1] = o->v[0][2] = 0;
  o->w[0] = wt[0];
  Q = 1;
  int lim[3] = {1, D >= 2 ? 1 : 0, D >= 3 ? 1 : 0};
  for (int a = -lim[0]; a <= lim[0]; a++)
    for (int b = -lim[1]; b <= lim[1]; b++)
      for (int c = -lim[2]; c <= lim[2]; c++) {
        int m = a * a + b * b + c * c;
        if (m == 0 || m > 2) continue;
        o->v[Q][0] = a; o->v[Q][1] = b; o->v[Q][2] = c;
        o->w[Q] = wt[m];
        Q++;
      }
  o->D = D; o->Q = Q; o->lattice = lattice;
  for (int q = 0; q < Q; q++) {
    o->opp[q] = -1;
    for (int r = 0; r < Q; r++)
      if (o->v[r][0] == -o->v[q][0] && o->v[r][1] == -o->v[q][1] && o->v[r][2] == -o->v[q][2])
        o->opp[q] = r;
  }
  return 0;
}

/* ------------------------------------------------------------- equilibria */

static double dotv(const orc *o, int q, const double *u) {
  return o->v[q][0] * u[0] + o->v[q][1] * u[1] + o->v[q][2] * u[2];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Eq. (eta) with Eq. (delta): the rest weight absorbs the (1-phi) part. */
static double eta(const orc *o, int q, double phi) {
  double w0 = o->w[0];
  if (q == 0) return 1.0 + (1.0 - w0) / w0 * (1.0 - phi);
  return phi;
}

/* Incompressible equilibrium, Eq. (equilibriumI). */
static double feq_I(const orc *o, int q, double phi, double eps, const double *u) {
  double vu = dotv(o, q, u), uu = dot3(u, u);
  return o->w[q] * (eps * eta(o, q, phi) + vu / CS2 + (vu * vu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* Standard equilibrium, Eq. (equilibrium). */
static double feq_S(const orc *o, int q, double alpha, const double *u) {
  double vu = dotv(o, q, u), uu = dot3(u, u);
  return o->w[q] * alpha * (1.0 + vu / CS2 + (vu * vu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* Linearised forcing operator, Eq. (forcingoperator). */
static double feq_L(const orc *o, int q, double psi, double S, const double *G) {
  return o->w[q] * (S * eta(o, q, psi) + dotv(o, q, G) / CS2);
}

/* B(x) of Eq. (spalding).  reading: H(0) = 1/2 makes B continuous, i.e. B is
 * x clamped to [0,1]. */
static double spalding_B(double x) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  return x;
}

/* Eq. (transient); a non-positive n_t means no ramp (the maximum at once). */
static double ramp(const double mm[2], long t, int nt) {
  if (nt <= 0) return mm[1];
  return (mm[1] - mm[0]) * tanh((double)t / (double)nt) + mm[0];
}

static void coords(const orc *o, long i, int x[3]) {
  x[0] = (int)(i % o->n[0]);
  x[1] = (int)((i / o->n[0]) % o->n[1]);
  x[2] = (int)(i / ((long)o->n[0] * o->n[1]));
}
static long node_of(const orc *o, const int x[3]) {
  return x[0] + (long)o->n[0] * (x[1] + (long)o->n[1] * x[2]);
}

/* -------------------------------------------------------------- collision */

static void collide_node(orc *o, long i, int latch) {
  const int Q = o->Q, D = o->D;
  const orc_params *p = &o->p;
  const double *fg = o->f[S_G] + i * Q, *fl = o->f[S_L] + i * Q;
  const double *fag = o->f[S_AG] + i * Q, *fal = o->f[S_AL] + i * Q;
  const double *fbg = o->f[S_BG] + i * Q, *fbl = o->f[S_BL] + i * Q;

  /* Moments: Eqs. (momentzero), (momentfirst); second-order tensor Pi of
   * Sec. 2.1.2; Eq. (momentzeroapha) and the first moment of f_alpha,
   * Eq. (momentfirstalpha); Eq. (momentzerobeta). */
  double eps_g = 0, eps_l = 0, a_g = 0, a_l = 0, b_g = 0, b_l = 0;
  double u_g[3] = {0, 0, 0}, u_l[3] = {0, 0, 0}, J_g[3] = {0, 0, 0}, J_l[3] = {0, 0, 0};
  double Pi_g[3][3], Pi_l[3][3];
  memset(Pi_g, 0, sizeof Pi_g);
  memset(Pi_l, 0, sizeof Pi_l);
  for (int q = 0; q < Q; q++) {
    eps_g += fg[q]; eps_l += fl[q];
    a_g += fag[q]; a_l += fal[q];
    b_g += fbg[q]; b_l += fbl[q];
    for (int a = 0; a < D; a++) {
      u_g[a] += o->v[q][a] * fg[q];
      u_l[a] += o->v[q][a] * fl[q];
      J_g[a] += o->v[q][a] * fag[q];
      J_l[a] += o->v[q][a] * fal[q];
      for (int b = 0; b < D; b++) {
        Pi_g[a][b] += o->v[q][a] * o->v[q][b] * fg[q];
        Pi_l[a][b] += o->v[q][a] * o->v[q][b] * fl[q];
      }
    }
  }

  /* Continuity sources from the beta schemes, Eq. (lbmbetataylorzeroth5):
   * beta = 1 at the start of every step, so S = 1 - beta(t). */
  double S_g = 1.0 - b_g, S_l = 1.0 - b_l;

  /* Spalding renormalisation, Eq. (spalding); alpha_l^B = 1 - alpha_g^B.
   * reading: if B(a_g) + B(a_l) = 0 the node takes alpha_g^B = 1/2. */
  double al_g, al_l;
  if (p->spalding_mode == 0) {
    al_g = a_g; al_l = a_l;
  } else {
    double Bg = spalding_B(a_g), Bl = spalding_B(a_l);
    al_g = (Bg + Bl > 0.0) ? Bg / (Bg + Bl) : 0.5;
    al_l = 1.0 - al_g;
  }

  /* Pressure coupling, Eq. (lbm-phi-l); the gas uses phi_g = 1. */
  double phi = (1.0 + (eps_g - 1.0) / p->R) / eps_l;

  /* Ohwada dashpot, Eq. (lbm-cont-g1Dhat) and the third strategy of
   * Eq. (lbm-cont-l1Dhat), Gamma_l = phi*eps_l - 1.  reading: u^2 = |u|^2. */
  double Sp_g = S_g - p->gamma * dot3(u_g, u_g) * (eps_g - 1.0);
  double Sp_l = S_l - p->gamma * dot3(u_l, u_l) * (phi * eps_l - 1.0);

  /* Lagged update, Eqs. (lbm-cont-1D-update) and (Lambda-update), with
   * Lambda of Eq. (Lambda).  reading: latch when t is a multiple of n_gamma. */
  if (latch) {
    o->Spp_g[i] = Sp_g;
    o->Spp_l[i] = Sp_l;
    o->Lam[i] = al_g * al_l * (al_g + al_l * p->R);
  }
  double Spp_g = o->Spp_g[i], Spp_l = o->Spp_l[i], Lam = o->Lam[i];

  /* grad(alpha) from the first-moment non-equilibrium of f_alpha,
   * Eq. (gradlnalpha) multiplied by alpha.  reading: alpha*upsilon is the raw
   * first moment J and alpha is the raw zeroth moment a, so
   * grad(alpha) = (omega_alpha/cs2) (a u - J).  Then Eq. (spalding2). */
  double kgrad = p->omega_alpha / CS2;
  double gr_g[3] = {0, 0, 0}, gr_l[3] = {0, 0, 0}, dl[3], gG_g[3], gG_l[3];
  for (int a = 0; a < D; a++) {
    gr_g[a] = kgrad * (a_g * u_g[a] - J_g[a]);
    gr_l[a] = kgrad * (a_l * u_l[a] - J_l[a]);
  }
  for (int a = 0; a < 3; a++) {
    dl[a] = gr_g[a] + gr_l[a];
    gG_g[a] = gr_g[a] - 0.5 * dl[a];
    gG_l[a] = gr_l[a] - 0.5 * dl[a];
  }

  /* Stress from the non-equilibrium second moment.  Pi^eq from
   * Eq. (secondtensoreq).  D >= 2: Eq. (lbm-sigma3).  D = 1: Eq.
   * (taylor-second31Db) with nu^ef of Eq. (lbm-ef-viscosity).
   * reading: the source in the stress is the lagged S''. */
  double sg[3][3], sl[3][3];
  memset(sg, 0, sizeof sg);
  memset(sl, 0, sizeof sl);
  for (int a = 0; a < D; a++)
    for (int b = 0; b < D; b++) {
      double Peq_g = (a == b ? CS2 * eps_g : 0.0) + u_g[a] * u_g[b];
      double Peq_l = (a == b ? CS2 * phi * eps_l : 0.0) + u_l[a] * u_l[b];
      if (D == 1) {
        double nuef_g = (1.0 / p->omega_g - 0.5) - CS2 * p->psi_g / p->omega_g;
        double nuef_l = (1.0 / p->omega_l - 0.5) - CS2 * p->psi_l / p->omega_l;
        sg[a][b] = nuef_g * (p->omega_g * (Peq_g - Pi_g[a][b]) + p->psi_g * CS2 * Spp_g);
        sl[a][b] = nuef_l * (p->omega_l * (Peq_l - Pi_l[a][b]) + p->psi_l * CS2 * Spp_l);
      } else {
        sg[a][b] = (1.0 - 0.5 * p->omega_g) * (Peq_g - Pi_g[a][b]) - (a == b ? 0.5 * CS2 * p->psi_g * Spp_g : 0.0);
        sl[a][b] = (1.0 - 0.5 * p->omega_l) * (Peq_l - Pi_l[a][b]) - (a == b ? 0.5 * CS2 * p->psi_l * Spp_l : 0.0);
      }
    }

  /* Drag, Eq. (interphasemomentum) divided by alpha_phi*rho_phi, with the
   * Clift-Grace-Weber coefficient of Eq. (CliftGraceWeber); liquid wall
   * friction, Eq. (wallmomentum1D) (reading: friction opposes u_l, and the
   * CGW case uses K_W = kappa_W*Lambda').  Denominators use
   * max(alpha, alpha_floor). */
  double KI = p->drag_model == 1 ? p->kappa_I * Lam : p->kappa_I;
  double KW = p->drag_model == 1 ? p->kappa_W * Lam : p->kappa_W;
  double du[3], ag_d = al_g > p->alpha_floor ? al_g : p->alpha_floor;
  double al_d = al_l > p->alpha_floor ? al_l : p->alpha_floor;
  for (int a = 0; a < 3; a++) du[a] = u_l[a] - u_g[a];
  double ndu = sqrt(dot3(du, du)), nul = sqrt(dot3(u_l, u_l));

  /* Forces, Eqs. (Gg), (Gl); buoyancy in kinematic-pressure form,
   * Eq. (Gg1D): (R-1) g on the gas only.  reading: same form in any D. */
  double G_g[3] = {0, 0, 0}, G_l[3] = {0, 0, 0};
  for (int a = 0; a < D; a++) {
    double sgg = 0, slg = 0;
    for (int b = 0; b < D; b++) {
      sgg += sg[a][b] * gG_g[b];
      slg += sl[a][b] * gG_l[b];
    }
    G_g[a] = Spp_g * u_g[a] + sgg / ag_d + (a == p->g_axis ? (p->R - 1.0) * p->g_hat : 0.0) + KI * ndu * du[a] / ag_d;
    G_l[a] = Spp_l * u_l[a] + slg / al_d - KI * ndu * du[a] / (p->R * al_d) - KW * nul * u_l[a] / (p->R * al_d);
  }

  /* Collisions, Eqs. (lbmg), (lbml) with (colloperator) and the forcing
   * operator; Eq. (lbmalpha); Eq. (lbmbeta) with beta = 1 and the imposed
   * velocity of Eq. (velocitybeta).  reading: Spalding mode 2 relaxes f_alpha
   * towards the renormalised alpha^B, mode 0/1 towards the raw a. */
  double aeq_g = p->spalding_mode == 2 ? al_g : a_g;
  double aeq_l = p->spalding_mode == 2 ? al_l : a_l;
  double c_g[3], c_l[3];
  for (int a = 0; a < 3; a++) {
    c_g[a] = al_l * (u_g[a] - u_l[a]);
    c_l[a] = al_g * (u_l[a] - u_g[a]);
  }
  double *pg = o->fp[S_G] + i * Q, *pl = o->fp[S_L] + i * Q;
  double *pag = o->fp[S_AG] + i * Q, *pal = o->fp[S_AL] + i * Q;
  double *pbg = o->fp[S_BG] + i * Q, *pbl = o->fp[S_BL] + i * Q;
  for (int q = 0; q < Q; q++) {
    pg[q] = fg[q] + p->omega_g * (feq_I(o, q, 1.0, eps_g, u_g) - fg[q]) + feq_L(o, q, p->psi_g, Spp_g, G_g);
    pl[q] = fl[q] + p->omega_l * (feq_I(o, q, phi, eps_l, u_l) - fl[q]) + feq_L(o, q, p->psi_l, Spp_l, G_l);
    pag[q] = fag[q] + p->omega_alpha * (feq_S(o, q, aeq_g, u_g) - fag[q]);
    pal[q] = fal[q] + p->omega_alpha * (feq_S(o, q, aeq_l, u_l) - fal[q]);
    pbg[q] = feq_S(o, q, 1.0, c_g);
    pbl[q] = feq_S(o, q, 1.0, c_l);
  }

  o->eps_g[i] = eps_g; o->eps_l[i] = eps_l;
  o->alB_g[i] = al_g; o->alB_l[i] = al_l;
  for (int a = 0; a < 3; a++) {
    o->ug[3 * i + a] = u_g[a]; o->ul[3 * i + a] = u_l[a];
    o->cg[3 * i + a] = c_g[a]; o->cl[3 * i + a] = c_l[a];
  }
}

/* ------------------------------------------------------ boundary rules */

static int first_transverse(const orc *o) {
  for (int d = 0; d < o->D; d++)
    if (d != o->p.g_axis) return d;
  return -1;
}

/* Value streamed into node i along opp(q) when q leaves the domain through a
 * non-periodic face.  Wall: half-way bounce-back (Eq. (BCINLET), BB with zero
 * wall velocity, so Delta^BB = 0).  Inlet: Table 1.  Outlet: Table 2.
 * Extrapolations are Eqs. (BCIN), (BCOUT); the neighbour is one node inwards. */
static double bc_value(const orc *o, int s, long i, const int x[3], int q, int type) {
  const orc_params *p = &o->p;
  const double fpost = o->fp[s][i * o->Q + q];
  const int Q = o->Q;
  int ax = p->g_axis;
  if (type == ORC_WALL) return fpost;
  if (type == ORC_INLET) {
    int xn[3] = {x[0], x[1], x[2]};
    xn[ax] += 1;
    long in_ = node_of(o, xn);
    double aIN = ramp(p->in_alpha, o->t, p->ramp_nt);
    double ugIN = ramp(p->in_ug, o->t, p->ramp_nt);
    double ulIN = p->inlet_ul_mode == 1 ? -aIN * ugIN / (1.0 - aIN) : ramp(p->in_ul, o->t, p->ramp_nt);
    double uB[3] = {0, 0, 0}, muB[3] = {0, 0, 0};
    if (s == S_G || s == S_L) {
      /* BB(I): density EX(hw), velocity Dirichlet, Eq. (BB). */
      double epsB_g = 1.5 * o->eps_g[i] - 0.5 * o->eps_g[in_];
      double epsB_l = 1.5 * o->eps_l[i] - 0.5 * o->eps_l[in_];
      uB[ax] = (s == S_G) ? ugIN : ulIN;
      muB[ax] = -uB[ax];
      if (s == S_G) return fpost + feq_I(o, q, 1.0, epsB_g, muB) - feq_I(o, q, 1.0, epsB_g, uB);
      double phiB = (1.0 + (epsB_g - 1.0) / p->R) / epsB_l;
      return fpost + feq_I(o, q, phiB, epsB_l, muB) - feq_I(o, q, phiB, epsB_l, uB);
    }
    if (s == S_AG || s == S_AL) {
      /* EQ(S): alpha and u Dirichlet. */
      uB[ax] = (s == S_AG) ? ugIN : ulIN;
      double aB = (s == S_AG) ? aIN : 1.0 - aIN;
      return feq_S(o, o->opp[q], aB, uB);
    }
    /* EQ(S) for the beta schemes: beta and c EX(fw).  reading: the beta that
     * is extrapolated is the start-of-step beta = 1 at both nodes. */
    const double *c = (s == S_BG) ? o->cg : o->cl;
    double betaB = 2.0 * 1.0 - 1.0, cB[3];
    for (int a = 0; a < 3; a++) cB[a] = 2.0 * c[3 * i + a] - c[3 * in_ + a];
    return feq_S(o, o->opp[q], betaB, cB);
  }
  if (type == ORC_OUTLET) {
    int xn[3] = {x[0], x[1], x[2]};
    xn[ax] -= 1;
    long in_ = node_of(o, xn);
    double uB[3], muB[3];
    if (s == S_G || s == S_L || s == S_AG || s == S_AL) {
      const double *u = (s == S_G || s == S_AG) ? o->ug : o->ul;
      for (int a = 0; a < 3; a++) {
        uB[a] = 1.5 * u[3 * i + a] - 0.5 * u[3 * in_ + a];
        muB[a] = -uB[a];
      }
      if (s == S_G || s == S_L) {
        /* ABB(I): eps = 1 Dirichlet (so phi = 1), velocity EX(hw), Eq. (ABB). */
        return -fpost + feq_I(o, q, 1.0, 1.0, muB) + feq_I(o, q, 1.0, 1.0, uB);
      }
      /* ABB(S): alpha and u EX(hw). */
      const double *al = (s == S_AG) ? o->alB_g : o->alB_l;
      double aB = 1.5 * al[i] - 0.5 * al[in_];
      return -fpost + feq_S(o, q, aB, muB) + feq_S(o, q, aB, uB);
    }
    const double *c = (s == S_BG) ? o->cg : o->cl;
    double cB[3];
    for (int a = 0; a < 3; a++) cB[a] = 2.0 * c[3 * i + a] - c[3 * in_ + a];
    return feq_S(o, o->opp[q], 2.0 * 1.0 - 1.0, cB);
  }
  (void)Q;
  return fpost;
}

static void stream_all(orc *o) {
  const int Q = o->Q, D = o->D;
  const orc_params *p = &o->p;
  int tr = first_transverse(o);
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
  for (long i = 0; i < o->N; i++) {
    int x[3];
    coords(o, i, x);
    for (int q = 0; q < Q; q++) {
      int y[3] = {x[0], x[1], x[2]};
      int crossed = 0, type = ORC_PERIODIC;
      for (int d = 0; d < D; d++) {
        y[d] += o->v[q][d];
        int bc = -1;
        if (y[d] < 0) {
          bc = p->bc_lo[d];
          if (bc == ORC_PERIODIC) y[d] += o->n[d];
        } else if (y[d] >= o->n[d]) {
          bc = p->bc_hi[d];
          if (bc == ORC_PERIODIC) y[d] -= o->n[d];
        }
        if (bc > 0) {
          /* an inlet face acts as a wall outside the strip */
          if (bc == ORC_INLET && tr >= 0 && (x[tr] < p->inlet_lo || x[tr] >= p->inlet_hi)) bc = ORC_WALL;
          if (!crossed || bc == ORC_WALL) type = bc; /* a wall wins over inlet/outlet */
          crossed = 1;
        }
      }
      for (int s = 0; s < 6; s++) {
        if (!crossed) {
          o->f[s][node_of(o, y) * Q + q] = o->fp[s][i * Q + q];
        } else {
          o->f[s][i * Q + o->opp[q]] = bc_value(o, s, i, x, q, type);
        }
      }
    }
  }
}

/* ---------------------------------------------------------------- API */

orc *orc_create(int lattice, int nx, int ny, int nz, const orc_params *p) {
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  if (!o) return NULL;
  if (lattice_build(o, lattice)) { free(o); return NULL; }
  if ((o->D < 2 && ny != 1) || (o->D < 3 && nz != 1)) { free(o); return NULL; }
  o->n[0] = nx; o->n[1] = ny; o->n[2] = nz;
  o->N = (long)nx * ny * nz;
  o->p = *p;
  if (o->p.n_gamma < 1) o->p.n_gamma = 1;
  o->nthreads = 1;
  long NQ = o->N * o->Q;
  for (int s = 0; s < 6; s++) {
    o->f[s] = (double *)calloc(NQ, sizeof(double));
    o->fp[s] = (double *)calloc(NQ, sizeof(double));
  }
  o->Spp_g = calloc(o->N, sizeof(double));
  o->Spp_l = calloc(o->N, sizeof(double));
  o->Lam = calloc(o->N, sizeof(double));
  o->eps_g = calloc(o->N, sizeof(double));
  o->eps_l = calloc(o->N, sizeof(double));
  o->alB_g = calloc(o->N, sizeof(double));
  o->alB_l = calloc(o->N, sizeof(double));
  o->ug = calloc(3 * o->N, sizeof(double));
  o->ul = calloc(3 * o->N, sizeof(double));
  o->cg = calloc(3 * o->N, sizeof(double));
  o->cl = calloc(3 * o->N, sizeof(double));
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  for (int s = 0; s < 6; s++) { free(o->f[s]); free(o->fp[s]); }
  free(o->Spp_g); free(o->Spp_l); free(o->Lam);
  free(o->eps_g); free(o->eps_l); free(o->alB_g); free(o->alB_l);
  free(o->ug); free(o->ul); free(o->cg); free(o->cl);
  free(o);
}

void orc_set_threads(orc *o, int n) { o->nthreads = n > 0 ? n : 1; }
int orc_Q(const orc *o) { return o->Q; }
long orc_time(const orc *o) { return o->t; }
void orc_lattice(const orc *o, int *v, double *w, int *opp) {
  for (int q = 0; q < o->Q; q++) {
    for (int a = 0; a < 3; a++) v[3 * q + a] = o->v[q][a];
    w[q] = o->w[q];
    opp[q] = o->opp[q];
  }
}

/* Initial state: every scheme at its equilibrium.  reading: eps_g = p_k/cs2
 * (Eq. (sigmag1D)), eps_l = 1, phi from Eq. (lbm-phi-l), alpha_l = 1 - alpha_g,
 * f_beta at f^eq(1, c) with c of Eq. (velocitybeta); held S'' = 0 and
 * Lambda' = Lambda(alpha_g) (both are latched again at t = 0).
 * Vector fields are D consecutive planes of N values. */
void orc_init(orc *o, const double *alpha_g, const double *u_g, const double *u_l, const double *p_k) {
  const int Q = o->Q, D = o->D;
  for (long i = 0; i < o->N; i++) {
    double ug[3] = {0, 0, 0}, ul[3] = {0, 0, 0}, cg[3], cl[3];
    for (int a = 0; a < D; a++) { ug[a] = u_g[a * o->N + i]; ul[a] = u_l[a * o->N + i]; }
    double ag = alpha_g[i], al = 1.0 - ag;
    double eps_g = p_k[i] / CS2, eps_l = 1.0;
    double phi = (1.0 + (eps_g - 1.0) / o->p.R) / eps_l;
    for (int a = 0; a < 3; a++) { cg[a] = al * (ug[a] - ul[a]); cl[a] = ag * (ul[a] - ug[a]); }
    for (int q = 0; q < Q; q++) {
      o->f[S_G][i * Q + q] = feq_I(o, q, 1.0, eps_g, ug);
      o->f[S_L][i * Q + q] = feq_I(o, q, phi, eps_l, ul);
      o->f[S_AG][i * Q + q] = feq_S(o, q, ag, ug);
      o->f[S_AL][i * Q + q] = feq_S(o, q, al, ul);
      o->f[S_BG][i * Q + q] = feq_S(o, q, 1.0, cg);
      o->f[S_BL][i * Q + q] = feq_S(o, q, 1.0, cl);
    }
    o->Spp_g[i] = 0.0;
    o->Spp_l[i] = 0.0;
    o->Lam[i] = ag * al * (ag + al * o->p.R);
  }
  o->t = 0;
}

void orc_step(orc *o, long nsteps) {
  for (long k = 0; k < nsteps; k++) {
    int latch = (o->t % o->p.n_gamma) == 0;
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
    for (long i = 0; i < o->N; i++) collide_node(o, i, latch);
    stream_all(o);
    o->t++;
  }
}

/* Macroscopic fields of the current state, as the next step would see them:
 * alpha_g^B (Eq. (spalding)), u_g, u_l (D planes each), p_k = cs2*eps_g
 * (Eq. (sigmag1D)), S_g, S_l = 1 - beta (Eq. (lbmbetataylorzeroth5)).
 * Any output pointer may be NULL. */
void orc_moments(const orc *o, double *alpha_g, double *u_g, double *u_l, double *p_k, double *S_g, double *S_l) {
  const int Q = o->Q, D = o->D;
  for (long i = 0; i < o->N; i++) {
    double eg = 0, ag = 0, al = 0, bg = 0, bl = 0, ug[3] = {0, 0, 0}, ul[3] = {0, 0, 0};
    for (int q = 0; q < Q; q++) {
      eg += o->f[S_G][i * Q + q];
      ag += o->f[S_AG][i * Q + q];
      al += o->f[S_AL][i * Q + q];
      bg += o->f[S_BG][i * Q + q];
      bl += o->f[S_BL][i * Q + q];
      for (int a = 0; a < D; a++) {
        ug[a] += o->v[q][a] * o->f[S_G][i * Q + q];
        ul[a] += o->v[q][a] * o->f[S_L][i * Q + q];
      }
    }
    double alg = ag;
    if (o->p.spalding_mode != 0) {
      double Bg = spalding_B(ag), Bl = spalding_B(al);
      alg = (Bg + Bl > 0.0) ? Bg / (Bg + Bl) : 0.5;
    }
    if (alpha_g) alpha_g[i] = alg;
    for (int a = 0; a < D; a++) {
      if (u_g) u_g[a * o->N + i] = ug[a];
      if (u_l) u_l[a * o->N + i] = ul[a];
    }
    if (p_k) p_k[i] = CS2 * eg;
    if (S_g) S_g[i] = 1.0 - bg;
    if (S_l) S_l[i] = 1.0 - bl;
  }
}

/* Populations of scheme s in [q][node] order (q-major planes). */
void orc_get_pops(const orc *o, int s, double *out) {
  for (long i = 0; i < o->N; i++)
    for (int q = 0; q < o->Q; q++) out[(long)q * o->N + i] = o->f[s][i * o->Q + q];
}
void orc_set_pops(orc *o, int s, const double *in) {
  for (long i = 0; i < o->N; i++)
    for (int q = 0; q < o->Q; q++) o->f[s][i * o->Q + q] = in[(long)q * o->N + i];
}
void orc_get_held(const orc *o, double *Spp_g, double *Spp_l, double *Lam) {
  memcpy(Spp_g, o->Spp_g, o->N * sizeof(double));
  memcpy(Spp_l, o->Spp_l, o->N * sizeof(double));
  memcpy(Lam, o->Lam, o->N * sizeof(double));
}

/* Diagnostics of the current state: [0] sum a_g, [1] sum a_l, [2] sum
 * alpha_g^B, [3] sum (a_g + a_l - 1)^2, [4] max |u| over both phases,
 * [5] number of nodes holding a non-finite population, [6] sum (eps_g - 1),
 * [7] sum (eps_l - 1). */
void orc_diag(const orc *o, double out[8]) {
  const int Q = o->Q, D = o->D;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long i = 0; i < o->N; i++) {
    double eg = 0, el = 0, ag = 0, al = 0, ug[3] = {0, 0, 0}, ul[3] = {0, 0, 0};
    int bad = 0;
    for (int q = 0; q < Q; q++) {
      for (int k = 0; k < 6; k++)
        if (!isfinite(o->f[k][i * Q + q])) bad = 1;
      eg += o->f[S_G][i * Q + q];
      el += o->f[S_L][i * Q + q];
      ag += o->f[S_AG][i * Q + q];
      al += o->f[S_AL][i * Q + q];
      for (int a = 0; a < D; a++) {
        ug[a] += o->v[q][a] * o->f[S_G][i * Q + q];
        ul[a] += o->v[q][a] * o->f[S_L][i * Q + q];
      }
    }
    double alg = ag;
    if (o->p.spalding_mode != 0) {
      double Bg = spalding_B(ag), Bl = spalding_B(al);
      alg = (Bg + Bl > 0.0) ? Bg / (Bg + Bl) : 0.5;
    }
    s[0] += ag; s[1] += al; s[2] += alg;
    s[3] += (ag + al - 1.0) * (ag + al - 1.0);
    double mg = sqrt(dot3(ug, ug)), ml = sqrt(dot3(ul, ul));
    double m = mg > ml ? mg : ml;
    if (m > s[4]) s[4] = m;
    s[5] += bad;
    s[6] += eg - 1.0;
    s[7] += el - 1.0;
  }
  memcpy(out, s, sizeof s);
}

/* Equilibria of one lattice at one argument set, for the pins of App. A and
 * of the moment identities: fI = f_I^eq(phi, eps, u), fS = f^eq(alpha, u),
 * fL = f_L^eq(psi, S, G), each of length Q in this oracle's velocity order. */
void orc_equilibria(const orc *o, double phi, double eps, const double *u, double alpha, double psi,
                    double S, const double *G, double *fI, double *fS, double *fL) {
  double uu[3] = {0, 0, 0}, GG[3] = {0, 0, 0};
  for (int a = 0; a < o->D; a++) { uu[a] = u[a]; GG[a] = G[a]; }
  for (int q = 0; q < o->Q; q++) {
    fI[q] = feq_I(o, q, phi, eps, uu);
    fS[q] = feq_S(o, q, alpha, uu);
    fL[q] = feq_L(o, q, psi, S, GG);
  }
}
