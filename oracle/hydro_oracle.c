/*
 * hydro_oracle.c -- plain, slow, FP64 CPU oracle of the GenASiS nonrelativistic
 * hydrodynamics update (Cardall et al., arXiv:1207.3392, Sections 3.1-3.6).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker of the CUDA path: it
 * shares no code, header, table or constant with paper_1207_3392_gb300/csrc,
 * and only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  The product path never calls it.
 *
 * What it computes, in the paper's order (Algorithm 1 of Section 3.3):
 *   primitive recovery            Eqs. BalancedBaryonDensity..balancedEnergy, p=(gamma-1)e (Sec. 3.5)
 *   ghost cells / boundaries      Algorithm 1 "Apply Boundary Conditions"; see the note below
 *   limited differences           Eq. MinMod (Sec. 3.1)
 *   reconstructed face values     the two equations preceding Eq. MinMod
 *   reconstructed balanced, fluxes  Eqs. FluxBaryon..FluxMomentumFluid and the energy flux (Sec. 3.5)
 *   Riemann states                Eqs. conservedLeft..conservedRight (Sec. 3.2)
 *   wave speeds alpha_+-          definition following Eq. JumpConditionHLLPlus, lambda = v -+ c_s (Sec. 3.5)
 *   HLL flux                      Eq. FluxHLL
 *   HLLC flux                     Eqs. MiddleWaveSpeed, NormalVelocityMiddle..EnergyMiddle, FluxHLLC
 *   divergence (update)           Eq. BalanceEquationAverage with A_q/V = 1/dq (Cartesian)
 *   TVD RK2 (Heun)                Eqs. Update, RungeKutta1..RungeKutta3 (Sec. 3.4)
 *   CFL time step                 Eq. courantTimeStep and the C_CFL factor after it (Sec. 3.6)
 *   conserved totals              sums over cells of U dV (Sec. 3.3, conservation on leaf cells)
 *   external-force source         the source vector of the Rayleigh-Taylor test (Sec. 4.3.2),
 *                                 potential at cell centres, gradient by centred differences
 *
 * Readings where the paper is garbled or silent:
 *   - Eq. PressureMiddle as printed violates p*_L = p*_R (stated right after
 *     Eq. EnergyMiddle).  Re-deriving it from the normal-momentum jump condition
 *     Eq. JumpConditionHLLCMinus/Plus gives
 *        p*_L = p_L - rho_L (alpha_- + v_L)(alpha_m - v_L)
 *        p*_R = p_R + rho_R (alpha_+ - v_R)(alpha_m - v_R),
 *     which is what is coded; the unit test of p*_L == p*_R pins it.
 *   - Eq. EnergyMiddle has G* on both sides; the energy jump condition gives
 *     G_K (not G*_K) in the numerator, which is coded.
 *   - Star fluxes come from the outer jump conditions:
 *        F*_L = F_L + alpha_-(U_L - U*_L),  F*_R = F_R + alpha_+(U*_R - U_R).
 *   - Eq. FluxHLLC case order: alpha_- == 0 -> F_L, then alpha_+ == 0 -> F_R,
 *     then alpha_m >= 0 -> F*_L, else F*_R.
 *   - Boundary conditions: the paper applies them to reconstructed values.  Two
 *     layers of ghost cells filled from the interior (periodic wrap; reflecting
 *     mirror with the normal momentum negated; outflow copy of the edge cell)
 *     and reconstructed like interior cells give the same face values for the
 *     periodic and reflecting cases, because the limited reconstruction of a
 *     mirrored/wrapped ghost is the mirror/wrap of its partner's.
 *   - Non-uniform widths: q_c - q_- = (d_{i-1}+d_i)/2, q_+ - q_- =
 *     d_{i-1}/2 + d_i + d_{i+1}/2, q_+ - q_c = (d_i+d_{i+1})/2, face offsets d_i/2
 *     (cell centre = geometric centre in Cartesian coordinates).
 *   - Reconstructed primitive set W = (n, v, e); p = (gamma-1) e afterwards.
 *   - No floors: a non-positive density or pressure, or a non-finite value, in
 *     an interior cell makes the call return OG_ENONPHYS.
 * *   - m (average baryon mass) = 1 throughout, so rho = n.
 *   - HLLC with the shock switch (solver 2): a face normal to q takes the HLL
 *     flux when either of its two cells lies on a shock moving along another
 *     axis r != q (detector above, from the stage's input state); a ghost cell
 *     carries the flags of the interior cell it is filled from.
 *   - The source vector of Sec. 4.3.2 is printed without a sign; the force
 *     -grad Phi must pull the fluid down the potential, so the source is
 *     S = -[0, m D dPhi/dx_q, (S . grad Phi)] (momentum q and energy).
 *
 * Layout: structure of arrays, U[var][k][j][i], x fastest; nvar = ndim + 2
 * (D, S_1..S_ndim, G).  Interior arrays only cross this interface; ghost layers
 * live in private scratch.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

#define OG_NG 2

enum { OG_PERIODIC = 0, OG_REFLECT = 1, OG_OUTFLOW = 2 };
enum { OG_HLL = 0, OG_HLLC = 1, OG_HLLC_SWITCH = 2 };

/* Shock detector of the HLLC -> HLL switch (Sec. 3.2 describes the switch but
 * not the detector; this criterion is this implementation's reading): a cell
 * lies on a shock moving along axis r when, across its two neighbours along r,
 * the flow is compressive (v_r(+) - v_r(-) < 0) and the pressure jumps by more
 * than OG_SHOCK_JUMP of the smaller pressure. */
#define OG_SHOCK_JUMP 0.5
enum { OG_OK = 0, OG_EINVAL = -1, OG_ENOMEM = -2, OG_ENONPHYS = -4 };

typedef struct {
  int ndim;
  int n[3];
  const double *width[3];
  int bc_lo[3], bc_hi[3];
  double gamma;
  double theta;
  int solver;
  double grad_phi[3];  /* gradient of a linear external potential Phi = grad_phi . x; 0: no source */
} og_desc;

/* Grid with ghost layers. */
typedef struct {
  int ndim, nvar;
  int n[3], e[3], g[3];
  size_t next;               /* cells in the ghost-extended box */
  double *w[3];              /* widths including ghosts, length e[q] */
} og_grid;

static size_t og_at(const og_grid *G, int i, int j, int k) {
  return ((size_t)(k + G->g[2]) * G->e[1] + (size_t)(j + G->g[1])) * G->e[0] + (size_t)(i + G->g[0]);
}

/* Source index of ghost cell c (outside [0,n)) for boundary code bc; *flip = 1
 * when the normal momentum changes sign (reflecting wall). */
static int og_ghost_src(int c, int n, int bc, int *flip) {
  *flip = 0;
  if (c >= 0 && c < n) return c;
  if (bc == OG_PERIODIC) return ((c % n) + n) % n;
  if (bc == OG_REFLECT) { *flip = 1; return c < 0 ? -1 - c : 2 * n - 1 - c; }
  return c < 0 ? 0 : n - 1;  /* outflow */
}

static int og_grid_init(og_grid *G, const og_desc *d) {
  if (d->ndim < 1 || d->ndim > 3) return OG_EINVAL;
  memset(G, 0, sizeof(*G));
  G->ndim = d->ndim;
  G->nvar = d->ndim + 2;
  G->next = 1;
  for (int q = 0; q < 3; ++q) {
    int active = q < d->ndim;
    G->n[q] = active ? d->n[q] : 1;
    if (G->n[q] < 1) return OG_EINVAL;
    if (active && G->n[q] < OG_NG) return OG_EINVAL;
    G->g[q] = active ? OG_NG : 0;
    G->e[q] = G->n[q] + 2 * G->g[q];
    G->next *= (size_t)G->e[q];
  }
  for (int q = 0; q < d->ndim; ++q) {
    G->w[q] = (double *)malloc(sizeof(double) * G->e[q]);
    if (!G->w[q]) return OG_ENOMEM;
    for (int c = -OG_NG; c < G->n[q] + OG_NG; ++c) {
      int flip;
      int bc = c < 0 ? d->bc_lo[q] : d->bc_hi[q];
      int s = og_ghost_src(c, G->n[q], bc, &flip);
      double wv = d->width[q][s];
      if (!(wv > 0.0)) return OG_EINVAL;
      G->w[q][c + OG_NG] = wv;
    }
  }
  return OG_OK;
}

static void og_grid_free(og_grid *G) {
  for (int q = 0; q < 3; ++q) free(G->w[q]);
}

/* ---------------------------------------------------------------------------
 * Variable relations (Section 3.5): D = n, S = m n v, G = e + m n |v|^2 / 2,
 * p = (gamma - 1) e, c_s = sqrt(gamma p / rho), m = 1.
 * W holds (n, v_1..v_ndim, e); U holds (D, S_1..S_ndim, G).
 * ------------------------------------------------------------------------- */
static void og_prim_from_cons(int nd, const double *U, double *W) {
  double n = U[0];
  double v2 = 0.0;
  W[0] = n;
  for (int a = 0; a < nd; ++a) {
    W[1 + a] = U[1 + a] / n;
    v2 += W[1 + a] * W[1 + a];
  }
  W[nd + 1] = U[nd + 1] - 0.5 * n * v2;
}

static void og_cons_from_prim(int nd, const double *W, double *U) {
  double n = W[0];
  double v2 = 0.0;
  U[0] = n;
  for (int a = 0; a < nd; ++a) {
    U[1 + a] = n * W[1 + a];
    v2 += W[1 + a] * W[1 + a];
  }
  U[nd + 1] = W[nd + 1] + 0.5 * n * v2;
}

/* Physical flux along axis q (Eqs. FluxBaryon, FluxMomentumFluid, energy flux). */
static void og_phys_flux(int nd, int q, double gamma, const double *W, const double *U, double *F) {
  double vq = W[1 + q];
  double p = (gamma - 1.0) * W[nd + 1];
  F[0] = U[0] * vq;
  for (int a = 0; a < nd; ++a) F[1 + a] = U[1 + a] * vq + (a == q ? p : 0.0);
  F[nd + 1] = (U[nd + 1] + p) * vq;  /* (e + p + n|v|^2/2) v^q */
}

/* Riemann flux at one face (Section 3.2 and its hydrodynamic specialisation in
 * Section 3.5).  WL, WR: reconstructed primitives (n, v, e) on the left and
 * right of the face; q: normal axis.  diag (optional): alpha_+, alpha_-,
 * alpha_m, p*_L, p*_R (alpha_m and p* only for subsonic HLLC faces, else 0). */
static void og_face_flux(int solver, double gamma, int nd, int q,
                         const double *WL, const double *WR, double *F, double *diag) {
  int nv = nd + 2;
  double UL[5], UR[5], FL[5], FR[5];
  og_cons_from_prim(nd, WL, UL);
  og_cons_from_prim(nd, WR, UR);
  og_phys_flux(nd, q, gamma, WL, UL, FL);
  og_phys_flux(nd, q, gamma, WR, UR, FR);
  double pL = (gamma - 1.0) * WL[nd + 1], pR = (gamma - 1.0) * WR[nd + 1];
  double cL = sqrt(gamma * pL / WL[0]), cR = sqrt(gamma * pR / WR[0]);
  double vL = WL[1 + q], vR = WR[1 + q];
  /* alpha_+- = max[0, +-lambda_+-(U_L), +-lambda_+-(U_R)], lambda_+- = v +- c_s */
  double ap = fmax(0.0, fmax(vL + cL, vR + cR));
  double am = fmax(0.0, fmax(-(vL - cL), -(vR - cR)));
  if (diag) { diag[0] = ap; diag[1] = am; diag[2] = 0.0; diag[3] = 0.0; diag[4] = 0.0; }

  if (solver == OG_HLL) {
    /* Eq. FluxHLL */
    for (int v = 0; v < nv; ++v)
      F[v] = (ap * FL[v] + am * FR[v] - ap * am * (UR[v] - UL[v])) / (ap + am);
    return;
  }

  /* Eq. FluxHLLC */
  if (am == 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
  if (ap == 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }

  /* Eq. MiddleWaveSpeed (Batten et al.), m = 1 */
  double SL = UL[1 + q], SR = UR[1 + q];
  double DL = UL[0], DR = UR[0];
  double alpha_m = (SR * (ap - vR) + SL * (am + vL) - (pR - pL))
                 / (DR * (ap - vR) + DL * (am + vL));
  double pstarL = pL - DL * (am + vL) * (alpha_m - vL);
  double pstarR = pR + DR * (ap - vR) * (alpha_m - vR);
  if (diag) { diag[2] = alpha_m; diag[3] = pstarL; diag[4] = pstarR; }

  double Us[5];
  if (alpha_m >= 0.0) {
    /* left middle state: density jump, v*^q = alpha_m, transverse v unchanged,
     * energy jump; then F*_L = F_L + alpha_-(U_L - U*_L). */
    double Ds = DL * (am + vL) / (am + alpha_m);
    Us[0] = Ds;
    for (int a = 0; a < nd; ++a) Us[1 + a] = Ds * (a == q ? alpha_m : WL[1 + a]);
    Us[nd + 1] = ((am + vL) * UL[nd + 1] + vL * pL - alpha_m * pstarL) / (am + alpha_m);
    for (int v = 0; v < nv; ++v) F[v] = FL[v] + am * (UL[v] - Us[v]);
  } else {
    double Ds = DR * (ap - vR) / (ap - alpha_m);
    Us[0] = Ds;
    for (int a = 0; a < nd; ++a) Us[1 + a] = Ds * (a == q ? alpha_m : WR[1 + a]);
    Us[nd + 1] = ((ap - vR) * UR[nd + 1] - vR * pR + alpha_m * pstarR) / (ap - alpha_m);
    for (int v = 0; v < nv; ++v) F[v] = FR[v] + ap * (Us[v] - UR[v]);
  }
}

/* Minmod of three arguments (Eq. MinMod): zero unless all share a strict sign,
 * else the argument of smallest magnitude. */
static double og_minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

static int og_bad_state(int nd, const double *W, double gamma) {
  double p = (gamma - 1.0) * W[nd + 1];
  for (int v = 0; v < nd + 2; ++v)
    if (!isfinite(W[v])) return 1;
  return !(W[0] > 0.0) || !(p > 0.0);
}

/* Fill the two ghost layers of every active axis from the interior. */
static void og_fill_ghosts(const og_grid *G, const og_desc *d, double *Ue) {
  int nd = G->ndim;
  for (int q = 0; q < nd; ++q) {
    int lo[3] = {0, 0, 0}, hi[3] = {G->n[0], G->n[1], G->n[2]};
    lo[q] = -OG_NG; hi[q] = G->n[q] + OG_NG;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int c[3] = {i, j, k};
          if (c[q] >= 0 && c[q] < G->n[q]) continue;
          int flip;
          int bc = c[q] < 0 ? d->bc_lo[q] : d->bc_hi[q];
          int s[3] = {i, j, k};
          s[q] = og_ghost_src(c[q], G->n[q], bc, &flip);
          size_t dst = og_at(G, i, j, k), src = og_at(G, s[0], s[1], s[2]);
          for (int v = 0; v < G->nvar; ++v) {
            double val = Ue[(size_t)v * G->next + src];
            if (flip && v == 1 + q) val = -val;
            Ue[(size_t)v * G->next + dst] = val;
          }
        }
  }
}

/* L[U] = -sum_q (F_{q,i+1/2} - F_{q,i-1/2}) / dq_i  (Eq. BalanceEquationAverage,
 * Cartesian, no sources).  U and L are interior arrays. */
static int og_rhs_grid(const og_grid *G, const og_desc *d, const double *U, double *L) {
  int nd = G->ndim, nv = G->nvar;
  size_t ne = G->next;
  size_t nin = (size_t)G->n[0] * G->n[1] * G->n[2];
  double *Ue = (double *)malloc(sizeof(double) * nv * ne);
  double *We = (double *)malloc(sizeof(double) * nv * ne);
  double *Win = (double *)malloc(sizeof(double) * nv * ne);   /* inner-face values */
  double *Wout = (double *)malloc(sizeof(double) * nv * ne);  /* outer-face values */
  if (!Ue || !We || !Win || !Wout) { free(Ue); free(We); free(Win); free(Wout); return OG_ENOMEM; }
  for (size_t t = 0; t < nv * ne; ++t) Ue[t] = NAN;  /* corners stay NaN: never used */

  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        size_t src = ((size_t)k * G->n[1] + j) * G->n[0] + i, dst = og_at(G, i, j, k);
        for (int v = 0; v < nv; ++v) Ue[(size_t)v * ne + dst] = U[(size_t)v * nin + src];
      }
  og_fill_ghosts(G, d, Ue);

  /* primitive recovery on every cell of the extended box */
  int bad = 0;
  for (size_t t = 0; t < ne; ++t) {
    double u[5] = {0, 0, 0, 0, 0}, w[5];
    for (int v = 0; v < nv; ++v) u[v] = Ue[(size_t)v * ne + t];
    og_prim_from_cons(nd, u, w);
    for (int v = 0; v < nv; ++v) We[(size_t)v * ne + t] = w[v];
  }
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        double w[5];
        size_t t = og_at(G, i, j, k);
        for (int v = 0; v < nv; ++v) w[v] = We[(size_t)v * ne + t];
        if (og_bad_state(nd, w, d->gamma)) bad = 1;
      }

  for (size_t t = 0; t < nv * nin; ++t) L[t] = 0.0;

  /* shock flags of the interior cells (bit r: on a shock moving along r) */
  unsigned char *flag = NULL;
  if (d->solver == OG_HLLC_SWITCH) {
    flag = (unsigned char *)calloc(nin, 1);
    if (!flag) { free(Ue); free(We); free(Win); free(Wout); return OG_ENOMEM; }
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          unsigned char bits = 0;
          for (int r = 0; r < nd; ++r) {
            int cm[3] = {i, j, k}, cp[3] = {i, j, k};
            cm[r] -= 1; cp[r] += 1;
            size_t tm = og_at(G, cm[0], cm[1], cm[2]), tp = og_at(G, cp[0], cp[1], cp[2]);
            double pm = (d->gamma - 1.0) * We[(size_t)(nd + 1) * ne + tm];
            double pp = (d->gamma - 1.0) * We[(size_t)(nd + 1) * ne + tp];
            double vm = We[(size_t)(1 + r) * ne + tm], vp = We[(size_t)(1 + r) * ne + tp];
            if (vp - vm < 0.0 && fabs(pp - pm) > OG_SHOCK_JUMP * fmin(pp, pm)) bits |= (unsigned char)(1u << r);
          }
          flag[((size_t)k * G->n[1] + j) * G->n[0] + i] = bits;
        }
  }

  for (int q = 0; q < nd; ++q) {
    const double *wq = G->w[q];  /* wq[c + NG] = width of cell c along q */
    /* differences and reconstructed face values: interior cells plus one
     * ghost on each side along q */
    int lo[3] = {0, 0, 0}, hi[3] = {G->n[0], G->n[1], G->n[2]};
    lo[q] = -1; hi[q] = G->n[q] + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int c[3] = {i, j, k};
          int cq = c[q];
          int cm[3] = {i, j, k}, cp[3] = {i, j, k};
          cm[q] -= 1; cp[q] += 1;
          size_t tc = og_at(G, i, j, k), tm = og_at(G, cm[0], cm[1], cm[2]), tp = og_at(G, cp[0], cp[1], cp[2]);
          double dm = wq[cq - 1 + OG_NG], dc = wq[cq + OG_NG], dp = wq[cq + 1 + OG_NG];
          double dist_cm = 0.5 * (dm + dc);          /* q_c - q_- */
          double dist_pm = 0.5 * dm + dc + 0.5 * dp; /* q_+ - q_- */
          double dist_pc = 0.5 * (dc + dp);          /* q_+ - q_c */
          for (int v = 0; v < nv; ++v) {
            double Wc = We[(size_t)v * ne + tc], Wm = We[(size_t)v * ne + tm], Wp = We[(size_t)v * ne + tp];
            double D = og_minmod3(d->theta * ((Wc - Wm) / dist_cm),
                                  (Wp - Wm) / dist_pm,
                                  d->theta * ((Wp - Wc) / dist_pc));
            Win[(size_t)v * ne + tc] = Wc - D * (0.5 * dc);
            Wout[(size_t)v * ne + tc] = Wc + D * (0.5 * dc);
          }
        }
    /* faces i-1/2 for i in [0, n_q]: left state = outer value of cell i-1,
     * right state = inner value of cell i (Eqs. conservedLeft..conservedRight).
     * Each face flux is applied to both neighbours. */
    int flo[3] = {0, 0, 0}, fhi[3] = {G->n[0], G->n[1], G->n[2]};
    fhi[q] = G->n[q] + 1;
    /* Loop over lines along q so the two updates of one face stay in one thread. */
    int t1 = (q == 0) ? 1 : 0, t2 = (q == 2) ? 1 : 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < G->n[t2]; ++b)
      for (int a = 0; a < G->n[t1]; ++a)
        for (int f = flo[q]; f < fhi[q]; ++f) {
          int c[3];
          c[q] = f; c[t1] = a; c[t2] = b;
          int cl[3] = {c[0], c[1], c[2]};
          cl[q] -= 1;
          size_t tr = og_at(G, c[0], c[1], c[2]), tl = og_at(G, cl[0], cl[1], cl[2]);
          double WL[5], WR[5], F[5];
          for (int v = 0; v < nv; ++v) { WL[v] = Wout[(size_t)v * ne + tl]; WR[v] = Win[(size_t)v * ne + tr]; }
          int solver = d->solver;
          if (solver == OG_HLLC_SWITCH) {
            /* flags of the two cells; a ghost (along q) takes its source cell's */
            int fl_, sl[3] = {cl[0], cl[1], cl[2]}, sr[3] = {c[0], c[1], c[2]};
            if (sl[q] < 0) sl[q] = og_ghost_src(sl[q], G->n[q], d->bc_lo[q], &fl_);
            if (sr[q] >= G->n[q]) sr[q] = og_ghost_src(sr[q], G->n[q], d->bc_hi[q], &fl_);
            unsigned char bits = flag[((size_t)sl[2] * G->n[1] + sl[1]) * G->n[0] + sl[0]] |
                                 flag[((size_t)sr[2] * G->n[1] + sr[1]) * G->n[0] + sr[0]];
            solver = (bits & (unsigned char)~(1u << q)) ? OG_HLL : OG_HLLC;
          }
          og_face_flux(solver, d->gamma, nd, q, WL, WR, F, NULL);
          if (f >= 1) {          /* outer face of cell f-1 */
            size_t li = ((size_t)cl[2] * G->n[1] + cl[1]) * G->n[0] + cl[0];
            double inv = 1.0 / wq[f - 1 + OG_NG];
            for (int v = 0; v < nv; ++v) L[(size_t)v * nin + li] -= F[v] * inv;
          }
          if (f < G->n[q]) {     /* inner face of cell f */
            size_t li = ((size_t)c[2] * G->n[1] + c[1]) * G->n[0] + c[0];
            double inv = 1.0 / wq[f + OG_NG];
            for (int v = 0; v < nv; ++v) L[(size_t)v * nin + li] += F[v] * inv;
          }
        }
  }
  /* External-force source (Sec. 4.3.2): Phi = grad_phi . x at the cell centres,
   * its gradient along q by the centred difference over the two neighbour
   * centres (exact for this linear potential up to rounding), then
   * S_q += -D dPhi/dq and G += -S_q dPhi/dq from the cell's own U. */
  if (d->grad_phi[0] != 0.0 || d->grad_phi[1] != 0.0 || d->grad_phi[2] != 0.0) {
    for (int q = 0; q < nd; ++q) {
      if (d->grad_phi[q] == 0.0) continue;
      const double *wq = G->w[q];
      /* centre coordinates of cells -1 .. n_q (origin at the low face of cell 0) */
      double *xc = (double *)malloc(sizeof(double) * (G->n[q] + 2));
      if (!xc) { free(flag); free(Ue); free(We); free(Win); free(Wout); return OG_ENOMEM; }
      xc[1] = 0.5 * wq[OG_NG];
      for (int c = 1; c < G->n[q]; ++c) xc[c + 1] = xc[c] + 0.5 * (wq[c - 1 + OG_NG] + wq[c + OG_NG]);
      xc[0] = xc[1] - 0.5 * (wq[OG_NG - 1] + wq[OG_NG]);
      xc[G->n[q] + 1] = xc[G->n[q]] + 0.5 * (wq[G->n[q] - 1 + OG_NG] + wq[G->n[q] + OG_NG]);
      for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
          for (int i = 0; i < G->n[0]; ++i) {
            int c[3] = {i, j, k};
            int cq = c[q];
            double phim = d->grad_phi[q] * xc[cq], phip = d->grad_phi[q] * xc[cq + 2];
            double dphi = (phip - phim) / (xc[cq + 2] - xc[cq]);
            size_t li = ((size_t)k * G->n[1] + j) * G->n[0] + i;
            double D = U[li], Sq = U[(size_t)(1 + q) * nin + li];
            L[(size_t)(1 + q) * nin + li] -= D * dphi;
            L[(size_t)(nv - 1) * nin + li] -= Sq * dphi;
          }
      free(xc);
    }
  }
  free(flag);
  free(Ue); free(We); free(Win); free(Wout);
  return bad ? OG_ENONPHYS : OG_OK;
}

/* ------------------------------- public API -------------------------------- */

int og_rhs(const og_desc *d, const double *U, double *L) {
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc == OG_OK) rc = og_rhs_grid(&G, d, U, L);
  og_grid_free(&G);
  return rc;
}

/* One TVD RK2 (Heun) step, in place: K1 = dt L[U^n], U1 = U^n + K1,
 * K2 = dt L[U1], U^{n+1} = U^n + (K1 + K2)/2  (Eqs. Update, RungeKutta1-3). */
int og_step(const og_desc *d, double *U, double dt) {
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc != OG_OK) { og_grid_free(&G); return rc; }
  size_t nin = (size_t)G.n[0] * G.n[1] * G.n[2], tot = nin * G.nvar;
  double *K1 = (double *)malloc(sizeof(double) * tot);
  double *K2 = (double *)malloc(sizeof(double) * tot);
  double *U1 = (double *)calloc(tot, sizeof(double));
  if (!K1 || !K2 || !U1) { rc = OG_ENOMEM; goto out; }
  rc = og_rhs_grid(&G, d, U, K1);
  if (rc != OG_OK) goto out;
  for (size_t t = 0; t < tot; ++t) { K1[t] *= dt; U1[t] = U[t] + K1[t]; }
  rc = og_rhs_grid(&G, d, U1, K2);
  if (rc != OG_OK) goto out;
  for (size_t t = 0; t < tot; ++t) { K2[t] *= dt; U[t] = U[t] + 0.5 * (K1[t] + K2[t]); }
out:
  free(K1); free(K2); free(U1);
  og_grid_free(&G);
  return rc;
}

/* dt_CFL = min over cells of min_q dq / max(|lambda_-|, |lambda_+|)
 * (Eq. courantTimeStep); the caller multiplies by C_CFL. */
int og_cfl_dt(const og_desc *d, const double *U, double *dt_cfl) {
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc != OG_OK) { og_grid_free(&G); return rc; }
  int nd = G.ndim, nv = G.nvar;
  size_t nin = (size_t)G.n[0] * G.n[1] * G.n[2];
  double best = INFINITY;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        size_t t = ((size_t)k * G.n[1] + j) * G.n[0] + i;
        double u[5], w[5];
        for (int v = 0; v < nv; ++v) u[v] = U[(size_t)v * nin + t];
        og_prim_from_cons(nd, u, w);
        if (og_bad_state(nd, w, d->gamma)) rc = OG_ENONPHYS;
        double p = (d->gamma - 1.0) * w[nd + 1];
        double cs = sqrt(d->gamma * p / w[0]);
        int c[3] = {i, j, k};
        for (int q = 0; q < nd; ++q) {
          double lm = w[1 + q] - cs, lp = w[1 + q] + cs;
          double s = fmax(fabs(lm), fabs(lp));
          double val = d->width[q][c[q]] / s;
          if (val < best) best = val;
        }
      }
  *dt_cfl = best;
  og_grid_free(&G);
  return rc;
}

/* Conserved totals: sum over interior cells of U_v * dV, dV = prod_q dq. */
int og_totals(const og_desc *d, const double *U, double *tot) {
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc != OG_OK) { og_grid_free(&G); return rc; }
  int nd = G.ndim, nv = G.nvar;
  size_t nin = (size_t)G.n[0] * G.n[1] * G.n[2];
  for (int v = 0; v < nv; ++v) tot[v] = 0.0;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        size_t t = ((size_t)k * G.n[1] + j) * G.n[0] + i;
        double dV = d->width[0][i];
        if (nd > 1) dV *= d->width[1][j];
        if (nd > 2) dV *= d->width[2][k];
        for (int v = 0; v < nv; ++v) tot[v] += U[(size_t)v * nin + t] * dV;
      }
  og_grid_free(&G);
  return rc;
}

/* Evolve from t = 0: repeat { dt = C_CFL dt_CFL; clamp the last step to t_end;
 * one RK2 step } while t < t_end (Algorithm Evolve, single level).  With
 * t_end <= 0 it takes exactly max_steps steps. */
int og_evolve(const og_desc *d, double *U, double cfl, double t_end, int max_steps,
              double *t_out, int *steps_out) {
  double t = 0.0;
  int steps = 0, rc = OG_OK;
  while ((t_end > 0.0 ? t < t_end : 1) && steps < max_steps) {
    double dtc;
    rc = og_cfl_dt(d, U, &dtc);
    if (rc != OG_OK) break;
    double dt = cfl * dtc;
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    rc = og_step(d, U, dt);
    if (rc != OG_OK) break;
    t += dt;
    ++steps;
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return rc;
}

/* Conversions for whole interior arrays.  vel holds ndim planes. */
int og_prim_to_cons(const og_desc *d, const double *rho, const double *vel, const double *p, double *U) {
  int nd = d->ndim;
  size_t nin = 1;
  for (int q = 0; q < nd; ++q) nin *= (size_t)d->n[q];
  for (size_t t = 0; t < nin; ++t) {
    double w[5], u[5];
    w[0] = rho[t];
    for (int a = 0; a < nd; ++a) w[1 + a] = vel[(size_t)a * nin + t];
    w[nd + 1] = p[t] / (d->gamma - 1.0);
    og_cons_from_prim(nd, w, u);
    for (int v = 0; v < nd + 2; ++v) U[(size_t)v * nin + t] = u[v];
  }
  return OG_OK;
}

int og_cons_to_prim(const og_desc *d, const double *U, double *rho, double *vel, double *p) {
  int nd = d->ndim, rc = OG_OK;
  size_t nin = 1;
  for (int q = 0; q < nd; ++q) nin *= (size_t)d->n[q];
  for (size_t t = 0; t < nin; ++t) {
    double w[5], u[5];
    for (int v = 0; v < nd + 2; ++v) u[v] = U[(size_t)v * nin + t];
    og_prim_from_cons(nd, u, w);
    if (og_bad_state(nd, w, d->gamma)) rc = OG_ENONPHYS;
    rho[t] = w[0];
    for (int a = 0; a < nd; ++a) vel[(size_t)a * nin + t] = w[1 + a];
    p[t] = (d->gamma - 1.0) * w[nd + 1];
  }
  return rc;
}

/* Single-face Riemann flux from primitive (rho, v[ndim], p) states, for unit
 * tests of the solvers in isolation.  diag as in og_face_flux. */
int og_riemann_flux(int solver, double gamma, int nd, int q,
                    const double *primL, const double *primR, double *F, double *diag) {
  double WL[5], WR[5];
  WL[0] = primL[0]; WR[0] = primR[0];
  for (int a = 0; a < nd; ++a) { WL[1 + a] = primL[1 + a]; WR[1 + a] = primR[1 + a]; }
  WL[nd + 1] = primL[nd + 1] / (gamma - 1.0);
  WR[nd + 1] = primR[nd + 1] / (gamma - 1.0);
  og_face_flux(solver, gamma, nd, q, WL, WR, F, diag);
  return OG_OK;
}

/* Physical flux F^q(U(prim)) for tests. */
int og_physical_flux(double gamma, int nd, int q, const double *prim, double *F) {
  double W[5], U[5];
  W[0] = prim[0];
  for (int a = 0; a < nd; ++a) W[1 + a] = prim[1 + a];
  W[nd + 1] = prim[nd + 1] / (gamma - 1.0);
  og_cons_from_prim(nd, W, U);
  og_phys_flux(nd, q, gamma, W, U, F);
  return OG_OK;
}

/* Plain face fluxes of a 2D state (the fluxes og_rhs differences), for the
 * learned-correction reference: Fx [nv][ny][nx+1] (face i between cells i-1
 * and i of row j), Fy [nv][ny+1][nx].  Same ghost filling, recovery,
 * reconstruction and Riemann solver as og_rhs_grid. */
int og_face_fluxes_2d(const og_desc *d, const double *U, double *Fx, double *Fy) {
  if (d->ndim != 2) return OG_EINVAL;
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc != OG_OK) { og_grid_free(&G); return rc; }
  int nv = G.nvar;
  size_t ne = G.next, nin = (size_t)G.n[0] * G.n[1];
  double *Ue = (double *)malloc(sizeof(double) * nv * ne);
  double *We = (double *)malloc(sizeof(double) * nv * ne);
  double *Win = (double *)malloc(sizeof(double) * nv * ne);
  double *Wout = (double *)malloc(sizeof(double) * nv * ne);
  if (!Ue || !We || !Win || !Wout) { rc = OG_ENOMEM; goto out; }
  for (size_t t = 0; t < nv * ne; ++t) Ue[t] = NAN;
  for (int j = 0; j < G.n[1]; ++j)
    for (int i = 0; i < G.n[0]; ++i)
      for (int v = 0; v < nv; ++v) Ue[(size_t)v * ne + og_at(&G, i, j, 0)] = U[(size_t)v * nin + (size_t)j * G.n[0] + i];
  og_fill_ghosts(&G, d, Ue);
  for (size_t t = 0; t < ne; ++t) {
    double u[5] = {0, 0, 0, 0, 0}, w[5];
    for (int v = 0; v < nv; ++v) u[v] = Ue[(size_t)v * ne + t];
    og_prim_from_cons(2, u, w);
    for (int v = 0; v < nv; ++v) We[(size_t)v * ne + t] = w[v];
  }
  for (int q = 0; q < 2; ++q) {
    const double *wq = G.w[q];
    int lo[2] = {0, 0}, hi[2] = {G.n[0], G.n[1]};
    lo[q] = -1; hi[q] = G.n[q] + 1;
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i) {
        int c[2] = {i, j}, cm[2] = {i, j}, cp[2] = {i, j};
        cm[q] -= 1; cp[q] += 1;
        size_t tc = og_at(&G, i, j, 0), tm = og_at(&G, cm[0], cm[1], 0), tp = og_at(&G, cp[0], cp[1], 0);
        double dm = wq[c[q] - 1 + OG_NG], dc = wq[c[q] + OG_NG], dp = wq[c[q] + 1 + OG_NG];
        double dist_cm = 0.5 * (dm + dc), dist_pm = 0.5 * dm + dc + 0.5 * dp, dist_pc = 0.5 * (dc + dp);
        for (int v = 0; v < nv; ++v) {
          double Wc = We[(size_t)v * ne + tc], Wm = We[(size_t)v * ne + tm], Wp = We[(size_t)v * ne + tp];
          double D = og_minmod3(d->theta * ((Wc - Wm) / dist_cm), (Wp - Wm) / dist_pm, d->theta * ((Wp - Wc) / dist_pc));
          Win[(size_t)v * ne + tc] = Wc - D * (0.5 * dc);
          Wout[(size_t)v * ne + tc] = Wc + D * (0.5 * dc);
        }
      }
    int nfx = q == 0 ? G.n[0] + 1 : G.n[0], nfy = q == 0 ? G.n[1] : G.n[1] + 1;
    double *Fo = q == 0 ? Fx : Fy;
    for (int j = 0; j < nfy; ++j)
      for (int i = 0; i < nfx; ++i) {
        int cr[2] = {i, j}, cl[2] = {i, j};
        cl[q] -= 1;
        double WL[5], WR[5], F[5];
        for (int v = 0; v < nv; ++v) {
          WL[v] = Wout[(size_t)v * ne + og_at(&G, cl[0], cl[1], 0)];
          WR[v] = Win[(size_t)v * ne + og_at(&G, cr[0], cr[1], 0)];
        }
        og_face_flux(d->solver, d->gamma, 2, q, WL, WR, F, NULL);
        for (int v = 0; v < nv; ++v) Fo[((size_t)v * nfy + j) * nfx + i] = F[v];
      }
  }
out:
  free(Ue); free(We); free(Win); free(Wout);
  og_grid_free(&G);
  return rc;
}

/* Plain face fluxes of a state in 1, 2 or 3 dimensions: F[q] holds, for axis
 * q, [nv][faces] with the faces of axis q in x-fastest order over
 * (n_0 + (q==0)) x (n_1 + (q==1)) x (n_2 + (q==2)); face index f along q lies
 * between cells f-1 and f.  Same ghost filling, recovery, reconstruction and
 * Riemann solver (including the shock switch) as og_rhs_grid, which this
 * repeats without the divergence. */
int og_face_fluxes(const og_desc *d, const double *U, double *F0, double *F1, double *F2) {
  og_grid G;
  int rc = og_grid_init(&G, d);
  if (rc != OG_OK) { og_grid_free(&G); return rc; }
  int nd = G.ndim, nv = G.nvar;
  size_t ne = G.next, nin = (size_t)G.n[0] * G.n[1] * G.n[2];
  double *Fq[3] = {F0, F1, F2};
  double *Ue = (double *)malloc(sizeof(double) * nv * ne);
  double *We = (double *)malloc(sizeof(double) * nv * ne);
  double *Win = (double *)malloc(sizeof(double) * nv * ne);
  double *Wout = (double *)malloc(sizeof(double) * nv * ne);
  double *L = (double *)malloc(sizeof(double) * nv * nin);
  unsigned char *flag = NULL;
  if (!Ue || !We || !Win || !Wout || !L) { rc = OG_ENOMEM; goto done; }
  /* the divergence is not needed, but og_rhs_grid's flags and face loops are
   * reproduced here face by face */
  for (size_t t = 0; t < nv * ne; ++t) Ue[t] = NAN;
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i)
        for (int v = 0; v < nv; ++v)
          Ue[(size_t)v * ne + og_at(&G, i, j, k)] = U[(size_t)v * nin + ((size_t)k * G.n[1] + j) * G.n[0] + i];
  og_fill_ghosts(&G, d, Ue);
  for (size_t t = 0; t < ne; ++t) {
    double u[5] = {0, 0, 0, 0, 0}, w[5];
    for (int v = 0; v < nv; ++v) u[v] = Ue[(size_t)v * ne + t];
    og_prim_from_cons(nd, u, w);
    for (int v = 0; v < nv; ++v) We[(size_t)v * ne + t] = w[v];
  }
  if (d->solver == OG_HLLC_SWITCH) {
    flag = (unsigned char *)calloc(nin, 1);
    if (!flag) { rc = OG_ENOMEM; goto done; }
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          unsigned char bits = 0;
          for (int r = 0; r < nd; ++r) {
            int cm[3] = {i, j, k}, cp[3] = {i, j, k};
            cm[r] -= 1; cp[r] += 1;
            size_t tm = og_at(&G, cm[0], cm[1], cm[2]), tp = og_at(&G, cp[0], cp[1], cp[2]);
            double pm = (d->gamma - 1.0) * We[(size_t)(nd + 1) * ne + tm];
            double pp = (d->gamma - 1.0) * We[(size_t)(nd + 1) * ne + tp];
            double vm = We[(size_t)(1 + r) * ne + tm], vp = We[(size_t)(1 + r) * ne + tp];
            if (vp - vm < 0.0 && fabs(pp - pm) > OG_SHOCK_JUMP * fmin(pp, pm)) bits |= (unsigned char)(1u << r);
          }
          flag[((size_t)k * G.n[1] + j) * G.n[0] + i] = bits;
        }
  }
  for (int q = 0; q < nd; ++q) {
    const double *wq = G.w[q];
    int lo[3] = {0, 0, 0}, hi[3] = {G.n[0], G.n[1], G.n[2]};
    lo[q] = -1; hi[q] = G.n[q] + 1;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int c[3] = {i, j, k}, cm[3] = {i, j, k}, cp[3] = {i, j, k};
          cm[q] -= 1; cp[q] += 1;
          size_t tc = og_at(&G, i, j, k), tm = og_at(&G, cm[0], cm[1], cm[2]), tp = og_at(&G, cp[0], cp[1], cp[2]);
          double dm = wq[c[q] - 1 + OG_NG], dc = wq[c[q] + OG_NG], dp = wq[c[q] + 1 + OG_NG];
          double dist_cm = 0.5 * (dm + dc), dist_pm = 0.5 * dm + dc + 0.5 * dp, dist_pc = 0.5 * (dc + dp);
          for (int v = 0; v < nv; ++v) {
            double Wc = We[(size_t)v * ne + tc], Wm = We[(size_t)v * ne + tm], Wp = We[(size_t)v * ne + tp];
            double D = og_minmod3(d->theta * ((Wc - Wm) / dist_cm), (Wp - Wm) / dist_pm, d->theta * ((Wp - Wc) / dist_pc));
            Win[(size_t)v * ne + tc] = Wc - D * (0.5 * dc);
            Wout[(size_t)v * ne + tc] = Wc + D * (0.5 * dc);
          }
        }
    int nf[3] = {G.n[0], G.n[1], G.n[2]};
    nf[q] += 1;
    size_t nfaces = (size_t)nf[0] * nf[1] * nf[2];
    for (int k = 0; k < nf[2]; ++k)
      for (int j = 0; j < nf[1]; ++j)
        for (int i = 0; i < nf[0]; ++i) {
          int cr[3] = {i, j, k}, cl[3] = {i, j, k};
          cl[q] -= 1;
          double WL[5], WR[5], F[5];
          for (int v = 0; v < nv; ++v) {
            WL[v] = Wout[(size_t)v * ne + og_at(&G, cl[0], cl[1], cl[2])];
            WR[v] = Win[(size_t)v * ne + og_at(&G, cr[0], cr[1], cr[2])];
          }
          int solver = d->solver;
          if (solver == OG_HLLC_SWITCH) {
            int fl_, sl[3] = {cl[0], cl[1], cl[2]}, sr[3] = {cr[0], cr[1], cr[2]};
            if (sl[q] < 0) sl[q] = og_ghost_src(sl[q], G.n[q], d->bc_lo[q], &fl_);
            if (sr[q] >= G.n[q]) sr[q] = og_ghost_src(sr[q], G.n[q], d->bc_hi[q], &fl_);
            unsigned char bits = flag[((size_t)sl[2] * G.n[1] + sl[1]) * G.n[0] + sl[0]] |
                                 flag[((size_t)sr[2] * G.n[1] + sr[1]) * G.n[0] + sr[0]];
            solver = (bits & (unsigned char)~(1u << q)) ? OG_HLL : OG_HLLC;
          }
          og_face_flux(solver, d->gamma, nd, q, WL, WR, F, NULL);
          for (int v = 0; v < nv; ++v) Fq[q][(size_t)v * nfaces + ((size_t)k * nf[1] + j) * nf[0] + i] = F[v];
        }
  }
  free(flag);
done:
  free(Ue); free(We); free(Win); free(Wout); free(L);
  og_grid_free(&G);
  return rc;
}

/* Exposed for the limiter unit test. */
double og_minmod(double a, double b, double c) { return og_minmod3(a, b, c); }
