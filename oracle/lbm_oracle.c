/*
 * CPU FP64 oracle of one time step of the coupled pseudopotential LBM + FD energy
 * equation of arXiv 2201.04560 (Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference the
 * CUDA library is checked against. Only tests/, __graft_entry__.smoke() and the CPU
 * baseline of bench.py may build, load or run it. It shares no code, header,
 * table or helper with the CUDA path. Compile with -ffp-contract=off.
 *
 * Every quantity is a full-grid FP64 array and every stage is a plain loop over all
 * nodes, in the order of the paper's model:
 *   rho (Eq. DensityAndVelocityRelationToF) -> p_EOS (Eq. peng-robinson) -> psi (Eq. psi)
 *   -> F^m with the wall form (Eqs. shanchen, shanchen-walls, psi-based-formula)
 *   -> F^b (Eq. gravitational_force) -> u (Eq. DensityAndVelocityRelationToF)
 *   -> m = M f, m^eq = M f^eq (Eq. EquilibriumDistribution, matrix M of Sec. 2)
 *   -> S (Eq. S), Q and C (Eqs. surface-tension-correction-term-Q/-C, Q-psi-based)
 *   -> m* = m - Lambda (m - m^eq) + (I - Lambda/2) S + C, f* = M^-1 m* (Eqs. lbm,
 *      collisionMRT, li_source_terms)
 *   -> streaming f(x + c_i) = f*(x), Zou-He wet-node walls, zero-gradient outflow
 *   -> temperature: Heun RK2 of Eq. (energy-equation) with lattice-weight stencils.
 *
 * Readings where the paper is silent or garbled (each one is listed in the design
 * notes of the repository):
 *  - Eq. (S): the sigma term is 12 sigma |F^m|^2 / (psi^2 (tau - 1/2)) (printed as
 *    (F^m . F^m)^2); the sigma term uses F^m (with the wall adhesion), the linear
 *    terms the total force F.
 *  - tau_v in Eq. (C) is tau_eta of Lambda; weights of Q and F^ads are the force
 *    weights W = 1/3, 1/12.
 *  - rho_bar is the mean of rho^n over all nodes at the start of the step.
 *  - psi-based wall: every solid link of a wall node x uses psi(rho_w(x), T(x)).
 *  - Zou-He no-slip closure with the half-force momentum sum_i f_i c_i = -F/2, F being
 *    the wall node's force of the step that streamed the populations in.
 *  - Outflow (zero gradient): after streaming, all f and T of the outflow column are
 *    copies of the first interior column; neighbours beyond it are copies too.
 *  - FD stencils: d_a th = 3 sum_i w_i c_ia th(x+c_i), lap th = 6 sum_i w_i (th(x+c_i)-th(x)),
 *    div(lambda grad T) = lambda lap T + grad lambda . grad T.
 *  - RK2 is Heun with rho, u (and lambda) frozen at time n; dp/dT is evaluated at the
 *    stage temperature. Dirichlet nodes are held; adiabatic walls mirror rho, T and the
 *    tangential u across the wall row (normal u flips sign).
 *  - lambda(rho) and eta(rho) are linear in rho and not clamped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- lattice of Sec. 2 (D2Q9, c_i ordering as printed) ---- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WEQ[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* interaction weights W(|c|^2): 1/3 for |c|^2 = 1, 1/12 for |c|^2 = 2 (below Eq. shanchen) */
static const double WF[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                             1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
/* transformation matrix M of Sec. 2 (Lallemand & Luo), rows as printed */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_OUTFLOW = 2 };
enum { ORC_T_PERIODIC = 0, ORC_T_DIRICHLET = 1, ORC_T_ADIABATIC = 2 };
/* side order: 0 = x-min, 1 = x-max, 2 = y-min, 3 = y-max */

typedef struct {
  int32_t nx, ny;
  double a, b, R, omega, G;
  double s[9];
  double eta_l, eta_v; /* if both > 0: s_eta per node from eta(rho) (Eq. eta-rho) */
  double rho_l, rho_v; /* interpolation anchors of eta(rho) and lambda(rho) */
  double sigma, kappa, gx, gy, cv, lambda_l, lambda_v;
  int32_t energy_on;
  int64_t iso_steps;
  int32_t hydro_bc[4], thermal_bc[4];
  double T_side[4], rho_w_side[4];
  const double *rho_w[4];       /* optional per-boundary-node wall density */
  const double *T_w[4];         /* optional per-boundary-node Dirichlet value */
  const uint8_t *T_dirichlet[4]; /* optional per-boundary-node kind: 1 Dirichlet, 0 adiabatic */
  double rho_bar_fixed; /* finite: the domain-mean density of Eq. (gravitational_force) is given
                           (the grid is a window of a larger domain); NaN: mean over this grid */
  int32_t contact_model; /* 0: psi-based (Eq. psi-based-formula); 1: modified psi-based
                            (Eq. mod-psi-based-formula) with the constant G_w below */
  double G_w;
} orc_params;

/* M^-1 = M^T diag(1/|row_k|^2): rows of M are orthogonal */
static double MINV[9][9];
static int minv_ready = 0;
static void build_minv(void) {
  if (minv_ready) return;
  for (int k = 0; k < 9; ++k) {
    double n2 = 0.0;
    for (int j = 0; j < 9; ++j) n2 += MM[k][j] * MM[k][j];
    for (int i = 0; i < 9; ++i) MINV[i][k] = MM[k][i] / n2;
  }
  minv_ready = 1;
}

/* ---- Eq. (peng-robinson) and Eq. (psi) ---- */
static double pr_tc(const orc_params *P) { return 0.0778 * P->a / (0.45724 * P->b * P->R); }
static double pr_k(const orc_params *P) {
  return 0.37464 + 1.54226 * P->omega - 0.2699 * P->omega * P->omega;
}
static double pr_p(const orc_params *P, double rho, double T) {
  double tc = pr_tc(P), k = pr_k(P);
  double al = 1.0 + k * (1.0 - sqrt(T / tc));
  al = al * al;
  return rho * P->R * T / (1.0 - P->b * rho) -
         P->a * al * rho * rho / (1.0 + 2.0 * P->b * rho - P->b * P->b * rho * rho);
}
static double pr_dpdT(const orc_params *P, double rho, double T) {
  double tc = pr_tc(P), k = pr_k(P);
  double dal = -k * (1.0 + k * (1.0 - sqrt(T / tc))) / sqrt(T * tc);
  return rho * P->R / (1.0 - P->b * rho) -
         P->a * dal * rho * rho / (1.0 + 2.0 * P->b * rho - P->b * P->b * rho * rho);
}
/* returns 0 and psi, or 1 when 2 (p - rho/3)/G < 0 */
static int pr_psi(const orc_params *P, double rho, double T, double *psi) {
  double arg = 2.0 * (pr_p(P, rho, T) - rho / 3.0) / P->G;
  if (!(arg >= 0.0)) return 1;
  *psi = sqrt(arg);
  return 0;
}

/* ---- boundary classification ---- */

/* Where does the neighbour (x+dx, y+dy) of an in-domain node lie?
 * Returns 0 in-domain (coordinates written, periodic wrap / outflow clamp applied),
 * 1 solid (beyond a wall; *side set). */
static int neighbour(const orc_params *P, int x, int y, int dx, int dy, int *ox, int *oy, int *side) {
  int X = x + dx, Y = y + dy;
  int nx = P->nx, ny = P->ny;
  if (X < 0 || X >= nx) {
    int sd = X < 0 ? 0 : 1;
    if (P->hydro_bc[sd] == ORC_PERIODIC) X = (X + nx) % nx;
    else if (P->hydro_bc[sd] == ORC_OUTFLOW) X = X < 0 ? 0 : nx - 1;
    else { *side = sd; return 1; }
  }
  if (Y < 0 || Y >= ny) {
    int sd = Y < 0 ? 2 : 3;
    if (P->hydro_bc[sd] == ORC_PERIODIC) Y = (Y + ny) % ny;
    else if (P->hydro_bc[sd] == ORC_OUTFLOW) Y = Y < 0 ? 0 : ny - 1;
    else { *side = sd; return 1; }
  }
  *ox = X;
  *oy = Y;
  return 0;
}

/* wall side a node sits on (-1 if none) */
static int wall_side_of(const orc_params *P, int x, int y) {
  if (x == 0 && P->hydro_bc[0] == ORC_WALL) return 0;
  if (x == P->nx - 1 && P->hydro_bc[1] == ORC_WALL) return 1;
  if (y == 0 && P->hydro_bc[2] == ORC_WALL) return 2;
  if (y == P->ny - 1 && P->hydro_bc[3] == ORC_WALL) return 3;
  return -1;
}
static int pos_on_side(int side, int x, int y) { return side < 2 ? y : x; }

static double wall_rho_w(const orc_params *P, int side, int x, int y) {
  if (P->rho_w[side]) return P->rho_w[side][pos_on_side(side, x, y)];
  return P->rho_w_side[side];
}

/* Dirichlet temperature node? y-sides take precedence over x-sides at corners;
 * thermally periodic sides are skipped. */
static int t_fixed(const orc_params *P, int x, int y, double *Tval) {
  int order[4] = {3, 2, 1, 0};
  for (int o = 0; o < 4; ++o) {
    int sd = order[o];
    int on = (sd == 0 && x == 0) || (sd == 1 && x == P->nx - 1) || (sd == 2 && y == 0) ||
             (sd == 3 && y == P->ny - 1);
    if (!on) continue;
    int pos = pos_on_side(sd, x, y);
    int dir;
    if (P->hydro_bc[sd] == ORC_OUTFLOW) return 0;
    /* a periodic side is no boundary for T: look at the other sides */
    if (P->hydro_bc[sd] == ORC_PERIODIC && P->thermal_bc[sd] == ORC_T_PERIODIC) continue;
    if (P->T_dirichlet[sd]) dir = P->T_dirichlet[sd][pos] != 0;
    else dir = P->thermal_bc[sd] == ORC_T_DIRICHLET;
    if (dir) {
      *Tval = P->T_w[sd] ? P->T_w[sd][pos] : P->T_side[sd];
      return 1;
    }
    return 0;
  }
  return 0;
}

static int outflow_col(const orc_params *P, int x, int y, int *sx, int *sy) {
  /* outflow node: returns 1 and the first interior node it copies */
  if (x == P->nx - 1 && P->hydro_bc[1] == ORC_OUTFLOW) { *sx = P->nx - 2; *sy = y; return 1; }
  if (x == 0 && P->hydro_bc[0] == ORC_OUTFLOW) { *sx = 1; *sy = y; return 1; }
  if (y == P->ny - 1 && P->hydro_bc[3] == ORC_OUTFLOW) { *sx = x; *sy = P->ny - 2; return 1; }
  if (y == 0 && P->hydro_bc[2] == ORC_OUTFLOW) { *sx = x; *sy = 1; return 1; }
  return 0;
}

#define IDX(x, y) ((size_t)(y) * (size_t)P->nx + (size_t)(x))
#define FI(i, x, y) ((size_t)(i) * N + IDX(x, y))

/* ---- Eq. (EquilibriumDistribution) ---- */
static void feq(double rho, double ux, double uy, double out[9]) {
  const double cs2 = 1.0 / 3.0;
  for (int i = 0; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = 0.0;
    double ua[2] = {ux, uy};
    int ca[2] = {CX[i], CY[i]};
    for (int al = 0; al < 2; ++al)
      for (int be = 0; be < 2; ++be)
        uu += (ca[al] * ca[be] - cs2 * (al == be)) * ua[al] * ua[be];
    out[i] = WEQ[i] * (rho + cu * rho / cs2 + uu * rho / (2.0 * cs2 * cs2));
  }
}

/* ---- the FD operator of Eq. (energy-equation) at one node ----
 * L(th) = -u.grad th + (lambda lap th + grad lambda . grad th)/(rho c_v)
 *         - th (dp/dT)_rho(rho, th) div u / (rho c_v)
 * with neighbour values taken through the boundary rules. */
static double lambda_of(const orc_params *P, double rho) {
  return (P->lambda_l * (rho - P->rho_v) + P->lambda_v * (P->rho_l - rho)) / (P->rho_l - P->rho_v);
}

static void nb_fields(const orc_params *P, const double *rho, const double *ux, const double *uy,
                      const double *th, int x, int y, int i, double *r, double *vx, double *vy,
                      double *t) {
  int ox, oy, side;
  if (neighbour(P, x, y, CX[i], CY[i], &ox, &oy, &side) == 0) {
    size_t k = IDX(ox, oy);
    *r = rho[k]; *vx = ux[k]; *vy = uy[k]; *t = th[k];
    return;
  }
  /* solid ghost: mirror across the wall row (adiabatic wall) */
  int mx = x + CX[i], my = y + CY[i];
  if (side == 0) mx = -mx;
  if (side == 1) mx = 2 * (P->nx - 1) - mx;
  if (side == 2) my = -my;
  if (side == 3) my = 2 * (P->ny - 1) - my;
  /* the mirrored point lies in the domain along the wall axis; wrap the other axis */
  int ox2, oy2, side2;
  neighbour(P, mx, my, 0, 0, &ox2, &oy2, &side2);
  size_t k = IDX(ox2, oy2);
  *r = rho[k]; *t = th[k];
  *vx = (side < 2) ? -ux[k] : ux[k];
  *vy = (side < 2) ? uy[k] : -uy[k];
}

static double energy_L(const orc_params *P, const double *rho, const double *ux, const double *uy,
                       const double *th, int x, int y) {
  size_t k0 = IDX(x, y);
  double r0 = rho[k0], t0 = th[k0];
  double gt[2] = {0, 0}, gl[2] = {0, 0}, div = 0.0, lap = 0.0;
  for (int i = 1; i < 9; ++i) {
    double r, vx, vy, t;
    nb_fields(P, rho, ux, uy, th, x, y, i, &r, &vx, &vy, &t);
    gt[0] += 3.0 * WEQ[i] * CX[i] * t;
    gt[1] += 3.0 * WEQ[i] * CY[i] * t;
    gl[0] += 3.0 * WEQ[i] * CX[i] * lambda_of(P, r);
    gl[1] += 3.0 * WEQ[i] * CY[i] * lambda_of(P, r);
    div += 3.0 * WEQ[i] * (CX[i] * vx + CY[i] * vy);
    lap += 6.0 * WEQ[i] * (t - t0);
  }
  double rcv = r0 * P->cv;
  return -(ux[k0] * gt[0] + uy[k0] * gt[1]) +
         (lambda_of(P, r0) * lap + gl[0] * gt[0] + gl[1] * gt[1]) / rcv -
         t0 * pr_dpdT(P, r0, t0) * div / rcv;
}

/* exported for the unit pin of the FD operator: out[k] = L(th) at every node */
int orc_energy_rhs(const orc_params *P, const double *rho, const double *ux, const double *uy,
                   const double *th, double *out) {
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) out[IDX(x, y)] = energy_L(P, rho, ux, uy, th, x, y);
  return 0;
}

/* ---- initial state: f = f^eq(rho0, u0), T = T0, then the boundary invariants ---- */
int orc_init(const orc_params *P, const double *rho0, const double *ux0, const double *uy0,
             const double *T0, double *f, double *T) {
  size_t N = (size_t)P->nx * P->ny;
  build_minv();
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      double fe[9];
      size_t k = IDX(x, y);
      feq(rho0[k], ux0[k], uy0[k], fe);
      for (int i = 0; i < 9; ++i) f[FI(i, x, y)] = fe[i];
      T[k] = T0[k];
    }
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      int sx, sy;
      if (outflow_col(P, x, y, &sx, &sy)) {
        for (int i = 0; i < 9; ++i) f[FI(i, x, y)] = f[FI(i, sx, sy)];
        T[IDX(x, y)] = T[IDX(sx, sy)];
      }
      double tv;
      if (t_fixed(P, x, y, &tv)) T[IDX(x, y)] = tv;
    }
  return 0;
}

/* work arrays, allocated per call (the oracle favours clarity over speed) */
typedef struct {
  double *rho, *psi, *Fmx, *Fmy, *Fx, *Fy, *ux, *uy, *fs, *k1, *Ts;
} work_t;

static int alloc_work(work_t *w, size_t N) {
  memset(w, 0, sizeof(*w));
  w->rho = malloc(N * sizeof(double)); w->psi = malloc(N * sizeof(double));
  w->Fmx = malloc(N * sizeof(double)); w->Fmy = malloc(N * sizeof(double));
  w->Fx = malloc(N * sizeof(double)); w->Fy = malloc(N * sizeof(double));
  w->ux = malloc(N * sizeof(double)); w->uy = malloc(N * sizeof(double));
  w->fs = malloc(9 * N * sizeof(double));
  w->k1 = malloc(N * sizeof(double)); w->Ts = malloc(N * sizeof(double));
  return (w->rho && w->psi && w->Fmx && w->Fmy && w->Fx && w->Fy && w->ux && w->uy && w->fs &&
          w->k1 && w->Ts) ? 0 : 1;
}
static void free_work(work_t *w) {
  free(w->rho); free(w->psi); free(w->Fmx); free(w->Fmy); free(w->Fx); free(w->Fy);
  free(w->ux); free(w->uy); free(w->fs); free(w->k1); free(w->Ts);
}

/* Moments, psi, forces and velocity of a state (steps 1-5). Returns 0, or 2 + node
 * index when the psi argument is negative. */
static long macro(const orc_params *P, const double *f, const double *T, work_t *w, double *rho_bar) {
  size_t N = (size_t)P->nx * P->ny;
  /* 1. rho = sum_i f_i */
  for (size_t k = 0; k < N; ++k) {
    double r = 0.0;
    for (int i = 0; i < 9; ++i) r += f[(size_t)i * N + k];
    w->rho[k] = r;
  }
  /* rho_bar: spatial mean over the whole domain (Eq. gravitational_force) */
  double sr = 0.0;
  for (size_t k = 0; k < N; ++k) sr += w->rho[k];
  *rho_bar = isnan(P->rho_bar_fixed) ? sr / (double)N : P->rho_bar_fixed;
  /* 2. psi (Eq. psi) */
  for (size_t k = 0; k < N; ++k)
    if (pr_psi(P, w->rho[k], T[k], &w->psi[k])) return 2 + (long)k;
  /* 3-4. F^m with the psi-based wall form, F^b, total F */
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      size_t k = IDX(x, y);
      double sx = 0.0, sy = 0.0;
      double ax = 0.0, ay = 0.0; /* sum of w_i s(x + c_i) c_i over the solid links */
      for (int i = 1; i < 9; ++i) {
        int ox, oy, side;
        double pn;
        if (neighbour(P, x, y, CX[i], CY[i], &ox, &oy, &side) == 0) {
          pn = w->psi[IDX(ox, oy)];
        } else if (P->contact_model == 1) {
          ax += WF[i] * CX[i];
          ay += WF[i] * CY[i];
          continue;
        } else if (pr_psi(P, wall_rho_w(P, side, x, y), T[k], &pn)) {
          return 2 + (long)k;
        }
        sx += WF[i] * pn * CX[i];
        sy += WF[i] * pn * CY[i];
      }
      /* Eq. (shanchen-walls): fluid links plus F^ads; the modified model's F^ads is
         -G_w psi^2 sum_solid w_i c_i (Eq. mod-psi-based-formula) */
      const double ps = w->psi[k];
      w->Fmx[k] = -P->G * ps * sx - P->G_w * ps * ps * ax;
      w->Fmy[k] = -P->G * ps * sy - P->G_w * ps * ps * ay;
      w->Fx[k] = w->Fmx[k] + P->gx * (w->rho[k] - *rho_bar);
      w->Fy[k] = w->Fmy[k] + P->gy * (w->rho[k] - *rho_bar);
    }
  /* 5. u = (sum_i f_i c_i + F/2) / rho */
  for (size_t k = 0; k < N; ++k) {
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
      jx += f[(size_t)i * N + k] * CX[i];
      jy += f[(size_t)i * N + k] * CY[i];
    }
    w->ux[k] = (jx + 0.5 * w->Fx[k]) / w->rho[k];
    w->uy[k] = (jy + 0.5 * w->Fy[k]) / w->rho[k];
  }
  return 0;
}

/* Zou-He no-slip wet node: the populations entering from the solid are closed by
 * bounce-back of the normal non-equilibrium part and by prescribing the population
 * momentum J = sum_i f_i c_i. No slip with the half-force velocity of
 * Eq. (DensityAndVelocityRelationToF) means J = -F/2; F is the force of the step that
 * produced these populations (the wall node's own F at the new time would make the
 * closure implicit in rho_wall and in its neighbours). */
static void zou_he(int side, double *fl, double Jx, double Jy) {
  if (side == 2) {        /* y-min: unknown 2, 5, 6 */
    fl[2] = fl[4] + 2.0 / 3.0 * Jy;
    fl[5] = fl[7] - 0.5 * (fl[1] - fl[3]) + Jy / 6.0 + 0.5 * Jx;
    fl[6] = fl[8] + 0.5 * (fl[1] - fl[3]) + Jy / 6.0 - 0.5 * Jx;
  } else if (side == 3) { /* y-max: unknown 4, 7, 8 */
    fl[4] = fl[2] - 2.0 / 3.0 * Jy;
    fl[7] = fl[5] + 0.5 * (fl[1] - fl[3]) - Jy / 6.0 - 0.5 * Jx;
    fl[8] = fl[6] - 0.5 * (fl[1] - fl[3]) - Jy / 6.0 + 0.5 * Jx;
  } else if (side == 0) { /* x-min: unknown 1, 5, 8 */
    fl[1] = fl[3] + 2.0 / 3.0 * Jx;
    fl[5] = fl[7] - 0.5 * (fl[2] - fl[4]) + Jx / 6.0 + 0.5 * Jy;
    fl[8] = fl[6] + 0.5 * (fl[2] - fl[4]) + Jx / 6.0 - 0.5 * Jy;
  } else {                /* x-max: unknown 3, 6, 7 */
    fl[3] = fl[1] - 2.0 / 3.0 * Jx;
    fl[6] = fl[8] - 0.5 * (fl[2] - fl[4]) - Jx / 6.0 + 0.5 * Jy;
    fl[7] = fl[5] + 0.5 * (fl[2] - fl[4]) - Jx / 6.0 - 0.5 * Jy;
  }
}

/* One time step in place. f: [9][ny][nx] post-stream state, T: [ny][nx].
 * Returns 0, or 2 + node index of a negative psi argument (state untouched then). */
long orc_step(const orc_params *P, double *f, double *T, int64_t step) {
  size_t N = (size_t)P->nx * P->ny;
  build_minv();
  work_t w;
  if (alloc_work(&w, N)) { free_work(&w); return 1; }
  double rho_bar;
  long err = macro(P, f, T, &w, &rho_bar);
  if (err) { free_work(&w); return err; }

  const double se = P->s[1], sz = P->s[2];
  const int var_eta = P->eta_l > 0.0 && P->eta_v > 0.0;
  /* 6-8. MRT collision with the Li source terms, node by node */
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      size_t k = IDX(x, y);
      double fl[9], fe[9], m[9], meq[9], S[9], C[9], ms[9], lam[9];
      for (int i = 0; i < 9; ++i) fl[i] = f[FI(i, x, y)];
      double rho = w.rho[k], ux = w.ux[k], uy = w.uy[k];
      double Fx = w.Fx[k], Fy = w.Fy[k], psi = w.psi[k];
      feq(rho, ux, uy, fe);
      for (int r = 0; r < 9; ++r) {
        m[r] = 0.0;
        meq[r] = 0.0;
        for (int j = 0; j < 9; ++j) {
          m[r] += MM[r][j] * fl[j];
          meq[r] += MM[r][j] * fe[j];
        }
      }
      for (int r = 0; r < 9; ++r) lam[r] = P->s[r];
      if (var_eta) {
        /* Eq. (eta-rho) in lattice units, eta = c_s^2 (tau_eta - 1/2) */
        double eta = ((rho - P->rho_v) * P->eta_l + (P->rho_l - rho) * P->eta_v) / (P->rho_l - P->rho_v);
        lam[7] = lam[8] = 1.0 / (3.0 * eta + 0.5);
      }
      double sv = lam[7];
      /* Eq. (S) */
      double uF = ux * Fx + uy * Fy;
      double Fm2 = w.Fmx[k] * w.Fmx[k] + w.Fmy[k] * w.Fmy[k];
      double tau_e = 1.0 / se, tau_z = 1.0 / sz;
      S[0] = 0.0;
      S[1] = 6.0 * uF + 12.0 * P->sigma * Fm2 / (psi * psi * (tau_e - 0.5));
      S[2] = -6.0 * uF - 12.0 * P->sigma * Fm2 / (psi * psi * (tau_z - 0.5));
      S[3] = Fx;
      S[4] = -Fx;
      S[5] = Fy;
      S[6] = -Fy;
      S[7] = 2.0 * (ux * Fx - uy * Fy);
      S[8] = ux * Fy + uy * Fx;
      /* Eqs. (Q), (Q-psi-based): solid links use psi(rho_w(x), T(x)); Eq. (Q-mod-psi-based):
         the modified model drops them (psi(x + c_i) replaced by psi(x)) */
      double Qxx = 0.0, Qyy = 0.0, Qxy = 0.0;
      for (int i = 1; i < 9; ++i) {
        int ox, oy, side;
        double pn;
        if (neighbour(P, x, y, CX[i], CY[i], &ox, &oy, &side) == 0) pn = w.psi[IDX(ox, oy)];
        else if (P->contact_model == 1) pn = psi;
        else pr_psi(P, wall_rho_w(P, side, x, y), T[k], &pn);
        double d = WF[i] * (pn - psi);
        Qxx += d * CX[i] * CX[i];
        Qyy += d * CY[i] * CY[i];
        Qxy += d * CX[i] * CY[i];
      }
      double qf = P->kappa * (P->G / 2.0) * psi;
      Qxx *= qf; Qyy *= qf; Qxy *= qf;
      /* Eq. (C) */
      C[0] = 0.0;
      C[1] = 1.5 * se * (Qxx + Qyy);
      C[2] = -1.5 * sz * (Qxx + Qyy);
      C[3] = C[4] = C[5] = C[6] = 0.0;
      C[7] = -sv * (Qxx - Qyy);
      C[8] = -sv * Qxy;
      /* m* = m - Lambda (m - m^eq) + (I - Lambda/2) S + C */
      for (int r = 0; r < 9; ++r) ms[r] = m[r] - lam[r] * (m[r] - meq[r]) + (1.0 - 0.5 * lam[r]) * S[r] + C[r];
      for (int i = 0; i < 9; ++i) {
        double v = 0.0;
        for (int r = 0; r < 9; ++r) v += MINV[i][r] * ms[r];
        w.fs[FI(i, x, y)] = v;
      }
    }

  /* 9. streaming f_i(x + c_i) = f*_i(x); destinations beyond walls/outflow are dropped */
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x)
      for (int i = 0; i < 9; ++i) {
        int X = x + CX[i], Y = y + CY[i];
        if (X < 0 || X >= P->nx) {
          if (P->hydro_bc[X < 0 ? 0 : 1] != ORC_PERIODIC) continue;
          X = (X + P->nx) % P->nx;
        }
        if (Y < 0 || Y >= P->ny) {
          if (P->hydro_bc[Y < 0 ? 2 : 3] != ORC_PERIODIC) continue;
          Y = (Y + P->ny) % P->ny;
        }
        f[FI(i, X, Y)] = w.fs[FI(i, x, y)];
      }
  /* Zou-He at the wall nodes, then the outflow copy */
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      int sd = wall_side_of(P, x, y);
      if (sd < 0) continue;
      double fl[9];
      for (int i = 0; i < 9; ++i) fl[i] = f[FI(i, x, y)];
      zou_he(sd, fl, -0.5 * w.Fx[IDX(x, y)], -0.5 * w.Fy[IDX(x, y)]);
      for (int i = 0; i < 9; ++i) f[FI(i, x, y)] = fl[i];
    }
  for (int y = 0; y < P->ny; ++y)
    for (int x = 0; x < P->nx; ++x) {
      int sx, sy;
      if (outflow_col(P, x, y, &sx, &sy))
        for (int i = 0; i < 9; ++i) f[FI(i, x, y)] = f[FI(i, sx, sy)];
    }

  /* 10. temperature: Heun RK2 of Eq. (energy-equation), rho^n and u^n frozen */
  if (P->energy_on && step >= P->iso_steps) {
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) {
        size_t k = IDX(x, y);
        double tv;
        w.k1[k] = energy_L(P, w.rho, w.ux, w.uy, T, x, y);
        w.Ts[k] = t_fixed(P, x, y, &tv) ? tv : T[k] + w.k1[k];
      }
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) {
        int sx, sy;
        if (outflow_col(P, x, y, &sx, &sy)) w.Ts[IDX(x, y)] = w.Ts[IDX(sx, sy)];
      }
    /* second stage into a scratch array (w.Fx is free now) */
    double *Tn = w.Fx;
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) {
        size_t k = IDX(x, y);
        double tv;
        if (t_fixed(P, x, y, &tv)) Tn[k] = tv;
        else Tn[k] = T[k] + 0.5 * (w.k1[k] + energy_L(P, w.rho, w.ux, w.uy, w.Ts, x, y));
      }
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) {
        int sx, sy;
        if (outflow_col(P, x, y, &sx, &sy)) Tn[IDX(x, y)] = Tn[IDX(sx, sy)];
      }
    memcpy(T, Tn, N * sizeof(double));
  }
  free_work(&w);
  return 0;
}

/* rho, u (with the half-force correction) and the mean density of a state */
long orc_fields(const orc_params *P, const double *f, const double *T, double *rho, double *ux,
                double *uy, double *rho_bar) {
  size_t N = (size_t)P->nx * P->ny;
  work_t w;
  if (alloc_work(&w, N)) { free_work(&w); return 1; }
  long err = macro(P, f, T, &w, rho_bar);
  if (!err) {
    memcpy(rho, w.rho, N * sizeof(double));
    memcpy(ux, w.ux, N * sizeof(double));
    memcpy(uy, w.uy, N * sizeof(double));
  }
  free_work(&w);
  return err;
}

/* exported for the pins of the oracle */
void orc_matrix(double *m_out, double *minv_out) {
  build_minv();
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      m_out[r * 9 + c] = MM[r][c];
      minv_out[r * 9 + c] = MINV[r][c];
    }
}
double orc_tc(const orc_params *P) { return pr_tc(P); }
size_t orc_params_size(void) { return sizeof(orc_params); }
