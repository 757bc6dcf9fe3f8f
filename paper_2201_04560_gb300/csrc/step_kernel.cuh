// Fused per-node update of the coupled pseudopotential LBM + FD energy equation
// (arXiv 2201.04560, Sec. 2) for sm_103a.
//
// One launch advances the whole grid by one time step. Each CTA owns a TX x TY tile
// and stages in shared memory everything its tile needs from a 3-node halo:
//   phase 1 (tile + 3 rings): load f, T once; rho, j = sum f c, psi(rho, T) (Eqs. psi,
//            peng-robinson)
//   phase 2 (tile + 2 rings): F^m with the psi-based wall form (Eqs. shanchen,
//            shanchen-walls, psi-based-formula), F^b (Eq. gravitational_force),
//            u = (j + F/2)/rho (Eq. DensityAndVelocityRelationToF)
//   phase 3 (tile + 1 ring): MRT collision with the Li source terms S and C
//            (Eqs. collisionMRT, li_source_terms, S, C, Q, Q-psi-based) -> f* in smem;
//            first Heun stage of Eq. (energy-equation) -> T*
//   phase 4 (tile): pull streaming f(x) = f*(x - c_i), Zou-He at wall nodes (J = -F/2), second Heun
//            stage, store f^{n+1}, T^{n+1}; FP64 block partial of sum rho^{n+1}, reduced
//            by the last CTA into rho_bar for the next launch.
// The halo recompute keeps DRAM traffic at one read and one write of (f, T) per node.
//
// Populations are stored as deviations f~_i = f_i - w_i rho_ref and the temperature as
// T - T_ref (rho_ref = T_ref = 0 for the FP64 path, so both precisions share one
// arithmetic): the moments carry rho_ref only in m_0, m_1, m_2, which the collision
// handles explicitly; the FD stencils act on the deviation directly and only the EOS
// and the compression term use T_ref + (T - T_ref).
#pragma once

#include <cstdint>

namespace ppl_dev {

enum { PERIODIC = 0, WALL = 1, OUTFLOW = 2 };
enum { T_PERIODIC = 0, T_DIRICHLET = 1, T_ADIABATIC = 2 };
enum : unsigned { FLAG_PSI_NEG = 1u, FLAG_NAN = 2u, FLAG_RHO_NONPOS = 4u };

template <typename real>
struct Params {
  int nx, ny;
  long long plane;  // nx * ny
  real a, b, R, Tc, k, G;
  real sqrt_Tc_inv;  // 1/sqrt(Tc)
  real s[9];
  int var_eta;
  real eta_l, eta_v, rho_l, rho_v, inv_drho;
  real sigma12_e, sigma12_z;  // 12 sigma / (tau_e - 1/2), 12 sigma / (tau_zeta - 1/2)
  real kappa_G2;              // kappa G / 2
  real gx, gy, cv, lam_l, lam_v, dlam;  // dlam = (lam_l - lam_v)/(rho_l - rho_v)
  int hbc[4], tbc[4];
  real T_side[4], rho_w_side[4];
  const real *rho_w[4];
  const real *T_w[4];
  const uint8_t *T_dir[4];
  real rho_ref;
  real T_ref;        // T is stored as T - T_ref (0 for the FP64 path)
  double inv_nodes;  // 1 / (nx ny)
};

struct StepIO {
  const void *f_in;
  const void *T_in;
  void *f_out;
  void *T_out;
  const double *stats_in;  // [0] rho_bar of this step
  double *stats_out;       // [0] rho_bar of the next step, [1] mass
  double *partials;        // one FP64 partial per CTA
  unsigned *counter;       // CTAs done (reset by the last one)
  unsigned *status;        // PPL_FLAG_* bits
};

// lattice of Sec. 2
__device__ __constant__ const int kCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ const int kCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename real>
__device__ __forceinline__ real wgt(int i) {
  return i == 0 ? real(4) / real(9) : (i < 5 ? real(1) / real(9) : real(1) / real(36));
}

// ---- Peng-Robinson EOS (Eq. peng-robinson) and the psi argument (Eq. psi) ----
template <typename real>
__device__ __forceinline__ real pr_alpha_root(const Params<real> &P, real T) {
  return real(1) + P.k * (real(1) - sqrt(T) * P.sqrt_Tc_inv);
}
template <typename real>
__device__ __forceinline__ real psi_arg(const Params<real> &P, real rho, real T) {
  const real ar = pr_alpha_root(P, T);
  const real den = real(1) + real(2) * P.b * rho - P.b * P.b * rho * rho;
  const real p = rho * P.R * T / (real(1) - P.b * rho) - P.a * ar * ar * rho * rho / den;
  return real(2) * (p - rho / real(3)) / P.G;
}
template <typename real>
__device__ __forceinline__ real dp_dT(const Params<real> &P, real rho, real T) {
  const real ar = pr_alpha_root(P, T);
  const real dal = -P.k * ar / (sqrt(T) * P.sqrt_Tc_inv * P.Tc);  // -k (1 + k(1 - sqrt(T/Tc)))/sqrt(T Tc)
  const real den = real(1) + real(2) * P.b * rho - P.b * P.b * rho * rho;
  return rho * P.R / (real(1) - P.b * rho) - P.a * dal * rho * rho / den;
}

// ---- boundary mapping of a (possibly out-of-domain) node coordinate ----
// Periodic axes wrap. An outflow line and everything beyond it read the first interior
// line (the zero-gradient copy). Beyond a wall the node is solid; its coordinates are
// mirrored across the wall row so that rho, T (and u) ghosts of adiabatic walls read the
// mirror image.
struct NodeMap {
  int x, y;
  int solid;  // 1 if beyond a wall
};

template <typename real>
__device__ __forceinline__ NodeMap map_node(const Params<real> &P, int gx, int gy) {
  NodeMap m;
  m.solid = 0;
  const int nx = P.nx, ny = P.ny;
  if (gx < 0 || gx >= nx) {
    const int sd = gx < 0 ? 0 : 1;
    const int k = P.hbc[sd];
    if (k == PERIODIC) {
      gx %= nx;
      if (gx < 0) gx += nx;
    } else if (k == OUTFLOW) {
      gx = sd == 0 ? 1 : nx - 2;
    } else {
      m.solid = 1;
      gx = sd == 0 ? -gx : 2 * (nx - 1) - gx;
    }
  } else if ((gx == nx - 1 && P.hbc[1] == OUTFLOW)) {
    gx = nx - 2;
  } else if (gx == 0 && P.hbc[0] == OUTFLOW) {
    gx = 1;
  }
  if (gy < 0 || gy >= ny) {
    const int sd = gy < 0 ? 2 : 3;
    const int k = P.hbc[sd];
    if (k == PERIODIC) {
      gy %= ny;
      if (gy < 0) gy += ny;
    } else if (k == OUTFLOW) {
      gy = sd == 2 ? 1 : ny - 2;
    } else {
      m.solid = 1;
      gy = sd == 2 ? -gy : 2 * (ny - 1) - gy;
    }
  } else if (gy == ny - 1 && P.hbc[3] == OUTFLOW) {
    gy = ny - 2;
  } else if (gy == 0 && P.hbc[2] == OUTFLOW) {
    gy = 1;
  }
  // ghosts far beyond a wall (ragged tiles) are never used; keep their address in range
  m.x = min(max(gx, 0), nx - 1);
  m.y = min(max(gy, 0), ny - 1);
  return m;
}

template <typename real>
__device__ __forceinline__ bool beyond_wall(const Params<real> &P, int gx, int gy) {
  return (gx < 0 && P.hbc[0] == WALL) || (gx >= P.nx && P.hbc[1] == WALL) || (gy < 0 && P.hbc[2] == WALL) ||
         (gy >= P.ny && P.hbc[3] == WALL);
}

// side of the wall a node lies on, or -1
template <typename real>
__device__ __forceinline__ int wall_side(const Params<real> &P, int gx, int gy) {
  if (gx == 0 && P.hbc[0] == WALL) return 0;
  if (gx == P.nx - 1 && P.hbc[1] == WALL) return 1;
  if (gy == 0 && P.hbc[2] == WALL) return 2;
  if (gy == P.ny - 1 && P.hbc[3] == WALL) return 3;
  return -1;
}

template <typename real>
__device__ __forceinline__ real wall_rho_w(const Params<real> &P, int side, int gx, int gy) {
  const int pos = side < 2 ? gy : gx;
  return P.rho_w[side] ? P.rho_w[side][pos] : P.rho_w_side[side];
}

// Dirichlet temperature node (y-sides decide at corners; thermally periodic sides skipped).
// (gx, gy) must be in-domain coordinates (periodic images already wrapped).
template <typename real>
__device__ __forceinline__ int t_side_kind(const Params<real> &P, int sd, int pos, real *val) {
  // -1: not a boundary for T (look further), 0: not Dirichlet, 1: Dirichlet
  if (P.hbc[sd] == OUTFLOW) return 0;
  if (P.hbc[sd] == PERIODIC && P.tbc[sd] == T_PERIODIC) return -1;
  const bool dir = P.T_dir[sd] ? (P.T_dir[sd][pos] != 0) : (P.tbc[sd] == T_DIRICHLET);
  if (!dir) return 0;
  *val = P.T_w[sd] ? P.T_w[sd][pos] : P.T_side[sd];
  return 1;
}
template <typename real>
__device__ __forceinline__ bool t_fixed(const Params<real> &P, int gx, int gy, real *val) {
  int r = -1;
  if (gy == P.ny - 1) r = t_side_kind(P, 3, gx, val);
  if (r < 0 && gy == 0) r = t_side_kind(P, 2, gx, val);
  if (r < 0 && gx == P.nx - 1) r = t_side_kind(P, 1, gy, val);
  if (r < 0 && gx == 0) r = t_side_kind(P, 0, gy, val);
  return r == 1;
}

template <typename real>
__device__ __forceinline__ bool is_outflow_line(const Params<real> &P, int gx, int gy) {
  return (gx >= P.nx - 1 && P.hbc[1] == OUTFLOW) || (gx <= 0 && P.hbc[0] == OUTFLOW) ||
         (gy >= P.ny - 1 && P.hbc[3] == OUTFLOW) || (gy <= 0 && P.hbc[2] == OUTFLOW);
}

// weight of a node in the domain sums: an outflow line is stored implicitly as a copy
// of the first interior line, which therefore counts twice
template <typename real>
__device__ __forceinline__ double sum_weight(const Params<real> &P, int gx, int gy) {
  double w = 1.0;
  if (P.hbc[1] == OUTFLOW) { if (gx == P.nx - 1) w = 0.0; else if (gx == P.nx - 2) w *= 2.0; }
  if (P.hbc[0] == OUTFLOW) { if (gx == 0) w = 0.0; else if (gx == 1) w *= 2.0; }
  if (P.hbc[3] == OUTFLOW) { if (gy == P.ny - 1) w = 0.0; else if (gy == P.ny - 2) w *= 2.0; }
  if (P.hbc[2] == OUTFLOW) { if (gy == 0) w = 0.0; else if (gy == 1) w *= 2.0; }
  return w;
}

// ---- Zou-He no-slip wet node ----
// Unknown populations (entering from the solid) from bounce-back of the normal
// non-equilibrium part and the prescribed population momentum J = sum_i f_i c_i; no slip
// with the half-force velocity (Eq. DensityAndVelocityRelationToF) is J = -F/2, F being
// the wall node's force of the step that produced the populations. The w_i rho_ref parts
// of opposite populations are equal, so the same closure holds for the deviations.
template <typename real>
__device__ __forceinline__ void zou_he(int side, real f[9], real Jx, real Jy) {
  const real h = real(0.5), t23 = real(2) / real(3), s6 = real(1) / real(6);
  if (side == 2) {
    f[2] = f[4] + t23 * Jy;
    f[5] = f[7] - h * (f[1] - f[3]) + s6 * Jy + h * Jx;
    f[6] = f[8] + h * (f[1] - f[3]) + s6 * Jy - h * Jx;
  } else if (side == 3) {
    f[4] = f[2] - t23 * Jy;
    f[7] = f[5] + h * (f[1] - f[3]) - s6 * Jy - h * Jx;
    f[8] = f[6] - h * (f[1] - f[3]) - s6 * Jy + h * Jx;
  } else if (side == 0) {
    f[1] = f[3] + t23 * Jx;
    f[5] = f[7] - h * (f[2] - f[4]) + s6 * Jx + h * Jy;
    f[8] = f[6] + h * (f[2] - f[4]) + s6 * Jx - h * Jy;
  } else {
    f[3] = f[1] - t23 * Jx;
    f[6] = f[8] - h * (f[2] - f[4]) - s6 * Jx + h * Jy;
    f[7] = f[5] + h * (f[2] - f[4]) - s6 * Jx - h * Jy;
  }
}

// ---- MRT collision in deviation form (Eqs. collisionMRT, li_source_terms, S, C) ----
// fd: deviations f~ on entry, post-collision deviations on exit. rho = rho_ref + sum f~.
template <typename real>
__device__ __forceinline__ void collide(const Params<real> &P, real fd[9], real rho, real delta, real ux,
                                        real uy, real Fx, real Fy, real Fm2_over_psi2, real Qxx, real Qyy,
                                        real Qxy, real s_eta) {
  // deviation moments m~ = M f~ (rows of M, Sec. 2)
  const real ax = fd[1] + fd[2] + fd[3] + fd[4];
  const real dg = fd[5] + fd[6] + fd[7] + fd[8];
  const real m1 = -real(4) * fd[0] - ax + real(2) * dg;
  const real m2 = real(4) * fd[0] - real(2) * ax + dg;
  const real m3 = fd[1] - fd[3] + fd[5] - fd[6] - fd[7] + fd[8];
  const real m4 = -real(2) * fd[1] + real(2) * fd[3] + fd[5] - fd[6] - fd[7] + fd[8];
  const real m5 = fd[2] - fd[4] + fd[5] + fd[6] - fd[7] - fd[8];
  const real m6 = -real(2) * fd[2] + real(2) * fd[4] + fd[5] + fd[6] - fd[7] - fd[8];
  const real m7 = fd[1] - fd[2] + fd[3] - fd[4];
  const real m8 = fd[5] - fd[6] + fd[7] - fd[8];
  // non-equilibrium parts m - m^eq (m^eq = M f^eq of Eq. EquilibriumDistribution);
  // the rho_ref w_i part contributes (rho_ref, -2 rho_ref, rho_ref, 0, ...) to m
  const real u2 = ux * ux + uy * uy;
  const real ru2 = rho * u2;
  const real n1 = m1 + real(2) * delta - real(3) * ru2;
  const real n2 = m2 - delta + real(3) * ru2;
  const real n3 = m3 - rho * ux;
  const real n4 = m4 + rho * ux;
  const real n5 = m5 - rho * uy;
  const real n6 = m6 + rho * uy;
  const real n7 = m7 - rho * (ux * ux - uy * uy);
  const real n8 = m8 - rho * ux * uy;
  // Li forcing S (Eq. S, sigma term with |F^m|^2) and the kappa correction C (Eq. C)
  const real uF = ux * Fx + uy * Fy;
  const real S1 = real(6) * uF + P.sigma12_e * Fm2_over_psi2;
  const real S2 = -real(6) * uF - P.sigma12_z * Fm2_over_psi2;
  const real S7 = real(2) * (ux * Fx - uy * Fy);
  const real S8 = ux * Fy + uy * Fx;
  const real qs = Qxx + Qyy;
  const real C1 = real(1.5) * P.s[1] * qs;
  const real C2 = -real(1.5) * P.s[2] * qs;
  const real C7 = -s_eta * (Qxx - Qyy);
  const real C8 = -s_eta * Qxy;
  // post-collision deviation moments m~* = m~ - Lambda (m - m^eq) + (I - Lambda/2) S + C
  const real h = real(0.5);
  const real p0 = delta;
  const real p1 = m1 - P.s[1] * n1 + (real(1) - h * P.s[1]) * S1 + C1;
  const real p2 = m2 - P.s[2] * n2 + (real(1) - h * P.s[2]) * S2 + C2;
  const real p3 = m3 - P.s[3] * n3 + (real(1) - h * P.s[3]) * Fx;
  const real p4 = m4 - P.s[4] * n4 - (real(1) - h * P.s[4]) * Fx;
  const real p5 = m5 - P.s[5] * n5 + (real(1) - h * P.s[5]) * Fy;
  const real p6 = m6 - P.s[6] * n6 - (real(1) - h * P.s[6]) * Fy;
  const real p7 = m7 - s_eta * n7 + (real(1) - h * s_eta) * S7 + C7;
  const real p8 = m8 - s_eta * n8 + (real(1) - h * s_eta) * S8 + C8;
  // f~* = M^-1 m~* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  const real a0 = p0 / real(9), a1 = p1 / real(36), a2 = p2 / real(36), a3 = p3 / real(6), a4 = p4 / real(12);
  const real a5 = p5 / real(6), a6 = p6 / real(12), a7 = p7 / real(4), a8 = p8 / real(4);
  const real ca = a0 - a1 - real(2) * a2;
  const real cd = a0 + real(2) * a1 + a2;
  fd[0] = a0 - real(4) * a1 + real(4) * a2;
  fd[1] = ca + a3 - real(2) * a4 + a7;
  fd[2] = ca + a5 - real(2) * a6 - a7;
  fd[3] = ca - a3 + real(2) * a4 + a7;
  fd[4] = ca - a5 + real(2) * a6 - a7;
  fd[5] = cd + a3 + a4 + a5 + a6 + a8;
  fd[6] = cd - a3 - a4 + a5 + a6 - a8;
  fd[7] = cd - a3 - a4 - a5 - a6 + a8;
  fd[8] = cd + a3 + a4 - a5 - a6 - a8;
}

// ---- FD operator of Eq. (energy-equation) with lattice-weight stencils ----
// th: temperature deviation T - T_ref with row stride WT, centre index it; rho/ux/uy:
// coefficient fields (frozen at time n) with row stride W3, centre index i3.
template <typename real, int WT, int W3>
__device__ __forceinline__ real energy_L(const Params<real> &P, const real *th, int it, const real *rho,
                                         const real *ux, const real *uy, int i3) {
  const real t0 = th[it];
  const real t1 = th[it + 1], t2 = th[it + WT], t3 = th[it - 1], t4 = th[it - WT];
  const real t5 = th[it + WT + 1], t6 = th[it + WT - 1], t7 = th[it - WT - 1], t8 = th[it - WT + 1];
  const real third = real(1) / real(3), twelfth = real(1) / real(12);
  const real gtx = third * (t1 - t3) + twelfth * (t5 - t6 - t7 + t8);
  const real gty = third * (t2 - t4) + twelfth * (t5 + t6 - t7 - t8);
  const real lap = (real(2) / real(3)) * (t1 + t2 + t3 + t4 - real(4) * t0) +
                   (real(1) / real(6)) * (t5 + t6 + t7 + t8 - real(4) * t0);
  const real r0 = rho[i3];
  const real grx = third * (rho[i3 + 1] - rho[i3 - 1]) +
                   twelfth * (rho[i3 + W3 + 1] - rho[i3 + W3 - 1] - rho[i3 - W3 - 1] + rho[i3 - W3 + 1]);
  const real gry = third * (rho[i3 + W3] - rho[i3 - W3]) +
                   twelfth * (rho[i3 + W3 + 1] + rho[i3 + W3 - 1] - rho[i3 - W3 - 1] - rho[i3 - W3 + 1]);
  const real div = third * (ux[i3 + 1] - ux[i3 - 1]) +
                   twelfth * (ux[i3 + W3 + 1] - ux[i3 + W3 - 1] - ux[i3 - W3 - 1] + ux[i3 - W3 + 1]) +
                   third * (uy[i3 + W3] - uy[i3 - W3]) +
                   twelfth * (uy[i3 + W3 + 1] + uy[i3 + W3 - 1] - uy[i3 - W3 - 1] - uy[i3 - W3 + 1]);
  const real lam = P.lam_v + P.dlam * (r0 - P.rho_v);
  const real inv_rcv = real(1) / (r0 * P.cv);
  const real t_abs = P.T_ref + t0;
  return -(ux[i3] * gtx + uy[i3] * gty) + (lam * lap + P.dlam * (grx * gtx + gry * gty)) * inv_rcv -
         t_abs * dp_dT(P, r0, t_abs) * div * inv_rcv;
}

template <typename real>
__device__ __forceinline__ real ld_real(const void *p, long long k) {
  return __ldg(reinterpret_cast<const real *>(p) + k);
}

template <typename real, bool ENERGY, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) fused_step(const Params<real> P, const StepIO io) {
  constexpr int W3 = TX + 6, H3 = TY + 6, R3 = W3 * H3;
  constexpr int W2 = TX + 4, H2 = TY + 4, R2 = W2 * H2;
  constexpr int W1 = TX + 2, H1 = TY + 2, R1 = W1 * H1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *s_rho = reinterpret_cast<real *>(smem_raw);
  real *s_psi = s_rho + R3;
  real *s_T = s_psi + R3;
  real *s_jx = s_T + R3;
  real *s_jy = s_jx + R3;
  real *s_ux = s_jy + R3;
  real *s_uy = s_ux + R3;
  real *s_fmx = s_uy + R3;
  real *s_fmy = s_fmx + R3;
  real *s_fs = s_fmy + R3;  // 9 * R1 post-collision populations
  real *s_Ts = s_jx;         // T* (R1 layout), reuses j after phase 2
  real *s_k1 = s_jy;         // first Heun stage (R1 layout)

  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const long long plane = P.plane;
  const real rho_bar = real(io.stats_in[0]);
  const bool touches_wall = ((P.hbc[0] == WALL) && x0 - 3 < 0) || ((P.hbc[1] == WALL) && x0 + TX + 3 > P.nx - 1) ||
                            ((P.hbc[2] == WALL) && y0 - 3 < 0) || ((P.hbc[3] == WALL) && y0 + TY + 3 > P.ny - 1);
  const bool touches_outflow = ((P.hbc[0] == OUTFLOW) && x0 - 3 <= 0) ||
                               ((P.hbc[1] == OUTFLOW) && x0 + TX + 3 >= P.nx - 1) ||
                               ((P.hbc[2] == OUTFLOW) && y0 - 3 <= 0) ||
                               ((P.hbc[3] == OUTFLOW) && y0 + TY + 3 >= P.ny - 1);
  unsigned flags = 0;

  // ---- phase 1: rho, j, T, psi on tile + 3 rings ----
  for (int i = threadIdx.x; i < R3; i += NT) {
    const int lx = i % W3, ly = i / W3;
    const NodeMap m = map_node(P, x0 - 3 + lx, y0 - 3 + ly);
    const long long k = (long long)m.y * P.nx + m.x;
    real f[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = ld_real<real>(io.f_in, q * plane + k);
    const real delta = ((f[0] + (f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
    const real rho = P.rho_ref + delta;
    const real T = ld_real<real>(io.T_in, k);  // T - T_ref
    s_rho[i] = rho;
    s_T[i] = T;
    s_jx[i] = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    s_jy[i] = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    real psi = real(0);
    if (!m.solid) {
      const real arg = psi_arg(P, rho, P.T_ref + T);
      if (!(arg >= real(0))) flags |= FLAG_PSI_NEG;
      psi = sqrt(fmax(arg, real(0)));
    }
    s_psi[i] = psi;
  }
  __syncthreads();

  // ---- phase 2: F^m, u on tile + 2 rings ----
  for (int t = threadIdx.x; t < R2; t += NT) {
    const int lx = t % W2 + 1, ly = t / W2 + 1;
    const int i = ly * W3 + lx;
    const int gx = x0 - 3 + lx, gy = y0 - 3 + ly;
    if (touches_wall && beyond_wall(P, gx, gy)) continue;
    const real psi_c = s_psi[i];
    real sx, sy;
    const NodeMap mm = map_node(P, gx, gy);  // periodic image -> in-domain coordinates
    const int ws = touches_wall ? wall_side(P, mm.x, mm.y) : -1;
    if (ws < 0) {
      const real p1 = s_psi[i + 1], p2 = s_psi[i + W3], p3 = s_psi[i - 1], p4 = s_psi[i - W3];
      const real p5 = s_psi[i + W3 + 1], p6 = s_psi[i + W3 - 1], p7 = s_psi[i - W3 - 1], p8 = s_psi[i - W3 + 1];
      sx = (p1 - p3) / real(3) + (p5 - p6 - p7 + p8) / real(12);
      sy = (p2 - p4) / real(3) + (p5 + p6 - p7 - p8) / real(12);
    } else {
      const real argw = psi_arg(P, wall_rho_w(P, ws, mm.x, mm.y), P.T_ref + s_T[i]);
      if (!(argw >= real(0))) flags |= FLAG_PSI_NEG;
      const real psi_w = sqrt(fmax(argw, real(0)));
      sx = real(0);
      sy = real(0);
#pragma unroll
      for (int q = 1; q < 9; ++q) {
        const int cx = kCX[q], cy = kCY[q];
        const real pn = beyond_wall(P, gx + cx, gy + cy) ? psi_w : s_psi[i + cy * W3 + cx];
        const real w = q < 5 ? real(1) / real(3) : real(1) / real(12);
        sx += w * pn * real(cx);
        sy += w * pn * real(cy);
      }
    }
    const real fmx = -P.G * psi_c * sx, fmy = -P.G * psi_c * sy;
    const real rho = s_rho[i];
    const real Fx = fmx + P.gx * (rho - rho_bar);
    const real Fy = fmy + P.gy * (rho - rho_bar);
    s_fmx[i] = fmx;
    s_fmy[i] = fmy;
    s_ux[i] = (s_jx[i] + real(0.5) * Fx) / rho;
    s_uy[i] = (s_jy[i] + real(0.5) * Fy) / rho;
  }
  __syncthreads();
  if (ENERGY && touches_wall) {
    // velocity ghosts one node beyond a wall (the only ones a fluid stencil reaches):
    // mirror image across the wall row, normal component flipped
    for (int t = threadIdx.x; t < R2; t += NT) {
      const int lx = t % W2 + 1, ly = t / W2 + 1;
      const int gx = x0 - 3 + lx, gy = y0 - 3 + ly;
      int mx = lx, my = ly;
      bool xwall;
      if (gx == -1 && P.hbc[0] == WALL) { mx = lx + 2; xwall = true; }
      else if (gx == P.nx && P.hbc[1] == WALL) { mx = lx - 2; xwall = true; }
      else if (gy == -1 && P.hbc[2] == WALL) { my = ly + 2; xwall = false; }
      else if (gy == P.ny && P.hbc[3] == WALL) { my = ly - 2; xwall = false; }
      else continue;
      if (mx < 0 || mx >= W3 || my < 0 || my >= H3) continue;
      const int i = ly * W3 + lx, im = my * W3 + mx;
      s_ux[i] = xwall ? -s_ux[im] : s_ux[im];
      s_uy[i] = xwall ? s_uy[im] : -s_uy[im];
    }
    __syncthreads();
  }

  // ---- phase 3: collision (and first Heun stage) on tile + 1 ring ----
  for (int t = threadIdx.x; t < R1; t += NT) {
    const int lx = t % W1 + 2, ly = t / W1 + 2;
    const int i = ly * W3 + lx;
    const int gx = x0 - 3 + lx, gy = y0 - 3 + ly;
    if (touches_wall && beyond_wall(P, gx, gy)) continue;
    const NodeMap m = map_node(P, gx, gy);
    const long long k = (long long)m.y * P.nx + m.x;
    real fd[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) fd[q] = ld_real<real>(io.f_in, q * plane + k);
    const real rho = s_rho[i];
    const real delta = rho - P.rho_ref;
    const real psi_c = s_psi[i];
    const int ws = touches_wall ? wall_side(P, m.x, m.y) : -1;
    real Qxx, Qyy, Qxy;
    {
      real pn[9];
      if (ws < 0) {
#pragma unroll
        for (int q = 1; q < 9; ++q) pn[q] = s_psi[i + kCY[q] * W3 + kCX[q]];
      } else {
        const real psi_w = sqrt(fmax(psi_arg(P, wall_rho_w(P, ws, m.x, m.y), P.T_ref + s_T[i]), real(0)));
#pragma unroll
        for (int q = 1; q < 9; ++q)
          pn[q] = beyond_wall(P, gx + kCX[q], gy + kCY[q]) ? psi_w : s_psi[i + kCY[q] * W3 + kCX[q]];
      }
      const real d1 = pn[1] - psi_c, d2 = pn[2] - psi_c, d3 = pn[3] - psi_c, d4 = pn[4] - psi_c;
      const real d5 = pn[5] - psi_c, d6 = pn[6] - psi_c, d7 = pn[7] - psi_c, d8 = pn[8] - psi_c;
      const real dd = (d5 + d6 + d7 + d8) / real(12);
      const real qf = P.kappa_G2 * psi_c;
      Qxx = qf * ((d1 + d3) / real(3) + dd);
      Qyy = qf * ((d2 + d4) / real(3) + dd);
      Qxy = qf * ((d5 - d6 + d7 - d8) / real(12));
    }
    const real ux = s_ux[i], uy = s_uy[i];
    const real fmx = s_fmx[i], fmy = s_fmy[i];
    const real Fx = fmx + P.gx * (rho - rho_bar);
    const real Fy = fmy + P.gy * (rho - rho_bar);
    const real fm2 = (fmx * fmx + fmy * fmy) / (psi_c * psi_c);
    real s_eta = P.s[7];
    if (P.var_eta) {
      const real eta = P.eta_v + (P.eta_l - P.eta_v) * (rho - P.rho_v) * P.inv_drho;
      s_eta = real(1) / (real(3) * eta + real(0.5));
    }
    collide(P, fd, rho, delta, ux, uy, Fx, Fy, fm2, Qxx, Qyy, Qxy, s_eta);
#pragma unroll
    for (int q = 0; q < 9; ++q) s_fs[q * R1 + t] = fd[q];
    if (ENERGY) {
      real Tw;
      real k1 = real(0), Ts;
      if (t_fixed(P, m.x, m.y, &Tw)) {
        Ts = Tw - P.T_ref;
      } else {
        k1 = energy_L<real, W3, W3>(P, s_T, i, s_rho, s_ux, s_uy, i);
        Ts = s_T[i] + k1;
      }
      s_Ts[t] = Ts;
      s_k1[t] = k1;
    }
  }
  __syncthreads();
  if (ENERGY && (touches_wall || touches_outflow)) {
    // T* ghosts: mirror one node beyond a wall; outflow lines copy the first interior line
    for (int t = threadIdx.x; t < R1; t += NT) {
      const int lx1 = t % W1, ly1 = t / W1;
      const int gx = x0 - 1 + lx1, gy = y0 - 1 + ly1;
      int sx = lx1, sy = ly1;
      if (gx == -1 && P.hbc[0] == WALL) sx = lx1 + 2;
      else if (gx == P.nx && P.hbc[1] == WALL) sx = lx1 - 2;
      else if (gy == -1 && P.hbc[2] == WALL) sy = ly1 + 2;
      else if (gy == P.ny && P.hbc[3] == WALL) sy = ly1 - 2;
      else if (P.hbc[1] == OUTFLOW && gx >= P.nx - 1) sx = lx1 - (gx - (P.nx - 2));
      else if (P.hbc[0] == OUTFLOW && gx <= 0) sx = lx1 + (1 - gx);
      else if (P.hbc[3] == OUTFLOW && gy >= P.ny - 1) sy = ly1 - (gy - (P.ny - 2));
      else if (P.hbc[2] == OUTFLOW && gy <= 0) sy = ly1 + (1 - gy);
      else continue;
      if (sx >= 0 && sx < W1 && sy >= 0 && sy < H1) s_Ts[t] = s_Ts[sy * W1 + sx];
    }
    __syncthreads();
  }

  // ---- phase 4: stream, boundary conditions, second Heun stage, store, reduce ----
  double acc = 0.0;
  for (int t = threadIdx.x; t < TX * TY; t += NT) {
    const int tx = t % TX, ty = t / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= P.nx || gy >= P.ny) continue;
    // an outflow line is an implicit copy of the first interior line: never stored
    if (touches_outflow && is_outflow_line(P, gx, gy)) continue;
    const int lx1 = tx + 1, ly1 = ty + 1;  // R1 coordinates
    const int i3 = (ty + 3) * W3 + (tx + 3);
    const int t1 = ly1 * W1 + lx1;
    real fd[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) fd[q] = s_fs[q * R1 + (ly1 - kCY[q]) * W1 + (lx1 - kCX[q])];
    const int ws = touches_wall ? wall_side(P, gx, gy) : -1;
    if (ws >= 0) {
      const real r0 = s_rho[i3];
      zou_he(ws, fd, -real(0.5) * (s_fmx[i3] + P.gx * (r0 - rho_bar)), -real(0.5) * (s_fmy[i3] + P.gy * (r0 - rho_bar)));
    }
    const real delta = ((fd[0] + (fd[1] + fd[2]) + (fd[3] + fd[4])) + ((fd[5] + fd[6]) + (fd[7] + fd[8])));
    const real rho_new = P.rho_ref + delta;
    real T_new = s_T[i3];
    if (ENERGY) {
      real Tw;
      if (!t_fixed(P, gx, gy, &Tw)) {
        const real k2 = energy_L<real, W1, W3>(P, s_Ts, t1, s_rho, s_ux, s_uy, i3);
        T_new = s_T[i3] + real(0.5) * (s_k1[t1] + k2);
      }
    }
    const long long k = (long long)gy * P.nx + gx;
    real *fo = reinterpret_cast<real *>(io.f_out);
#pragma unroll
    for (int q = 0; q < 9; ++q) fo[q * plane + k] = fd[q];
    reinterpret_cast<real *>(io.T_out)[k] = T_new;
    if (!(rho_new == rho_new) || !(T_new == T_new) || isinf(double(rho_new)) || isinf(double(T_new)))
      flags |= FLAG_NAN;
    if (!(rho_new > real(0))) flags |= FLAG_RHO_NONPOS;
    acc += sum_weight(P, gx, gy) * double(rho_new);
  }
  if (flags) atomicOr(io.status, flags);

  // ---- deterministic FP64 reduction of sum rho^{n+1} ----
  __shared__ double red[NT / 32];
  __shared__ bool am_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    io.partials[bid] = s;
    __threadfence();
    const unsigned done = atomicAdd(io.counter, 1u);
    am_last = (done == nblk - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < nblk; b += NT) s += __ldcg(io.partials + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < NT / 32; ++w) tot += red[w];
      io.stats_out[0] = tot * P.inv_nodes;
      io.stats_out[1] = tot;
      *io.counter = 0u;
    }
  }
}

template <typename real, int TX, int TY>
constexpr size_t step_smem_bytes() {
  return (size_t)(9 * (TX + 6) * (TY + 6) + 9 * (TX + 2) * (TY + 2)) * sizeof(real);
}

}  // namespace ppl_dev
