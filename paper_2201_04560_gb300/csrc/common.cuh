// Device-side building blocks of the coupled pseudopotential LBM + FD energy step
// (arXiv 2201.04560, Sec. 2): parameter block, Peng-Robinson EOS and psi, boundary
// classification, Zou-He closure, MRT collision with the Li source terms, and the FD
// operator of the energy equation. Shared by the fused step kernel (row_step.cuh) and
// the auxiliary kernels (initial state, export, norms).
//
// Populations are stored as deviations f~_i = f_i - w_i rho_ref and the temperature as
// T - T_ref (rho_ref = T_ref = 0 for the FP64 path, so both precisions share one
// arithmetic): the moments carry rho_ref only in m_0, m_1, m_2, which the collision
// handles explicitly; the FD stencils act on the deviation directly and only the EOS
// and the compression term use T_ref + (T - T_ref).
#pragma once

#include <cstdint>

#include "dual.cuh"

namespace ppl_dev {

enum { PERIODIC = 0, WALL = 1, OUTFLOW = 2 };
enum { T_PERIODIC = 0, T_DIRICHLET = 1, T_ADIABATIC = 2 };
enum : unsigned { FLAG_PSI_NEG = 1u, FLAG_NAN = 2u, FLAG_RHO_NONPOS = 4u, FLAG_STALL = 8u };

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
  real twoG_inv;     // 2 / G
  real cv_inv;       // 1 / c_v
  double inv_nodes;  // 1 / (nx ny)
  int mod_psi;       // wall adhesion: 0 psi-based, 1 modified psi-based
  real Gw_over_G;    // G_w / G of the modified model
  // coefficients of collide() with the relaxation rates and the row norms of M^-1 folded in
  real c1n, c1q, c1u, c1f;  // energy e:         a_1 = dm_1 / 36
  real c2n, c2q, c2u, c2f;  // energy square:    a_2 = dm_2 / 36
  real c4n, c4f, c6n, c6f;  // energy fluxes:    a_4 = dm_4 / 12, a_6 = dm_6 / 12
  real e_c0, e_c1;          // s_eta / 4 = 1 / (e_c0 + e_c1 rho) for a density-dependent viscosity
  real e_const;             // s_eta / 4 otherwise
};

struct StepIO {
  const void *f_in;
  const void *T_in;
  void *f_out;
  void *T_out;
  const double *stats_in;  // [0] rho_bar of this step, [2] its derivative (tangent step)
  double *stats_out;       // [0] rho_bar of the next step, [1] mass, [2] d rho_bar (tangent)
  double *partials;        // one FP64 partial per CTA (two for the tangent step)
  unsigned *counter;       // CTAs done (reset by the last one)
  unsigned *status;        // PPL_FLAG_* bits
  // TMA descriptors (CUtensorMap, global memory) of f_in as [9][ny][nx] and T_in as [ny][nx]
  // with a box of one row of the FP32 two-column strip, or null (per-thread row copies)
  const void *tmap_f;
  const void *tmap_T;
  // row blocks of the launch (two-column step): the first blocks_a have the kernel's H rows,
  // the others fill_rows rows; fill_rows = 0: all have H rows
  int blocks_a;
  int fill_rows;
};

// lattice of Sec. 2
__device__ __constant__ const int kCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ const int kCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename real>
__device__ __forceinline__ real wgt(int i) {
  return i == 0 ? real(4) / real(9) : (i < 5 ? real(1) / real(9) : real(1) / real(36));
}

// ---- Peng-Robinson EOS (Eq. peng-robinson) and the psi argument (Eq. psi) ----
// (PT: the parameter precision; real: the value type, PT itself or two packed FP32 lanes)
// The pressure is split as p = T A(rho) - alpha(T) B(rho) with A = rho R / (1 - b rho),
// B = a rho^2 / (1 + 2 b rho - b^2 rho^2) and alpha = (1 + k (1 - sqrt(T/Tc)))^2; the
// compression term of the energy equation is then T (dp/dT)_rho = T A + E(rho, T) with
// E = -T alpha'(T) B = k B alpha^(1/2) sqrt(T/Tc).
template <typename PT, typename real>
__device__ __forceinline__ void pr_parts(const Params<PT> &P, real rho, real *A, real *B) {
  const PT nb = -P.b, twob = P.b + P.b, nbb = -(P.b * P.b);
  const real omb = rho * nb + real(1);
  const real den = rho * (rho * nbb + twob) + real(1);  // 1 + 2 b rho - b^2 rho^2
  const real inv = real(1) / (omb * den);  // one division for both parts
  *A = rho * P.R * den * inv;
  *B = P.a * rho * rho * omb * inv;
}
// psi argument 2 (p - rho/3) / G of Eq. psi, with the parts A, B, E of the same (rho, T)
template <typename PT, typename real>
__device__ __forceinline__ real psi_arg_eos(const Params<PT> &P, real rho, real T, real *A, real *B, real *E) {
  const real st = sqrt(T) * P.sqrt_Tc_inv;
  const real ar = real(1) + P.k * (real(1) - st);
  pr_parts(P, rho, A, B);
  *E = P.k * *B * ar * st;
  const real TA = T * *A, ar2B = ar * ar * *B;
  return ((TA - (real(1) / real(3)) * rho) - ar2B) * P.twoG_inv;  // (p - rho/3) 2/G
}
template <typename PT, typename real>
__device__ __forceinline__ real psi_arg(const Params<PT> &P, real rho, real T) {
  real A, B, E;
  return psi_arg_eos(P, rho, T, &A, &B, &E);
}
template <typename PT, typename real>
__device__ __forceinline__ real T_dpdT(const Params<PT> &P, real A, real B, real T) {
  const real st = sqrt(T) * P.sqrt_Tc_inv;
  return T * A + P.k * B * (real(1) + P.k * (real(1) - st)) * st;
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
// fd: deviations f~ on entry, post-collision deviations on exit. rho = rho_ref + sum f~ (the
// value of the row's first stage), (ux, uy) the half-force velocity of the same populations
// (Eq. DensityAndVelocityRelationToF), F the total force, fm2 = |F^m|^2 / psi^2, Q of Eq. Q
// as qs = Qxx + Qyy, qd = Qxx - Qyy and qxy = Qxy, e = s_eta / 4.
//
// The moment increments dm = -Lambda (m - m^eq) + (I - Lambda/2) S + C are formed in closed
// form, with the rows of M of Sec. 2 (e: -4, -1 x4, 2 x4; eps: 4, -2 x4, 1 x4):
//  - momentum: m_j - rho u = -F/2 by the definition of u, so dm_jx = Fx and dm_jy = Fy
//    whatever s_j is;
//  - e and eps: with delta = sum f~, the rho_ref w_i parts cancel and the non-equilibrium
//    parts m_e - m_e^eq = m~_e + 2 delta - 3 rho u^2 and m_eps - m_eps^eq = m~_eps - delta +
//    3 rho u^2 reduce to -2 f~0 + (f~1 + .. + f~4) + 4 (f~5 + .. + f~8) - 3 rho u^2 and
//    3 (f~0 - (f~1 + .. + f~4) + rho u^2), free of the mass sum;
//  - dm_0 = 0, so f* = f + M^-1 dm leaves the mass untouched by construction.
// M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4); its row norms and the
// relaxation rates are folded into the coefficients Params::c* (a_k = dm_k / |M_k|^2), and
// the sums over the nine rows of M^T are factored into shared pairs.
template <typename PT, typename real>
__device__ __forceinline__ void collide(const Params<PT> &P, real fd[9], real rho, real ux, real uy, real Fx,
                                        real Fy, real fm2, real qs, real qd, real qxy, real e) {
  const real s13 = fd[1] + fd[3], d13 = fd[1] - fd[3];
  const real s24 = fd[2] + fd[4], d24 = fd[2] - fd[4];
  const real s57 = fd[5] + fd[7], d57 = fd[5] - fd[7];
  const real s68 = fd[6] + fd[8], d68 = fd[6] - fd[8];
  const real ax = s13 + s24, dg = s57 + s68;
  const real jx = rho * ux, jy = rho * uy;  // rho u = m_j + F/2
  const real y2 = jy * uy;
  const real ru2 = jx * ux + y2;  // rho u^2
  const real ne = real(4) * dg + (ax - real(2) * fd[0]) - real(3) * ru2;  // m_e - m_e^eq
  const real nz = (fd[0] - ax) + ru2;                                     // (m_eps - m_eps^eq) / 3
  const real nqx = ((d57 - d68) - real(2) * d13) + jx;                    // m_qx^eq = -rho ux
  const real nqy = ((d57 + d68) - real(2) * d24) + jy;
  // pxx, pxy enter with -s_eta: their non-equilibrium parts are formed negated
  const real mxx = (ru2 - real(2) * y2) - (s13 - s24);  // m_pxx^eq - m_pxx, m_pxx^eq = rho (ux^2 - uy^2)
  const real mxy = jx * uy + (s68 - s57);               // m_pxy^eq - m_pxy, m_pxy^eq = rho ux uy
  // Li source S (Eq. S): (0, 6 u.F + sigma term, -6 u.F - sigma term, Fx, -Fx, Fy, -Fy,
  // 2 (ux Fx - uy Fy), ux Fy + uy Fx); kappa correction C (Eq. C) on e, eps, pxx, pxy
  const real yF = uy * Fy;
  const real uF = ux * Fx + yF;
  const real a1 = P.c1n * ne + P.c1q * qs + P.c1u * uF + P.c1f * fm2;
  const real a2 = P.c2n * nz + P.c2q * qs + P.c2u * uF + P.c2f * fm2;
  const real a3 = Fx * (real(1) / real(6)), a5 = Fy * (real(1) / real(6));
  const real a4 = P.c4n * nqx + P.c4f * Fx;
  const real a6 = P.c6n * nqy + P.c6f * Fy;
  const real g = real(0.25) - real(0.5) * e;  // (1 - s_eta / 2) / 4
  const real a7 = e * (mxx - qd) + (g + g) * (uF - real(2) * yF);
  const real a8 = e * (mxy - qxy) + g * (ux * Fy + uy * Fx);
  // f* = f + M^T a: f1, f3 get a7 - (a1 + 2 a2) +- (a3 - 2 a4); f2, f4 get -(a1 + 2 a2 + a7) +-
  // (a5 - 2 a6); the diagonals get 2 a1 + a2 +- a8 +- (a3 + a4) +- (a5 + a6)
  const real b1 = a1 + real(2) * a2, cd = real(2) * a1 + a2;
  const real u4 = a3 - real(2) * a4, v6 = a5 - real(2) * a6;
  const real cp = a7 - b1, cn = b1 + a7;
  const real p34 = a3 + a4, p56 = a5 + a6;
  const real e5 = cd + a8, e6 = cd - a8;
  const real pp = p56 + p34, pm = p56 - p34;
  fd[0] += real(4) * (a2 - a1);
  fd[1] += cp + u4;
  fd[3] += cp - u4;
  fd[2] += v6 - cn;
  fd[4] -= cn + v6;
  fd[5] += e5 + pp;
  fd[7] += e5 - pp;
  fd[6] += e6 + pm;
  fd[8] += e6 - pm;
}

template <typename real>
__device__ __forceinline__ real ld_real(const void *p, long long k) {
  return __ldg(reinterpret_cast<const real *>(p) + k);
}
template <>
__device__ __forceinline__ Dual ld_real<Dual>(const void *p, long long k) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
  return Dual(v.x, v.y);
}
template <>
__device__ __forceinline__ DualF ld_real<DualF>(const void *p, long long k) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(p) + k);
  return DualF(v.x, v.y);
}


}  // namespace ppl_dev
