// Host side of libppl: the C ABI declared in include/ppl.h, device buffers, CUDA-graph
// step chunks, and the auxiliary kernels (initial state, field export, FP64 norms).
// The hot path is the fused step kernel of row_step.cuh (one column per thread; FP32, FP64
// and the FP64 sensitivity step) and row_step_pair.cuh (FP32, two columns per thread),
// instantiated in step_fp32.cu, step_fp64.cu and step_tangent.cu. The refinement tools
// built on it are in tools.cu.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled: the encoder is taken from the driver at run time

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sim.cuh"

namespace {

// ---------------------------------------------------------------------------------
// auxiliary kernels
// ---------------------------------------------------------------------------------

// Eq. (EquilibriumDistribution): f^eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
// stored as the deviation f^eq_i - w_i rho_ref. Dirichlet nodes take their wall value.
template <typename real>
__global__ void init_state(const Params<real> P, const double *rho0, const double *ux0, const double *uy0,
                           const double *T0, real *f, real *T) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  const int gx = (int)(k % P.nx), gy = (int)(k / P.nx);
  const double r = rho0[k], ux = ux0[k], uy = uy0[k];
  const double uu = ux * ux + uy * uy;
  const double rr = (double)P.rho_ref;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const double w = q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double cu = kCX[q] * ux + kCY[q] * uy;
    const double fe = w * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    f[q * P.plane + k] = (real)(fe - w * rr);
  }
  real tv;
  const double Tabs = t_fixed(P, gx, gy, &tv) ? (double)tv : T0[k];
  T[k] = (real)(Tabs - (double)P.T_ref);
}

// Per-node diagnostics of the stored state, reduced per block into kStats FP64 partials:
// sum rho, sum |rho|, sum |T|, min rho, max rho, min T, max T, and the sum of d rho of a
// tangent state. Also checks that psi is defined everywhere (including the wall values
// psi(rho_w, T)).
constexpr int kStats = 8;

template <typename real>
__global__ void stats_partials(const Params<real> P, const real *f, const real *T, double *part,
                               unsigned *status) {
  constexpr int NT = 256;
  __shared__ double red[kStats][NT / 32];
  double s[kStats] = {0.0, 0.0, 0.0, 1e300, -1e300, 1e300, -1e300, 0.0};
  unsigned flags = 0;
  for (long long k = (long long)blockIdx.x * NT + threadIdx.x; k < P.plane; k += (long long)gridDim.x * NT) {
    const int gx = (int)(k % P.nx), gy = (int)(k / P.nx);
    const double w = sum_weight(P, gx, gy);
    if (w == 0.0) continue;
    real d = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) d += f[q * P.plane + k];
    const real rho = P.rho_ref + d;
    const real t = P.T_ref + T[k];
    const real arg = psi_arg(P, rho, t);
    if (!(arg >= real(0))) flags |= FLAG_PSI_NEG;
    const int ws = wall_side(P, gx, gy);
    if (ws >= 0 && !(psi_arg(P, wall_rho_w(P, ws, gx, gy), t) >= real(0))) flags |= FLAG_PSI_NEG;
    if (!(rho == rho) || !(t == t) || isinf((double)rho) || isinf((double)t)) flags |= FLAG_NAN;
    if (!(rho > real(0))) flags |= FLAG_RHO_NONPOS;
    s[0] += w * (double)rho;
    s[1] += w * fabs((double)rho);
    s[2] += w * fabs((double)t);
    s[3] = fmin(s[3], (double)rho);
    s[4] = fmax(s[4], (double)rho);
    s[5] = fmin(s[5], (double)t);
    s[6] = fmax(s[6], (double)t);
    s[7] += w * tangent_of(rho);
  }
  if (flags) atomicOr(status, flags);
  auto is_sum = [](int j) { return j < 3 || j == 7; };
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    for (int j = 0; j < kStats; ++j) {
      const double x = __shfl_down_sync(0xffffffffu, s[j], o);
      s[j] = is_sum(j) ? s[j] + x : (j == 3 || j == 5 ? fmin(s[j], x) : fmax(s[j], x));
    }
  }
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < kStats; ++j) red[j][threadIdx.x >> 5] = s[j];
  __syncthreads();
  if (threadIdx.x < kStats) {
    const int j = threadIdx.x;
    double v = red[j][0];
    for (int w = 1; w < NT / 32; ++w) {
      const double x = red[j][w];
      v = is_sum(j) ? v + x : (j == 3 || j == 5 ? fmin(v, x) : fmax(v, x));
    }
    part[(long long)blockIdx.x * kStats + j] = v;
  }
}

// fixed-order finalize of the partials: out = {sum rho, sum|rho|, sum|T|, min/max rho, min/max T};
// stats[0] = rho_bar, stats[1] = mass, stats[2] = d rho_bar (tangent states, else 0).
// One block of kFinNT threads: thread j folds the partials j, j + kFinNT, ... in that order,
// then the block combines the threads by a fixed shared-memory tree (the same order on every
// run: the result is bitwise reproducible).
constexpr int kFinNT = 256;
__global__ void __launch_bounds__(kFinNT) stats_finalize(const double *part, int nblk, double inv_nodes, double *out,
                                                         double *stats) {
  __shared__ double red[kStats][kFinNT];
  const int j = threadIdx.x;
  double s[kStats] = {0.0, 0.0, 0.0, 1e300, -1e300, 1e300, -1e300, 0.0};
  for (int b = j; b < nblk; b += kFinNT) {
    const double *p = part + (long long)b * kStats;
    s[0] += p[0];
    s[1] += p[1];
    s[2] += p[2];
    s[3] = fmin(s[3], p[3]);
    s[4] = fmax(s[4], p[4]);
    s[5] = fmin(s[5], p[5]);
    s[6] = fmax(s[6], p[6]);
    s[7] += p[7];
  }
  for (int k = 0; k < kStats; ++k) red[k][j] = s[k];
  __syncthreads();
  for (int h = kFinNT / 2; h > 0; h >>= 1) {
    if (j < h) {
      double *r = &red[0][0];
      for (int k = 0; k < kStats; ++k) {
        const double a = r[k * kFinNT + j], c = r[k * kFinNT + j + h];
        r[k * kFinNT + j] = (k == 3 || k == 5) ? fmin(a, c) : (k == 4 || k == 6) ? fmax(a, c) : a + c;
      }
    }
    __syncthreads();
  }
  if (j == 0) {
    for (int k = 0; k < 7; ++k) out[k] = red[k][0];
    if (stats) {
      stats[0] = red[0][0] * inv_nodes;
      stats[1] = red[0][0];
      stats[2] = red[7][0] * inv_nodes;
    }
  }
}

// rho, u = (sum f c + F/2)/rho and T at every node (the outflow line reads its copy)
template <typename real>
__global__ void export_fields(const Params<real> P, const real *f, const real *T, const double *stats,
                              void *o_rho, void *o_ux, void *o_uy, void *o_T, int dtype) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  const int gx = (int)(k % P.nx), gy = (int)(k / P.nx);
  const NodeMap c = map_node(P, gx, gy);
  const long long kc = (long long)c.y * P.nx + c.x;
  real fl[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) fl[q] = f[q * P.plane + kc];
  real d = 0;
#pragma unroll
  for (int q = 0; q < 9; ++q) d += fl[q];
  const real rho = P.rho_ref + d;
  const real t = P.T_ref + T[kc];
  const real jx = fl[1] - fl[3] + fl[5] - fl[6] - fl[7] + fl[8];
  const real jy = fl[2] - fl[4] + fl[5] + fl[6] - fl[7] - fl[8];
  const real psi_c = sqrt(fmax(psi_arg(P, rho, t), real(0)));
  const int ws = wall_side(P, gx, gy);
  // solid links: psi(rho_w, T) (psi-based model) or (G_w / G) psi (modified model, whose
  // F^ads = -G_w psi^2 sum w c has that form)
  const real psi_w = ws < 0 ? real(0)
                     : P.mod_psi ? P.Gw_over_G * psi_c
                                 : sqrt(fmax(psi_arg(P, wall_rho_w(P, ws, gx, gy), t), real(0)));
  real sx = 0, sy = 0;
  for (int q = 1; q < 9; ++q) {
    const int nxp = gx + kCX[q], nyp = gy + kCY[q];
    real pn;
    if (beyond_wall(P, nxp, nyp)) {
      pn = psi_w;
    } else {
      const NodeMap m = map_node(P, nxp, nyp);
      const long long kn = (long long)m.y * P.nx + m.x;
      real dn = 0;
      for (int r = 0; r < 9; ++r) dn += f[r * P.plane + kn];
      pn = sqrt(fmax(psi_arg(P, P.rho_ref + dn, P.T_ref + T[kn]), real(0)));
    }
    const real w = q < 5 ? real(1) / real(3) : real(1) / real(12);
    sx += w * pn * real(kCX[q]);
    sy += w * pn * real(kCY[q]);
  }
  real rho_bar = (real)stats[0];
  if constexpr (is_dual<real>::value) rho_bar = real(stats[0], stats[2]);  // with d rho_bar
  const real Fx = -P.G * psi_c * sx + P.gx * (rho - rho_bar);
  const real Fy = -P.G * psi_c * sy + P.gy * (rho - rho_bar);
  const real ux = (jx + real(0.5) * Fx) / rho, uy = (jy + real(0.5) * Fy) / rho;
  if (dtype == 2) {  // derivatives of the tangent state (FP64)
    if (o_rho) ((double *)o_rho)[k] = tangent_of(rho);
    if (o_ux) ((double *)o_ux)[k] = tangent_of(ux);
    if (o_uy) ((double *)o_uy)[k] = tangent_of(uy);
    if (o_T) ((double *)o_T)[k] = tangent_of(t);
  } else if (dtype == 0) {
    if (o_rho) ((double *)o_rho)[k] = (double)rho;
    if (o_ux) ((double *)o_ux)[k] = (double)ux;
    if (o_uy) ((double *)o_uy)[k] = (double)uy;
    if (o_T) ((double *)o_T)[k] = (double)t;
  } else {
    if (o_rho) ((float *)o_rho)[k] = (float)value_of(rho);
    if (o_ux) ((float *)o_ux)[k] = (float)value_of(ux);
    if (o_uy) ((float *)o_uy)[k] = (float)value_of(uy);
    if (o_T) ((float *)o_T)[k] = (float)value_of(t);
  }
}

template <typename real>
__global__ void export_populations(const Params<real> P, const real *f, double *out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  const NodeMap c = map_node(P, (int)(k % P.nx), (int)(k / P.nx));
  const long long kc = (long long)c.y * P.nx + c.x;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const double w = q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    out[q * P.plane + k] = (double)f[q * P.plane + kc] + w * (double)P.rho_ref;
  }
}

}  // namespace


namespace ppl_host {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return PPL_OK;
  if (e == cudaErrorMemoryAllocation) return PPL_E_NOMEM;
  return PPL_E_CUDA;
}
uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *c = (const unsigned char *)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t hash_config(const ppl_sim *h) {
  const ppl_config &c = h->cfg;
  uint64_t x = 1469598103934665603ull;
  x = fnv(x, &c.nx, sizeof(c.nx));
  x = fnv(x, &c.ny, sizeof(c.ny));
  x = fnv(x, &c.precision, sizeof(c.precision));
  const double sc[] = {c.rho_ref, c.T_ref, c.a, c.b, c.R, c.omega, c.G, c.eta_l, c.eta_v, c.rho_l, c.rho_v,
                       c.sigma, c.kappa, c.gx, c.gy, c.cv, c.lambda_l, c.lambda_v, c.G_w};
  x = fnv(x, sc, sizeof(sc));
  x = fnv(x, c.s, sizeof(c.s));
  x = fnv(x, &c.energy_on, sizeof(c.energy_on));
  x = fnv(x, &c.iso_steps, sizeof(c.iso_steps));
  x = fnv(x, c.hydro_bc, sizeof(c.hydro_bc));
  x = fnv(x, c.thermal_bc, sizeof(c.thermal_bc));
  x = fnv(x, c.T_side, sizeof(c.T_side));
  x = fnv(x, c.rho_w_side, sizeof(c.rho_w_side));
  x = fnv(x, &c.contact_model, sizeof(c.contact_model));
  for (int s = 0; s < 4; ++s) {
    if (!h->h_rho_w[s].empty()) x = fnv(x, h->h_rho_w[s].data(), h->h_rho_w[s].size() * 8);
    if (!h->h_T_w[s].empty()) x = fnv(x, h->h_T_w[s].data(), h->h_T_w[s].size() * 8);
    if (!h->h_T_dir[s].empty()) x = fnv(x, h->h_T_dir[s].data(), h->h_T_dir[s].size());
  }
  return x;
}

// a state carrying d/d(sigma) or d/d(kappa), FP64 or FP32
bool is_tangent(int prec) {
  return prec == PPL_FP64_DSIGMA || prec == PPL_FP64_DKAPPA || prec == PPL_FP32_DSIGMA || prec == PPL_FP32_DKAPPA;
}
bool is_tangent32(int prec) { return prec == PPL_FP32_DSIGMA || prec == PPL_FP32_DKAPPA; }
// FP32 storage: f_i - w_i rho_ref and T - T_ref
bool stores_deviation(int prec) { return prec == PPL_FP32DEV || is_tangent32(prec); }

// The two-column FP32 kernel needs x periodic for the hydrodynamics (no wall or outflow
// columns; the temperature may be held on the x lines) and an even nx (8-byte aligned
// column pairs that never straddle the periodic seam).
bool pair_applicable(const ppl_config &c) {
  return c.precision == PPL_FP32DEV && c.hydro_bc[0] == PPL_PERIODIC && c.hydro_bc[1] == PPL_PERIODIC &&
         c.nx % 2 == 0 && c.nx >= 8;
}

// kernel: PPL_KERNEL_AUTO, PPL_KERNEL_COLUMN or PPL_KERNEL_PAIR (checked by the caller)
StepVariant pick_variant(const ppl_config &c, int kernel) {
  if (c.precision == PPL_FP64) return step_variant_fp64();
  if (is_tangent32(c.precision)) return step_variant_tangent32();
  if (c.precision != PPL_FP32DEV) return step_variant_tangent();
  const bool pair = kernel == PPL_KERNEL_PAIR || (kernel == PPL_KERNEL_AUTO && pair_applicable(c));
  return pair ? step_variant_fp32_pair() : step_variant_fp32();
}

int validate(const ppl_config *c) {
  if (!c) return PPL_E_INVAL;
  if (c->nx < 3 || c->ny < 3) return PPL_E_INVAL;
  if ((long long)c->nx * c->ny > (1ll << 34)) return PPL_E_INVAL;
  if (c->precision != PPL_FP64 && c->precision != PPL_FP32DEV && !is_tangent(c->precision)) return PPL_E_INVAL;
  if (!(c->a > 0) || !(c->b > 0) || !(c->R > 0) || !(c->G < 0)) return PPL_E_INVAL;
  for (int i = 0; i < 9; ++i)
    if (!(c->s[i] > 0 && c->s[i] < 2)) return PPL_E_INVAL;
  if (!(c->rho_l != c->rho_v)) return PPL_E_INVAL;
  if (c->contact_model != PPL_CONTACT_PSI && c->contact_model != PPL_CONTACT_MOD_PSI) return PPL_E_INVAL;
  if (!std::isfinite(c->G_w)) return PPL_E_INVAL;
  if (c->energy_on && !(c->cv > 0)) return PPL_E_INVAL;
  if (c->iso_steps < 0) return PPL_E_INVAL;
  for (int s = 0; s < 4; ++s) {
    if (c->hydro_bc[s] < 0 || c->hydro_bc[s] > 2) return PPL_E_INVAL;
    if (c->thermal_bc[s] < 0 || c->thermal_bc[s] > 2) return PPL_E_INVAL;
  }
  int nonper_axes = 0;
  for (int ax = 0; ax < 2; ++ax) {
    const int s0 = 2 * ax, s1 = 2 * ax + 1;
    const bool p0 = c->hydro_bc[s0] == PPL_PERIODIC, p1 = c->hydro_bc[s1] == PPL_PERIODIC;
    if (p0 != p1) return PPL_E_INVAL;
    const int len = ax == 0 ? c->nx : c->ny;
    if (!p0) {
      ++nonper_axes;
      if (len < 4) return PPL_E_INVAL;
      for (int s : {s0, s1})
        if (c->thermal_bc[s] == PPL_T_PERIODIC && c->hydro_bc[s] == PPL_WALL) return PPL_E_INVAL;
    } else {
      // a periodic axis: temperature periodic, or Dirichlet rings on both sides
      const bool t0 = c->thermal_bc[s0] == PPL_T_PERIODIC, t1 = c->thermal_bc[s1] == PPL_T_PERIODIC;
      if (t0 != t1) return PPL_E_INVAL;
      if (!t0 && (c->thermal_bc[s0] != PPL_T_DIRICHLET || c->thermal_bc[s1] != PPL_T_DIRICHLET))
        return PPL_E_INVAL;
      if (c->rho_w[s0] || c->rho_w[s1]) return PPL_E_INVAL;
    }
  }
  if (nonper_axes > 1) return PPL_E_INVAL;
  return PPL_OK;
}

template <typename real>
void fill_params(ppl_sim *h, Params<real> &P, const real *const *rw, const real *const *tw,
                 const uint8_t *const *td) {
  const ppl_config &c = h->cfg;
  memset(&P, 0, sizeof(P));
  P.nx = c.nx;
  P.ny = c.ny;
  P.plane = (long long)c.nx * c.ny;
  const double Tc = ppl_tc(c.a, c.b, c.R);
  P.a = (real)c.a;
  P.b = (real)c.b;
  P.R = (real)c.R;
  P.Tc = (real)Tc;
  P.k = (real)(0.37464 + 1.54226 * c.omega - 0.2699 * c.omega * c.omega);
  P.G = (real)c.G;
  P.twoG_inv = (real)(2.0 / c.G);
  P.cv_inv = (real)(1.0 / c.cv);
  P.sqrt_Tc_inv = (real)(1.0 / std::sqrt(Tc));
  for (int i = 0; i < 9; ++i) P.s[i] = (real)c.s[i];
  // eta(rho) enters as a per-node rate only where the two phases' viscosities differ; equal
  // ones give the constant s_eta = 1 / (3 eta + 1/2) (below)
  P.var_eta = (c.eta_l > 0 && c.eta_v > 0 && c.eta_l != c.eta_v) ? 1 : 0;
  P.eta_l = (real)c.eta_l;
  P.eta_v = (real)c.eta_v;
  P.rho_l = (real)c.rho_l;
  P.rho_v = (real)c.rho_v;
  P.inv_drho = (real)(1.0 / (c.rho_l - c.rho_v));
  // 12 sigma / (tau - 1/2) with tau = 1/s (Eq. S)
  P.sigma12_e = (real)(12.0 * c.sigma / (1.0 / c.s[1] - 0.5));
  P.sigma12_z = (real)(12.0 * c.sigma / (1.0 / c.s[2] - 0.5));
  P.kappa_G2 = (real)(c.kappa * c.G / 2.0);
  if constexpr (is_dual<real>::value) {  // seed the parameter the tangent is taken with
    if (h->prec == PPL_FP64_DSIGMA || h->prec == PPL_FP32_DSIGMA) {
      P.sigma12_e.d = 12.0 / (1.0 / c.s[1] - 0.5);
      P.sigma12_z.d = 12.0 / (1.0 / c.s[2] - 0.5);
    } else {
      P.kappa_G2.d = c.G / 2.0;
    }
  }
  // collide() coefficients: a_1 = dm_1 / 36, a_2 = dm_2 / 36 (eps enters as a third of its
  // non-equilibrium part), a_4 = dm_4 / 12, a_6 = dm_6 / 12, with dm = -s n + (1 - s/2) S + C
  // and C_1 = 3/2 s_1 (Qxx + Qyy), C_2 = -3/2 s_2 (Qxx + Qyy) (Eqs. collisionMRT, S, C); the
  // sigma terms are formed in real arithmetic so that a sigma tangent carries through
  {
    const double *s = c.s;
    P.c1n = (real)(-s[1] / 36.0);
    P.c1q = (real)(s[1] / 24.0);
    P.c1u = (real)((1.0 - 0.5 * s[1]) / 6.0);
    P.c1f = P.sigma12_e * (real)((1.0 - 0.5 * s[1]) / 36.0);
    P.c2n = (real)(-s[2] / 12.0);
    P.c2q = (real)(-s[2] / 24.0);
    P.c2u = (real)(-(1.0 - 0.5 * s[2]) / 6.0);
    P.c2f = P.sigma12_z * (real)(-(1.0 - 0.5 * s[2]) / 36.0);
    P.c4n = (real)(-s[4] / 12.0);
    P.c4f = (real)(-(1.0 - 0.5 * s[4]) / 12.0);
    P.c6n = (real)(-s[6] / 12.0);
    P.c6f = (real)(-(1.0 - 0.5 * s[6]) / 12.0);
    // s_eta = 1 / (3 nu + 1/2) with nu linear in rho between the phases
    const double e1 = P.var_eta ? 12.0 * (c.eta_l - c.eta_v) / (c.rho_l - c.rho_v) : 0.0;
    P.e_c1 = (real)e1;
    P.e_c0 = (real)(12.0 * c.eta_v + 2.0 - e1 * c.rho_v);
    P.e_const = (c.eta_l > 0 && c.eta_v > 0 && c.eta_l == c.eta_v) ? (real)(0.25 / (3.0 * c.eta_l + 0.5))
                                                                    : (real)(0.25 * s[7]);
  }
  P.mod_psi = c.contact_model == PPL_CONTACT_MOD_PSI ? 1 : 0;
  P.Gw_over_G = (real)(c.G_w / c.G);
  P.gx = (real)c.gx;
  P.gy = (real)c.gy;
  P.cv = (real)c.cv;
  P.lam_l = (real)c.lambda_l;
  P.lam_v = (real)c.lambda_v;
  P.dlam = (real)((c.lambda_l - c.lambda_v) / (c.rho_l - c.rho_v));
  for (int s = 0; s < 4; ++s) {
    P.hbc[s] = c.hydro_bc[s];
    P.tbc[s] = c.thermal_bc[s];
    P.T_side[s] = (real)c.T_side[s];
    P.rho_w_side[s] = (real)c.rho_w_side[s];
    P.rho_w[s] = rw[s];
    P.T_w[s] = tw[s];
    P.T_dir[s] = td[s];
  }
  P.rho_ref = stores_deviation(h->prec) ? (real)c.rho_ref : (real)0;
  P.T_ref = stores_deviation(h->prec) ? (real)c.T_ref : (real)0;
  P.inv_nodes = 1.0 / (double)P.plane;
}




template <typename real>
int launch_step_t(ppl_sim *h, bool energy) {
  const Params<real> &P = params_of<real>(h);
  StepIO io;
  io.f_in = h->f[h->cur];
  io.T_in = h->T[h->cur];
  io.f_out = h->f[1 - h->cur];
  io.T_out = h->T[1 - h->cur];
  io.stats_in = h->stats[h->cur];
  io.stats_out = h->stats[1 - h->cur];
  io.partials = h->partials;
  io.counter = h->counter;
  io.status = h->status;
  io.tmap_f = h->tmaps ? (const unsigned char *)h->tmaps + h->cur * sizeof(CUtensorMap) : nullptr;
  io.tmap_T = h->tmaps ? (const unsigned char *)h->tmaps + (2 + h->cur) * sizeof(CUtensorMap) : nullptr;
  io.blocks_a = h->tall_blocks;
  io.fill_rows = h->fill_rows;
  int H = h->rows_per_cta;
  void *args[] = {(void *)&P, (void *)&io, (void *)&H};
  CK(cudaLaunchKernel(h->var.fn[energy ? 1 : 0], h->grid, dim3(h->var.nt), args, h->var.smem, h->stream));
  h->cur = 1 - h->cur;
  h->step += 1;
  h->launches += 1;
  return PPL_OK;
}

// Tensor maps of the FP32 state for the TMA row staging of the two-column step: f as
// [9][ny][nx] with a box of one row of the 2 kNTP-column strip over all nine planes, T as
// [ny][nx] with a box of one row; one pair per ping-pong buffer, in device memory. Left
// unset (the step then stages rows with per-thread copies) where the driver offers no
// encoder, the row pitch is not a multiple of 16 bytes (nx % 4 != 0) or no strip fits.
void build_tensor_maps(ppl_sim *h) {
  h->tmaps = nullptr;
  const int box = 2 * kNTP;
  if (h->prec != PPL_FP32DEV || h->nx % 4 != 0 || h->nx < box) return;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return;
  const auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  CUtensorMap maps[4];
  const cuuint64_t nx = (cuuint64_t)h->nx, ny = (cuuint64_t)h->ny;
  const cuuint32_t unit[3] = {1, 1, 1};
  for (int b = 0; b < 2; ++b) {
    const cuuint64_t fdim[3] = {nx, ny, 9}, fstride[2] = {nx * 4, nx * ny * 4};
    const cuuint32_t fbox[3] = {(cuuint32_t)box, 1, 9};
    const cuuint64_t tdim[2] = {nx, ny}, tstride[1] = {nx * 4};
    const cuuint32_t tbox[2] = {(cuuint32_t)box, 1};
    if (encode(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->f[b], fdim, fstride, fbox, unit,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        encode(&maps[2 + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->T[b], tdim, tstride, tbox, unit,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return;
  }
  void *d = nullptr;
  if (cudaMalloc(&d, sizeof(maps)) != cudaSuccess) return;
  if (cudaMemcpy(d, maps, sizeof(maps), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return;
  }
  h->tmaps = d;
}

int launch_step(ppl_sim *h, bool energy) {
  return h->prec == PPL_FP64        ? launch_step_t<double>(h, energy)
         : h->prec == PPL_FP32DEV   ? launch_step_t<float>(h, energy)
         : is_tangent32(h->prec)    ? launch_step_t<DualF>(h, energy)
                                    : launch_step_t<Dual>(h, energy);
}

bool energy_at(const ppl_sim *h, int64_t step) { return h->cfg.energy_on && step >= h->cfg.iso_steps; }

// capture kGraphLen[k] launches starting from parity p; host bookkeeping is restored
static int capture_graph(ppl_sim *h, int e, int p, int k) {
  const int cur0 = h->cur;
  const int64_t step0 = h->step, l0 = h->launches;
  h->cur = p;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = PPL_OK;
  for (int i = 0; i < kGraphLen[k] && rc == PPL_OK; ++i) rc = launch_step(h, e != 0);
  cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
  h->cur = cur0;
  h->step = step0;
  h->launches = l0;
  if (rc != PPL_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(ce);
  ce = cudaGraphInstantiate(&h->graph[e][p][k], g, 0);
  cudaGraphDestroy(g);
  CK(ce);
  return PPL_OK;
}

// every length and both parities of one energy setting, captured together on first use (so
// that the first run long enough for a graph, typically a warm-up, pays for all of them)
static int capture_graphs(ppl_sim *h, int e) {
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 5; ++k)
      if (!h->graph[e][p][k]) {
        const int rc = capture_graph(h, e, p, k);
        if (rc) return rc;
      }
  return PPL_OK;
}

void drop_graphs(ppl_sim *h) {
  for (auto &ep : h->graph)
    for (auto &pk : ep)
      for (auto &g : pk)
        if (g) {
          cudaGraphExecDestroy(g);
          g = nullptr;
        }
}

template <typename real>
int run_stats(ppl_sim *h, double *stats_dst) {
  const Params<real> &P = params_of<real>(h);
  stats_partials<real><<<h->stats_blocks, 256, 0, h->stream>>>(P, (const real *)h->f[h->cur],
                                                               (const real *)h->T[h->cur], h->partials,
                                                               h->status);
  CK(cudaGetLastError());
  stats_finalize<<<1, kFinNT, 0, h->stream>>>(h->partials, h->stats_blocks, P.inv_nodes, h->norm_out, stats_dst);
  CK(cudaGetLastError());
  return PPL_OK;
}

int stats(ppl_sim *h, double *stats_dst) {
  return h->prec == PPL_FP64        ? run_stats<double>(h, stats_dst)
         : h->prec == PPL_FP32DEV   ? run_stats<float>(h, stats_dst)
         : is_tangent32(h->prec)    ? run_stats<DualF>(h, stats_dst)
                                    : run_stats<Dual>(h, stats_dst);
}

template <typename real>
int upload_state_t(ppl_sim *h, const double *rho0, const double *ux0, const double *uy0, const double *T0) {
  const size_t nb = (size_t)h->N * sizeof(double);
  CK(cudaMemcpyAsync(h->upload, rho0, nb, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->upload + h->N, ux0, nb, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->upload + 2 * h->N, uy0, nb, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->upload + 3 * h->N, T0, nb, cudaMemcpyHostToDevice, h->stream));
  const Params<real> &P = params_of<real>(h);
  const int nt = 256;
  const unsigned nb_blocks = (unsigned)((h->N + nt - 1) / nt);
  init_state<real><<<nb_blocks, nt, 0, h->stream>>>(P, h->upload, h->upload + h->N, h->upload + 2 * h->N,
                                                    h->upload + 3 * h->N, (real *)h->f[0], (real *)h->T[0]);
  CK(cudaGetLastError());
  return PPL_OK;
}

int upload_state(ppl_sim *h, const double *rho0, const double *ux0, const double *uy0, const double *T0) {
  if (!rho0 || !ux0 || !uy0 || !T0) return PPL_E_INVAL;
  h->cur = 0;
  h->step = 0;
  CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
  int rc = h->prec == PPL_FP64      ? upload_state_t<double>(h, rho0, ux0, uy0, T0)
           : h->prec == PPL_FP32DEV ? upload_state_t<float>(h, rho0, ux0, uy0, T0)
           : is_tangent32(h->prec)  ? upload_state_t<DualF>(h, rho0, ux0, uy0, T0)
                                    : upload_state_t<Dual>(h, rho0, ux0, uy0, T0);
  if (rc) return rc;
  rc = stats(h, h->stats[0]);
  if (rc) return rc;
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st & (FLAG_PSI_NEG | FLAG_NAN | FLAG_RHO_NONPOS)) {
    cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream);
    cudaStreamSynchronize(h->stream);
    return PPL_E_INVAL;
  }
  return PPL_OK;
}

// default launch shape: one wave of resident CTAs over the rows
int default_rows(const ppl_sim *h) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->var.fn[1], h->var.nt, h->var.smem);
  const int slots = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int strips = (h->nx + h->var.width - 1) / h->var.width;
  int yblocks = slots / strips;
  if (yblocks < 1) yblocks = 1;
  return (h->ny + yblocks - 1) / yblocks;  // small grids get short blocks: more CTAs in flight
}

// Default shape of the two-column step on a large grid: one wave of tall row blocks over the
// first ~86 % of the rows, then short blocks (~0.27 of the tall height) for the rest. The CTAs
// resident on an SM do not progress at one rate (the older ones are issued first), so in a
// single wave of equal blocks the SM's occupancy decays towards the end of the step; the short
// blocks take the freed slots and keep it full, at the price of their extra halo rows
// (measured on 2048 x 4096: 53.2 against 49.4 G node updates/s for one uniform wave).
void default_shape(const ppl_sim *h, int *rows, int *fill_rows) {
  *rows = default_rows(h);
  *fill_rows = 0;
  if (h->var.nt != kNTP || h->prec != PPL_FP32DEV) return;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->var.fn[1], h->var.nt, h->var.smem);
  const int strips = (h->nx + h->var.width - 1) / h->var.width;
  const int tall = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) / strips;
  if (tall < 1) return;
  const int H1 = (int)std::lround(0.86 * h->ny / tall);
  if (H1 < 24) return;  // short blocks would be mostly halo
  const int H2 = std::max(4, (int)std::lround(0.27 * H1));
  if ((long long)tall * H1 >= h->ny) return;
  *rows = H1;
  *fill_rows = H2;
}

// grid of a launch shape; *tall receives the row blocks of `rows` rows
dim3 shape_grid(const ppl_sim *h, int rows, int fill_rows, int *tall) {
  const int strips = (h->nx + h->var.width - 1) / h->var.width;
  if (fill_rows <= 0) {
    *tall = (h->ny + rows - 1) / rows;
    return dim3(strips, *tall);
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->var.fn[1], h->var.nt, h->var.smem);
  *tall = std::max(1, std::min((sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) / strips, (h->ny - 1) / rows));
  const int rest = h->ny - *tall * rows;
  return dim3(strips, *tall + (rest + fill_rows - 1) / fill_rows);
}

int check_status(ppl_sim *h) {
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st ? PPL_E_NUMERIC : PPL_OK;
}

void free_all(ppl_sim *h) {
  drop_graphs(h);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->f[i]);
    cudaFree(h->T[i]);
    cudaFree(h->stats[i]);
  }
  cudaFree(h->bnd);
  cudaFree(h->tmaps);
  cudaFree(h->partials);
  cudaFree(h->norm_out);
  cudaFree(h->counter);
  cudaFree(h->status);
  cudaFree(h->upload);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

}  // namespace ppl_host

using namespace ppl_host;

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------

extern "C" {

const char *ppl_strerror(int code) {
  switch (code) {
    case PPL_OK: return "ok";
    case PPL_E_INVAL: return "invalid argument, configuration or initial state";
    case PPL_E_CUDA: return "CUDA runtime error";
    case PPL_E_NUMERIC: return "numerical failure flagged on the device (NaN, rho <= 0 or negative psi argument)";
    case PPL_E_TIMEOUT: return "bounded device wait timed out";
    case PPL_E_IO: return "checkpoint I/O error or configuration mismatch";
    case PPL_E_NOMEM: return "out of memory";
    default: return "unknown error code";
  }
}

double ppl_tc(double a, double b, double R) { return 0.0778 * a / (0.45724 * b * R); }

double ppl_refine_a(double a_base, int32_t n_base, int32_t n) {
  const double r = (double)n_base / (double)n;
  return a_base * r * r;
}

// Maxwell equal-area rule for the PR isotherm (Sec. 3.2 target of the sigma tuning), using
// the closed-form integral of p dv with v = 1/rho:
//   int p dv = R T ln(v - b) - a alpha / (2 sqrt2 b) ln((v + b - sqrt2 b)/(v + b + sqrt2 b)).
// Spinodal points and phase densities by bisection, p_sat by bisection on the area balance.
int ppl_maxwell(double a, double b, double R, double omega, double T, double *rho_v, double *rho_l,
                double *p_sat) {
  if (!rho_v || !rho_l || !p_sat || !(a > 0) || !(b > 0) || !(R > 0) || !(T > 0)) return PPL_E_INVAL;
  const double Tc = ppl_tc(a, b, R);
  if (!(T < Tc)) return PPL_E_INVAL;
  const double k = 0.37464 + 1.54226 * omega - 0.2699 * omega * omega;
  const double ar = 1.0 + k * (1.0 - std::sqrt(T / Tc));
  const double aa = a * ar * ar;
  auto p = [&](double r) { return r * R * T / (1.0 - b * r) - aa * r * r / (1.0 + 2.0 * b * r - b * b * r * r); };
  auto dp = [&](double r) {
    const double d = 1.0 + 2.0 * b * r - b * b * r * r;
    return R * T / ((1.0 - b * r) * (1.0 - b * r)) - aa * (2.0 * r * d - r * r * (2.0 * b - 2.0 * b * b * r)) / (d * d);
  };
  // bracket the spinodal: first sign change of dp/drho from + to - and back
  const double rmax = 0.999999 / b;
  const int n = 20000;
  double ra = -1, rb = -1;
  for (int i = 1; i < n; ++i) {
    const double r0 = rmax * (i - 1) / n, r1 = rmax * i / n;
    if (ra < 0 && dp(r0 + 1e-300) > 0 && dp(r1) <= 0) ra = r1;
    if (ra > 0 && dp(r0) < 0 && dp(r1) >= 0) { rb = r1; break; }
  }
  if (ra < 0 || rb < 0) return PPL_E_INVAL;
  auto bis = [&](auto fn, double lo, double hi) {
    double flo = fn(lo);
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      const double fm = fn(mid);
      if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else hi = mid;
      if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi);
  };
  const double r_smax = bis(dp, ra - rmax / n, ra);  // local max of p
  const double r_smin = bis(dp, rb - rmax / n, rb);  // local min of p
  const double p_hi = p(r_smax), p_lo = std::fmax(p(r_smin), 1e-300);
  const double s2 = std::sqrt(2.0);
  auto prim = [&](double v) { return R * T * std::log(v - b) - aa / (2.0 * s2 * b) * std::log((v + b - s2 * b) / (v + b + s2 * b)); };
  double rv = 0, rl = 0;
  auto area = [&](double ps) {
    rv = bis([&](double r) { return p(r) - ps; }, 1e-300, r_smax);
    rl = bis([&](double r) { return p(r) - ps; }, r_smin, rmax);
    const double vv = 1.0 / rv, vl = 1.0 / rl;
    return prim(vv) - prim(vl) - ps * (vv - vl);
  };
  double lo = p_lo, hi = p_hi;
  double alo = area(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double am = area(mid);
    if ((am > 0) == (alo > 0)) { lo = mid; alo = am; } else hi = mid;
    if (hi - lo <= 1e-16 * hi) break;
  }
  const double ps = 0.5 * (lo + hi);
  area(ps);
  *rho_v = rv;
  *rho_l = rl;
  *p_sat = ps;
  return PPL_OK;
}

int ppl_init(const ppl_config *cfg, const double *rho0, const double *ux0, const double *uy0, const double *T0,
             ppl_t **out) {
  if (!out) return PPL_E_INVAL;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  ppl_sim *h = new (std::nothrow) ppl_sim();
  if (!h) return PPL_E_NOMEM;
  h->cfg = *cfg;
  h->prec = cfg->precision;
  h->nx = cfg->nx;
  h->ny = cfg->ny;
  h->N = (long long)cfg->nx * cfg->ny;
  h->rsz = h->prec == PPL_FP64        ? 8
           : h->prec == PPL_FP32DEV   ? 4
           : is_tangent32(h->prec)    ? sizeof(DualF)
                                      : sizeof(Dual);
  for (int s = 0; s < 4; ++s) {
    const int len = s < 2 ? cfg->ny : cfg->nx;
    if (cfg->rho_w[s]) h->h_rho_w[s].assign(cfg->rho_w[s], cfg->rho_w[s] + len);
    if (cfg->T_w[s]) h->h_T_w[s].assign(cfg->T_w[s], cfg->T_w[s] + len);
    if (cfg->T_dirichlet[s]) h->h_T_dir[s].assign(cfg->T_dirichlet[s], cfg->T_dirichlet[s] + len);
    h->cfg.rho_w[s] = h->h_rho_w[s].empty() ? nullptr : h->h_rho_w[s].data();
    h->cfg.T_w[s] = h->h_T_w[s].empty() ? nullptr : h->h_T_w[s].data();
    h->cfg.T_dirichlet[s] = h->h_T_dir[s].empty() ? nullptr : h->h_T_dir[s].data();
  }
  h->cfg_hash = hash_config(h);
  auto fail = [&](int code) {
    free_all(h);
    delete h;
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(PPL_E_CUDA);
  h->stream = h->own_stream;

  // launch shape: strips of var.width columns, one wave of CTAs over the rows
  h->var = pick_variant(h->cfg, PPL_KERNEL_AUTO);
  for (int e = 0; e < 2; ++e)
    if (cudaFuncSetAttribute(h->var.fn[e], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->var.smem) !=
        cudaSuccess)
      return fail(PPL_E_CUDA);
  default_shape(h, &h->rows_per_cta, &h->fill_rows);
  h->grid = shape_grid(h, h->rows_per_cta, h->fill_rows, &h->tall_blocks);
  h->stats_blocks = 608;
  const size_t nctas = (size_t)h->grid.x * h->grid.y;
  const size_t step_part = nctas * (is_tangent(h->prec) ? 2 : 1);
  const size_t npart = std::max(step_part, (size_t)h->stats_blocks * kStats);

  // device buffers
  const size_t fbytes = (size_t)9 * h->N * h->rsz, tbytes = (size_t)h->N * h->rsz;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&h->f[i], fbytes) != cudaSuccess || cudaMalloc(&h->T[i], tbytes) != cudaSuccess ||
        cudaMalloc(&h->stats[i], 4 * sizeof(double)) != cudaSuccess ||
        cudaMemset(h->stats[i], 0, 4 * sizeof(double)) != cudaSuccess)
      return fail(PPL_E_NOMEM);
  }
  h->npart = npart;
  if (cudaMalloc(&h->partials, npart * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->norm_out, 7 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->counter, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&h->status, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&h->upload, (size_t)4 * h->N * sizeof(double)) != cudaSuccess)
    return fail(PPL_E_NOMEM);
  if (cudaMemsetAsync(h->counter, 0, sizeof(unsigned), h->stream) != cudaSuccess) return fail(PPL_E_CUDA);
  build_tensor_maps(h);

  // boundary arrays in the working precision
  size_t bbytes = 0;
  for (int s = 0; s < 4; ++s) {
    const size_t len = s < 2 ? h->ny : h->nx;
    bbytes += (h->h_rho_w[s].empty() ? 0 : len * h->rsz) + (h->h_T_w[s].empty() ? 0 : len * h->rsz) +
              (h->h_T_dir[s].empty() ? 0 : ((len + 15) / 16) * 16);
  }
  const void *rw[4] = {nullptr, nullptr, nullptr, nullptr}, *tw[4] = {nullptr, nullptr, nullptr, nullptr};
  const uint8_t *td[4] = {nullptr, nullptr, nullptr, nullptr};
  if (bbytes) {
    if (cudaMalloc(&h->bnd, bbytes) != cudaSuccess) return fail(PPL_E_NOMEM);
    std::vector<unsigned char> host(bbytes);
    size_t off = 0;
    for (int s = 0; s < 4; ++s) {
      const size_t len = s < 2 ? h->ny : h->nx;
      auto put_real = [&](const std::vector<double> &v, const void **dst) {
        if (v.empty()) return;
        for (size_t i = 0; i < len; ++i) {
          if (h->prec == PPL_FP64) {
            memcpy(&host[off + i * 8], &v[i], 8);
          } else if (is_tangent32(h->prec)) {
            const DualF x(v[i]);
            memcpy(&host[off + i * sizeof(DualF)], &x, sizeof(DualF));
          } else if (is_tangent(h->prec)) {
            const Dual x(v[i]);
            memcpy(&host[off + i * sizeof(Dual)], &x, sizeof(Dual));
          } else {
            const float x = (float)v[i];
            memcpy(&host[off + i * 4], &x, 4);
          }
        }
        *dst = (const unsigned char *)h->bnd + off;
        off += len * h->rsz;
      };
      put_real(h->h_rho_w[s], &rw[s]);
      put_real(h->h_T_w[s], &tw[s]);
      if (!h->h_T_dir[s].empty()) {
        memcpy(&host[off], h->h_T_dir[s].data(), len);
        td[s] = (const uint8_t *)h->bnd + off;
        off += ((len + 15) / 16) * 16;
      }
    }
    if (cudaMemcpy(h->bnd, host.data(), bbytes, cudaMemcpyHostToDevice) != cudaSuccess) return fail(PPL_E_CUDA);
  }
  if (h->prec == PPL_FP64)
    fill_params<double>(h, h->pd, (const double *const *)rw, (const double *const *)tw, td);
  else if (h->prec == PPL_FP32DEV)
    fill_params<float>(h, h->pf, (const float *const *)rw, (const float *const *)tw, td);
  else if (is_tangent32(h->prec))
    fill_params<DualF>(h, h->ptf, (const DualF *const *)rw, (const DualF *const *)tw, td);
  else
    fill_params<Dual>(h, h->pt, (const Dual *const *)rw, (const Dual *const *)tw, td);

  rc = upload_state(h, rho0, ux0, uy0, T0);
  if (rc) return fail(rc);
  *out = h;
  return PPL_OK;
}

int ppl_reset(ppl_t *h, const double *rho0, const double *ux0, const double *uy0, const double *T0) {
  if (!h) return PPL_E_INVAL;
  return upload_state(h, rho0, ux0, uy0, T0);
}

int ppl_set_stream(ppl_t *h, void *cuda_stream) {
  if (!h) return PPL_E_INVAL;
  h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
  return PPL_OK;
}

int ppl_step_async(ppl_t *h, int64_t nsteps) {
  if (!h || nsteps < 0) return PPL_E_INVAL;
  int64_t left = nsteps;
  // inside a stream capture of the caller every step is launched on its own (the capture
  // records them); no graph is captured or replayed
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(h->stream, &cs));
  const int kmin = cs == cudaStreamCaptureStatusNone ? 0 : 5;
  while (left > 0) {
    const bool e = energy_at(h, h->step);
    int k = kmin;  // the longest graph that fits and does not cross the start of the energy equation
    while (k < 5 && (left < kGraphLen[k] || energy_at(h, h->step + kGraphLen[k] - 1) != e)) ++k;
    if (k < 5) {
      if (!h->graph[e][h->cur][k]) {
        int rc = capture_graphs(h, e ? 1 : 0);
        if (rc) return rc;
      }
      CK(cudaGraphLaunch(h->graph[e][h->cur][k], h->stream));
      h->step += kGraphLen[k];
      h->launches += kGraphLen[k];
      left -= kGraphLen[k];
    } else {
      int rc = launch_step(h, e);
      if (rc) return rc;
      left -= 1;
    }
  }
  return PPL_OK;
}

int ppl_sync(ppl_t *h) {
  if (!h) return PPL_E_INVAL;
  return check_status(h);
}

int ppl_step(ppl_t *h, int64_t nsteps) {
  int rc = ppl_step_async(h, nsteps);
  if (rc) return rc;
  return check_status(h);
}

static int export_device(ppl_t *h, void *rho, void *ux, void *uy, void *T, int dtype) {
  const int nt = 256;
  const unsigned nb = (unsigned)((h->N + nt - 1) / nt);
  if (h->prec == PPL_FP64)
    export_fields<double><<<nb, nt, 0, h->stream>>>(h->pd, (const double *)h->f[h->cur],
                                                    (const double *)h->T[h->cur], h->stats[h->cur], rho, ux, uy,
                                                    T, dtype);
  else if (h->prec == PPL_FP32DEV)
    export_fields<float><<<nb, nt, 0, h->stream>>>(h->pf, (const float *)h->f[h->cur],
                                                   (const float *)h->T[h->cur], h->stats[h->cur], rho, ux, uy, T,
                                                   dtype);
  else if (is_tangent32(h->prec))
    export_fields<DualF><<<nb, nt, 0, h->stream>>>(h->ptf, (const DualF *)h->f[h->cur],
                                                   (const DualF *)h->T[h->cur], h->stats[h->cur], rho, ux, uy, T,
                                                   dtype);
  else
    export_fields<Dual><<<nb, nt, 0, h->stream>>>(h->pt, (const Dual *)h->f[h->cur], (const Dual *)h->T[h->cur],
                                                  h->stats[h->cur], rho, ux, uy, T, dtype);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return PPL_OK;
}

static int fields_to_host(ppl_t *h, double *rho, double *ux, double *uy, double *T, int dtype) {
  double *d = nullptr;
  const size_t nb = (size_t)h->N * sizeof(double);
  CK(cudaMalloc(&d, 4 * nb));
  int rc = export_device(h, rho ? d : nullptr, ux ? d + h->N : nullptr, uy ? d + 2 * h->N : nullptr,
                         T ? d + 3 * h->N : nullptr, dtype);
  double *dst[4] = {rho, ux, uy, T};
  for (int i = 0; i < 4 && rc == PPL_OK; ++i)
    if (dst[i]) rc = cuda_err(cudaMemcpyAsync(dst[i], d + i * h->N, nb, cudaMemcpyDeviceToHost, h->stream));
  if (rc == PPL_OK) rc = cuda_err(cudaStreamSynchronize(h->stream));
  cudaFree(d);
  return rc;
}

int ppl_fields_device(ppl_t *h, void *rho, void *ux, void *uy, void *T, int dtype) {
  if (!h || (dtype != 0 && dtype != 1)) return PPL_E_INVAL;
  return export_device(h, rho, ux, uy, T, dtype);
}

int ppl_tangent_fields(ppl_t *h, double *drho, double *dux, double *duy, double *dT) {
  if (!h || !is_tangent(h->prec)) return PPL_E_INVAL;
  return fields_to_host(h, drho, dux, duy, dT, 2);
}

int ppl_fields(ppl_t *h, double *rho, double *ux, double *uy, double *T) {
  if (!h) return PPL_E_INVAL;
  return fields_to_host(h, rho, ux, uy, T, 0);
}

int ppl_populations(ppl_t *h, double *f) {
  if (!h || !f) return PPL_E_INVAL;
  double *d = nullptr;
  const size_t nb = (size_t)9 * h->N * sizeof(double);
  CK(cudaMalloc(&d, nb));
  const int nt = 256;
  const unsigned blocks = (unsigned)((h->N + nt - 1) / nt);
  if (h->prec == PPL_FP64)
    export_populations<double><<<blocks, nt, 0, h->stream>>>(h->pd, (const double *)h->f[h->cur], d);
  else if (h->prec == PPL_FP32DEV)
    export_populations<float><<<blocks, nt, 0, h->stream>>>(h->pf, (const float *)h->f[h->cur], d);
  else if (is_tangent32(h->prec))
    export_populations<DualF><<<blocks, nt, 0, h->stream>>>(h->ptf, (const DualF *)h->f[h->cur], d);
  else
    export_populations<Dual><<<blocks, nt, 0, h->stream>>>(h->pt, (const Dual *)h->f[h->cur], d);
  int rc = cuda_err(cudaGetLastError());
  if (rc == PPL_OK) rc = cuda_err(cudaMemcpyAsync(f, d, nb, cudaMemcpyDeviceToHost, h->stream));
  if (rc == PPL_OK) rc = cuda_err(cudaStreamSynchronize(h->stream));
  cudaFree(d);
  return rc;
}

int ppl_state_device(ppl_t *h, double *f, double *T) {
  if (!h || !f || !T || is_tangent(h->prec)) return PPL_E_INVAL;
  const int nt = 256;
  const unsigned blocks = (unsigned)((h->N + nt - 1) / nt);
  if (h->prec == PPL_FP64)
    export_populations<double><<<blocks, nt, 0, h->stream>>>(h->pd, (const double *)h->f[h->cur], f);
  else
    export_populations<float><<<blocks, nt, 0, h->stream>>>(h->pf, (const float *)h->f[h->cur], f);
  CK(cudaGetLastError());
  return export_device(h, nullptr, nullptr, nullptr, T, 0);
}

size_t ppl_snapshot_bytes(const ppl_t *h) {
  return h ? (size_t)10 * h->N * h->rsz + 4 * sizeof(double) : 0;
}

int ppl_snapshot(ppl_t *h, void *dst) {
  if (!h || !dst) return PPL_E_INVAL;
  unsigned char *d = (unsigned char *)dst;
  const size_t fb = (size_t)9 * h->N * h->rsz, tb = (size_t)h->N * h->rsz;
  CK(cudaMemcpyAsync(d, h->f[h->cur], fb, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(d + fb, h->T[h->cur], tb, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(d + fb + tb, h->stats[h->cur], 4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return PPL_OK;
}

int ppl_restore(ppl_t *h, const void *src, int64_t step) {
  if (!h || !src || step < 0) return PPL_E_INVAL;
  const unsigned char *d = (const unsigned char *)src;
  const size_t fb = (size_t)9 * h->N * h->rsz, tb = (size_t)h->N * h->rsz;
  h->cur = 0;
  CK(cudaMemcpyAsync(h->f[0], d, fb, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->T[0], d + fb, tb, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->stats[0], d + fb + tb, 4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
  h->step = step;
  return PPL_OK;
}

int ppl_norms(ppl_t *h, ppl_norms_t *out) {
  if (!h || !out) return PPL_E_INVAL;
  int rc = stats(h, nullptr);
  if (rc) return rc;
  double v[7];
  unsigned st = 0;
  CK(cudaMemcpyAsync(v, h->norm_out, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out->step = h->step;
  out->mass = v[0];
  out->rho_mean = v[0] / (double)h->N;
  out->sum_abs_rho = v[1];
  out->sum_abs_T = v[2];
  out->rho_min = v[3];
  out->rho_max = v[4];
  out->T_min = v[5];
  out->T_max = v[6];
  out->flags = st;
  return PPL_OK;
}

struct CkptHeader {
  char magic[8];
  int32_t version, nx, ny, precision, rsz, pad;
  int64_t step;
  uint64_t cfg_hash;
};

int ppl_save(ppl_t *h, const char *path) {
  if (!h || !path) return PPL_E_INVAL;
  CK(cudaStreamSynchronize(h->stream));
  const size_t fbytes = (size_t)9 * h->N * h->rsz, tbytes = (size_t)h->N * h->rsz;
  std::vector<unsigned char> buf(fbytes + tbytes);
  double st[2];
  CK(cudaMemcpy(buf.data(), h->f[h->cur], fbytes, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(buf.data() + fbytes, h->T[h->cur], tbytes, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(st, h->stats[h->cur], sizeof(st), cudaMemcpyDeviceToHost));
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "PPLCKPT1", 8);
  hd.version = 1;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.precision = h->prec;
  hd.rsz = (int32_t)h->rsz;
  hd.step = h->step;
  hd.cfg_hash = h->cfg_hash;
  FILE *fp = fopen(path, "wb");
  if (!fp) return PPL_E_IO;
  bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(st, sizeof(st), 1, fp) == 1 &&
            fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  ok = (fclose(fp) == 0) && ok;
  return ok ? PPL_OK : PPL_E_IO;
}

int ppl_load(ppl_t *h, const char *path) {
  if (!h || !path) return PPL_E_INVAL;
  FILE *fp = fopen(path, "rb");
  if (!fp) return PPL_E_IO;
  CkptHeader hd;
  double st[2];
  const size_t fbytes = (size_t)9 * h->N * h->rsz, tbytes = (size_t)h->N * h->rsz;
  std::vector<unsigned char> buf(fbytes + tbytes);
  bool ok = fread(&hd, sizeof(hd), 1, fp) == 1 && memcmp(hd.magic, "PPLCKPT1", 8) == 0 && hd.version == 1 &&
            hd.nx == h->nx && hd.ny == h->ny && hd.precision == h->prec && hd.rsz == (int32_t)h->rsz &&
            hd.cfg_hash == h->cfg_hash && fread(st, sizeof(st), 1, fp) == 1 &&
            fread(buf.data(), 1, buf.size(), fp) == buf.size();
  fclose(fp);
  if (!ok) return PPL_E_IO;
  CK(cudaStreamSynchronize(h->stream));
  h->cur = 0;
  CK(cudaMemcpy(h->f[0], buf.data(), fbytes, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->T[0], buf.data() + fbytes, tbytes, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->stats[0], st, sizeof(st), cudaMemcpyHostToDevice));
  CK(cudaMemset(h->status, 0, sizeof(unsigned)));
  h->step = hd.step;
  return PPL_OK;
}

int64_t ppl_launch_count(const ppl_t *h) { return h ? h->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------------
// ppl_step_noalloc: one fused step on caller-owned device buffers, allocating nothing.
// Its scratch (per-CTA FP64 partials of the mass sum and the CTA completion counter)
// lives in the file-scope array below, which every GPU that loads the library holds
// until the process exits.
// ---------------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxCtas = 4096;  // CTA partials the static scratch can hold
// [0, kNoAllocMaxCtas): CTA partials; [kNoAllocMaxCtas]: completion counter (as unsigned)
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxCtas + 1];

constexpr int kNoAllocMaxDevices = 256;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};  // device address of g_noalloc_scratch per device

// one-time set-up on the current device: the device address of the scratch (the host-side
// name of a __device__ array is not a device address) and the kernels' shared-memory limit
int noalloc_setup(double **scratch) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PPL_E_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    for (const StepVariant &v : {step_variant_fp64(), step_variant_fp32(), step_variant_fp32_pair()})
      for (int e = 0; e < 2; ++e)
        CK(cudaFuncSetAttribute(v.fn[e], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
    g_noalloc_addr[dev] = p;
  }
  *scratch = (double *)g_noalloc_addr[dev];
  return PPL_OK;
}

}  // namespace

extern "C" {

int ppl_step_noalloc(const ppl_config *cfg, const void *f_in, const void *T_in, void *f_out, void *T_out,
                     const double *stats_in, double *stats_out, uint32_t *status, void *cuda_stream) {
  int rc = validate(cfg);
  if (rc) return rc;
  if (is_tangent(cfg->precision)) return PPL_E_INVAL;  // plain FP64 / FP32 states only
  for (int s = 0; s < 4; ++s)
    if (cfg->rho_w[s] || cfg->T_w[s] || cfg->T_dirichlet[s]) return PPL_E_INVAL;  // would need device copies
  double *scratch = nullptr;
  rc = noalloc_setup(&scratch);
  if (rc) return rc;
  const StepVariant var = pick_variant(*cfg, PPL_KERNEL_AUTO);
  // the launch shape of ppl_init: strips of var.width columns, one wave of CTAs over the rows
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, var.fn[1], var.nt, var.smem));
  const int slots = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int strips = (cfg->nx + var.width - 1) / var.width;
  int yblocks = slots / strips;
  if (yblocks < 1) yblocks = 1;
  const int H = (cfg->ny + yblocks - 1) / yblocks;
  const dim3 grid(strips, (cfg->ny + H - 1) / H);
  if ((long long)grid.x * grid.y > kNoAllocMaxCtas) return PPL_E_NOMEM;  // beyond the static scratch
  // the caller's buffers (checked after the configuration, before anything is enqueued)
  if (!f_in || !T_in || !f_out || !T_out || !stats_in || !stats_out || !status) return PPL_E_INVAL;
  // 8-byte aligned state (the FP32 two-column kernel moves column pairs, FP64 moves doubles)
  for (const void *p : {f_in, T_in, (const void *)f_out, (const void *)T_out})
    if ((uintptr_t)p % 8 != 0) return PPL_E_INVAL;
  {
    // the step reads neighbours of what it writes: no output range may overlap another buffer
    const size_t es = cfg->precision == PPL_FP64 ? sizeof(double) : sizeof(float);
    const size_t nb = (size_t)cfg->nx * (size_t)cfg->ny * es;
    const uintptr_t fi = (uintptr_t)f_in, ti = (uintptr_t)T_in, fo = (uintptr_t)f_out, to = (uintptr_t)T_out;
    auto overlap = [](uintptr_t a, size_t na, uintptr_t b, size_t nb_) { return a < b + nb_ && b < a + na; };
    if (overlap(fo, 9 * nb, fi, 9 * nb) || overlap(fo, 9 * nb, ti, nb) || overlap(to, nb, fi, 9 * nb) ||
        overlap(to, nb, ti, nb) || overlap(fo, 9 * nb, to, nb))
      return PPL_E_INVAL;
  }
  // parameters of this configuration (a stack handle carries no device memory)
  ppl_sim tmp;
  tmp.cfg = *cfg;
  tmp.prec = cfg->precision;
  const void *none[4] = {nullptr, nullptr, nullptr, nullptr};
  const uint8_t *none8[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned *counter = (unsigned *)(scratch + kNoAllocMaxCtas);
  CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));  // the finalize relies on a zero counter
  StepIO io;
  io.f_in = f_in;
  io.T_in = T_in;
  io.f_out = f_out;
  io.T_out = T_out;
  io.stats_in = stats_in;
  io.stats_out = stats_out;
  io.partials = scratch;
  io.counter = counter;
  io.status = status;
  io.tmap_f = nullptr;  // caller-owned buffers: per-thread row copies
  io.tmap_T = nullptr;
  io.blocks_a = 0;
  io.fill_rows = 0;
  const int e = cfg->energy_on ? 1 : 0;
  if (cfg->precision == PPL_FP64) {
    Params<double> P;
    fill_params<double>(&tmp, P, (const double *const *)none, (const double *const *)none, none8);
    void *args[] = {(void *)&P, (void *)&io, (void *)&H};
    CK(cudaLaunchKernel(var.fn[e], grid, dim3(var.nt), args, var.smem, stream));
  } else {
    Params<float> P;
    fill_params<float>(&tmp, P, (const float *const *)none, (const float *const *)none, none8);
    void *args[] = {(void *)&P, (void *)&io, (void *)&H};
    CK(cudaLaunchKernel(var.fn[e], grid, dim3(var.nt), args, var.smem, stream));
  }
  return PPL_OK;
}

void ppl_destroy(ppl_t *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"

