// Reverse-mode (adjoint) sweep of the fused step, for the sigma / kappa calibration of Sec.
// 3.2 on the lattice: given the state f^n of a step and the adjoint fbar^{n+1} = dJ/df^{n+1}
// of its output, one call forms fbar^n = (d f^{n+1} / d f^n)^T fbar^{n+1} and adds
// (d f^{n+1} / d(sigma, kappa))^T fbar^{n+1} to an FP64 gradient. The forward map is the
// step of Sec. 2 on a periodic isothermal box without gravity (the calibration runs: a
// planar interface and a static droplet), with absolute populations in FP64:
//   rho = sum f, psi = sqrt(2 (p(rho, T) - rho/3) / G)                   Eqs. (psi), (peng-robinson)
//   s = sum_i W_i psi(x + c_i) c_i, F = -G psi s, |F|^2 = G^2 |s|^2       Eq. (shanchen)
//   Q = kappa G/2 psi sum_i W_i (psi(x + c_i) - psi(x)) c_i c_i           Eq. (Q)
//   u = (sum f c + F/2) / rho                                            Eq. (DensityAndVelocityRelationToF)
//   f* = f + M^-1 [-Lambda (m - m^eq) + (I - Lambda/2) S + C]            Eqs. (collisionMRT), (S), (C)
//   f^{n+1}_i(x + c_i) = f*_i(x)                                         Eq. (lbm)
// The collision is taken in the closed form of the step kernels (common.cuh: momentum
// increments equal to F, e / eps non-equilibrium parts without the mass sum), and its
// transpose is written out operation by operation below, in reverse order.
//
// Three kernels per step: (1) rho, psi and d psi / d rho of every node; (2) per node, the
// forward quantities again and their adjoints: the node's own share of fbar^n, its share of
// rho-bar, and the adjoints of the psi stencil sums (s, Q), which belong to the neighbours'
// psi; per-CTA FP64 partials of the parameter gradient; (3) per node, psi-bar gathered
// from the stencil sums of the neighbours, and fbar^n_i += (rho-bar + psi-bar dpsi/drho).
// A last one-block kernel adds the partials to the gradient in a fixed order, so a sweep
// is bitwise reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sim.cuh"

using namespace ppl_host;

namespace {

constexpr int kAdjNT = 128;
constexpr int kAdjScratch = 10;  // doubles per node: rho, psi, dpsi, rbar, pbar_c, sbx, sby, ts, td, txy

struct AdjParams {
  int nx, ny;
  long long N;
  double a, b, R, G, Tc, k;  // Peng-Robinson and the pseudopotential strength
  double kG2;                // kappa G / 2
  double G2;                 // G^2
  // closed-form collision coefficients (as the step kernels form them)
  double c1n, c1q, c1u, c1f, c2n, c2q, c2u, c2f, c4n, c4f, c6n, c6f, e;
  double dc1f_dsigma, dc2f_dsigma;  // c1f, c2f are linear in sigma
  double dkG2_dkappa;               // G / 2
};

__device__ __forceinline__ long long wrap(const AdjParams &P, int x, int y) {
  x %= P.nx;
  if (x < 0) x += P.nx;
  y %= P.ny;
  if (y < 0) y += P.ny;
  return (long long)y * P.nx + x;
}

__device__ __constant__ const int kAX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ const int kAY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Peng-Robinson p(rho, T) and dp/drho at fixed T (Eq. peng-robinson)
__device__ __forceinline__ void pr_p(const AdjParams &P, double rho, double T, double *p, double *dp) {
  const double st = sqrt(T / P.Tc);
  const double al = (1.0 + P.k * (1.0 - st)) * (1.0 + P.k * (1.0 - st));
  const double omb = 1.0 - P.b * rho;
  const double den = 1.0 + 2.0 * P.b * rho - P.b * P.b * rho * rho;
  *p = rho * P.R * T / omb - P.a * al * rho * rho / den;
  const double dden = 2.0 * P.b - 2.0 * P.b * P.b * rho;
  *dp = P.R * T / (omb * omb) - P.a * al * (2.0 * rho * den - rho * rho * dden) / (den * den);
}

// (1) rho, psi, d psi / d rho
__global__ void adj_psi(const AdjParams P, const double *f, const double *T, double *scr) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.N) return;
  double rho = 0.0;
  for (int i = 0; i < 9; ++i) rho += f[i * P.N + k];
  double p, dp;
  pr_p(P, rho, T[k], &p, &dp);
  const double arg = 2.0 * (p - rho / 3.0) / P.G;
  const double psi = sqrt(fmax(arg, 0.0));
  scr[0 * P.N + k] = rho;
  scr[1 * P.N + k] = psi;
  scr[2 * P.N + k] = psi > 0.0 ? (dp - 1.0 / 3.0) / (P.G * psi) : 0.0;  // d psi / d rho
}

// (2) the node's adjoint: fbar_out gets the node's own share, scr its stencil adjoints
__global__ void __launch_bounds__(kAdjNT) adj_node(const AdjParams P, const double *f, const double *fbar_in,
                                                   double *fbar_out, double *scr, double *part) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dsig = 0.0, dkap = 0.0;
  if (k < P.N) {
    const int x = (int)(k % P.nx), y = (int)(k / P.nx);
    const double *psi_f = scr + 1 * P.N;
    double fl[9], ps[9];
    for (int i = 0; i < 9; ++i) {
      fl[i] = f[i * P.N + k];
      ps[i] = psi_f[wrap(P, x + kAX[i], y + kAY[i])];
    }
    const double rho = scr[k], psi_c = ps[0];
    // ---- forward ----
    const double jx0 = fl[1] - fl[3] + fl[5] - fl[6] - fl[7] + fl[8];
    const double jy0 = fl[2] - fl[4] + fl[5] + fl[6] - fl[7] - fl[8];
    const double t3 = 1.0 / 3.0, t12 = 1.0 / 12.0, t6 = 1.0 / 6.0;
    const double sx = t3 * (ps[1] - ps[3]) + t12 * (ps[5] - ps[7] + ps[8] - ps[6]);
    const double sy = t3 * (ps[2] - ps[4]) + t12 * (ps[5] - ps[7] - ps[8] + ps[6]);
    const double Ss = t3 * (ps[1] + ps[2] + ps[3] + ps[4]) + t6 * (ps[5] + ps[6] + ps[7] + ps[8]) - 2.0 * psi_c;
    const double Sd = t3 * (ps[1] + ps[3] - ps[2] - ps[4]);
    const double Sxy = t12 * (ps[5] + ps[7] - ps[6] - ps[8]);
    const double Fx = -P.G * psi_c * sx, Fy = -P.G * psi_c * sy;
    const double fm2 = P.G2 * (sx * sx + sy * sy);
    const double ux = (jx0 + 0.5 * Fx) / rho, uy = (jy0 + 0.5 * Fy) / rho;
    // closed-form collision, forward values needed by its transpose
    const double jx = rho * ux, jy = rho * uy;
    const double e = P.e, g = 0.25 - 0.5 * e;
    // ---- transpose, from the post-collision populations back ----
    double fb[9];  // fbar*_i(x) = fbar^{n+1}_i(x + c_i)
    for (int i = 0; i < 9; ++i) fb[i] = fbar_in[i * P.N + wrap(P, x + kAX[i], y + kAY[i])];
    double gf[9];  // the node's own share of fbar^n
    for (int i = 0; i < 9; ++i) gf[i] = fb[i];  // f* = f + ...
    const double cpb = fb[1] + fb[3], u4b = fb[1] - fb[3];
    const double v6b = fb[2] - fb[4], cnb = -fb[2] - fb[4];
    const double e5b = fb[5] + fb[7], ppb = fb[5] - fb[7];
    const double e6b = fb[6] + fb[8], pmb = fb[6] - fb[8];
    double a1b = -4.0 * fb[0], a2b = 4.0 * fb[0];
    const double p56b = ppb + pmb, p34b = ppb - pmb;
    const double cdb = e5b + e6b, a8b = e5b - e6b;
    double a3b = p34b, a4b = p34b, a5b = p56b, a6b = p56b;
    const double a7b = cpb + cnb, b1b = cnb - cpb;
    a3b += u4b;
    a4b += -2.0 * u4b;
    a5b += v6b;
    a6b += -2.0 * v6b;
    a1b += 2.0 * cdb + b1b;
    a2b += cdb + 2.0 * b1b;
    double uxb = 0.0, uyb = 0.0, Fxb = 0.0, Fyb = 0.0, rhob = 0.0;
    double mxyb = 0.0, mxxb = 0.0, qsb = 0.0, qdb = 0.0, qxyb = 0.0, uFb = 0.0, yFb = 0.0, fm2b = 0.0;
    double nqyb = 0.0, nqxb = 0.0, nzb = 0.0, neb = 0.0, ru2b = 0.0, y2b = 0.0, jxb = 0.0, jyb = 0.0;
    // a8 = e (mxy - qxy) + g (ux Fy + uy Fx)
    mxyb += e * a8b;
    qxyb += -e * a8b;
    uxb += g * Fy * a8b;
    Fyb += g * ux * a8b;
    uyb += g * Fx * a8b;
    Fxb += g * uy * a8b;
    // a7 = e (mxx - qd) + 2 g (uF - 2 yF)
    mxxb += e * a7b;
    qdb += -e * a7b;
    uFb += 2.0 * g * a7b;
    yFb += -4.0 * g * a7b;
    // a6 = c6n nqy + c6f Fy, a4 = c4n nqx + c4f Fx, a5 = Fy / 6, a3 = Fx / 6
    nqyb += P.c6n * a6b;
    Fyb += P.c6f * a6b;
    nqxb += P.c4n * a4b;
    Fxb += P.c4f * a4b;
    Fyb += a5b / 6.0;
    Fxb += a3b / 6.0;
    // a2 = c2n nz + c2q qs + c2u uF + c2f fm2, a1 = c1n ne + c1q qs + c1u uF + c1f fm2
    nzb += P.c2n * a2b;
    qsb += P.c2q * a2b + P.c1q * a1b;
    uFb += P.c2u * a2b + P.c1u * a1b;
    fm2b += P.c2f * a2b + P.c1f * a1b;
    neb += P.c1n * a1b;
    dsig += (P.dc1f_dsigma * a1b + P.dc2f_dsigma * a2b) * fm2;
    // uF = ux Fx + yF, yF = uy Fy
    uxb += Fx * uFb;
    Fxb += ux * uFb;
    yFb += uFb;
    uyb += Fy * yFb;
    Fyb += uy * yFb;
    // mxy = jx uy + (s68 - s57), mxx = (ru2 - 2 y2) - (s13 - s24)
    jxb += uy * mxyb;
    uyb += jx * mxyb;
    double s68b = mxyb, s57b = -mxyb;
    ru2b += mxxb;
    y2b += -2.0 * mxxb;
    double s13b = -mxxb, s24b = mxxb;
    // nqy = (d57 + d68 - 2 d24) + jy, nqx = (d57 - d68 - 2 d13) + jx
    double d57b = nqyb + nqxb, d68b = nqyb - nqxb, d24b = -2.0 * nqyb, d13b = -2.0 * nqxb;
    jyb += nqyb;
    jxb += nqxb;
    // nz = (f0 - ax) + ru2, ne = 4 dg + (ax - 2 f0) - 3 ru2
    gf[0] += nzb - 2.0 * neb;
    const double axb = -nzb + neb;
    const double dgb = 4.0 * neb;
    ru2b += nzb - 3.0 * neb;
    // ru2 = jx ux + y2, y2 = jy uy
    jxb += ux * ru2b;
    uxb += jx * ru2b;
    y2b += ru2b;
    jyb += uy * y2b;
    uyb += jy * y2b;
    // jx = rho ux, jy = rho uy (the collision's rho u)
    rhob += ux * jxb + uy * jyb;
    uxb += rho * jxb;
    uyb += rho * jyb;
    // ax = s13 + s24, dg = s57 + s68
    s13b += axb;
    s24b += axb;
    s57b += dgb;
    s68b += dgb;
    gf[1] += s13b + d13b;
    gf[3] += s13b - d13b;
    gf[2] += s24b + d24b;
    gf[4] += s24b - d24b;
    gf[5] += s57b + d57b;
    gf[7] += s57b - d57b;
    gf[6] += s68b + d68b;
    gf[8] += s68b - d68b;
    // u = (j0 + F/2) / rho
    const double jx0b = uxb / rho, jy0b = uyb / rho;
    Fxb += 0.5 * uxb / rho;
    Fyb += 0.5 * uyb / rho;
    rhob += -(ux * uxb + uy * uyb) / rho;
    for (int i = 0; i < 9; ++i) gf[i] += jx0b * kAX[i] + jy0b * kAY[i];
    // F = -G psi_c s, fm2 = G^2 |s|^2
    double pcb = -P.G * (sx * Fxb + sy * Fyb);
    const double sxb = -P.G * psi_c * Fxb + 2.0 * P.G2 * sx * fm2b;
    const double syb = -P.G * psi_c * Fyb + 2.0 * P.G2 * sy * fm2b;
    // Q = kG2 psi_c (Ss, Sd, Sxy)
    pcb += P.kG2 * (Ss * qsb + Sd * qdb + Sxy * qxyb) - 2.0 * P.kG2 * psi_c * qsb;
    dkap += P.dkG2_dkappa * psi_c * (Ss * qsb + Sd * qdb + Sxy * qxyb);
    for (int i = 0; i < 9; ++i) fbar_out[i * P.N + k] = gf[i];
    scr[3 * P.N + k] = rhob;
    scr[4 * P.N + k] = pcb;
    scr[5 * P.N + k] = sxb;
    scr[6 * P.N + k] = syb;
    scr[7 * P.N + k] = P.kG2 * psi_c * qsb;  // adjoint weights of the neighbours' psi in Ss, Sd, Sxy
    scr[8 * P.N + k] = P.kG2 * psi_c * qdb;
    scr[9 * P.N + k] = P.kG2 * psi_c * qxyb;
  }
  // per-CTA FP64 partials of the gradient, in a fixed order
  __shared__ double red[2][kAdjNT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    dsig += __shfl_down_sync(0xffffffffu, dsig, o);
    dkap += __shfl_down_sync(0xffffffffu, dkap, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dsig;
    red[1][threadIdx.x >> 5] = dkap;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kAdjNT / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// weight of psi(x + c_i) in the stencil sums s_x, s_y, Ss, Sd, Sxy of node x
__device__ __forceinline__ void stencil_w(int i, double *wx, double *wy, double *ws, double *wd, double *wxy) {
  const double t3 = 1.0 / 3.0, t12 = 1.0 / 12.0, t6 = 1.0 / 6.0;
  const int cx = kAX[i], cy = kAY[i];
  const bool axis = (cx == 0) != (cy == 0);
  const double W = axis ? t3 : t12;
  *wx = W * cx;
  *wy = W * cy;
  *ws = axis ? t3 : t6;
  *wd = axis ? t3 * (double)(cx * cx - cy * cy) : 0.0;
  *wxy = axis ? 0.0 : t12 * (double)(cx * cy);
}

// (3) psi-bar of node z from its own use and from every neighbour x = z - c_i whose stencil
// reads psi(z); then fbar^n_i(z) += rho-bar(z) + psi-bar(z) d psi / d rho
__global__ void adj_gather(const AdjParams P, const double *scr, double *fbar_out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.N) return;
  const int x = (int)(k % P.nx), y = (int)(k / P.nx);
  double pb = scr[4 * P.N + k];
  for (int i = 1; i < 9; ++i) {
    const long long n = wrap(P, x - kAX[i], y - kAY[i]);
    double wx, wy, ws, wd, wxy;
    stencil_w(i, &wx, &wy, &ws, &wd, &wxy);
    pb += wx * scr[5 * P.N + n] + wy * scr[6 * P.N + n] + ws * scr[7 * P.N + n] + wd * scr[8 * P.N + n] +
          wxy * scr[9 * P.N + n];
  }
  const double rb = scr[3 * P.N + k] + pb * scr[2 * P.N + k];
  for (int i = 0; i < 9; ++i) fbar_out[i * P.N + k] += rb;
}

// grad[0..1] += the partials, in block order
__global__ void adj_accumulate(const double *part, int nblk, double *grad) {
  __shared__ double red[2][kAdjNT];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kAdjNT) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int h = kAdjNT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    grad[0] += red[0][0];
    grad[1] += red[1][0];
  }
}

bool adjoint_applicable(const ppl_config *c) {
  for (int s = 0; s < 4; ++s)
    if (c->hydro_bc[s] != PPL_PERIODIC || c->thermal_bc[s] != PPL_T_PERIODIC) return false;
  return !c->energy_on && c->gx == 0.0 && c->gy == 0.0 && !(c->eta_l > 0 && c->eta_v > 0);
}

long long adj_blocks(const ppl_config *c) { return ((long long)c->nx * c->ny + kAdjNT - 1) / kAdjNT; }

}  // namespace

extern "C" {

size_t ppl_adjoint_scratch_bytes(int32_t nx, int32_t ny) {
  if (nx <= 0 || ny <= 0) return 0;
  const long long N = (long long)nx * ny;
  return (size_t)(kAdjScratch * N + 2 * ((N + kAdjNT - 1) / kAdjNT)) * sizeof(double);
}

int ppl_adjoint_step(const ppl_config *cfg, const double *f, const double *T, const double *fbar_in,
                     double *fbar_out, double *grad, void *scratch, void *cuda_stream) {
  int rc = validate(cfg);
  if (rc) return rc;
  if (!adjoint_applicable(cfg)) return PPL_E_INVAL;
  if (!f || !T || !fbar_in || !fbar_out || !grad || !scratch || fbar_in == fbar_out) return PPL_E_INVAL;
  AdjParams P;
  P.nx = cfg->nx;
  P.ny = cfg->ny;
  P.N = (long long)cfg->nx * cfg->ny;
  P.a = cfg->a;
  P.b = cfg->b;
  P.R = cfg->R;
  P.G = cfg->G;
  P.Tc = ppl_tc(cfg->a, cfg->b, cfg->R);
  P.k = 0.37464 + 1.54226 * cfg->omega - 0.2699 * cfg->omega * cfg->omega;
  P.kG2 = cfg->kappa * cfg->G / 2.0;
  P.G2 = cfg->G * cfg->G;
  const double *s = cfg->s;
  // the coefficients of collide() (common.cuh), built as the step kernels build them
  const double se = 12.0 / (1.0 / s[1] - 0.5), sz = 12.0 / (1.0 / s[2] - 0.5);
  P.c1n = -s[1] / 36.0;
  P.c1q = s[1] / 24.0;
  P.c1u = (1.0 - 0.5 * s[1]) / 6.0;
  P.dc1f_dsigma = se * ((1.0 - 0.5 * s[1]) / 36.0);
  P.c1f = cfg->sigma * P.dc1f_dsigma;
  P.c2n = -s[2] / 12.0;
  P.c2q = -s[2] / 24.0;
  P.c2u = -(1.0 - 0.5 * s[2]) / 6.0;
  P.dc2f_dsigma = sz * (-(1.0 - 0.5 * s[2]) / 36.0);
  P.c2f = cfg->sigma * P.dc2f_dsigma;
  P.c4n = -s[4] / 12.0;
  P.c4f = -(1.0 - 0.5 * s[4]) / 12.0;
  P.c6n = -s[6] / 12.0;
  P.c6f = -(1.0 - 0.5 * s[6]) / 12.0;
  P.e = 0.25 * s[7];
  P.dkG2_dkappa = cfg->G / 2.0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *scr = (double *)scratch;
  double *part = scr + kAdjScratch * P.N;
  const unsigned nb = (unsigned)adj_blocks(cfg);
  adj_psi<<<nb, kAdjNT, 0, st>>>(P, f, T, scr);
  adj_node<<<nb, kAdjNT, 0, st>>>(P, f, fbar_in, fbar_out, scr, part);
  adj_gather<<<nb, kAdjNT, 0, st>>>(P, scr, fbar_out);
  adj_accumulate<<<1, kAdjNT, 0, st>>>(part, (int)nb, grad);
  return cuda_err(cudaGetLastError());
}

}  // extern "C"
