// Fused time step of the coupled pseudopotential LBM + FD energy equation
// (arXiv 2201.04560, Sec. 2) for sm_103a: the row-marching pipeline.
//
// A CTA owns a strip of NT columns (NT - 6 interior columns plus a 3-column halo on each
// side) and H rows. One thread per column marches up the rows; rows are staged
// asynchronously into shared memory PF rows ahead (cp.async), and every iteration runs
// four stages at fixed row lags:
//   S1 (row q):   rho, j = sum f c, psi(rho, T)                       Eqs. (psi), (peng-robinson)
//   S2 (row q-1): F^m with the psi-based wall form, F^b, u             Eqs. (shanchen), (shanchen-walls),
//                                                                      (psi-based-formula), (gravitational_force),
//                                                                      (DensityAndVelocityRelationToF)
//   S3 (row q-2): Q and the MRT collision with the Li source terms;    Eqs. (Q), (Q-psi-based), (collisionMRT),
//                 first Heun stage of the energy equation              (li_source_terms), (S), (C), (energy-equation)
//   S4 (row q-3): pull streaming f(x) = f*(x - c_i), Zou-He, second   Eq. (lbm), Sec. 2.2
//                 Heun stage, store, FP64 mass partial
// Per-row quantities live in small shared-memory ring buffers (rows q-3..q), so every
// node is computed once per CTA; only the x-halo columns and 3 rows at each end of the
// strip are recomputed. DRAM traffic is one read and one write of (f, T) per node.
#pragma once

#include "common.cuh"

namespace ppl_dev {

// classification of a line index g (a column or a row) against its axis boundaries
struct LineMap {
  int src;      // in-domain line the node's state is read from (wrap, outflow copy, wall mirror)
  int solid;    // beyond a wall
  int wall;     // side index if this line is a wall line, else -1
  int outflow;  // an outflow line or beyond: an implicit copy of the first interior line
};

__device__ __forceinline__ LineMap map_line(int g, int n, int bc_lo, int bc_hi, int side_lo) {
  LineMap m;
  m.solid = 0;
  m.wall = -1;
  m.outflow = 0;
  if (g < 0 || g >= n) {
    const int k = g < 0 ? bc_lo : bc_hi;
    if (k == PERIODIC) {
      g %= n;
      if (g < 0) g += n;
    } else if (k == OUTFLOW) {
      m.outflow = 1;
      g = g < 0 ? 1 : n - 2;
    } else {
      m.solid = 1;
      g = g < 0 ? -g : 2 * (n - 1) - g;
      g = min(max(g, 0), n - 1);  // far ghosts of ragged strips are never used
    }
  } else {
    if (g == 0 && bc_lo == WALL) m.wall = side_lo;
    else if (g == n - 1 && bc_hi == WALL) m.wall = side_lo + 1;
    if (g == n - 1 && bc_hi == OUTFLOW) {
      m.outflow = 1;
      g = n - 2;
    } else if (g == 0 && bc_lo == OUTFLOW) {
      m.outflow = 1;
      g = 1;
    }
  }
  m.src = g;
  return m;
}

// mass-sum weight of a line: the first interior line also stands for its outflow copy
__device__ __forceinline__ double line_weight(int g, int n, int bc_lo, int bc_hi) {
  double w = 1.0;
  if (bc_hi == OUTFLOW && g == n - 2) w += 1.0;
  if (bc_lo == OUTFLOW && g == 1) w += 1.0;
  return w;
}

template <typename real>
__device__ __forceinline__ void cp_async_real(real *smem_dst, const real *gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (sizeof(real) == 16)  // value + tangent of the sensitivity step
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else if (sizeof(real) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename real>
struct S3Carry {  // S2 (row r) -> S3 (row r, next iteration)
  real fmx, fmy, fm2, inv_rho;  // F^m, |F^m|^2 / psi^2 = G^2 |s|^2, 1/rho
  real qs, qd, qxy;             // Q of Eq. (Q) as Qxx + Qyy, Qxx - Qyy, Qxy
};
template <typename real>
struct S4Carry {  // S3 (row r) -> S4 (row r, next iteration)
  real k1, lam, gdx, gdy, div, inv_rcv, ux, uy, A, B, Fx, Fy;
};

// FP64 keeps the EOS parts A, B, E of each node from the first stage for the compression
// term of the collision stage (rings [4][NT]), where a division and a square root cost
// more than three shared-memory round trips; the other precisions recompute them
template <typename real>
__host__ __device__ constexpr bool eos_ring() {
  return std::is_same<real, double>::value;
}

template <int NT, int PF, typename real>
constexpr size_t row_step_smem_bytes() {
  return (size_t)((PF + 3) * 10 + 5 * 4 + 18 + 3 + (eos_ring<real>() ? 12 : 0)) * NT * sizeof(real);
}

// Deterministic FP64 reduction of sum rho^{n+1} over the grid: the CTA's partial (acc of
// every thread) is written to its slot; the last CTA to finish sums the slots in a fixed
// order and publishes rho_bar and the mass for the next step. TANGENT: dacc carries the
// derivative of the sum as well (two slots per CTA), published as d rho_bar.
// The tile of a step is CTA `bid` of `nblk` (blockIdx / gridDim for a step launch); `done`, if
// given, is set to `done_value` (release) by the last tile once rho_bar is published (the
// persistent batch's step-completion flag).
// Rows [ya, yb) of row block `by` of a launch: the first io.blocks_a blocks have H rows, the
// others io.fill_rows rows (io.fill_rows = 0: every block has H rows).
__device__ __forceinline__ void block_rows(const StepIO &io, int H, int by, int ny, int *ya, int *yb) {
  const bool tall = io.fill_rows <= 0 || by < io.blocks_a;
  *ya = tall ? by * H : io.blocks_a * H + (by - io.blocks_a) * io.fill_rows;
  *yb = min(*ya + (tall ? H : io.fill_rows), ny);
}

template <int NT, bool TANGENT, typename PT>
__device__ __forceinline__ void tile_mass_finalize(const Params<PT> &P, const StepIO &io, double acc, double dacc,
                                                   unsigned bid, unsigned nblk, unsigned *done = nullptr,
                                                   unsigned done_value = 0) {
  const int t = threadIdx.x;
  constexpr int K = TANGENT ? 2 : 1;
  __shared__ double red[K][NT / 32];
  __shared__ bool am_last;
  double v[K];
  v[0] = acc;
  if (TANGENT) v[K - 1] = dacc;
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    if ((t & 31) == 0) red[j][t >> 5] = v[j];
  }
  __syncthreads();
  if (t == 0) {
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[j][w];
      io.partials[(size_t)bid * K + j] = s;
    }
    __threadfence();
    const unsigned done = atomicAdd(io.counter, 1u);
    am_last = (done == nblk - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double s[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      s[j] = 0.0;
      // the partials in the order b = t, t + NT, ..., loaded eight at a time so that their
      // latencies overlap (this CTA runs alone at the end of the step)
      for (unsigned b0 = t; b0 < nblk; b0 += 8 * NT) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned b = b0 + u * NT;
          x[u] = b < nblk ? __ldcg(io.partials + (size_t)b * K + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) s[j] += x[u];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_down_sync(0xffffffffu, s[j], o);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j)
      if ((t & 31) == 0) red[j][t >> 5] = s[j];
    __syncthreads();
    if (t == 0) {
      double tot[K];
      for (int j = 0; j < K; ++j) {
        tot[j] = 0.0;
        for (int w = 0; w < NT / 32; ++w) tot[j] += red[j][w];
      }
      io.stats_out[0] = tot[0] * P.inv_nodes;
      io.stats_out[1] = tot[0];
      if (TANGENT) io.stats_out[2] = tot[K - 1] * P.inv_nodes;
      *io.counter = 0u;
      if (done) {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(done), "r"(done_value) : "memory");
      }
    }
  }
  __syncthreads();  // the shared reduction slots may be reused by the caller's next tile
}

template <int NT, bool TANGENT, typename PT>
__device__ __forceinline__ void block_mass_finalize(const Params<PT> &P, const StepIO &io, double acc,
                                                    double dacc) {
  tile_mass_finalize<NT, TANGENT>(P, io, acc, dacc, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}

// SIMPLE: every row the CTA touches is an interior row (no wall, outflow or periodic
// wrap in y), so all row classification folds away at compile time.
template <typename real, bool ENERGY, int NT, int PF, bool SIMPLE>
__device__ __forceinline__ void row_body(const Params<real> &P, const StepIO &io, const int H,
                                         unsigned char *smem_raw) {
  constexpr int D = PF + 3;  // staging depth in rows
  constexpr int W = NT - 6;  // interior columns per strip
  real *stg = reinterpret_cast<real *>(smem_raw);  // [D][10][NT]: f_0..f_8, T of staged rows
  real *rpsi = stg + D * 10 * NT;                   // rings [4][NT] indexed by row mod 4
  real *rrho = rpsi + 4 * NT;
  real *rT = rrho + 4 * NT;
  real *rux = rT + 4 * NT;
  real *ruy = rux + 4 * NT;
  // [3][6][NT] post-collision populations that stream sideways (c_x != 0: i = 1, 3, 5, 6,
  // 7, 8), row mod 3; f*_0, f*_2, f*_4 stay in the column and are handed over in registers
  real *rfs = ruy + 4 * NT;
  real *rTs = rfs + 18 * NT;  // [3][NT] first Heun stage T*, row mod 3
  real *rA = rTs + 3 * NT;    // [4][NT] EOS parts of the row (eos_ring), row mod 4
  real *rB = rA + 4 * NT;
  real *rE = rB + 4 * NT;
  const real third = real(1) / real(3), twelfth = real(1) / real(12);
  const real big = sizeof(real) == 4 ? real(3.0e38) : real(1.0e300);

  const int t = threadIdx.x;
  const int x0 = blockIdx.x * W;
  int ya, yb;
  block_rows(io, H, blockIdx.y, P.ny, &ya, &yb);
  const int gx = x0 - 3 + t;
  const LineMap cm = map_line(gx, P.nx, P.hbc[0], P.hbc[1], 0);
  const bool col_bnd = cm.src == 0 || cm.src == P.nx - 1;  // node may sit on an x boundary line
  const long long plane = P.plane;
  real rho_bar = real(io.stats_in[0]);
  if constexpr (is_dual<real>::value) rho_bar = real(io.stats_in[0], io.stats_in[2]);
  const bool xwall_strip = (P.hbc[0] == WALL && x0 - 3 < 0) || (P.hbc[1] == WALL && x0 + W + 3 > P.nx - 1);
  const bool xout_strip = (P.hbc[0] == OUTFLOW && x0 - 3 <= 0) || (P.hbc[1] == OUTFLOW && x0 + W + 3 >= P.nx - 1);
  const bool any_outflow = P.hbc[0] == OUTFLOW || P.hbc[1] == OUTFLOW || P.hbc[2] == OUTFLOW || P.hbc[3] == OUTFLOW;
  const bool t_s2 = t >= 1 && t < NT - 1;
  const bool t_s3 = t >= 2 && t < NT - 2;
  const bool t_s4 = t >= 3 && t < NT - 3 && gx < P.nx && !cm.solid && !cm.outflow;
  const double wcol = line_weight(gx, P.nx, P.hbc[0], P.hbc[1]);
  const real *fin = reinterpret_cast<const real *>(io.f_in) + cm.src;
  const real *Tin = reinterpret_cast<const real *>(io.T_in) + cm.src;
  real *fout = reinterpret_cast<real *>(io.f_out);
  real *Tout = reinterpret_cast<real *>(io.T_out);
  const int n_it = yb - ya + 6;  // rows ya-3 .. yb+2 pass through S1
  unsigned flags = 0;
  double acc = 0.0, dacc = 0.0;  // FP64 mass partial (and its tangent)
  real acc_s = real(0), acc_c = real(0);  // FP32 path: compensated per-thread sum

  auto row_map = [&](int g) -> LineMap {
    if (SIMPLE) {
      LineMap m;
      m.src = g;
      m.solid = 0;
      m.wall = -1;
      m.outflow = 0;
      return m;
    }
    return map_line(g, P.ny, P.hbc[2], P.hbc[3], 2);
  };
  auto stage_row = [&](int q, int slot) {
    const long long k = (long long)row_map(q).src * P.nx;
    real *dst = stg + slot * 10 * NT + t;
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async_real(dst + i * NT, fin + i * plane + k);
    cp_async_real(dst + 9 * NT, Tin + k);
  };

#pragma unroll
  for (int j = 0; j < PF; ++j) {
    if (j < n_it) stage_row(ya - 3 + j, j);
    cp_async_commit();
  }

  real c1jx = 0, c1jy = 0, n1jx = 0, n1jy = 0;  // S1 -> S2 (j of the row)
  real f0n = 0, f2n = 0, f4n = 0, f0c = 0, f2c1 = 0, f2c2 = 0;  // column-bound f* (S3 -> S4)
  S3Carry<real> c2{}, n2{};
  S4Carry<real> cur{}, nxt{};
  int f3 = 0;  // iq mod 3
  for (int iq = 0; iq < n_it; ++iq) {
    const int q = ya - 3 + iq;
    if (iq + PF < n_it) stage_row(q + PF, (iq + PF) % D);
    cp_async_commit();
    cp_async_wait<PF>();  // this thread's copies of row q have landed
    const int s4_0 = iq & 3, s4_1 = (iq + 3) & 3, s4_2 = (iq + 2) & 3, s4_3 = (iq + 1) & 3;  // rows q, q-1, q-2, q-3
    const int f_r3 = f3, f_r2 = f3 == 2 ? 0 : f3 + 1, f_r4 = f3 == 0 ? 2 : f3 - 1;  // f*/T* rows q-3, q-2, q-4

    // ---- S1: row q ----
    {
      const LineMap rm = row_map(q);
      const real *st = stg + (iq % D) * 10 * NT + t;
      real f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = st[i * NT];
      const real Tt = st[9 * NT];
      const real delta = ((f[0] + (f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
      const real rho = P.rho_ref + delta;
      real psi = real(0);
      const int i0 = s4_0 * NT + t;
      if (!cm.solid && !rm.solid) {
        real arg;
        if constexpr (eos_ring<real>()) {
          real A, B, E;
          arg = psi_arg_eos(P, rho, P.T_ref + Tt, &A, &B, &E);
          rA[i0] = A;
          rB[i0] = B;
          rE[i0] = E;
        } else {
          arg = psi_arg(P, rho, P.T_ref + Tt);
        }
        if (!(arg >= real(0))) flags |= FLAG_PSI_NEG;
        psi = sqrt(fmax(arg, real(0)));
      }
      rpsi[i0] = psi;
      rrho[i0] = rho;
      rT[i0] = Tt;
      n1jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
      n1jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    }
    __syncthreads();

    // ---- S2: row q-1 ----
    if (iq >= 2) {
      const int r = q - 1;
      const LineMap rm = row_map(r);
      const int i0 = s4_1 * NT + t, iu = s4_0 * NT + t, id = s4_2 * NT + t;
      if (t_s2) {
        if (!cm.solid && !rm.solid) {
          const real p1 = rpsi[i0 + 1], p3 = rpsi[i0 - 1], p2 = rpsi[iu], p4 = rpsi[id];
          const real p5 = rpsi[iu + 1], p6 = rpsi[iu - 1], p7 = rpsi[id - 1], p8 = rpsi[id + 1];
          const real psi_c = rpsi[i0];
          const real d57 = p5 - p7, d86 = p8 - p6, s57 = p5 + p7, s68 = p6 + p8, s13 = p1 + p3, s24 = p2 + p4;
          real sx = third * (p1 - p3) + twelfth * (d57 + d86);
          real sy = third * (p2 - p4) + twelfth * (d57 - d86);
          // Q (Eq. Q) from the same psi neighbourhood, as Qxx + Qyy, Qxx - Qyy and Qxy
          real qs = third * (s13 + s24) + (real(1) / real(6)) * (s57 + s68) - real(2) * psi_c;
          real qd = third * (s13 - s24);
          const real qxy = twelfth * (s57 - s68);
          const int ws = cm.wall >= 0 ? cm.wall : rm.wall;
          if (ws >= 0) {
            // solid links (psi = 0 in the ring): their force weights sum to 1/2 along the
            // outward normal; in Q they add (1/2, 1/6) times the link's psi to the normal and
            // tangential components. psi-based model (Eqs. shanchen-walls, psi-based-formula,
            // Q-psi-based): both use psi_w = psi(rho_w, T). Modified model (Eqs.
            // mod-psi-based-formula, Q-mod-psi-based): the force is -G_w psi^2 sum w c, i.e.
            // a link psi of (G_w / G) psi, and Q drops the links (link psi = psi).
            real pf, pq;
            if (P.mod_psi) {
              pf = P.Gw_over_G * psi_c;
              pq = psi_c;
            } else {
              const real argw = psi_arg(P, wall_rho_w(P, ws, cm.src, rm.src), P.T_ref + rT[i0]);
              if (!(argw >= real(0))) flags |= FLAG_PSI_NEG;
              pf = pq = sqrt(fmax(argw, real(0)));
            }
            const real hw = real(0.5) * pf;
            if (ws == 0) sx -= hw;
            else if (ws == 1) sx += hw;
            else if (ws == 2) sy -= hw;
            else sy += hw;
            qs += (real(2) / real(3)) * pq;
            if (ws < 2) qd += third * pq;
            else qd -= third * pq;
          }
          const real qf = P.kappa_G2 * psi_c;
          n2.qs = qf * qs;
          n2.qd = qf * qd;
          n2.qxy = qf * qxy;
          const real rho = rrho[i0];
          const real gps = -P.G * psi_c;
          const real fmx = gps * sx, fmy = gps * sy;
          const real Fx = fmx + P.gx * (rho - rho_bar), Fy = fmy + P.gy * (rho - rho_bar);
          const real inv_rho = real(1) / rho;
          const real ux = (c1jx + real(0.5) * Fx) * inv_rho;
          const real uy = (c1jy + real(0.5) * Fy) * inv_rho;
          rux[i0] = ux;
          ruy[i0] = uy;
          n2.fmx = fmx;
          n2.fmy = fmy;
          n2.fm2 = P.G * P.G * (sx * sx + sy * sy);  // |F^m|^2 / psi^2 (F^m is proportional to psi)
          n2.inv_rho = inv_rho;
          if (!SIMPLE && ENERGY && r == 1 && P.hbc[2] == WALL) {  // mirror ghost of row -1
            rux[s4_3 * NT + t] = ux;
            ruy[s4_3 * NT + t] = -uy;
          }
        } else if (!SIMPLE && ENERGY && rm.solid && r == P.ny && P.hbc[3] == WALL) {  // mirror ghost of row ny
          rux[i0] = rux[s4_3 * NT + t];
          ruy[i0] = -ruy[s4_3 * NT + t];
        }
      }
      __syncthreads();
      if (ENERGY && xwall_strip) {
        if (t_s2) {
          int src = -1;
          if (P.hbc[0] == WALL && gx == -1) src = t + 2;
          else if (P.hbc[1] == WALL && gx == P.nx) src = t - 2;
          if (src >= 1 && src < NT - 1) {
            rux[i0] = -rux[s4_1 * NT + src];
            ruy[i0] = ruy[s4_1 * NT + src];
          }
        }
        __syncthreads();
      }
    }

    // ---- S3: row q-2 ----
    if (iq >= 4) {
      const int r = q - 2;
      const LineMap rm = row_map(r);
      const int i0 = s4_2 * NT + t, iu = s4_1 * NT + t, id = s4_3 * NT + t;
      if (t_s3) {
        if (!cm.solid && !rm.solid) {
          const real *st = stg + ((iq + D - 2) % D) * 10 * NT + t;
          real fd[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) fd[i] = st[i * NT];
          const real rho = rrho[i0];
          const real ux = rux[i0], uy = ruy[i0];
          const real Fx = c2.fmx + P.gx * (rho - rho_bar), Fy = c2.fmy + P.gy * (rho - rho_bar);
          real e = P.e_const;  // s_eta / 4
          if (P.var_eta) e = real(1) / (P.e_c0 + P.e_c1 * rho);
          collide(P, fd, rho, ux, uy, Fx, Fy, c2.fm2, c2.qs, c2.qd, c2.qxy, e);
          real *fs = rfs + f_r2 * 6 * NT + t;
          fs[0 * NT] = fd[1];
          fs[1 * NT] = fd[3];
          fs[2 * NT] = fd[5];
          fs[3 * NT] = fd[6];
          fs[4 * NT] = fd[7];
          fs[5 * NT] = fd[8];
          f0n = fd[0];
          f2n = fd[2];
          f4n = fd[4];
          nxt.Fx = Fx;
          nxt.Fy = Fy;
          if (ENERGY) {
            real Tw, Ts;
            const real T0 = rT[i0];
            nxt.ux = ux;
            nxt.uy = uy;
            real E = real(0);
            if constexpr (eos_ring<real>()) {
              nxt.A = rA[i0];
              nxt.B = rB[i0];
              E = rE[i0];
            } else {
              pr_parts(P, rho, &nxt.A, &nxt.B);
            }
            nxt.inv_rcv = c2.inv_rho * P.cv_inv;
            nxt.lam = P.lam_v + P.dlam * (rho - P.rho_v);
            // frozen coefficients of Eq. (energy-equation): grad lambda = dlam grad rho, div u
            const real r1 = rrho[i0 + 1], r3 = rrho[i0 - 1], r2 = rrho[iu], r4 = rrho[id];
            const real r5 = rrho[iu + 1], r6 = rrho[iu - 1], r7 = rrho[id - 1], r8 = rrho[id + 1];
            nxt.gdx = P.dlam * (third * (r1 - r3) + twelfth * (r5 - r6 - r7 + r8));
            nxt.gdy = P.dlam * (third * (r2 - r4) + twelfth * (r5 + r6 - r7 - r8));
            nxt.div = third * (rux[i0 + 1] - rux[i0 - 1]) +
                      twelfth * (rux[iu + 1] - rux[iu - 1] - rux[id - 1] + rux[id + 1]) +
                      third * (ruy[iu] - ruy[id]) + twelfth * (ruy[iu + 1] + ruy[iu - 1] - ruy[id - 1] - ruy[id + 1]);
            const bool bnd = col_bnd || (!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1));
            if (bnd && t_fixed(P, cm.src, rm.src, &Tw)) {
              Ts = Tw - P.T_ref;
              nxt.k1 = real(0);
            } else if (rm.outflow) {
              Ts = rTs[f_r3 * NT + t];  // outflow row: copy of the first interior row
              nxt.k1 = real(0);
            } else {
              const real t1 = rT[i0 + 1], t3 = rT[i0 - 1], t2 = rT[iu], t4 = rT[id];
              const real t5 = rT[iu + 1], t6 = rT[iu - 1], t7 = rT[id - 1], t8 = rT[id + 1];
              const real gtx = third * (t1 - t3) + twelfth * (t5 - t6 - t7 + t8);
              const real gty = third * (t2 - t4) + twelfth * (t5 + t6 - t7 - t8);
              const real lap = (real(2) / real(3)) * (t1 + t2 + t3 + t4 - real(4) * T0) +
                               (real(1) / real(6)) * (t5 + t6 + t7 + t8 - real(4) * T0);
              const real TdpdT = eos_ring<real>() ? (P.T_ref + T0) * nxt.A + E : T_dpdT(P, nxt.A, nxt.B, P.T_ref + T0);
              const real k1 = -(ux * gtx + uy * gty) + (nxt.lam * lap + nxt.gdx * gtx + nxt.gdy * gty) * nxt.inv_rcv -
                              TdpdT * nxt.div * nxt.inv_rcv;
              nxt.k1 = k1;
              Ts = T0 + k1;
            }
            rTs[f_r2 * NT + t] = Ts;
            if (!SIMPLE && r == 1 && P.hbc[2] == WALL) rTs[f_r4 * NT + t] = Ts;  // mirror ghost of row -1
          }
        } else if (!SIMPLE && ENERGY && rm.solid && r == P.ny && P.hbc[3] == WALL) {
          rTs[f_r2 * NT + t] = rTs[f_r4 * NT + t];  // mirror ghost of row ny (copy of row ny-2)
        }
      }
      __syncthreads();
      if (ENERGY && (xwall_strip || xout_strip)) {
        if (t_s3) {
          int src = -1;
          if (P.hbc[0] == WALL && gx == -1) src = t + 2;
          else if (P.hbc[1] == WALL && gx == P.nx) src = t - 2;
          else if (P.hbc[1] == OUTFLOW && gx >= P.nx - 1) src = t - (gx - (P.nx - 2));
          else if (P.hbc[0] == OUTFLOW && gx <= 0) src = t + (1 - gx);
          if (src >= 2 && src < NT - 2) rTs[f_r2 * NT + t] = rTs[f_r2 * NT + src];
        }
        __syncthreads();
      }
    }

    // ---- S4: row q-3 ----
    if (iq >= 6 && t_s4) {
      const int r = q - 3;
      const LineMap rm = row_map(r);
      if (!rm.outflow) {
        // pull: f_i(x) = f*_i(x - c_i); ring rows r-1, r, r+1 are slots f_r4, f_r3, f_r2
        const real *lo = rfs + f_r4 * 6 * NT + t, *mid = rfs + f_r3 * 6 * NT + t, *hi = rfs + f_r2 * 6 * NT + t;
        real fd[9];
        fd[0] = f0c;       // f*_0 of row r (previous iteration's S3)
        fd[1] = mid[0 * NT - 1];
        fd[2] = f2c2;      // f*_2 of row r-1 (two iterations back)
        fd[3] = mid[1 * NT + 1];
        fd[4] = f4n;       // f*_4 of row r+1 (this iteration's S3)
        fd[5] = lo[2 * NT - 1];
        fd[6] = lo[3 * NT + 1];
        fd[7] = hi[4 * NT + 1];
        fd[8] = hi[5 * NT - 1];
        const int ws = cm.wall >= 0 ? cm.wall : rm.wall;
        if (ws >= 0) zou_he(ws, fd, -real(0.5) * cur.Fx, -real(0.5) * cur.Fy);
        const real delta = ((fd[0] + (fd[1] + fd[2]) + (fd[3] + fd[4])) + ((fd[5] + fd[6]) + (fd[7] + fd[8])));
        const real rho_new = P.rho_ref + delta;
        real T_new = rT[s4_3 * NT + t];
        if (ENERGY) {
          real Tw;
          const bool bnd = col_bnd || (!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1));
          if (!(bnd && t_fixed(P, cm.src, rm.src, &Tw))) {
            const real *m0 = rTs + f_r3 * NT + t, *u0 = rTs + f_r2 * NT + t, *d0 = rTs + f_r4 * NT + t;
            const real c = m0[0];
            const real t1 = m0[1], t3 = m0[-1], t2 = u0[0], t4 = d0[0];
            const real t5 = u0[1], t6 = u0[-1], t7 = d0[-1], t8 = d0[1];
            const real gtx = third * (t1 - t3) + twelfth * (t5 - t6 - t7 + t8);
            const real gty = third * (t2 - t4) + twelfth * (t5 + t6 - t7 - t8);
            const real lap = (real(2) / real(3)) * (t1 + t2 + t3 + t4 - real(4) * c) +
                             (real(1) / real(6)) * (t5 + t6 + t7 + t8 - real(4) * c);
            const real k2 = -(cur.ux * gtx + cur.uy * gty) + (cur.lam * lap + cur.gdx * gtx + cur.gdy * gty) * cur.inv_rcv -
                            T_dpdT(P, cur.A, cur.B, P.T_ref + c) * cur.div * cur.inv_rcv;
            T_new = T_new + real(0.5) * (cur.k1 + k2);
          }
        }
        const long long k = (long long)r * P.nx + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) fout[i * plane + k] = fd[i];
        Tout[k] = T_new;
        if (!(rho_new > real(0) && rho_new <= big && fabs(T_new) <= big))
          flags |= (rho_new == rho_new && fabs(T_new) <= big && rho_new <= big) ? FLAG_RHO_NONPOS : FLAG_NAN;
        const real wr = (!SIMPLE && any_outflow) ? real(wcol * line_weight(r, P.ny, P.hbc[2], P.hbc[3]))
                                                 : (any_outflow ? real(wcol) : real(1));
        if (sizeof(real) != 4) {
          acc += double(wr * rho_new);
          dacc += tangent_of(wr * rho_new);
        } else {
          // compensated FP32 sum of this thread's column (FP64 beyond the thread)
          const real yk = wr * rho_new - acc_c;
          const real tk = acc_s + yk;
          acc_c = (tk - acc_s) - yk;
          acc_s = tk;
        }
      }
    }
    c1jx = n1jx;
    c1jy = n1jy;
    c2 = n2;
    cur = nxt;
    f0c = f0n;
    f2c2 = f2c1;
    f2c1 = f2n;
    f3 = f3 == 2 ? 0 : f3 + 1;
  }
  cp_async_wait<0>();
  if (sizeof(real) == 4) acc = double(acc_s) - double(acc_c);
  if (flags) atomicOr(io.status, flags);

  block_mass_finalize<NT, is_dual<real>::value>(P, io, acc, dacc);
}


// FP32: 5 CTAs per SM fit in shared memory; ask the register allocator for the same
template <typename real, bool ENERGY, int NT, int PF>
__global__ void __launch_bounds__(NT, sizeof(real) == 4 ? 5 : 1) row_step(const Params<real> P, const StepIO io,
                                                                       const int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int ya, yb;
  block_rows(io, H, blockIdx.y, P.ny, &ya, &yb);
  if (ya - 3 >= 1 && yb + 2 <= P.ny - 2)
    row_body<real, ENERGY, NT, PF, true>(P, io, H, smem_raw);
  else
    row_body<real, ENERGY, NT, PF, false>(P, io, H, smem_raw);
}

}  // namespace ppl_dev
