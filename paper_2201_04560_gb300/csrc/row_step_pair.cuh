// FP32 fused step with two columns per thread (packed f32x2 arithmetic) for domains that
// are hydrodynamically periodic in x, with an even nx (the x lines may hold Dirichlet
// temperatures).
//
// The same row-marching pipeline as row_step.cuh (stages S1..S4 at row lags 0..3, rings
// of per-row quantities in shared memory), with each thread owning the adjacent columns
// (2t, 2t + 1) of a strip of 2 NT columns: 4 halo columns on each side, 2 NT - 8 interior
// columns. Both columns of a thread are computed by one packed instruction wherever the
// arithmetic allows (F2 in lane2.cuh), the staged rows and the stores move 8 bytes per
// thread, and a column's neighbours come from one 8-byte and two 4-byte shared-memory
// reads per pair (ring rows carry two zeroed pad floats on each side, so the reads of the
// strip's outermost threads need no clamping: those columns are halo, never stored). With
// x periodic and nx even, a pair never straddles the domain edge
// and its global address is 8-byte aligned. Rows (walls, outflow, Dirichlet lines in y)
// are handled exactly as in the one-column kernel; only per-node boundary data of a wall
// row (rho_w, T_w, the Dirichlet mask) is looked up column by column.
//
// Row staging: a strip that lies wholly inside the domain has each row brought in by TMA
// (one thread issues a 3-D tensor copy of the nine population rows and a 2-D copy of the
// temperature row, completing on the slot's mbarrier, which all threads wait on); strips
// that wrap across the periodic x seam, and domains without tensor maps, use per-thread
// 8-byte cp.async copies with the wrap applied per column.
#pragma once

#include "lane2.cuh"
#include "row_step.cuh"

namespace ppl_dev {

// values of the columns (2t - 1, 2t), (2t, 2t + 1), (2t + 1, 2t + 2) of one padded ring row
struct Trip {
  F2 l, c, r;
};
__device__ __forceinline__ Trip trip(const float *row, int t) {
  const float2 c = *reinterpret_cast<const float2 *>(row + 2 * t);
  const float l = row[2 * t - 1], r = row[2 * t + 2];
  return {F2(l, c.x), F2(c), F2(c.y, r)};
}
__device__ __forceinline__ F2 ld2(const float *p) { return F2(*reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ void st2(float *p, F2 v) { *reinterpret_cast<float2 *>(p) = v.v; }
__device__ __forceinline__ void cp_async8(float *smem_dst, const float *gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// staged rows [PF + 3][10][2 NT]; rings of row stride 2 NT + 4: psi, rho, T, ux, uy [4] (row
// mod 4) and [3][7] (row mod 3: the six sideways post-collision populations and the first
// Heun stage T*)
// ---- TMA row staging: bulk tensor copies completing on an mbarrier (sm_90+) ----
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void tmap_acquire(const void *m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(m) : "memory");
}
// waits for the phase of the given parity to complete; false after limit_ns (and at most 2^26
// polls), so that a copy that never lands cannot hang the kernel
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns = 1000000000ull) {
  unsigned long long t0 = 0;
  for (int i = 0; i < (1 << 26); ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(now));
    if (i == 0) t0 = now;
    else if (now - t0 > limit_ns) return false;
  }
  return false;
}
// one staged row: f_0..f_8 (box of 2 NT columns x 1 row x 9 planes) and T (2 NT columns x 1
// row) of row y from column x, into the slot at shared address dst ([10][2 NT] floats, 128-byte
// aligned), completing 10 x 2 NT x 4 bytes on the mbarrier bar
template <int NT>
__device__ __forceinline__ void tma_row(unsigned dst, unsigned bar, const void *mf, const void *mt, int x, int y) {
  constexpr unsigned kRow = 2 * NT * 4;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "n"(10 * kRow) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"(mf), "r"(x), "r"(y), "r"(0), "r"(bar)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(dst + 9 * kRow),
      "l"(mt), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int NT>
__host__ __device__ constexpr int pair_ring_stride() {
  return 2 * NT + 4;
}
template <int NT, int PF>
constexpr size_t row_step_pair_smem_bytes() {  // + 128: the staging base is aligned up to 128 bytes
  return (size_t)((PF + 3) * 10 * (2 * NT) + (5 * 4 + 3 * 7) * pair_ring_stride<NT>()) * sizeof(float) + 128;
}

template <bool ENERGY, int NT, int PF, bool SIMPLE>
__device__ __forceinline__ void row_body_pair(const Params<float> &P, const StepIO &io, const int H,
                                              unsigned char *smem_raw, unsigned long long *bars) {
  constexpr int D = PF + 3;
  constexpr int SW = 2 * NT;  // strip columns
  constexpr int W = SW - 8;   // interior columns
  static_assert(W % 4 == 0, "strip starts must stay 16-byte aligned for the TMA copies");
  constexpr int RS = pair_ring_stride<NT>();
  constexpr int NRING = 5 * 4 + 3 * 7;  // ring rows
  const unsigned raw_s = (unsigned)__cvta_generic_to_shared(smem_raw);
  float *stg = reinterpret_cast<float *>(smem_raw + ((128u - (raw_s & 127u)) & 127u));  // [D][10][SW]
  float *rings = stg + D * 10 * SW;
  // ring pointers address column 0 of slot 0; columns -2, -1, SW, SW + 1 are the pads
  float *rpsi = rings + 2;  // [4][RS], row mod 4
  float *rrho = rpsi + 4 * RS;
  float *rT = rrho + 4 * RS;
  float *rux = rT + 4 * RS;
  float *ruy = rux + 4 * RS;
  float *rfs = ruy + 4 * RS;  // [3][7][RS], row mod 3: f*_1, f*_3, f*_5, f*_6, f*_7, f*_8, T*
  const float third = 1.0f / 3.0f, twelfth = 1.0f / 12.0f;
  const float big = 3.0e38f;

  const int t = threadIdx.x;
  const int c2 = 2 * t;  // strip column of lane 0
  const int x0 = blockIdx.x * W;
  const int ya = blockIdx.y * H;
  const int yb = min(ya + H, P.ny);
  const int gx0 = x0 - 4 + c2;  // even
  int src0 = gx0 % P.nx;
  if (src0 < 0) src0 += P.nx;
  const int col0 = src0, col1 = src0 + 1;  // in-domain columns of the two lanes
  // a lane on a thermally non-periodic x line (e.g. a Dirichlet ring around a periodic box)
  const bool col_fix = (P.tbc[0] != T_PERIODIC || P.tbc[1] != T_PERIODIC) && (col0 == 0 || col1 == P.nx - 1);
  const long long plane = P.plane;
  const float rho_bar = (float)io.stats_in[0];
  const bool any_outflow = P.hbc[2] == OUTFLOW || P.hbc[3] == OUTFLOW;
  const bool t_s4 = t >= 2 && t < NT - 2 && gx0 < P.nx;  // both lanes interior and in the domain
  const float *fin = reinterpret_cast<const float *>(io.f_in) + src0;
  const float *Tin = reinterpret_cast<const float *>(io.T_in) + src0;
  float *fout = reinterpret_cast<float *>(io.f_out);
  float *Tout = reinterpret_cast<float *>(io.T_out);
  const int n_it = yb - ya + 6;
  unsigned flags = 0;
  F2 acc_s(0.0f), acc_n(0.0f);  // compensated per-lane mass sums (acc_n: minus the compensation)
  // status checks folded into running values, tested once at the end: the least psi argument
  // and density, and a sum of the new temperatures (NaN or Inf in rho or T reaches the sums)
  float arg_min = big, rho_min = big;
  F2 t_sum(0.0f);

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
  // TMA staging for strips wholly inside the domain, where the tensor maps exist
  const bool use_tma = io.tmap_f != nullptr && x0 - 4 >= 0 && x0 - 4 + SW <= P.nx;
  const unsigned stg_s = (unsigned)__cvta_generic_to_shared(stg);
  const unsigned bar_s = (unsigned)__cvta_generic_to_shared(bars);
  if (use_tma && t == 0) {
    for (int j = 0; j < D; ++j) mbar_init(bar_s + 8 * j, 1);
    mbar_fence_init();
    tmap_acquire(io.tmap_f);
    tmap_acquire(io.tmap_T);
  }
  __syncthreads();
  auto stage_row = [&](int q, int slot) {
    const int src = row_map(q).src;
    if (use_tma) {
      if (t == 0) tma_row<NT>(stg_s + slot * 10 * SW * 4, bar_s + 8 * slot, io.tmap_f, io.tmap_T, x0 - 4, src);
      return;
    }
    const long long k = (long long)src * P.nx;
    float *dst = stg + slot * 10 * SW + c2;
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async8(dst + i * SW, fin + i * plane + k);
    cp_async8(dst + 9 * SW, Tin + k);
  };
  for (int i = t; i < NRING * 4; i += NT) rings[(i >> 2) * RS + ((i & 3) < 2 ? (i & 3) : SW + (i & 3))] = 0.0f;

#pragma unroll
  for (int j = 0; j < PF; ++j) {
    if (j < n_it) stage_row(ya - 3 + j, j);
    cp_async_commit();
  }
  // TMA runs TL = D - 2 rows ahead: row q + TL goes into the slot of row q - 2 as soon as the
  // collision stage has read it, one stage earlier than a copy issued at the next iteration
  constexpr int TL = D - 2;
  if (use_tma)
    for (int j = PF; j < TL; ++j)
      if (j < n_it) stage_row(ya - 3 + j, j);

  F2 c1jx(0.0f), c1jy(0.0f), n1jx(0.0f), n1jy(0.0f);
  F2 f0n(0.0f), f2n(0.0f), f4n(0.0f), f0c(0.0f), f2c1(0.0f), f2c2(0.0f);
  S3Carry<F2> cc2{}, nn2{};
  S4Carry<F2> cur{}, nxt{};
  int f3 = 0;
  for (int iq = 0; iq < n_it; ++iq) {
    const int q = ya - 3 + iq;
    if (!use_tma && iq + PF < n_it) stage_row(q + PF, (iq + PF) % D);
    bool stalled = false;
    if (use_tma) {
      stalled = !mbar_wait(bar_s + 8 * (iq % D), (iq / D) & 1);  // row q has landed
    } else {
      cp_async_commit();
      cp_async_wait<PF>();  // this thread's copies of row q have landed
    }
    const int s4_0 = iq & 3, s4_1 = (iq + 3) & 3, s4_2 = (iq + 2) & 3, s4_3 = (iq + 1) & 3;
    const int f_r3 = f3, f_r2 = f3 == 2 ? 0 : f3 + 1, f_r4 = f3 == 0 ? 2 : f3 - 1;

    // ---- S1: row q ----
    {
      const LineMap rm = row_map(q);
      const float *st = stg + (iq % D) * 10 * SW + c2;
      F2 f[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = ld2(st + i * SW);
      const F2 Tt = ld2(st + 9 * SW);
      const F2 delta = ((f[0] + (f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
      const F2 rho = P.rho_ref + delta;
      F2 psi(0.0f);
      if (!rm.solid) {
        const F2 arg = psi_arg(P, rho, P.T_ref + Tt);
        arg_min = fminf(arg_min, fminf(arg.lo(), arg.hi()));
        psi = sqrt(fmax(arg, F2(0.0f)));
      }
      const int i0 = s4_0 * RS + c2;
      st2(rpsi + i0, psi);
      st2(rrho + i0, rho);
      st2(rT + i0, Tt);
      const F2 d57 = f[5] - f[7], d68 = f[6] - f[8];
      n1jx = (f[1] - f[3]) + (d57 - d68);
      n1jy = (f[2] - f[4]) + (d57 + d68);
    }
    if (use_tma) {
      // a row that did not land stops the CTA (uniformly): the copies already issued are
      // waited for (bounded) before it leaves, and the status word reports the step invalid
      if (__syncthreads_or(stalled)) {
        flags |= FLAG_STALL;
        if (t == 0)
          for (int n = iq; n <= min(iq + TL - 1, n_it - 1); ++n) mbar_wait(bar_s + 8 * (n % D), (n / D) & 1);
        break;
      }
    } else {
      __syncthreads();
    }

    // ---- S2: row q-1 ----
    if (iq >= 2) {
      const int r = q - 1;
      const LineMap rm = row_map(r);
      const int i0 = s4_1 * RS, iu = s4_0 * RS, id = s4_2 * RS;
      if (!rm.solid) {
        const Trip pu = trip(rpsi + iu, t), pm = trip(rpsi + i0, t), pd = trip(rpsi + id, t);
        const F2 p1 = pm.r, p3 = pm.l, p2 = pu.c, p4 = pd.c, p5 = pu.r, p6 = pu.l, p7 = pd.l, p8 = pd.r;
        const F2 psi_c = pm.c;
        const F2 d57 = p5 - p7, d86 = p8 - p6, s57 = p5 + p7, s68 = p6 + p8, s13 = p1 + p3, s24 = p2 + p4;
        F2 sx = third * (p1 - p3) + twelfth * (d57 + d86);
        F2 sy = third * (p2 - p4) + twelfth * (d57 - d86);
        // Q as Qxx + Qyy, Qxx - Qyy and Qxy
        F2 qs = third * (s13 + s24) + (1.0f / 6.0f) * (s57 + s68) - 2.0f * psi_c;
        F2 qd = third * (s13 - s24);
        const F2 qxy = twelfth * (s57 - s68);
        if (!SIMPLE && rm.wall >= 0) {
          // solid links of a y wall: see the one-column kernel (Eqs. shanchen-walls,
          // psi-based-formula, Q-psi-based, mod-psi-based-formula, Q-mod-psi-based)
          const int ws = rm.wall;
          F2 pf, pq;
          if (P.mod_psi) {
            pf = P.Gw_over_G * psi_c;
            pq = psi_c;
          } else {
            const F2 Tw = P.T_ref + ld2(rT + i0 + c2);
            const float a0 = psi_arg(P, wall_rho_w(P, ws, col0, rm.src), Tw.lo());
            const float a1 = psi_arg(P, wall_rho_w(P, ws, col1, rm.src), Tw.hi());
            if (!(a0 >= 0.0f) || !(a1 >= 0.0f)) flags |= FLAG_PSI_NEG;
            pf = pq = F2(sqrtf(fmaxf(a0, 0.0f)), sqrtf(fmaxf(a1, 0.0f)));
          }
          const F2 hw = 0.5f * pf;
          if (ws == 2) sy = sy - hw;
          else sy = sy + hw;
          qs = qs + (2.0f / 3.0f) * pq;
          qd = qd - third * pq;
        }
        const F2 qf = P.kappa_G2 * psi_c;
        nn2.qs = qf * qs;
        nn2.qd = qf * qd;
        nn2.qxy = qf * qxy;
        const F2 rho = ld2(rrho + i0 + c2);
        const F2 gps = (-P.G) * psi_c;
        const F2 fmx = gps * sx, fmy = gps * sy;
        const F2 Fx = fmx + P.gx * (rho - rho_bar), Fy = fmy + P.gy * (rho - rho_bar);
        const F2 inv_rho = 1.0f / rho;
        const F2 ux = (c1jx + 0.5f * Fx) * inv_rho;
        const F2 uy = (c1jy + 0.5f * Fy) * inv_rho;
        st2(rux + i0 + c2, ux);
        st2(ruy + i0 + c2, uy);
        nn2.fmx = fmx;
        nn2.fmy = fmy;
        nn2.fm2 = (P.G * P.G) * (sx * sx + sy * sy);
        nn2.inv_rho = inv_rho;
        if (!SIMPLE && ENERGY && r == 1 && P.hbc[2] == WALL) {  // mirror ghost of row -1
          st2(rux + s4_3 * RS + c2, ux);
          st2(ruy + s4_3 * RS + c2, -uy);
        }
      } else if (!SIMPLE && ENERGY && r == P.ny && P.hbc[3] == WALL) {  // mirror ghost of row ny
        st2(rux + i0 + c2, ld2(rux + s4_3 * RS + c2));
        st2(ruy + i0 + c2, -ld2(ruy + s4_3 * RS + c2));
      }
      __syncthreads();
    }

    // ---- S3: row q-2 ----
    if (iq >= 4) {
      const int r = q - 2;
      const LineMap rm = row_map(r);
      const int i0 = s4_2 * RS, iu = s4_1 * RS, id = s4_3 * RS;
      float *fs = rfs + f_r2 * 7 * RS + c2;  // this row's f* and T* slot
      if (!rm.solid) {
        const float *st = stg + ((iq + D - 2) % D) * 10 * SW + c2;
        F2 fd[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fd[i] = ld2(st + i * SW);
        const F2 rho = ld2(rrho + i0 + c2);
        const F2 ux = ld2(rux + i0 + c2), uy = ld2(ruy + i0 + c2);
        const F2 Fx = cc2.fmx + P.gx * (rho - rho_bar), Fy = cc2.fmy + P.gy * (rho - rho_bar);
        F2 e(P.e_const);  // s_eta / 4
        if (P.var_eta) e = 1.0f / (P.e_c0 + P.e_c1 * rho);
        collide(P, fd, rho, ux, uy, Fx, Fy, cc2.fm2, cc2.qs, cc2.qd, cc2.qxy, e);
        st2(fs + 0 * RS, fd[1]);
        st2(fs + 1 * RS, fd[3]);
        st2(fs + 2 * RS, fd[5]);
        st2(fs + 3 * RS, fd[6]);
        st2(fs + 4 * RS, fd[7]);
        st2(fs + 5 * RS, fd[8]);
        f0n = fd[0];
        f2n = fd[2];
        f4n = fd[4];
        nxt.Fx = Fx;
        nxt.Fy = Fy;
        if (ENERGY) {
          const F2 T0 = ld2(rT + i0 + c2);
          nxt.ux = ux;
          nxt.uy = uy;
          pr_parts(P, rho, &nxt.A, &nxt.B);
          nxt.inv_rcv = cc2.inv_rho * P.cv_inv;
          nxt.lam = P.lam_v + P.dlam * (rho - P.rho_v);
          const Trip ru = trip(rrho + iu, t), rmd = trip(rrho + i0, t), rd = trip(rrho + id, t);
          nxt.gdx = P.dlam * (third * (rmd.r - rmd.l) + twelfth * (ru.r - ru.l - rd.l + rd.r));
          nxt.gdy = P.dlam * (third * (ru.c - rd.c) + twelfth * (ru.r + ru.l - rd.l - rd.r));
          const Trip xu = trip(rux + iu, t), xm = trip(rux + i0, t), xd = trip(rux + id, t);
          const Trip yu = trip(ruy + iu, t), yd = trip(ruy + id, t);
          nxt.div = third * (xm.r - xm.l) + twelfth * (xu.r - xu.l - xd.l + xd.r) + third * (yu.c - yd.c) +
                    twelfth * (yu.r + yu.l - yd.l - yd.r);
          F2 Ts;
          if (!SIMPLE && rm.outflow) {
            Ts = ld2(rfs + f_r3 * 7 * RS + 6 * RS + c2);  // outflow row: copy of the first interior row
            nxt.k1 = F2(0.0f);
          } else {
            const Trip tu = trip(rT + iu, t), tm = trip(rT + i0, t), td = trip(rT + id, t);
            const F2 gtx = third * (tm.r - tm.l) + twelfth * (tu.r - tu.l - td.l + td.r);
            const F2 gty = third * (tu.c - td.c) + twelfth * (tu.r + tu.l - td.l - td.r);
            const F2 lap = (2.0f / 3.0f) * (tm.r + tu.c + tm.l + td.c - 4.0f * T0) +
                           (1.0f / 6.0f) * (tu.r + tu.l + td.l + td.r - 4.0f * T0);
            // (lambda lap T + grad lambda . grad T - T (dp/dT) div u) / (rho c_v) - u . grad T
            const F2 adv = ux * gtx + uy * gty;
            const F2 cond = nxt.lam * lap + nxt.gdx * gtx + nxt.gdy * gty;
            const F2 comp = T_dpdT(P, nxt.A, nxt.B, P.T_ref + T0) * nxt.div;
            const F2 k1 = ev((cond - comp) * nxt.inv_rcv) - adv;
            nxt.k1 = k1;
            Ts = T0 + k1;
            if ((!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1)) || col_fix) {  // Dirichlet nodes of a boundary line
              float tw0, tw1;
              const bool d0 = t_fixed(P, col0, rm.src, &tw0), d1 = t_fixed(P, col1, rm.src, &tw1);
              if (d0 || d1) {
                Ts = F2(d0 ? tw0 - P.T_ref : Ts.lo(), d1 ? tw1 - P.T_ref : Ts.hi());
                nxt.k1 = F2(d0 ? 0.0f : k1.lo(), d1 ? 0.0f : k1.hi());
              }
            }
          }
          st2(fs + 6 * RS, Ts);
          if (!SIMPLE && r == 1 && P.hbc[2] == WALL) st2(rfs + f_r4 * 7 * RS + 6 * RS + c2, Ts);  // mirror ghost of row -1
        }
      } else if (!SIMPLE && ENERGY && r == P.ny && P.hbc[3] == WALL) {
        st2(fs + 6 * RS, ld2(rfs + f_r4 * 7 * RS + 6 * RS + c2));  // mirror ghost of row ny
      }
      __syncthreads();
    }
    // the slot of row q - 2 is free (its last reader, the collision stage, is past a barrier;
    // before iteration 4 its row was read by the first stage only)
    if (use_tma && iq + TL < n_it) stage_row(q + TL, (iq + TL) % D);

    // ---- S4: row q-3 ----
    if (iq >= 6 && t_s4) {
      const int r = q - 3;
      const LineMap rm = row_map(r);
      if (!rm.outflow) {
        // pull f_i(x) = f*_i(x - c_i) from the ring rows r-1 (lo), r (mid), r+1 (hi)
        const float *lo = rfs + f_r4 * 7 * RS, *mid = rfs + f_r3 * 7 * RS, *hi = rfs + f_r2 * 7 * RS;
        F2 fd[9];
        fd[0] = f0c;
        fd[1] = trip(mid + 0 * RS, t).l;
        fd[2] = f2c2;
        fd[3] = trip(mid + 1 * RS, t).r;
        fd[4] = f4n;
        fd[5] = trip(lo + 2 * RS, t).l;
        fd[6] = trip(lo + 3 * RS, t).r;
        fd[7] = trip(hi + 4 * RS, t).r;
        fd[8] = trip(hi + 5 * RS, t).l;
        if (!SIMPLE && rm.wall >= 0) zou_he<F2>(rm.wall, fd, ev(-0.5f * cur.Fx), ev(-0.5f * cur.Fy));
        const F2 delta = ((fd[0] + (fd[1] + fd[2]) + (fd[3] + fd[4])) + ((fd[5] + fd[6]) + (fd[7] + fd[8])));
        const F2 rho_new = P.rho_ref + delta;
        const F2 T_old = ld2(rT + s4_3 * RS + c2);
        F2 T_new = T_old;
        if (ENERGY) {
          const Trip tm = trip(mid + 6 * RS, t), tu = trip(hi + 6 * RS, t), td = trip(lo + 6 * RS, t);
          const F2 gtx = third * (tm.r - tm.l) + twelfth * (tu.r - tu.l - td.l + td.r);
          const F2 gty = third * (tu.c - td.c) + twelfth * (tu.r + tu.l - td.l - td.r);
          const F2 lap = (2.0f / 3.0f) * (tm.r + tu.c + tm.l + td.c - 4.0f * tm.c) +
                         (1.0f / 6.0f) * (tu.r + tu.l + td.l + td.r - 4.0f * tm.c);
          const F2 adv = cur.ux * gtx + cur.uy * gty;
          const F2 cond = cur.lam * lap + cur.gdx * gtx + cur.gdy * gty;
          const F2 comp = T_dpdT(P, cur.A, cur.B, P.T_ref + tm.c) * cur.div;
          const F2 k2 = ev((cond - comp) * cur.inv_rcv) - adv;
          T_new = T_new + 0.5f * (cur.k1 + k2);
          if ((!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1)) || col_fix) {  // Dirichlet nodes keep their value
            float tw;
            const bool d0 = t_fixed(P, col0, rm.src, &tw), d1 = t_fixed(P, col1, rm.src, &tw);
            T_new = F2(d0 ? T_old.lo() : T_new.lo(), d1 ? T_old.hi() : T_new.hi());
          }
        }
        const long long k = (long long)r * P.nx + gx0;
#pragma unroll
        for (int i = 0; i < 9; ++i) st2(fout + i * plane + k, fd[i]);
        st2(Tout + k, T_new);
        rho_min = fminf(rho_min, fminf(rho_new.lo(), rho_new.hi()));
        t_sum = t_sum + T_new;
        const float wr = (!SIMPLE && any_outflow) ? (float)line_weight(r, P.ny, P.hbc[2], P.hbc[3]) : 1.0f;
        const F2 yk = wr * rho_new + acc_n;
        const F2 tk = acc_s + yk;
        acc_n = yk - (tk - acc_s);
        acc_s = tk;
      }
    }
    c1jx = n1jx;
    c1jy = n1jy;
    cc2 = nn2;
    cur = nxt;
    f0c = f0n;
    f2c2 = f2c1;
    f2c1 = f2n;
    f3 = f3 == 2 ? 0 : f3 + 1;
  }
  cp_async_wait<0>();
  double acc = ((double)acc_s.lo() + (double)acc_n.lo()) + ((double)acc_s.hi() + (double)acc_n.hi());
  if (!(arg_min >= 0.0f)) flags |= FLAG_PSI_NEG;
  if (!(rho_min > 0.0f)) flags |= FLAG_RHO_NONPOS;
  if (!isfinite(acc) || !isfinite((double)t_sum.lo() + (double)t_sum.hi())) flags |= FLAG_NAN;
  if (flags) atomicOr(io.status, flags);
  block_mass_finalize<NT, false>(P, io, acc, 0.0);
}

template <bool ENERGY, int NT, int PF>
__global__ void __launch_bounds__(NT, 320 / NT) row_step_pair(const Params<float> P, const StepIO io, const int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long bars[PF + 3];  // mbarriers of the TMA staging slots
  const int ya = blockIdx.y * H;
  const int yb = min(ya + H, P.ny);
  if (ya - 3 >= 1 && yb + 2 <= P.ny - 2)
    row_body_pair<ENERGY, NT, PF, true>(P, io, H, smem_raw, bars);
  else
    row_body_pair<ENERGY, NT, PF, false>(P, io, H, smem_raw, bars);
}

}  // namespace ppl_dev
