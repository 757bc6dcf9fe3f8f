// FP32 fused step with two columns per thread (packed f32x2 arithmetic) for domains that
// are hydrodynamically periodic in x, with an even nx (the x lines may hold Dirichlet
// temperatures).
//
// The row-marching pipeline of row_step.cuh with each thread owning the adjacent columns
// (2t, 2t + 1) of a strip of 2 NT columns: 4 halo columns on each side, 2 NT - 8 interior
// columns. Both columns of a thread are computed by one packed instruction wherever the
// arithmetic allows (F2 in lane2.cuh), the staged rows and the stores move 8 bytes per
// thread. Ring rows keep the even columns in one half and the odd columns in the other, so
// that each of a column pair's neighbour pairs (2t - 1, 2t), (2t, 2t + 1), (2t + 1, 2t + 2)
// is two conflict-free 4-byte reads straight into a register pair (each half carries a
// zeroed pad float at both ends, so the reads of the strip's outermost threads need no
// clamping: those columns are halo, never stored). With
// x periodic and nx even, a pair never straddles the domain edge and its global address is
// 8-byte aligned. Rows (walls, outflow, Dirichlet lines in y) are handled as in the
// one-column kernel; only per-node boundary data of a wall row (rho_w, T_w, the Dirichlet
// mask) is looked up column by column.
//
// Stages and row lags of one iteration (row q staged):
//   S1 (row q):   rho, j = sum f c, psi                                   Eqs. (psi), (peng-robinson)
//   S2 (row q-1): F^m (+ psi-based wall form), F^b, Q, u, and the MRT     Eqs. (shanchen), (shanchen-walls),
//                 collision with the Li source terms                      (psi-based-formula), (Q), (Q-psi-based),
//                                                                         (gravitational_force), (collisionMRT),
//                                                                         (li_source_terms), (S), (C)
//   S3 (row q-2): pull streaming, Zou-He, store of f and the mass        Eq. (lbm), Sec. 2.2;
//                 partial; first Heun stage of the energy equation        Eq. (energy-equation)
//   S4 (row q-3): second Heun stage, store of T
// Every per-row quantity lives in a ring of three rows (row mod 3): psi and rho (rows q .. q-2),
// T (rows q .. q-2), u (rows q-1 .. q-3), the sideways post-collision populations (rows q-1 ..
// q-3), the first Heun stage T* (rows q-2 .. q-4) and the staged rows (q-1 .. q+1). The
// stencils of the first Heun stage reach rho and T one row further down (q-3); that row's
// share of each stencil is formed one iteration earlier, when the row is the stencil's
// centre, and kept in registers (each thread's own columns). With every ring of period three, the
// slots are addressed through three per-thread pointers that rotate once per iteration,
// so every ring access is a fixed offset from one of them.
//
// Row staging: a strip that lies wholly inside the domain has each row brought in by TMA
// (one thread issues a 3-D tensor copy of the nine population rows and a 2-D copy of the
// temperature row, completing on the slot's mbarrier, which all threads wait on) two rows
// ahead; strips that wrap across the periodic x seam, and domains without tensor maps, use
// per-thread 8-byte cp.async copies, also two rows ahead (one copy group per row; a thread
// reads only the columns it copied), with the wrap applied per column.
#pragma once

#include "lane2.cuh"
#include "row_step.cuh"

namespace ppl_dev {

// the pairs of columns (2t - 1, 2t), (2t, 2t + 1), (2t + 1, 2t + 2) around a thread's own pair
struct Trip {
  F2 l, c, r;
};
__device__ __forceinline__ F2 ld2(const float *p) { return F2(*reinterpret_cast<const float2 *>(p)); }
// a ring row holds [pad, E_0 .. E_{NT-1}, pad, pad, O_0 .. O_{NT-1}, pad] with E_t, O_t the
// columns 2t, 2t + 1; a thread's pointer addresses its E_t, and O_t lies NT + 2 floats further
template <int NT>
__device__ __forceinline__ F2 rld(const float *p) { return F2(p[0], p[NT + 2]); }
template <int NT>
__device__ __forceinline__ void rst(float *p, F2 v) { p[0] = v.lo(); p[NT + 2] = v.hi(); }
template <int NT>
__device__ __forceinline__ Trip rtrip(const float *p) {
  const float e = p[0], o = p[NT + 2];
  return {F2(p[NT + 1], e), F2(e, o), F2(o, p[1])};
}

__device__ __forceinline__ void st2(float *p, F2 v) { *reinterpret_cast<float2 *>(p) = v.v; }
__device__ __forceinline__ void cp_async8(float *smem_dst, const float *gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

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
constexpr int kPairSlots = 3;      // staged rows and ring rows per quantity
constexpr int kPairRingRows = 8;  // ring rows per slot: psi, rho, T, ux, uy, f*_5, f*_6, T*
// Post-collision populations that stream sideways or down are read sooner than the slot period:
// f*_7, f*_8 of row q - 1 by the streaming of row q - 2 in the same iteration (one buffer), and
// f*_1, f*_3 in the next iteration (two buffers, alternating)
constexpr int kPairBufRows = 6;
template <int NT>
constexpr size_t row_step_pair_smem_bytes() {  // + 128: the staging base is aligned up to 128 bytes
  return (size_t)(kPairSlots * 10 * (2 * NT) + (kPairSlots * kPairRingRows + kPairBufRows) * pair_ring_stride<NT>()) *
             sizeof(float) +
         128;
}

// Specialisation a tile takes: 1 (no boundary logic) if its rows and their 3-row halo lie inside
// the domain and its strip holds no column of a thermally non-periodic x line (Dirichlet
// temperatures on x = 0 or x = nx - 1); 2 if the rows are inside but the strip holds such a
// column (only the per-column Dirichlet checks remain); 0 otherwise.
template <int NT>
__device__ __forceinline__ int pair_tile_kind(const Params<float> &P, int ya, int yb, int bx) {
  const int g0 = bx * (2 * NT - 8) - 4, g1 = g0 + 2 * NT - 1;  // first and last strip column
  const bool xfix = (P.tbc[0] != T_PERIODIC || P.tbc[1] != T_PERIODIC) && (g0 <= 0 || g1 >= P.nx - 1);
  if (ya - 3 < 1 || yb + 2 > P.ny - 2) return 0;
  return xfix ? 2 : 1;
}

// The right-hand side of the energy equation (Eq. energy-equation) at a node, with the
// pressure split p = T A(rho) - alpha(T) B(rho) (alpha = (1 + k (1 - sqrt(T / Tc)))^2):
//   L(T) = (lambda lap T + grad lambda . grad T - T (dp/dT)_rho div u) / (rho c_v) - u . grad T
// and T (dp/dT)_rho = T (A - k^2 B / Tc) + k (1 + k) B sqrt(T / Tc). Both Heun stages of a row
// evaluate L with the same rho and u, so the first stage folds them into five coefficients
//   L(T) = lr lap T + vx dT/dx + vy dT/dy + T nA + sqrt(T) nB
// (lr = lambda / (rho c_v), v = grad lambda / (rho c_v) - u, nA and nB the compression term
// times -div u / (rho c_v)), which it hands to the second stage with h = T^n + L(T^n) / 2.
struct PairHeun {
  F2 h, lr, vx, vy, nA, nB;
};

// One tile of the step: strip bx (2 NT - 8 interior columns) and rows [ya, yb), CTA bid of
// nblk for the mass reduction; `done` as in tile_mass_finalize.
// reduce = false skips the mass reduction (a step whose domain mean nobody reads).
template <bool ENERGY, int NT, bool SIMPLE, bool XFIX = false>
__device__ __forceinline__ void row_body_pair(const Params<float> &P, const StepIO &io, const int ya, const int yb, int bx,
                                              unsigned bid, unsigned nblk, unsigned char *smem_raw,
                                              unsigned long long *bars, unsigned *done = nullptr,
                                              unsigned done_value = 0, bool reduce = true) {
  constexpr int SW = 2 * NT;  // strip columns
  constexpr int W = SW - 8;   // interior columns
  static_assert(W % 4 == 0, "strip starts must stay 16-byte aligned for the TMA copies");
  constexpr int RS = pair_ring_stride<NT>();
  constexpr int NRING = kPairSlots * kPairRingRows + kPairBufRows;
  const unsigned raw_s = (unsigned)__cvta_generic_to_shared(smem_raw);
  float *stg = reinterpret_cast<float *>(smem_raw + ((128u - (raw_s & 127u)) & 127u));  // [3][10][SW]
  float *rings = stg + kPairSlots * 10 * SW;
  // ring row of quantity k in slot s at rings + (s * kPairRingRows + k) * RS, laid out as
  // [pad, even columns, pad, pad, odd columns, pad]; after the three slots the two f*_1, f*_3
  // buffers (two rows each) and the f*_7, f*_8 buffer. The slots are addressed by role through
  // three rotating per-thread pointers (below), so every ring access is a fixed offset from one
  // of them
  enum { R_PSI = 0, R_RHO = 1, R_T = 2, R_UX = 3, R_UY = 4, R_F5 = 5, R_F6 = 6, R_TS = 7 };
  const float third = 1.0f / 3.0f, twelfth = 1.0f / 12.0f;
  const float big = 3.0e38f;
  // T (dp/dT)_rho = T (A + kA B) + sqrt(T) (kB B)
  const float kA = -P.k * P.k / P.Tc, kB = P.k * (1.0f + P.k) * P.sqrt_Tc_inv;

  const int t = threadIdx.x;
  const int c2 = 2 * t;  // strip column of lane 0
  const int x0 = bx * W;
  const int gx0 = x0 - 4 + c2;  // even
  int src0 = gx0 % P.nx;
  if (src0 < 0) src0 += P.nx;
  const int col0 = src0, col1 = src0 + 1;  // in-domain columns of the two lanes
  // a lane on a thermally non-periodic x line (e.g. a Dirichlet ring around a periodic box)
  // (never in the SIMPLE specialisation, which such strips do not take)
  const bool col_fix = (!SIMPLE || XFIX) && (P.tbc[0] != T_PERIODIC || P.tbc[1] != T_PERIODIC) &&
                       (col0 == 0 || col1 == P.nx - 1);
  const long long plane = P.plane;
  const float rho_bar = (float)io.stats_in[0];
  const bool any_outflow = P.hbc[2] == OUTFLOW || P.hbc[3] == OUTFLOW;
  const bool t_in = t >= 2 && t < NT - 2 && gx0 < P.nx;  // both lanes interior and in the domain
  const float *fin = reinterpret_cast<const float *>(io.f_in) + src0;
  const float *Tin = reinterpret_cast<const float *>(io.T_in) + src0;
  float *fout = reinterpret_cast<float *>(io.f_out) + gx0;
  float *Tout = reinterpret_cast<float *>(io.T_out) + gx0;
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
    for (int j = 0; j < kPairSlots; ++j) mbar_init(bar_s + 8 * j, 1);
    mbar_fence_init();
    tmap_acquire(io.tmap_f);
    tmap_acquire(io.tmap_T);
  }
  for (int i = t; i < NRING * 4; i += NT) {
    const int k = i & 3;
    rings[(i >> 2) * RS + (k == 0 ? 0 : k == 1 ? NT + 1 : k == 2 ? NT + 2 : 2 * NT + 3)] = 0.0f;
  }
  __syncthreads();
  // row q into staging slot `slot` (TMA, one thread), or into this thread's columns at dst
  auto stage_row = [&](int q, int slot, const float *dst_c) {
    const int src = row_map(q).src;
    if (use_tma) {
      if (t == 0) tma_row<NT>(stg_s + slot * 10 * SW * 4, bar_s + 8 * slot, io.tmap_f, io.tmap_T, x0 - 4, src);
      return;
    }
    const long long k = (long long)src * P.nx;
    float *dst = const_cast<float *>(dst_c);
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async8(dst + i * SW, fin + i * plane + k);
    cp_async8(dst + 9 * SW, Tin + k);
  };
  // rows ya - 3 and ya - 2 go out before the loop; each iteration then stages the row two
  // ahead of its first stage, once the collision has read the slot it goes into (one
  // cp.async group per row)
  stage_row(ya - 3, 0, stg + c2);
  cp_async_commit();
  if (n_it > 1) stage_row(ya - 2, 1, stg + 10 * SW + c2);
  cp_async_commit();

  // Slot roles: 0 holds rows q and q - 3, 1 rows q - 1 and q - 4, 2 rows q - 2 and q + 1.
  // Each iteration rotates the roles (0, 1, 2) <- (2, 0, 1).
  float *r0 = rings + 0 * kPairRingRows * RS + 1 + t, *r1 = rings + 2 * kPairRingRows * RS + 1 + t,
        *r2 = rings + 1 * kPairRingRows * RS + 1 + t;
  // f*_1, f*_3 buffers: written for row q - 1 (f13w), read for row q - 2 (f13r); f*_7, f*_8: f78
  float *f13w = rings + kPairSlots * kPairRingRows * RS + 1 + t, *f13r = f13w + 2 * RS, *const f78 = f13w + 4 * RS;
  const float *g0 = stg + 0 * 10 * SW + c2, *g1 = stg + 2 * 10 * SW + c2, *g2 = stg + 1 * 10 * SW + c2;
  int k0 = 0, k1 = 2, k2 = 1;  // slot numbers of the roles (TMA destination, mbarrier)
  unsigned ph = 0;              // mbarrier parity per slot (bit k)
  // values carried between stages and iterations, by row
  F2 f0n(0.0f), f0c(0.0f);                             // S2 (row q - 1) -> S3 (row q - 2, next)
  F2 f2n(0.0f), f2c(0.0f), f2cc(0.0f);                 // f_2 of rows q - 1, q - 2, q - 3
  F2 Fxn(0.0f), Fyn(0.0f), Fxc(0.0f), Fyc(0.0f), irn(0.0f), irc(0.0f);  // F and 1/rho, S2 -> S3
  F2 f4(0.0f);  // post-collision f_4 of row q - 1, streamed down into row q - 2 in the same iteration
  PairHeun nxt{}, cur{};  // S3 (row q - 2) -> S4 (row q - 3, next iteration)
  // shares of the stencils of the first Heun stage that the row below the centre contributes
  // (grad rho x, y; grad T x, y; Laplacian of T), formed when that row was the centre (S3 reads
  // them before it forms the next row's, so they need no second set of registers)
  F2 sh0(0.0f), sh1(0.0f), sh2(0.0f), sh3(0.0f), sh4(0.0f);

  for (int iq = 0; iq < n_it; ++iq) {
    const int q = ya - 3 + iq;
    if (!use_tma) cp_async_wait<1>();  // this thread's copies of row q have landed (row q + 1 may not)
    bool stalled = false;
    if (use_tma) stalled = !mbar_wait(bar_s + 8 * k0, (ph >> k0) & 1u);  // row q has landed

    // ---- S1: row q ----
    {
      const LineMap rm = row_map(q);
      const float *st = g0;
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
      rst<NT>(r0 + (R_PSI) * RS, psi);
      rst<NT>(r0 + (R_RHO) * RS, rho);
      rst<NT>(r0 + (R_T) * RS, Tt);
    }
    if (use_tma) {
      // a row that did not land stops the CTA (uniformly): the copies already issued are
      // waited for (bounded) before it leaves, and the status word reports the step invalid
      if (__syncthreads_or(stalled)) {
        flags |= FLAG_STALL;
        if (t == 0) {
          mbar_wait(bar_s + 8 * k0, (ph >> k0) & 1u);
          if (iq + 1 < n_it) mbar_wait(bar_s + 8 * k2, (ph >> k2) & 1u);
        }
        break;
      }
    } else {
      __syncthreads();
    }

    // ---- S2: row q-1 (forces, velocity, collision) ----
    if (iq >= 2) {
      const int r = q - 1;
      const LineMap rm = row_map(r);
      if (!rm.solid) {
        const Trip pu = rtrip<NT>(r0 + (R_PSI) * RS), pm = rtrip<NT>(r1 + (R_PSI) * RS), pd = rtrip<NT>(r2 + (R_PSI) * RS);
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
            const F2 Tw = P.T_ref + rld<NT>(r1 + (R_T) * RS);
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
        const F2 rho = rld<NT>(r1 + (R_RHO) * RS);
        const F2 gps = (-P.G) * psi_c;
        const F2 fmx = gps * sx, fmy = gps * sy;
        const F2 Fx = fmx + P.gx * (rho - rho_bar), Fy = fmy + P.gy * (rho - rho_bar);
        const F2 inv_rho = 1.0f / rho;
        // the staged row q - 1 (collided below), and its momentum j = sum f c
        const float *st = g1;
        F2 fd[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fd[i] = ld2(st + i * SW);
        const F2 g57 = fd[5] - fd[7], g68 = fd[6] - fd[8];
        const F2 ux = ((fd[1] - fd[3]) + (g57 - g68) + 0.5f * Fx) * inv_rho;
        const F2 uy = ((fd[2] - fd[4]) + (g57 + g68) + 0.5f * Fy) * inv_rho;
        rst<NT>(r1 + (R_UX) * RS, ux);
        rst<NT>(r1 + (R_UY) * RS, uy);
        if (!SIMPLE && ENERGY && r == 1 && P.hbc[2] == WALL) {  // mirror ghost of row -1 (slot of row q - 3)
          rst<NT>(r0 + (R_UX) * RS, ux);
          rst<NT>(r0 + (R_UY) * RS, -uy);
        }
        // collision of the staged row q - 1
        F2 e(P.e_const);  // s_eta / 4
        if (P.var_eta) e = 1.0f / (P.e_c0 + P.e_c1 * rho);
        const F2 fm2 = (P.G * P.G) * (sx * sx + sy * sy);
        collide(P, fd, rho, ux, uy, Fx, Fy, fm2, ev(qf * qs), ev(qf * qd), ev(qf * qxy), e);
        rst<NT>(f13w, fd[1]);
        rst<NT>(f13w + RS, fd[3]);
        rst<NT>(r1 + (R_F5) * RS, fd[5]);
        rst<NT>(r1 + (R_F6) * RS, fd[6]);
        rst<NT>(f78, fd[7]);
        rst<NT>(f78 + RS, fd[8]);
        f0n = fd[0];
        f2n = fd[2];
        f4 = fd[4];
        Fxn = Fx;
        Fyn = Fy;
        irn = inv_rho;
      } else if (!SIMPLE && ENERGY && r == P.ny && P.hbc[3] == WALL) {  // mirror ghost of row ny = row ny - 2
        rst<NT>(r1 + (R_UX) * RS, rld<NT>(r0 + (R_UX) * RS));
        rst<NT>(r1 + (R_UY) * RS, -rld<NT>(r0 + (R_UY) * RS));
      }
      __syncthreads();
    }
    // the slot of row q - 1 is free (its last reader, the collision, is past a barrier; before
    // iteration 2 its row was read by the first stage only): row q + 2 goes into it (a thread's
    // own copies only replace what the thread itself read)
    if (iq + 2 < n_it) stage_row(q + 2, k1, g1);
    if (!use_tma) cp_async_commit();

    // ---- S3: row q-2 (streaming, store of f; first Heun stage) ----
    if (iq >= 3) {
      const int r = q - 2;
      const LineMap rm = row_map(r);
      if (iq >= 5 && r < yb && !rm.outflow) {
        // pull f_i(x) = f*_i(x - c_i) from the ring rows r-1 (lo), r (mid), r+1 (hi); the halo
        // lanes compute alongside and store nothing
        F2 fd[9];
        fd[0] = f0c;
        fd[1] = rtrip<NT>(f13r).l;
        fd[2] = f2cc;
        fd[3] = rtrip<NT>(f13r + RS).r;
        fd[4] = f4;
        fd[5] = rtrip<NT>(r0 + (R_F5) * RS).l;
        fd[6] = rtrip<NT>(r0 + (R_F6) * RS).r;
        fd[7] = rtrip<NT>(f78).r;
        fd[8] = rtrip<NT>(f78 + RS).l;
        if (!SIMPLE && rm.wall >= 0) zou_he<F2>(rm.wall, fd, ev(-0.5f * Fxc), ev(-0.5f * Fyc));
        const F2 delta = ((fd[0] + (fd[1] + fd[2]) + (fd[3] + fd[4])) + ((fd[5] + fd[6]) + (fd[7] + fd[8])));
        const F2 rho_new = P.rho_ref + delta;
        const long long k = (long long)r * P.nx;
        if (t_in) {
#pragma unroll
          for (int i = 0; i < 9; ++i) st2(fout + i * plane + k, fd[i]);
          if (!ENERGY) {
            const F2 T_old = rld<NT>(r2 + (R_T) * RS);
            st2(Tout + k, T_old);
            t_sum = t_sum + T_old;
          }
          rho_min = fminf(rho_min, fminf(rho_new.lo(), rho_new.hi()));
          const float wr = (!SIMPLE && any_outflow) ? (float)line_weight(r, P.ny, P.hbc[2], P.hbc[3]) : 1.0f;
          const F2 yk = wr * rho_new + acc_n;
          const F2 tk = acc_s + yk;
          acc_n = yk - (tk - acc_s);
          acc_s = tk;
        }
      }
      if (ENERGY) {
        const Trip rmd = rtrip<NT>(r2 + (R_RHO) * RS), tm = rtrip<NT>(r2 + (R_T) * RS);
        if (iq >= 4) {
          if (!rm.solid) {
            PairHeun &c = nxt;
            const Trip ru = rtrip<NT>(r1 + (R_RHO) * RS), tu = rtrip<NT>(r1 + (R_T) * RS);
            const F2 rho = rmd.c, T0 = tm.c;
            const Trip xu = rtrip<NT>(r1 + (R_UX) * RS), xm = rtrip<NT>(r2 + (R_UX) * RS), xd = rtrip<NT>(r0 + (R_UX) * RS);
            const Trip yu = rtrip<NT>(r1 + (R_UY) * RS), ym = rtrip<NT>(r2 + (R_UY) * RS), yd = rtrip<NT>(r0 + (R_UY) * RS);
            F2 A, B;
            pr_parts(P, rho, &A, &B);
            const F2 ir = irc * P.cv_inv;  // 1 / (rho c_v)
            const F2 di = P.dlam * ir;     // d lambda / d rho / (rho c_v)
            c.lr = (P.lam_v + P.dlam * (rho - P.rho_v)) * ir;
            // 9-point stencils; the lower row's share was formed when it was the centre
            c.vx = di * (third * (rmd.r - rmd.l) + twelfth * (ru.r - ru.l) + sh0) - xm.c;
            c.vy = di * (third * ru.c + twelfth * (ru.r + ru.l) + sh1) - ym.c;
            const F2 ndiv = (-third) * (xm.r - xm.l) + (-twelfth) * (xu.r - xu.l - xd.l + xd.r) +
                            (-third) * (yu.c - yd.c) + (-twelfth) * (yu.r + yu.l - yd.l - yd.r);
            const F2 s = ndiv * ir;  // -div u / (rho c_v)
            c.nA = s * (A + kA * B);
            c.nB = s * ev(kB * B);
            F2 Ts;
            if (!SIMPLE && rm.outflow) {
              Ts = rld<NT>(r0 + (R_TS) * RS);  // outflow row: copy of the first interior row
              c.h = T0;
            } else {
              const F2 gtx = third * (tm.r - tm.l) + twelfth * (tu.r - tu.l) + sh2;
              const F2 gty = third * tu.c + twelfth * (tu.r + tu.l) + sh3;
              const F2 lap = (2.0f / 3.0f) * (tm.r + tu.c + tm.l - 4.0f * T0) +
                             (1.0f / 6.0f) * (tu.r + tu.l - 4.0f * T0) + sh4;
              const F2 Ta = P.T_ref + T0;
              const F2 k1 = c.lr * lap + c.vx * gtx + c.vy * gty + Ta * c.nA + sqrt(Ta) * c.nB;
              Ts = T0 + k1;
              c.h = T0 + 0.5f * k1;
              if ((!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1)) || col_fix) {  // Dirichlet nodes of a boundary line
                float tw0, tw1;
                const bool d0 = t_fixed(P, col0, rm.src, &tw0), d1 = t_fixed(P, col1, rm.src, &tw1);
                if (d0 || d1) {
                  Ts = F2(d0 ? tw0 - P.T_ref : Ts.lo(), d1 ? tw1 - P.T_ref : Ts.hi());
                  c.h = F2(d0 ? T0.lo() : c.h.lo(), d1 ? T0.hi() : c.h.hi());
                }
              }
            }
            rst<NT>(r2 + (R_TS) * RS, Ts);
            if (!SIMPLE && r == 1 && P.hbc[2] == WALL) rst<NT>(r1 + (R_TS) * RS, Ts);  // mirror ghost of row -1
          } else if (!SIMPLE && r == P.ny && P.hbc[3] == WALL) {
            rst<NT>(r2 + (R_TS) * RS, rld<NT>(r1 + (R_TS) * RS));  // mirror ghost of row ny
          }
        }
        // this row's share of the stencils of the row above (used by the next iteration)
        sh0 = twelfth * (rmd.r - rmd.l);
        sh1 = -(third * rmd.c + twelfth * (rmd.l + rmd.r));
        sh2 = twelfth * (tm.r - tm.l);
        sh3 = -(third * tm.c + twelfth * (tm.l + tm.r));
        sh4 = (2.0f / 3.0f) * tm.c + (1.0f / 6.0f) * (tm.l + tm.r);
        // the second Heun stage reads this iteration's T*, and the next first stage overwrites
        // the rho and T ring rows read above
        __syncthreads();
      }
    }

    // ---- S4: row q-3 (second Heun stage, store of T) ----
    if (ENERGY && iq >= 6) {  // the halo lanes compute alongside and store nothing
      const int r = q - 3;
      const LineMap rm = row_map(r);
      if (!rm.outflow) {
        const PairHeun &c = cur;
        const Trip tm = rtrip<NT>(r0 + (R_TS) * RS), tu = rtrip<NT>(r2 + (R_TS) * RS), td = rtrip<NT>(r1 + (R_TS) * RS);
        const F2 gtx = third * (tm.r - tm.l) + twelfth * (tu.r - tu.l - td.l + td.r);
        const F2 gty = third * (tu.c - td.c) + twelfth * (tu.r + tu.l - td.l - td.r);
        const F2 lap = (2.0f / 3.0f) * (tm.r + tu.c + tm.l + td.c - 4.0f * tm.c) +
                       (1.0f / 6.0f) * (tu.r + tu.l + td.l + td.r - 4.0f * tm.c);
        const F2 Ta = P.T_ref + tm.c;
        const F2 k2 = c.lr * lap + c.vx * gtx + c.vy * gty + Ta * c.nA + sqrt(Ta) * c.nB;
        F2 T_new = c.h + 0.5f * k2;
        if ((!SIMPLE && (rm.src == 0 || rm.src == P.ny - 1)) || col_fix) {  // Dirichlet nodes keep their value
          float tw;
          const bool d0 = t_fixed(P, col0, rm.src, &tw), d1 = t_fixed(P, col1, rm.src, &tw);
          T_new = F2(d0 ? c.h.lo() : T_new.lo(), d1 ? c.h.hi() : T_new.hi());  // h = T^n there
        }
        if (t_in) {
          st2(Tout + (long long)r * P.nx, T_new);
          t_sum = t_sum + T_new;
        }
      }
    }
    // hand over to the next iteration: carried values by row, slot roles rotated
    if (use_tma) ph ^= 1u << k0;
    f0c = f0n;
    f2cc = f2c;
    f2c = f2n;
    Fxc = Fxn;
    Fyc = Fyn;
    irc = irn;
    cur = nxt;
    {
      float *rt = r2;
      r2 = r1;
      r1 = r0;
      r0 = rt;
      const float *gt = g2;
      g2 = g1;
      g1 = g0;
      g0 = gt;
      const int kt = k2;
      k2 = k1;
      k1 = k0;
      k0 = kt;
      float *ft = f13w;
      f13w = f13r;
      f13r = ft;
    }
  }
  cp_async_wait<0>();
  double acc = ((double)acc_s.lo() + (double)acc_n.lo()) + ((double)acc_s.hi() + (double)acc_n.hi());
  if (!(arg_min >= 0.0f)) flags |= FLAG_PSI_NEG;
  if (!(rho_min > 0.0f)) flags |= FLAG_RHO_NONPOS;
  if (!isfinite(acc) || !isfinite((double)t_sum.lo() + (double)t_sum.hi())) flags |= FLAG_NAN;
  if (flags) atomicOr(io.status, flags);
  if (reduce)
    tile_mass_finalize<NT, false>(P, io, acc, 0.0, bid, nblk, done, done_value);
  else
    __syncthreads();  // every thread's stores of this tile precede what the caller does next
}

template <bool ENERGY, int NT>
__global__ void __launch_bounds__(NT, 448 / NT) row_step_pair(const Params<float> P, const StepIO io, const int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long bars[kPairSlots];  // mbarriers of the TMA staging slots
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x, nblk = gridDim.x * gridDim.y;
  int ya, yb;
  block_rows(io, H, blockIdx.y, P.ny, &ya, &yb);
  // (strips with a Dirichlet x line take the general form here: a third specialisation in
  // this kernel costs the others registers at its 128-register budget)
  if (pair_tile_kind<NT>(P, ya, yb, blockIdx.x) == 1)
    row_body_pair<ENERGY, NT, true>(P, io, ya, yb, blockIdx.x, bid, nblk, smem_raw, bars);
  else
    row_body_pair<ENERGY, NT, false>(P, io, ya, yb, blockIdx.x, bid, nblk, smem_raw, bars);
}

}  // namespace ppl_dev
