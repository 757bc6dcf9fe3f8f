// The mesh-refinement sequence (Sec. 3: dx, dx/2, dx/4 ... with dt ~ dx^2, so 1 : 4 : 16
// steps per coarse step) as one persistent launch: a grid of resident CTAs takes work items
// from a ticket counter in a fixed order and runs each as one tile of one step of one mesh
// with the FP32 two-column step (row_step_pair.cuh), on the same tiles as that mesh's own
// launch grid, so results are bitwise those of stepping each handle by itself.
//
// Items are ordered by the time of the step they belong to (step j of a mesh with s
// substeps per coarse step sits at j / s), all tiles of one step together. With gravity, a
// tile of step j waits until every tile of step j - 1 of its mesh is done: the last of those
// publishes the step's domain-mean density (Eq. gravitational_force) and then releases the
// mesh's step counter. Without gravity no step reads that mean, and a tile of step j waits
// only for the tiles of step j - 1 within its reach (the 4-column and 3-row halo of the
// step; those are also the tiles that read the rows it overwrites), so steps overlap in a
// wavefront; the mass is then reduced on the launch's last step only. Items are handed
// out in order to CTAs that are already running, so every item a CTA waits for is held by
// a running CTA and the waits end. Each wait is bounded (a time limit read from
// %globaltimer); a wait that runs out raises the batch's abort flag, every CTA leaves at
// its next item, and the host reports PPL_E_TIMEOUT.
#include <cuda_runtime.h>

#include "row_step_pair.cuh"
#include "step_variants.h"

namespace ppl_dev {

// control words of one persistent launch (device memory, cleared before each launch)
struct PersistCtl {
  unsigned ticket;  // next work item
  unsigned abort;   // a wait ran out
  unsigned done[kPersistMaxMeshes];  // steps of each mesh completed in this launch
  unsigned tile_done[1];             // steps of each tile completed (meshes without gravity)
};

// waits (thread 0, bounded) until *flag >= target; false if the wait ran out or the batch aborts
__device__ __forceinline__ bool wait_at_least(const unsigned *flag, unsigned target, const PersistCtl *ctl,
                                              unsigned long long wait_ns) {
  unsigned long long t0 = 0;
  for (long long i = 0;; ++i) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return true;
    if (i >= (1ll << 28)) return false;  // a clock that does not advance still ends the wait
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(now));
    if (i == 0) t0 = now;
    else if (now - t0 > wait_ns) return false;
    unsigned ab;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(ab) : "l"(&ctl->abort) : "memory");
    if (ab) return false;
    __nanosleep(64);
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int NT>
__global__ void __launch_bounds__(NT, 384 / NT) persistent_batch(const PersistMesh *meshes, const PersistItem *items,
                                                                 int n_items, int n_outer, PersistCtl *ctl,
                                                                 unsigned long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long bars[kPairSlots];
  __shared__ Params<float> P;
  __shared__ int item_s;
  const int total = n_items * n_outer;
  for (;;) {
    if (threadIdx.x == 0) {
      int it = (int)atomicAdd(&ctl->ticket, 1u);
      if (it >= total || ld_acquire(&ctl->abort)) it = -1;
      item_s = it;
    }
    __syncthreads();
    const int it = item_s;
    if (it < 0) break;
    const PersistItem e = items[it % n_items];
    const int outer = it / n_items;
    const PersistMesh &M = meshes[e.mesh];
    const unsigned j = (unsigned)(outer * M.sub + e.step);  // the mesh's step within this launch
    const int bx = e.tile % M.gx, by = e.tile / M.gx;
    // the previous step has finished where this tile reads (bounded waits)
    bool ok = true;
    if (j > 0 && M.local) {
      // thread i watches the i-th tile within reach (3 strips x 2 reach_y + 1 row blocks), so
      // one round of loads covers them all
      const int span = 2 * M.reach_y + 1;
      const unsigned *flag = nullptr;
      if ((int)threadIdx.x < 3 * span) {
        int ny_ = by + (int)threadIdx.x / 3 - M.reach_y;
        const int nx_ = ((bx + (int)threadIdx.x % 3 - 1) % M.gx + M.gx) % M.gx;
        if (M.periodic_y) ny_ = ((ny_ % M.gy) + M.gy) % M.gy;
        if (ny_ >= 0 && ny_ < M.gy) flag = &ctl->tile_done[M.tile0 + ny_ * M.gx + nx_];
      }
      unsigned long long t0 = 0;
      for (long long i = 0;; ++i) {
        bool ready = true;
        if (flag) {
          unsigned v;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
          ready = v >= j;
        }
        if (__syncthreads_and(ready)) break;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(now));
        if (i == 0) t0 = now;
        const bool out = i >= (1ll << 28) || (i > 0 && now - t0 > wait_ns) || ld_acquire(&ctl->abort);
        if (__syncthreads_or(out)) {
          ok = false;
          break;
        }
        __nanosleep(64);
      }
    }
    if (threadIdx.x == 0) {
      if (ok && j > 0 && !M.local) ok = wait_at_least(&ctl->done[e.mesh], j, ctl, wait_ns);
      if (!ok) {
        atomicExch(&ctl->abort, 1u);
        atomicOr(M.status, FLAG_STALL);
        item_s = -1;
      }
    }
    // the mesh's parameters for this tile
    for (int k = threadIdx.x; k < (int)(sizeof(Params<float>) / 4); k += NT)
      reinterpret_cast<unsigned *>(&P)[k] = reinterpret_cast<const unsigned *>(&M.P)[k];
    __syncthreads();
    if (item_s < 0) break;
    const int par = (M.cur0 + (int)j) & 1;  // ping-pong buffer read by this step
    StepIO io;
    io.f_in = M.f[par];
    io.T_in = M.T[par];
    io.f_out = M.f[1 - par];
    io.T_out = M.T[1 - par];
    io.stats_in = M.stats[par];
    io.stats_out = M.stats[1 - par];
    io.partials = M.partials;
    io.counter = M.counter;
    io.status = M.status;
    // rows are staged by per-thread cp.async (generic proxy): the populations a tile reads
    // were written by other CTAs of this launch, which TMA (async proxy) reads would need
    // cross-proxy fences to see; the staging path does not change the results
    io.tmap_f = nullptr;
    io.tmap_T = nullptr;
    io.blocks_a = 0;
    io.fill_rows = 0;
    const int ya = by * M.H, yb = min(ya + M.H, P.ny);
    const int kind = pair_tile_kind<NT>(P, ya, yb, bx);
    const bool energy = M.energy_on && M.step0 + (long long)j >= M.iso_steps;
    unsigned *done = &ctl->done[e.mesh];
    const unsigned nblk = (unsigned)(M.gx * M.gy);
    // without gravity the mass is reduced on the launch's last step only (its counter and
    // partials then serve one step)
    const bool reduce = !M.local || j + 1 == (unsigned)(n_outer * M.sub);
    const unsigned tile = (unsigned)e.tile, dv = j + 1;
    if (energy) {
      if (kind == 1)
        row_body_pair<true, NT, true>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
      else if (kind == 2)
        row_body_pair<true, NT, true, true>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
      else
        row_body_pair<true, NT, false>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
    } else {
      if (kind == 1)
        row_body_pair<false, NT, true>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
      else if (kind == 2)
        row_body_pair<false, NT, true, true>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
      else
        row_body_pair<false, NT, false>(P, io, ya, yb, bx, tile, nblk, smem_raw, bars, done, dv, reduce);
    }
    if (M.local && threadIdx.x == 0) {  // this tile's step is complete (all its threads passed a barrier)
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(&ctl->tile_done[M.tile0 + e.tile]), "r"(j + 1)
                   : "memory");
    }
  }
}

size_t persistent_batch_smem() { return row_step_pair_smem_bytes<kNTP>(); }

cudaError_t launch_persistent_batch(const PersistMesh *meshes, const PersistItem *items, int n_items, int n_outer,
                                    void *ctl, unsigned long long wait_ns, int ctas, cudaStream_t stream) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(persistent_batch<kNTP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)persistent_batch_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  persistent_batch<kNTP><<<ctas, kNTP, persistent_batch_smem(), stream>>>(meshes, items, n_items, n_outer,
                                                                         (PersistCtl *)ctl, wait_ns);
  return cudaGetLastError();
}

int persistent_batch_ctas_per_sm() {
  int n = 0;
  if (cudaFuncSetAttribute(persistent_batch<kNTP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)persistent_batch_smem()) != cudaSuccess)
    return 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_batch<kNTP>, kNTP, persistent_batch_smem());
  return n;
}

size_t persistent_ctl_bytes(int tiles) { return sizeof(PersistCtl) + (size_t)(tiles > 0 ? tiles : 0) * sizeof(unsigned); }

}  // namespace ppl_dev
