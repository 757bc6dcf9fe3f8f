// Launch shapes of the fused row step and the host-side handles of its instantiations.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "common.cuh"

namespace ppl_dev {

constexpr int kNT32 = 128;  // threads (columns incl. the 3 + 3 halo) per CTA, FP32
constexpr int kPF32 = 1;    // rows staged ahead, FP32
constexpr int kNT64 = 128;
constexpr int kPF64 = 1;
constexpr int kNTD = 128;  // tangent (Dual) step
constexpr int kPFD = 1;
constexpr int kNTDF = 128;  // FP32 tangent (DualF) step
constexpr int kPFDF = 1;
constexpr int kNTP = 64;   // FP32 two-column kernel: threads per CTA (2 kNTP columns)

struct StepVariant {
  int nt;        // threads per CTA
  int width;     // interior columns per CTA (strip width minus the halo)
  size_t smem;   // dynamic shared memory per CTA
  const void *fn[2];  // [energy on]
};

StepVariant step_variant_fp32();
StepVariant step_variant_fp32_pair();  // two columns per thread: hydrodynamically x-periodic, nx even
StepVariant step_variant_fp64();
StepVariant step_variant_tangent();    // FP64 value + derivative (Dual)
StepVariant step_variant_tangent32();  // FP32 value + derivative (DualF)

// one CTA waiting on an mbarrier that nothing completes, with the step's bounded wait
cudaError_t launch_stall_probe(unsigned long long limit_ns, unsigned *status);

// ---- the persistent batched launch of the refinement sequence (batch_persist.cu) ----
constexpr int kPersistMaxMeshes = 16;
// one mesh of the batch: its FP32 handle's parameters, buffers and launch grid
struct PersistMesh {
  Params<float> P;
  void *f[2], *T[2];    // ping-pong state
  double *stats[2];     // rho_bar and mass of each buffer's state
  double *partials;     // per-tile mass partials
  unsigned *counter;    // tiles done in the current step
  unsigned *status;     // PPL_FLAG_* bits
  const void *tmaps;    // 4 tensor maps (f[0], f[1], T[0], T[1]) or null
  int gx, gy, H;        // tiles: gx strips x gy row blocks of H rows
  int sub;              // steps per outer step
  int cur0;             // buffer holding the state at launch
  int energy_on;
  long long step0, iso_steps;
  // no gravity: no step reads the domain mean, so a tile depends only on the tiles within the
  // step's reach (one strip, reach_y row blocks each way) of the previous step
  int local, reach_y, periodic_y;
  int tile0;            // first of this mesh's per-tile step counters in the control block
};
struct PersistItem {  // one tile of one step of one mesh within an outer step
  int mesh, step, tile;
};
size_t persistent_batch_smem();
size_t persistent_ctl_bytes(int tiles);  // control block with per-tile counters for `tiles` tiles
int persistent_batch_ctas_per_sm();
// n_outer outer steps of every mesh: items (n_items per outer step) handed out in order
cudaError_t launch_persistent_batch(const PersistMesh *meshes, const PersistItem *items, int n_items, int n_outer,
                                    void *ctl, unsigned long long wait_ns, int ctas, cudaStream_t stream);

}  // namespace ppl_dev
