// Internal host-side declarations shared by the translation units of libppl (not part of
// the C ABI): the handle, the step launch and status helpers, the launch-shape helpers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/ppl.h"
#include "common.cuh"
#include "step_variants.h"

using namespace ppl_dev;

struct ppl_sim {
  ppl_config cfg;  // boundary-array pointers re-pointed at the owned copies below
  std::vector<double> h_rho_w[4], h_T_w[4];
  std::vector<uint8_t> h_T_dir[4];
  int prec = 0;
  int nx = 0, ny = 0;
  long long N = 0;
  size_t rsz = 8;  // sizeof(real)
  void *f[2] = {nullptr, nullptr};
  void *T[2] = {nullptr, nullptr};
  void *bnd = nullptr;  // device copies of the per-node boundary arrays
  void *tmaps = nullptr;  // FP32: 4 CUtensorMap (f[0], f[1], T[0], T[1]) for the TMA row staging, or null
  double *stats[2] = {nullptr, nullptr};
  double *partials = nullptr;  // max(#step CTAs (x2 for tangents), kStats * #stats blocks)
  size_t npart = 0;            // doubles in partials
  uint64_t shape_gen = 0;      // bumped when the launch shape or partials change
  double *norm_out = nullptr;  // 7 doubles
  unsigned *counter = nullptr;
  unsigned *status = nullptr;
  double *upload = nullptr;  // 4 * N doubles staging for init / reset
  int cur = 0;
  int64_t step = 0;
  int64_t launches = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  // captured step sequences [energy][starting parity][length index] (lengths kGraphLen)
  cudaGraphExec_t graph[2][2][5] = {};
  StepVariant var;
  dim3 grid;
  int rows_per_cta = 0;
  // two-height shape of the two-column step: grid.y = tall_blocks row blocks of rows_per_cta
  // rows, then row blocks of fill_rows rows up to ny (fill_rows = 0: all rows_per_cta)
  int tall_blocks = 0;
  int fill_rows = 0;
  int stats_blocks = 0;
  Params<double> pd;
  Params<float> pf;
  Params<Dual> pt;    // FP64 tangent modes
  Params<DualF> ptf;  // FP32 tangent modes
  uint64_t cfg_hash = 0;
};

namespace ppl_host {

// steps per captured CUDA graph, longest first (even: the ping-pong parity returns); a run
// of n steps replays the longest graphs that fit and launches at most one step on its own
constexpr int kGraphSteps = 32;
constexpr int kGraphLen[5] = {32, 16, 8, 4, 2};
void drop_graphs(ppl_sim *h);

int cuda_err(cudaError_t e);
#define CK(x)                                   \
  do {                                          \
    int _rc = cuda_err(x);                      \
    if (_rc != PPL_OK) return _rc;              \
  } while (0)

// checks a configuration (sizes, parameters, boundary combinations): PPL_OK or PPL_E_INVAL
int validate(const ppl_config *c);
// a state carrying d/d(sigma) or d/d(kappa) (FP64 or FP32)
bool is_tangent(int prec);
bool is_tangent32(int prec);
// the two-column FP32 kernel applies (x periodic for rho and T, even nx)
bool pair_applicable(const ppl_config &c);
// step kernel variant for a configuration and PPL_KERNEL_* choice
StepVariant pick_variant(const ppl_config &c, int kernel);
// one step launch on the handle's stream (advances cur / step / launches)
int launch_step(ppl_sim *h, bool energy);
// the energy equation is advanced at this step
bool energy_at(const ppl_sim *h, int64_t step);
// synchronises the handle's stream and maps the device status word to PPL_OK / PPL_E_NUMERIC
int check_status(ppl_sim *h);
// default rows per CTA: one wave of resident CTAs over the rows
int default_rows(const ppl_sim *h);
// the default launch shape: rows per CTA and, for the two-column step of a large grid, the
// height of the short row blocks that follow one wave of tall ones (0: uniform)
void default_shape(const ppl_sim *h, int *rows, int *fill_rows);
// applies a launch shape (fill_rows = 0: uniform row blocks of `rows` rows)
int apply_shape(ppl_sim *h, int rows, int fill_rows);
// grid of a launch shape; *tall receives the number of row blocks of `rows` rows
dim3 shape_grid(const ppl_sim *h, int rows, int fill_rows, int *tall);

template <typename real>
const Params<real> &params_of(const ppl_sim *h);
template <>
inline const Params<double> &params_of<double>(const ppl_sim *h) { return h->pd; }
template <>
inline const Params<float> &params_of<float>(const ppl_sim *h) { return h->pf; }
template <>
inline const Params<Dual> &params_of<Dual>(const ppl_sim *h) { return h->pt; }
template <>
inline const Params<DualF> &params_of<DualF>(const ppl_sim *h) { return h->ptf; }

}  // namespace ppl_host
