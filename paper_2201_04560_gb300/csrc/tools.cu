// Host side of libppl, part 2: the mesh-refinement tools built on the step (Secs. 3-4):
// cross-mesh differences, the batched refinement sequence, the launch shape and its
// autotuner, the droplet area, the wall heat flux, the contact angle and the time shift.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sim.cuh"

using namespace ppl_host;

// ---------------------------------------------------------------------------------
// Cross-grid relative difference (Eqs. rel-diff-timestep and global-rel-diff): the coarse
// field interpolated bilinearly onto the fine grid against the fine field.
// ---------------------------------------------------------------------------------
namespace {

// coarse coordinate of fine line g: cell-centred on periodic axes, node-aligned (ends on
// ends) on bounded axes
__device__ __forceinline__ double coarse_coord(int g, int nf, int nc, bool periodic) {
  if (periodic) return (g + 0.5) * ((double)nc / nf) - 0.5;
  return nf > 1 ? g * ((double)(nc - 1) / (nf - 1)) : 0.0;
}

template <typename real>
__device__ __forceinline__ double node_value(const Params<real> &P, const real *f, const real *T, int x, int y,
                                             int field) {
  const NodeMap m = map_node(P, x, y);  // outflow lines read their first-interior copy
  const long long k = (long long)m.y * P.nx + m.x;
  if (field == 1) return (double)P.T_ref + (double)T[k];
  if (field == 2) return ((double)P.T_ref + (double)T[k]) / (double)P.Tc;  // reduced T / T_c
  double d = 0.0;
  for (int q = 0; q < 9; ++q) d += (double)f[q * P.plane + k];
  return (double)P.rho_ref + d;
}

template <typename rc, typename rf>
__global__ void cross_norm_partials(const Params<rc> Pc, const rc *fc, const rc *Tc, const Params<rf> Pf,
                                    const rf *ff, const rf *Tf, int field, double *part) {
  constexpr int NT = 256;
  __shared__ double red[2][NT / 32];
  double num = 0.0, den = 0.0;
  const bool perx = Pc.hbc[0] == PERIODIC, pery = Pc.hbc[2] == PERIODIC;
  const int fv = field == 1 ? 2 : field;  // temperatures compare as T / T_c of each mesh
  for (long long k = (long long)blockIdx.x * NT + threadIdx.x; k < Pf.plane; k += (long long)gridDim.x * NT) {
    const int x = (int)(k % Pf.nx), y = (int)(k / Pf.nx);
    const double X = coarse_coord(x, Pf.nx, Pc.nx, perx), Y = coarse_coord(y, Pf.ny, Pc.ny, pery);
    int x0 = (int)floor(X), y0 = (int)floor(Y);
    const double wx = X - x0, wy = Y - y0;
    int x1 = x0 + 1, y1 = y0 + 1;
    if (perx) {
      x0 = (x0 % Pc.nx + Pc.nx) % Pc.nx;
      x1 = (x1 % Pc.nx + Pc.nx) % Pc.nx;
    } else {
      x0 = min(max(x0, 0), Pc.nx - 1);
      x1 = min(max(x1, 0), Pc.nx - 1);
    }
    if (pery) {
      y0 = (y0 % Pc.ny + Pc.ny) % Pc.ny;
      y1 = (y1 % Pc.ny + Pc.ny) % Pc.ny;
    } else {
      y0 = min(max(y0, 0), Pc.ny - 1);
      y1 = min(max(y1, 0), Pc.ny - 1);
    }
    const double c00 = node_value(Pc, fc, Tc, x0, y0, fv), c10 = node_value(Pc, fc, Tc, x1, y0, fv);
    const double c01 = node_value(Pc, fc, Tc, x0, y1, fv), c11 = node_value(Pc, fc, Tc, x1, y1, fv);
    const double I = (1.0 - wy) * ((1.0 - wx) * c00 + wx * c10) + wy * ((1.0 - wx) * c01 + wx * c11);
    const double v = node_value(Pf, ff, Tf, x, y, fv);
    num += fabs(I - v);
    den += fabs(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[threadIdx.x][w];
    part[(long long)blockIdx.x * 2 + threadIdx.x] = s;
  }
}

__global__ void pair_finalize(const double *part, int nblk, double *out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
}

template <typename rc, typename rf>
int launch_cross_norm(const ppl_sim *c, const ppl_sim *f, int field, double *dpart, int nblk, cudaStream_t s) {
  cross_norm_partials<rc, rf><<<nblk, 256, 0, s>>>(params_of<rc>(c), (const rc *)c->f[c->cur],
                                                   (const rc *)c->T[c->cur], params_of<rf>(f),
                                                   (const rf *)f->f[f->cur], (const rf *)f->T[f->cur], field, dpart);
  CK(cudaGetLastError());
  return PPL_OK;
}

}  // namespace

extern "C" {

int ppl_cross_norm(const ppl_t *coarse, const ppl_t *fine, int field, double *num, double *den) {
  if (!coarse || !fine || !num || !den || (field != 0 && field != 1)) return PPL_E_INVAL;
  if (is_tangent(coarse->prec) || is_tangent(fine->prec)) return PPL_E_INVAL;
  for (int s = 0; s < 4; ++s)
    if (coarse->cfg.hydro_bc[s] != fine->cfg.hydro_bc[s]) return PPL_E_INVAL;  // same domain, two meshes
  CK(cudaStreamSynchronize(coarse->stream));
  cudaStream_t s = fine->stream;
  const int nblk = 608;
  double *d = nullptr;
  CK(cudaMalloc(&d, (2 * nblk + 2) * sizeof(double)));
  int rc;
  const bool c64 = coarse->prec == PPL_FP64, f64 = fine->prec == PPL_FP64;
  if (c64 && f64) rc = launch_cross_norm<double, double>(coarse, fine, field, d, nblk, s);
  else if (c64) rc = launch_cross_norm<double, float>(coarse, fine, field, d, nblk, s);
  else if (f64) rc = launch_cross_norm<float, double>(coarse, fine, field, d, nblk, s);
  else rc = launch_cross_norm<float, float>(coarse, fine, field, d, nblk, s);
  double out[2] = {0.0, 0.0};
  if (rc == PPL_OK) {
    pair_finalize<<<1, 32, 0, s>>>(d, nblk, d + 2 * nblk);
    rc = cuda_err(cudaGetLastError());
  }
  if (rc == PPL_OK) rc = cuda_err(cudaMemcpyAsync(out, d + 2 * nblk, sizeof(out), cudaMemcpyDeviceToHost, s));
  if (rc == PPL_OK) rc = cuda_err(cudaStreamSynchronize(s));
  cudaFree(d);
  if (rc == PPL_OK) {
    *num = out[0];
    *den = out[1];
  }
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batched refinement sequence: several handles advanced together, sim k taking
// substeps[k] steps per outer step (dt ~ dx^2: 1, 4, 16 for dx, dx/2, dx/4). One outer
// step (or two, to bring every ping-pong parity back) is one CUDA graph whose branches
// run the grids concurrently.
// ---------------------------------------------------------------------------------
struct ppl_batch {
  std::vector<ppl_sim *> sims;
  std::vector<int32_t> sub;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> done;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;      // joins of the handles' streams, outside capture
  cudaEvent_t cap_fork = nullptr;  // fork inside a capture
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [energy pattern is uniform on]
  std::vector<int> graph_energy[2];
  std::vector<uint64_t> graph_gen[2];  // shape_gen of each sim at capture
  int period = 1;  // outer steps per graph
  // persistent mode: one launch for all meshes and outer steps (batch_persist.cu)
  int mode = PPL_BATCH_AUTO;
  unsigned long long wait_ns = 1000000000ull;  // bound of every dependency wait
  PersistMesh *h_meshes = nullptr;             // pinned staging of the mesh table
  PersistMesh *d_meshes = nullptr;
  PersistItem *d_items = nullptr;
  void *d_ctl = nullptr;
  size_t ctl_bytes = 0;
  unsigned *h_abort = nullptr;  // pinned copy of the abort word
  int n_items = 0;
  std::vector<uint64_t> items_gen;  // shape_gen of each sim when the item list was built
  cudaGraphExec_t pgraph = nullptr;
  int64_t pgraph_outer = -1;
};

namespace {

void batch_free(ppl_batch *b) {
  for (int i = 0; i < 2; ++i)
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
  if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
  if (b->h_meshes) cudaFreeHost(b->h_meshes);
  if (b->h_abort) cudaFreeHost(b->h_abort);
  cudaFree(b->d_meshes);
  cudaFree(b->d_items);
  cudaFree(b->d_ctl);
  for (auto s : b->branch) cudaStreamDestroy(s);
  for (auto e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap_fork) cudaEventDestroy(b->cap_fork);
  if (b->main) cudaStreamDestroy(b->main);
}

// energy flags of each sim over the next `period` outer steps, or empty if not uniform
std::vector<int> energy_pattern(const ppl_batch *b) {
  std::vector<int> pat;
  for (size_t k = 0; k < b->sims.size(); ++k) {
    const ppl_sim *h = b->sims[k];
    const int64_t n = (int64_t)b->period * b->sub[k];
    const bool e0 = energy_at(h, h->step), e1 = energy_at(h, h->step + n - 1);
    if (e0 != e1) return {};
    pat.push_back(e0 ? 1 : 0);
  }
  return pat;
}

int batch_capture(ppl_batch *b, const std::vector<int> &pat, cudaGraphExec_t *out) {
  // host bookkeeping of every sim is restored after capture
  std::vector<int> cur0;
  std::vector<int64_t> step0, l0;
  std::vector<cudaStream_t> s0;
  for (auto h : b->sims) {
    cur0.push_back(h->cur);
    step0.push_back(h->step);
    l0.push_back(h->launches);
    s0.push_back(h->stream);
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
  int rc = cuda_err(cudaEventRecord(b->cap_fork, b->main));
  for (size_t k = 0; k < b->sims.size() && rc == PPL_OK; ++k) {
    ppl_sim *h = b->sims[k];
    rc = cuda_err(cudaStreamWaitEvent(b->branch[k], b->cap_fork, 0));
    h->stream = b->branch[k];
    for (int64_t i = 0; i < (int64_t)b->period * b->sub[k] && rc == PPL_OK; ++i) rc = launch_step(h, pat[k] != 0);
    if (rc == PPL_OK) rc = cuda_err(cudaEventRecord(b->done[k], b->branch[k]));
    if (rc == PPL_OK) rc = cuda_err(cudaStreamWaitEvent(b->main, b->done[k], 0));
  }
  cudaError_t ce = cudaStreamEndCapture(b->main, &g);
  for (size_t k = 0; k < b->sims.size(); ++k) {
    ppl_sim *h = b->sims[k];
    h->cur = cur0[k];
    h->step = step0[k];
    h->launches = l0[k];
    h->stream = s0[k];
  }
  if (rc != PPL_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(ce);
  ce = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(ce);
  return PPL_OK;
}

// Every handle steps with the FP32 two-column kernel: the persistent mode applies.
bool persistent_applicable(const ppl_batch *b) {
  if (b->sims.size() > (size_t)kPersistMaxMeshes) return false;
  for (auto h : b->sims)
    if (h->prec != PPL_FP32DEV || h->var.fn[0] != step_variant_fp32_pair().fn[0] || h->fill_rows > 0)
      return false;  // (the persistent items address uniform row blocks)
  return true;
}

// work items of one outer step: all tiles of a step together, steps ordered by their time
// j / sub within the outer step (ties: the larger number of substeps first)
std::vector<PersistItem> persistent_items(const ppl_batch *b) {
  struct Key {
    double t;
    int sub, mesh, step;
  };
  std::vector<Key> keys;
  for (size_t m = 0; m < b->sims.size(); ++m)
    for (int j = 0; j < b->sub[m]; ++j) keys.push_back({(double)j / b->sub[m], b->sub[m], (int)m, j});
  std::stable_sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
    return x.t < y.t || (x.t == y.t && x.sub > y.sub);
  });
  std::vector<PersistItem> items;
  for (const Key &k : keys) {
    const ppl_sim *h = b->sims[k.mesh];
    const int tiles = (int)(h->grid.x * h->grid.y);
    for (int i = 0; i < tiles; ++i) items.push_back({k.mesh, k.step, i});
  }
  return items;
}

int persistent_step(ppl_batch *b, int64_t outer) {
  if (!persistent_applicable(b)) return PPL_E_INVAL;
  const int n = (int)b->sims.size();
  if (!b->h_meshes) {
    CK(cudaMallocHost((void **)&b->h_meshes, kPersistMaxMeshes * sizeof(PersistMesh)));
    CK(cudaMallocHost((void **)&b->h_abort, sizeof(unsigned)));
    CK(cudaMalloc((void **)&b->d_meshes, kPersistMaxMeshes * sizeof(PersistMesh)));
  }
  std::vector<uint64_t> gen;
  int tiles = 0;
  for (auto h : b->sims) {
    gen.push_back(h->shape_gen);
    tiles += (int)(h->grid.x * h->grid.y);
  }
  if (gen != b->items_gen || !b->d_items) {
    CK(cudaStreamSynchronize(b->main));
    cudaFree(b->d_ctl);
    b->d_ctl = nullptr;
    CK(cudaMalloc(&b->d_ctl, persistent_ctl_bytes(tiles)));
    b->ctl_bytes = persistent_ctl_bytes(tiles);
    std::vector<PersistItem> items = persistent_items(b);
    CK(cudaStreamSynchronize(b->main));
    cudaFree(b->d_items);
    b->d_items = nullptr;
    CK(cudaMalloc((void **)&b->d_items, items.size() * sizeof(PersistItem)));
    CK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(PersistItem), cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    b->items_gen = gen;
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    b->pgraph = nullptr;
  }
  // the mesh table of this launch (read by the graph's copy node when it runs)
  CK(cudaStreamSynchronize(b->main));
  int tile0 = 0;
  for (int m = 0; m < n; ++m) {
    ppl_sim *h = b->sims[m];
    PersistMesh &M = b->h_meshes[m];
    M.local = h->cfg.gx == 0.0 && h->cfg.gy == 0.0;
    M.reach_y = (3 + h->rows_per_cta - 1) / h->rows_per_cta;  // rows of the halo, in row blocks
    M.periodic_y = h->cfg.hydro_bc[2] == PPL_PERIODIC;
    M.tile0 = tile0;
    tile0 += (int)(h->grid.x * h->grid.y);
    M.P = h->pf;
    for (int i = 0; i < 2; ++i) {
      M.f[i] = h->f[i];
      M.T[i] = h->T[i];
      M.stats[i] = h->stats[i];
    }
    M.partials = h->partials;
    M.counter = h->counter;
    M.status = h->status;
    M.tmaps = h->tmaps;
    M.gx = (int)h->grid.x;
    M.gy = (int)h->grid.y;
    M.H = h->rows_per_cta;
    M.sub = b->sub[m];
    M.cur0 = h->cur;
    M.energy_on = h->cfg.energy_on;
    M.step0 = h->step;
    M.iso_steps = h->cfg.iso_steps;
  }
  if (!b->pgraph || b->pgraph_outer != outer) {
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    b->pgraph = nullptr;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm = persistent_batch_ctas_per_sm();
    if (per_sm < 1) return PPL_E_CUDA;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    int rc = cuda_err(cudaMemcpyAsync(b->d_meshes, b->h_meshes, n * sizeof(PersistMesh), cudaMemcpyHostToDevice,
                                      b->main));
    if (rc == PPL_OK) rc = cuda_err(cudaMemsetAsync(b->d_ctl, 0, b->ctl_bytes, b->main));
    if (rc == PPL_OK)
      rc = cuda_err(launch_persistent_batch(b->d_meshes, b->d_items, b->n_items, (int)outer, b->d_ctl, b->wait_ns,
                                            sms * per_sm, b->main));
    cudaError_t ce = cudaStreamEndCapture(b->main, &g);
    if (rc != PPL_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    CK(ce);
    ce = cudaGraphInstantiate(&b->pgraph, g, 0);
    cudaGraphDestroy(g);
    CK(ce);
    b->pgraph_outer = outer;
  }
  CK(cudaGraphLaunch(b->pgraph, b->main));
  CK(cudaMemcpyAsync(b->h_abort, (const char *)b->d_ctl + sizeof(unsigned), sizeof(unsigned),
                     cudaMemcpyDeviceToHost, b->main));
  CK(cudaStreamSynchronize(b->main));
  for (int m = 0; m < n; ++m) {
    ppl_sim *h = b->sims[m];
    const int64_t k = outer * b->sub[m];
    h->step += k;
    h->launches += k;
    if (k & 1) h->cur = 1 - h->cur;
  }
  if (*b->h_abort) {
    // a stopped launch leaves steps half done: clear each mesh's tile counter so that the
    // handles can be reset or reloaded and stepped again
    for (auto h : b->sims) CK(cudaMemsetAsync(h->counter, 0, sizeof(unsigned), b->main));
    CK(cudaStreamSynchronize(b->main));
    return PPL_E_TIMEOUT;
  }
  return PPL_OK;
}

}  // namespace

extern "C" {

int ppl_batch_create(ppl_t *const *sims, const int32_t *substeps, int32_t n, ppl_batch_t **out) {
  if (!out || !sims || !substeps || n < 1 || n > 64) return PPL_E_INVAL;
  *out = nullptr;
  ppl_batch *b = new (std::nothrow) ppl_batch();
  if (!b) return PPL_E_NOMEM;
  bool odd = false;
  for (int k = 0; k < n; ++k) {
    if (!sims[k] || substeps[k] < 1) {
      delete b;
      return PPL_E_INVAL;
    }
    for (int j = 0; j < k; ++j)
      if (sims[j] == sims[k]) {
        delete b;
        return PPL_E_INVAL;
      }
    b->sims.push_back(sims[k]);
    b->sub.push_back(substeps[k]);
    odd = odd || (substeps[k] & 1);
  }
  b->period = odd ? 2 : 1;  // every sim's ping-pong parity returns after one graph
  bool ok = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->cap_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < n && ok; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (s) b->branch.push_back(s);
    if (e) b->done.push_back(e);
  }
  if (!ok) {
    batch_free(b);
    delete b;
    return PPL_E_CUDA;
  }
  *out = b;
  return PPL_OK;
}

int ppl_batch_set_mode(ppl_batch_t *b, int mode) {
  if (!b || (mode != PPL_BATCH_GRAPH && mode != PPL_BATCH_PERSISTENT && mode != PPL_BATCH_AUTO)) return PPL_E_INVAL;
  if (mode == PPL_BATCH_PERSISTENT && !persistent_applicable(b)) return PPL_E_INVAL;
  b->mode = mode;
  return PPL_OK;
}

int ppl_batch_get_mode(const ppl_batch_t *b) { return b ? b->mode : PPL_E_INVAL; }

int ppl_batch_set_wait_limit(ppl_batch_t *b, int64_t ns) {
  if (!b || ns < 0) return PPL_E_INVAL;
  b->wait_ns = (unsigned long long)ns;
  if (b->pgraph) cudaGraphExecDestroy(b->pgraph);  // the limit is a kernel argument of the captured launch
  b->pgraph = nullptr;
  return PPL_OK;
}

int ppl_batch_step(ppl_batch_t *b, int64_t outer) {
  if (!b || outer < 0) return PPL_E_INVAL;
  // the batch stream starts after everything already queued on the sims' own streams
  for (auto h : b->sims) {
    CK(cudaEventRecord(b->fork, h->stream));
    CK(cudaStreamWaitEvent(b->main, b->fork, 0));
  }
  bool persistent = b->mode == PPL_BATCH_PERSISTENT;
  if (b->mode == PPL_BATCH_AUTO) {
    // the persistent launch where it applies and every mesh is free of gravity (tiles then
    // wait only for their neighbours: measured faster than the graph branches); else graphs
    persistent = persistent_applicable(b);
    for (auto h : b->sims) persistent = persistent && h->cfg.gx == 0.0 && h->cfg.gy == 0.0;
  }
  if (persistent && outer > 0) {
    int prc = persistent_step(b, outer);
    CK(cudaEventRecord(b->fork, b->main));
    for (auto h : b->sims) CK(cudaStreamWaitEvent(h->stream, b->fork, 0));
    if (prc != PPL_OK) return prc;
    int rc = PPL_OK;
    for (auto h : b->sims) {
      const int r = check_status(h);
      if (r != PPL_OK && rc == PPL_OK) rc = r;
    }
    return rc;
  }
  int64_t left = outer;
  while (left > 0) {
    std::vector<int> pat = energy_pattern(b);
    bool parity_ok = true;
    for (auto h : b->sims) parity_ok = parity_ok && h->cur == 0;
    if (left >= b->period && !pat.empty() && parity_ok) {
      std::vector<uint64_t> gen;
      for (auto h : b->sims) gen.push_back(h->shape_gen);
      int slot = -1;
      for (int i = 0; i < 2; ++i)
        if (b->graph[i] && b->graph_energy[i] == pat && b->graph_gen[i] == gen) slot = i;
      if (slot < 0) {
        slot = b->graph[0] ? 1 : 0;
        if (b->graph[slot]) cudaGraphExecDestroy(b->graph[slot]);
        b->graph[slot] = nullptr;
        int rc = batch_capture(b, pat, &b->graph[slot]);
        if (rc) return rc;
        b->graph_energy[slot] = pat;
        b->graph_gen[slot] = gen;
      }
      CK(cudaGraphLaunch(b->graph[slot], b->main));
      for (size_t k = 0; k < b->sims.size(); ++k) {
        ppl_sim *h = b->sims[k];
        const int64_t n = (int64_t)b->period * b->sub[k];
        h->step += n;
        h->launches += n;
        if (n & 1) h->cur = 1 - h->cur;
      }
      left -= b->period;
    } else {
      // one outer step, launched directly on the batch stream
      for (size_t k = 0; k < b->sims.size(); ++k) {
        ppl_sim *h = b->sims[k];
        cudaStream_t s0 = h->stream;
        h->stream = b->main;
        int rc = PPL_OK;
        for (int i = 0; i < b->sub[k] && rc == PPL_OK; ++i) rc = launch_step(h, energy_at(h, h->step));
        h->stream = s0;
        if (rc) return rc;
      }
      left -= 1;
    }
  }
  // the sims' own streams continue after the batch; status of every sim
  CK(cudaEventRecord(b->fork, b->main));
  for (auto h : b->sims) CK(cudaStreamWaitEvent(h->stream, b->fork, 0));
  int rc = PPL_OK;
  for (auto h : b->sims) {
    const int r = check_status(h);
    if (r != PPL_OK && rc == PPL_OK) rc = r;
  }
  return rc;
}

void ppl_batch_destroy(ppl_batch_t *b) {
  if (!b) return;
  cudaStreamSynchronize(b->main);
  batch_free(b);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Launch shape: rows per CTA, and a timing autotuner over it
// ---------------------------------------------------------------------------------
namespace {

int apply_rows(ppl_sim *h, int H) { return apply_shape(h, H, 0); }

int apply_default_shape(ppl_sim *h) {
  int H, F;
  default_shape(h, &H, &F);
  return apply_shape(h, H, F);
}

}  // namespace

int ppl_host::apply_shape(ppl_sim *h, int H, int fill_rows) {
  int tall = 0;
  const dim3 grid = shape_grid(h, H, fill_rows, &tall);
  const size_t nctas = (size_t)grid.x * grid.y;
  CK(cudaStreamSynchronize(h->stream));
  const size_t need = nctas * (is_tangent(h->prec) ? 2 : 1);
  if (need > h->npart) {
    double *p = nullptr;
    if (cudaMalloc(&p, need * sizeof(double)) != cudaSuccess) return PPL_E_NOMEM;
    cudaFree(h->partials);
    h->partials = p;
    h->npart = need;
  }
  drop_graphs(h);
  h->rows_per_cta = H;
  h->fill_rows = fill_rows > 0 ? fill_rows : 0;
  h->tall_blocks = tall;
  h->grid = grid;
  h->shape_gen += 1;
  return PPL_OK;
}

extern "C" {

int ppl_set_launch(ppl_t *h, int32_t rows_per_cta) {
  if (!h || rows_per_cta < 0 || rows_per_cta > h->ny) return PPL_E_INVAL;
  return rows_per_cta == 0 ? apply_default_shape(h) : apply_rows(h, rows_per_cta);
}

int ppl_select_kernel(ppl_t *h, int kernel) {
  if (!h || kernel < PPL_KERNEL_AUTO || kernel > PPL_KERNEL_PAIR) return PPL_E_INVAL;
  if (kernel == PPL_KERNEL_PAIR && !pair_applicable(h->cfg)) return PPL_E_INVAL;
  const StepVariant v = pick_variant(h->cfg, kernel);
  for (int e = 0; e < 2; ++e)
    CK(cudaFuncSetAttribute(v.fn[e], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
  CK(cudaStreamSynchronize(h->stream));
  h->var = v;
  return apply_default_shape(h);
}

int ppl_get_kernel(const ppl_t *h) {
  if (!h) return PPL_E_INVAL;
  return h->var.fn[0] == step_variant_fp32_pair().fn[0] ? PPL_KERNEL_PAIR : PPL_KERNEL_COLUMN;
}

}  // extern "C"

namespace {

// FP64 FMA rate: eight independent chains of dependent DFMAs per thread, four 256-thread CTAs
// per SM, so that the FP64 pipe (not latency) bounds the loop; the roofline denominator of the
// FP64 step
constexpr int kDfmaPerIter = 128;
__global__ void dfma_loop(double *out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kDfmaPerIter / 8; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

cudaError_t launch_dfma_loop(double *out, int blocks, int threads, int iters, cudaStream_t stream) {
  dfma_loop<<<blocks, threads, 0, stream>>>(out, iters, 0.999999, 1e-9);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int ppl_fp64_rate(int32_t iters, double *dfma_per_s) {
  if (iters < 1 || iters > 1000000 || !dfma_per_s) return PPL_E_INVAL;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * (sms > 0 ? sms : 1), threads = 256;
  double *d = nullptr;
  CK(cudaMalloc(&d, (size_t)blocks * threads * sizeof(double)));
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_dfma_loop(d, blocks, threads, 8, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_dfma_loop(d, blocks, threads, iters, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(d);
  CK(e);
  *dfma_per_s = (double)blocks * threads * iters * kDfmaPerIter / (ms * 1e-3);
  return PPL_OK;
}

int ppl_stall_probe(int64_t limit_ns, uint32_t *flags) {
  if (limit_ns <= 0 || limit_ns > 1000000000LL || !flags) return PPL_E_INVAL;
  unsigned *d = nullptr;
  CK(cudaMalloc(&d, sizeof(unsigned)));
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = launch_stall_probe((unsigned long long)limit_ns, d);
  unsigned st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(d);
  CK(e);
  *flags = st;
  return PPL_OK;
}

int ppl_tma_staging(const ppl_t *h) {
  if (!h) return PPL_E_INVAL;
  return h->tmaps ? 1 : 0;
}

int ppl_get_launch(const ppl_t *h, int32_t *rows_per_cta, int32_t *ctas) {
  if (!h) return PPL_E_INVAL;
  if (rows_per_cta) *rows_per_cta = h->rows_per_cta;
  if (ctas) *ctas = (int32_t)(h->grid.x * h->grid.y);
  return PPL_OK;
}

int ppl_autotune(ppl_t *h, int32_t steps, int32_t *best_rows, double *best_ms) {
  if (!h || steps < 1) return PPL_E_INVAL;
  int rc = check_status(h);
  if (rc) return rc;
  // state aside: populations, temperature and the mass sum of the current slot
  const int c0 = h->cur;
  const int64_t step0 = h->step, l0 = h->launches;
  const size_t fbytes = (size_t)9 * h->N * h->rsz, tbytes = (size_t)h->N * h->rsz;
  void *sf = nullptr, *sT = nullptr, *ss = nullptr;
  if (cudaMalloc(&sf, fbytes) != cudaSuccess || cudaMalloc(&sT, tbytes) != cudaSuccess ||
      cudaMalloc(&ss, 4 * sizeof(double)) != cudaSuccess) {
    cudaFree(sf);
    cudaFree(sT);
    cudaFree(ss);
    return PPL_E_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = cuda_err(cudaEventCreate(&e0));
  if (rc == PPL_OK) rc = cuda_err(cudaEventCreate(&e1));
  if (rc == PPL_OK) rc = cuda_err(cudaMemcpyAsync(sf, h->f[c0], fbytes, cudaMemcpyDeviceToDevice, h->stream));
  if (rc == PPL_OK) rc = cuda_err(cudaMemcpyAsync(sT, h->T[c0], tbytes, cudaMemcpyDeviceToDevice, h->stream));
  if (rc == PPL_OK)
    rc = cuda_err(cudaMemcpyAsync(ss, h->stats[c0], 4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));

  auto restore = [&]() -> int {
    CK(cudaMemcpyAsync(h->f[c0], sf, fbytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->T[c0], sT, tbytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->stats[c0], ss, 4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    h->cur = c0;
    h->step = step0;
    h->launches = l0;
    return PPL_OK;
  };

  // candidates: each applicable kernel (FP32: two-column and one-column) x rows per CTA
  std::vector<int> kernels = {PPL_KERNEL_COLUMN};
  if (pair_applicable(h->cfg)) kernels.insert(kernels.begin(), PPL_KERNEL_PAIR);
  int best = 0, best_fill = 0, best_kernel = kernels[0];
  float best_t = -1.0f;
  for (size_t kk = 0; kk < kernels.size() && rc == PPL_OK; ++kk) {
    const StepVariant v = pick_variant(h->cfg, kernels[kk]);
    for (int e = 0; e < 2 && rc == PPL_OK; ++e)
      rc = cuda_err(cudaFuncSetAttribute(v.fn[e], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
    if (rc != PPL_OK) break;
    h->var = v;
    // the default shape (two heights where it applies) and uniform row blocks
    int dH = 0, dF = 0;
    default_shape(h, &dH, &dF);
    std::vector<std::pair<int, int>> cand = {{dH, dF}};
    for (int H : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256})
      if (H <= h->ny && std::find(cand.begin(), cand.end(), std::make_pair(H, 0)) == cand.end()) cand.push_back({H, 0});
    for (size_t i = 0; i < cand.size() && rc == PPL_OK; ++i) {
      rc = apply_shape(h, cand[i].first, cand[i].second);
      if (rc == PPL_OK) rc = ppl_step_async(h, 2);  // warm-up (and graph capture below)
      if (rc == PPL_OK && steps >= kGraphSteps) rc = ppl_step_async(h, kGraphSteps);
      if (rc == PPL_OK) rc = restore();
      if (rc == PPL_OK) rc = cuda_err(cudaEventRecord(e0, h->stream));
      if (rc == PPL_OK) rc = ppl_step_async(h, steps);
      if (rc == PPL_OK) rc = cuda_err(cudaEventRecord(e1, h->stream));
      if (rc == PPL_OK) rc = cuda_err(cudaEventSynchronize(e1));
      float ms = 0.0f;
      if (rc == PPL_OK) rc = cuda_err(cudaEventElapsedTime(&ms, e0, e1));
      if (rc == PPL_OK) rc = restore();
      if (rc == PPL_OK && (best_t < 0.0f || ms < best_t)) {
        best_t = ms;
        best = cand[i].first;
        best_fill = cand[i].second;
        best_kernel = kernels[kk];
      }
    }
  }
  if (rc == PPL_OK) h->var = pick_variant(h->cfg, best_kernel);
  if (rc == PPL_OK) rc = apply_shape(h, best, best_fill);
  if (rc == PPL_OK) rc = cuda_err(cudaStreamSynchronize(h->stream));
  cudaFree(sf);
  cudaFree(sT);
  cudaFree(ss);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == PPL_OK) {
    if (best_rows) *best_rows = best;
    if (best_ms) *best_ms = (double)best_t / steps;
  }
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Droplet radius of Sec. 4.1: liquid area from the density field, and the relative
// change of two R(t) series, Eq. (relative-change-R)
// ---------------------------------------------------------------------------------
namespace {

template <typename real>
__global__ void phase_area_partials(const Params<real> P, const real *f, double lo, double inv_span, double *part) {
  constexpr int NT = 256;
  __shared__ double red[NT / 32];
  double acc = 0.0;
  for (long long k = (long long)blockIdx.x * NT + threadIdx.x; k < P.plane; k += (long long)gridDim.x * NT) {
    const int x = (int)(k % P.nx), y = (int)(k / P.nx);
    const double rho = node_value(P, f, f, x, y, 0);
    acc += fmin(fmax((rho - lo) * inv_span, 0.0), 1.0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void sum_finalize(const double *part, int nblk, double *out) {
  if (threadIdx.x != 0) return;
  double a = 0.0;
  for (int i = 0; i < nblk; ++i) a += part[i];
  out[0] = a;
}

}  // namespace

extern "C" {

int ppl_phase_area(ppl_t *h, double rho_lo, double rho_hi, double *area) {
  if (!h || !area || !(rho_hi > rho_lo)) return PPL_E_INVAL;
  const int nblk = h->stats_blocks;  // partials holds >= kStats * stats_blocks doubles
  const double inv = 1.0 / (rho_hi - rho_lo);
  if (h->prec == PPL_FP64)
    phase_area_partials<double><<<nblk, 256, 0, h->stream>>>(h->pd, (const double *)h->f[h->cur], rho_lo, inv,
                                                             h->partials);
  else if (h->prec == PPL_FP32DEV)
    phase_area_partials<float><<<nblk, 256, 0, h->stream>>>(h->pf, (const float *)h->f[h->cur], rho_lo, inv,
                                                            h->partials);
  else if (is_tangent32(h->prec))
    phase_area_partials<DualF><<<nblk, 256, 0, h->stream>>>(h->ptf, (const DualF *)h->f[h->cur], rho_lo, inv,
                                                            h->partials);
  else
    phase_area_partials<Dual><<<nblk, 256, 0, h->stream>>>(h->pt, (const Dual *)h->f[h->cur], rho_lo, inv,
                                                           h->partials);
  CK(cudaGetLastError());
  sum_finalize<<<1, 32, 0, h->stream>>>(h->partials, nblk, h->norm_out);
  CK(cudaGetLastError());
  double out = 0.0;
  CK(cudaMemcpyAsync(&out, h->norm_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *area = out;
  return PPL_OK;
}

int ppl_relative_change(const double *R, const double *R_star, int64_t n, double *out) {
  if (!R || !R_star || !out || n < 1) return PPL_E_INVAL;
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    num += std::fabs(R[i] - R_star[i]);
    den += std::fabs(R_star[i]);
  }
  if (!(den > 0.0)) return PPL_E_INVAL;
  *out = num / den;
  return PPL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Wall heat flux of Eq. (pool-heat-flux): mean over a boundary line of the conductive flux
// into the domain, lambda(rho) times the inward normal derivative of T, second-order
// one-sided difference
// ---------------------------------------------------------------------------------
namespace {

template <typename real>
__global__ void wall_flux_partials(const Params<real> P, const real *f, const real *T, int side, double *part) {
  constexpr int NT = 256;
  __shared__ double red[NT / 32];
  const bool xs = side < 2;
  const int len = xs ? P.ny : P.nx;
  double acc = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < len; i += gridDim.x * NT) {
    int x[3], y[3];
    for (int k = 0; k < 3; ++k) {
      const int d = (side & 1) ? -k : k;  // k nodes inward from the boundary line
      x[k] = xs ? ((side & 1) ? P.nx - 1 : 0) + d : i;
      y[k] = xs ? i : ((side & 1) ? P.ny - 1 : 0) + d;
    }
    const double t0 = node_value(P, f, T, x[0], y[0], 1), t1 = node_value(P, f, T, x[1], y[1], 1),
                 t2 = node_value(P, f, T, x[2], y[2], 1);
    const double rho = node_value(P, f, T, x[0], y[0], 0);
    const double lam = (double)P.lam_v + (double)P.dlam * (rho - (double)P.rho_v);
    const double dTdn = 0.5 * (-3.0 * t0 + 4.0 * t1 - t2);  // inward normal derivative
    acc += -lam * dTdn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

}  // namespace

extern "C" {

int ppl_wall_heat_flux(ppl_t *h, int side, double *q) {
  if (!h || !q || side < 0 || side > 3 || is_tangent(h->prec)) return PPL_E_INVAL;
  if (h->cfg.hydro_bc[side] == PPL_PERIODIC && h->cfg.thermal_bc[side] == PPL_T_PERIODIC) return PPL_E_INVAL;
  const int len = side < 2 ? h->ny : h->nx;
  if ((side < 2 ? h->nx : h->ny) < 3) return PPL_E_INVAL;
  const int nblk = (len + 255) / 256 < h->stats_blocks ? (len + 255) / 256 : h->stats_blocks;
  if (h->prec == PPL_FP64)
    wall_flux_partials<double><<<nblk, 256, 0, h->stream>>>(h->pd, (const double *)h->f[h->cur],
                                                            (const double *)h->T[h->cur], side, h->partials);
  else
    wall_flux_partials<float><<<nblk, 256, 0, h->stream>>>(h->pf, (const float *)h->f[h->cur],
                                                           (const float *)h->T[h->cur], side, h->partials);
  CK(cudaGetLastError());
  sum_finalize<<<1, 32, 0, h->stream>>>(h->partials, nblk, h->norm_out);
  CK(cudaGetLastError());
  double out = 0.0;
  CK(cudaMemcpyAsync(&out, h->norm_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *q = out / len;
  return PPL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Contact angle of a droplet on a wall (Sec. 4.3.1), from a host density field
// ---------------------------------------------------------------------------------
namespace {

// first crossing of `level` walking from index 0 along a strided profile; NaN if none
double first_crossing(const double *v, long long stride, int n, double level) {
  for (int i = 0; i + 1 < n; ++i) {
    const double a = v[(long long)i * stride], b = v[(long long)(i + 1) * stride];
    if ((a - level) * (b - level) <= 0.0 && a != b) return i + (a - level) / (a - b);
  }
  return std::nan("");
}

}  // namespace

extern "C" {

int ppl_contact_angle(const double *rho, int32_t nx, int32_t ny, int side, double rho_mid, double *theta) {
  if (!rho || !theta || nx < 3 || ny < 3 || side < 0 || side > 3) return PPL_E_INVAL;
  // walk the wall line (index s) and the inward direction (index n) with strides
  const bool xs = side < 2;
  const int L = xs ? ny : nx, D = xs ? nx : ny;
  const long long s_stride = xs ? nx : 1;
  const long long n_stride = (xs ? 1 : (long long)nx) * ((side & 1) ? -1 : 1);
  const long long origin = (side & 1) ? (xs ? nx - 1 : (long long)(ny - 1) * nx) : 0;
  // base line: the first line from the wall inward whose densest node is liquid with a
  // crossing on each side (a density layer on the wall line can hide the foot there)
  for (int n0 = 0; n0 < D / 2; ++n0) {
    const double *line = rho + origin + n0 * n_stride;
    int cx = 0;
    for (int s = 1; s < L; ++s)
      if (line[s * s_stride] > line[cx * s_stride]) cx = s;
    if (!(line[cx * s_stride] > rho_mid)) continue;
    const double *foot = line + cx * s_stride;
    const double right = cx + first_crossing(foot, s_stride, L - cx, rho_mid);
    const double left = cx - first_crossing(foot, -s_stride, cx + 1, rho_mid);
    if (!std::isfinite(right) || !std::isfinite(left)) continue;
    const double a = 0.5 * (right - left);
    const int centre = (int)std::lround(0.5 * (right + left));
    if (centre < 0 || centre >= L) return PPL_E_INVAL;
    const double up = first_crossing(line + centre * s_stride, n_stride, D - n0, rho_mid);
    if (!std::isfinite(up) || !(up > 0.0)) return PPL_E_INVAL;
    // circle through (+-a, n0) and (0, n0 + up); its centre sits at height h - Rc
    const double Rc = (a * a + up * up) / (2.0 * up);
    const double yc = n0 + up - Rc;
    const double q = std::fmax(-1.0, std::fmin(1.0, yc / Rc));
    *theta = 90.0 + std::asin(q) * (180.0 / 3.14159265358979323846);
    return PPL_OK;
  }
  return PPL_E_INVAL;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Time-shift search of Eq. (rel-diff-minimize)
// ---------------------------------------------------------------------------------
extern "C" {

int ppl_time_shift(ppl_t *coarse, const ppl_t *finest, int field, int64_t m, int64_t stride, int64_t *delta,
                   double *num_min) {
  if (!coarse || !finest || !delta || (field != 0 && field != 1) || m < 0 || stride < 1) return PPL_E_INVAL;
  for (int s = 0; s < 4; ++s)
    if (coarse->cfg.hydro_bc[s] != finest->cfg.hydro_bc[s]) return PPL_E_INVAL;
  int64_t best_d = 0;
  double best = -1.0;
  for (int64_t d = -m; d <= m; d += stride) {
    double num = 0.0, den = 0.0;
    int rc = ppl_cross_norm(coarse, finest, field, &num, &den);
    if (rc) return rc;
    if (best < 0.0 || num < best) {
      best = num;
      best_d = d;
    }
    if (d + stride <= m) {
      rc = ppl_step(coarse, stride);
      if (rc) return rc;
    }
  }
  *delta = best_d;
  if (num_min) *num_min = best;
  return PPL_OK;
}

}  // extern "C"
