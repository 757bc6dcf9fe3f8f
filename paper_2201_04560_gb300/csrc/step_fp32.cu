// FP32 instantiations of the fused row step (compiled with approximate division and
// square root: the FP32 path's error budget is set against the FP64 oracle).
#include "row_step.cuh"
#include "row_step_pair.cuh"
#include "step_variants.h"

namespace ppl_dev {

template <bool ENERGY>
static const void *fp32_fn() {
  return (const void *)row_step<float, ENERGY, kNT32, kPF32>;
}

StepVariant step_variant_fp32() {
  StepVariant v;
  v.nt = kNT32;
  v.width = kNT32 - 6;
  v.smem = row_step_smem_bytes<kNT32, kPF32, float>();
  v.fn[0] = fp32_fn<false>();
  v.fn[1] = fp32_fn<true>();
  return v;
}

template <bool ENERGY>
static const void *fp32_pair_fn() {
  return (const void *)row_step_pair<ENERGY, kNTP>;
}

StepVariant step_variant_fp32_pair() {
  StepVariant v;
  v.nt = kNTP;
  v.width = 2 * kNTP - 8;
  v.smem = row_step_pair_smem_bytes<kNTP>();
  v.fn[0] = fp32_pair_fn<false>();
  v.fn[1] = fp32_pair_fn<true>();
  return v;
}

// Wait-limit probe: one CTA waits, through the bounded mbarrier wait of the TMA row staging,
// on an mbarrier that nothing arrives at; the wait runs out after limit_ns and the CTA reports
// FLAG_STALL in the status word, as the step kernel does for a row that never lands.
__global__ void stall_probe(unsigned long long limit_ns, unsigned *status) {
  __shared__ unsigned long long bar;
  const unsigned b = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool landed = mbar_wait(b, 0, limit_ns);
  if (__syncthreads_or(!landed) && threadIdx.x == 0) atomicOr(status, FLAG_STALL);
}

cudaError_t launch_stall_probe(unsigned long long limit_ns, unsigned *status) {
  stall_probe<<<1, 64>>>(limit_ns, status);
  return cudaGetLastError();
}

}  // namespace ppl_dev
