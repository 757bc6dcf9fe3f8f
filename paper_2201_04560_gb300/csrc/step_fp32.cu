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
  return (const void *)row_step_pair<ENERGY, kNTP, kPFP>;
}

StepVariant step_variant_fp32_pair() {
  StepVariant v;
  v.nt = kNTP;
  v.width = 2 * kNTP - 8;
  v.smem = row_step_pair_smem_bytes<kNTP, kPFP>();
  v.fn[0] = fp32_pair_fn<false>();
  v.fn[1] = fp32_pair_fn<true>();
  return v;
}

}  // namespace ppl_dev
