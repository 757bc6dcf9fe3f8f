// FP64 instantiations of the fused row step (IEEE division and square root).
#include "row_step.cuh"
#include "step_variants.h"

namespace ppl_dev {

template <bool ENERGY>
static const void *fp64_fn() {
  return (const void *)row_step<double, ENERGY, kNT64, kPF64>;
}

StepVariant step_variant_fp64() {
  StepVariant v;
  v.nt = kNT64;
  v.width = kNT64 - 6;
  v.smem = row_step_smem_bytes<kNT64, kPF64, double>();
  v.fn[0] = fp64_fn<false>();
  v.fn[1] = fp64_fn<true>();
  return v;
}

}  // namespace ppl_dev
