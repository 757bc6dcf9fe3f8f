// FP32 sensitivity instantiation of the fused row step: FP32 values (stored as deviations,
// like the FP32 step) carrying their derivative with respect to sigma or kappa; compiled
// like the FP32 step (approximate division and square root).
#include "row_step.cuh"
#include "step_variants.h"

namespace ppl_dev {

template <bool ENERGY>
static const void *tangent32_fn() {
  return (const void *)row_step<DualF, ENERGY, kNTDF, kPFDF>;
}

StepVariant step_variant_tangent32() {
  StepVariant v;
  v.nt = kNTDF;
  v.width = kNTDF - 6;
  v.smem = row_step_smem_bytes<kNTDF, kPFDF, DualF>();
  v.fn[0] = tangent32_fn<false>();
  v.fn[1] = tangent32_fn<true>();
  return v;
}

}  // namespace ppl_dev
