// Sensitivity instantiation of the fused row step: FP64 values carrying their derivative
// with respect to sigma or kappa (forward mode, IEEE arithmetic).
#include "row_step.cuh"
#include "step_variants.h"

namespace ppl_dev {

template <bool ENERGY>
static const void *tangent_fn() {
  return (const void *)row_step<Dual, ENERGY, kNTD, kPFD>;
}

StepVariant step_variant_tangent() {
  StepVariant v;
  v.nt = kNTD;
  v.width = kNTD - 6;
  v.smem = row_step_smem_bytes<kNTD, kPFD, Dual>();
  v.fn[0] = tangent_fn<false>();
  v.fn[1] = tangent_fn<true>();
  return v;
}

}  // namespace ppl_dev
