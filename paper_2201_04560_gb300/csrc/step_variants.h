// Launch shapes of the fused row step and the host-side handles of its instantiations.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

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
constexpr int kPFP = 1;

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

}  // namespace ppl_dev
