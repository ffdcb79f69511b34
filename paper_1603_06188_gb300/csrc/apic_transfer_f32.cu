// FP32 instantiation of the per-step kernels (particle and grid state in float; momentum
// totals still accumulate in double).
#include "apic_batch.cuh"

namespace apic {
APIC_DEFINE_PRECISION(float, f32)
APIC_DEFINE_BATCH(float, f32)
}  // namespace apic
