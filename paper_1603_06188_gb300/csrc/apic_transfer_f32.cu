// FP32 instantiation of the per-step kernels (particle and grid state in float; momentum
// totals still accumulate in double).
#include "apic_transfer.cuh"

namespace apic {
APIC_DEFINE_PRECISION(float, f32)
}  // namespace apic
