// FP64 instantiation of the per-step kernels (particle and grid state in double).
#include "apic_batch.cuh"

namespace apic {
APIC_DEFINE_PRECISION(double, f64)
APIC_DEFINE_BATCH(double, f64)
}  // namespace apic
