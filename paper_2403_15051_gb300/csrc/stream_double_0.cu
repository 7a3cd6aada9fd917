// Instantiation of the fused stage kernel for double populations, geometry 0 (0 cylinder, 1 sphere).
#include "stream_kernel.cuh"

namespace fdlb {
FDLB_STREAM_INSTANCE(double, 0)
}  // namespace fdlb
