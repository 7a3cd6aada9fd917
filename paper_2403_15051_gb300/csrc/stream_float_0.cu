// Instantiation of the fused stage kernel for float populations, geometry 0 (0 cylinder, 1 sphere).
#include "stream_kernel.cuh"

namespace fdlb {
FDLB_STREAM_INSTANCE(float, 0)
}  // namespace fdlb
