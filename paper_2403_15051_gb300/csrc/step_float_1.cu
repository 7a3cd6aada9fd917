// Instantiation of the persistent step kernel for float populations, geometry 1 (0 cylinder, 1 sphere).
#include "step_kernel.cuh"

namespace fdlb {
FDLB_STEP_INSTANCE(float, 1)
}  // namespace fdlb
