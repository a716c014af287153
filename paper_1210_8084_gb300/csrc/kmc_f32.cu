// kmc_f32.cu -- binary32-state instantiation of the step kernels.
#include "kmc_kernels.cuh"

namespace kmc {
KMC_INSTANTIATE(float)
}  // namespace kmc
