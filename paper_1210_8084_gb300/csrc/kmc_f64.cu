// kmc_f64.cu -- binary64-state instantiation of the step kernels.
#include "kmc_kernels.cuh"

namespace kmc {
KMC_INSTANTIATE(double)
}  // namespace kmc
