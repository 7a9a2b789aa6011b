// DG operator kernels on triangles (D = 2): instantiation of dg_kernels.cuh.
#include "dg_kernels.cuh"

namespace pcexp {
PCEXP_INST_D(double, 2)
PCEXP_INST_D(float, 2)
}  // namespace pcexp
