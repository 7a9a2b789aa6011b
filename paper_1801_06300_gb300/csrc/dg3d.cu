// DG operator kernels on tetrahedra (D = 3): instantiation of dg_kernels.cuh.
#include "dg_kernels.cuh"

namespace pcexp {
PCEXP_INST_D(double, 3)
PCEXP_INST_D(float, 3)
template cudaError_t launch_tan_tables_d<3>(const DGData<float>&, cudaStream_t);
}  // namespace pcexp
