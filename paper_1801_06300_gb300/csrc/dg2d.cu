// DG operator kernels on triangles (D = 2): instantiation of dg_kernels.cuh.
#include "dg_kernels.cuh"

namespace pcexp {
PCEXP_INST_D(double, 2)
PCEXP_INST_D(float, 2)
template cudaError_t launch_tan_tables_d<2>(const DGData<float>&, cudaStream_t);
}  // namespace pcexp
