// inst_3d_k4.cu -- kernels of the 3D operator at order 4 (5 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_4() { return Ops<3, 5>::table(); }
}  // namespace feod
