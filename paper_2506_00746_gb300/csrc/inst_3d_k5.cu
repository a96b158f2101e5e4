// inst_3d_k5.cu -- kernels of the 3D operator at order 5 (6 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_5() { return Ops<3, 6>::table(); }
}  // namespace feod
