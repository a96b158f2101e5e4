// inst_3d_k3.cu -- kernels of the 3D operator at order 3 (4 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_3() { return Ops<3, 4>::table(); }
}  // namespace feod
