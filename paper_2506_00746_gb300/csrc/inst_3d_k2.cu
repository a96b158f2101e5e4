// inst_3d_k2.cu -- kernels of the 3D operator at order 2 (3 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_2() { return Ops<3, 3>::table(); }
}  // namespace feod
