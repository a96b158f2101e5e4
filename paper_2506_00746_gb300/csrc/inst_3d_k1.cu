// inst_3d_k1.cu -- kernels of the 3D operator at order 1 (2 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_1() { return Ops<3, 2>::table(); }
}  // namespace feod
