// inst_3d_k6.cu -- kernels of the 3D operator at order 6 (7 nodes / Gauss points per direction).
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_3d_6() { return Ops<3, 7>::table(); }
}  // namespace feod
