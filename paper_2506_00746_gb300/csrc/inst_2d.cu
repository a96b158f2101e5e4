// inst_2d.cu -- kernels of the 2D operator, orders 1..6.
#include "element_kernels.cuh"

namespace feod {
const OpTable *ops_2d(int d1)
{
    switch (d1) {
    case 2: return Ops<2, 2>::table();
    case 3: return Ops<2, 3>::table();
    case 4: return Ops<2, 4>::table();
    case 5: return Ops<2, 5>::table();
    case 6: return Ops<2, 6>::table();
    case 7: return Ops<2, 7>::table();
    default: return nullptr;
    }
}
}  // namespace feod
