// Kernel instantiations: dimension 3, PDE 0 (0 Euler, 1 MHD-GLM), M = 1..3,
// FP64 and FP32-mixed; M = 4 in kern_euler3_p4.cu and kern_euler3_p4f.cu.
#include "kernels.cuh"

namespace cw {

std::unique_ptr<Ops> make_ops_euler3(int M, int fp32, const RefElem& re) {
  switch (M * 2 + (fp32 ? 1 : 0)) {
    case 2: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 1, 0, double>>(re));
    case 3: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 1, 0, float>>(re));
    case 4: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 2, 0, double>>(re));
    case 5: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 2, 0, float>>(re));
    case 6: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 3, 0, double>>(re));
    case 7: return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 3, 0, float>>(re));
    case 8:
    case 9: return make_ops_euler3_p4(fp32, re);
    default: return nullptr;
  }
}

}  // namespace cw
