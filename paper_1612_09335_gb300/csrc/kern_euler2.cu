// Kernel instantiations: dimension 2, Euler, M = 1..4, FP64 and FP32-mixed.
#include "kernels.cuh"

namespace cw {

std::unique_ptr<Ops> make_ops_euler2(int M, int fp32, const RefElem& re) {
  switch (M * 2 + (fp32 ? 1 : 0)) {
    case 2: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 1, 0, double>>(re));
    case 3: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 1, 0, float>>(re));
    case 4: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 2, 0, double>>(re));
    case 5: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 2, 0, float>>(re));
    case 6: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 3, 0, double>>(re));
    case 7: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 3, 0, float>>(re));
    case 8: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 4, 0, double>>(re));
    case 9: return std::unique_ptr<Ops>(new OpsImpl<Cfg<2, 4, 0, float>>(re));
    default: return nullptr;
  }
}

}  // namespace cw
