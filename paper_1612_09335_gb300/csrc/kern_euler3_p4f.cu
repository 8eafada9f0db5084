// Kernel instantiations: dimension 3, Euler, M = 4 (fifth order), FP32-mixed.
#include "kernels.cuh"

namespace cw {

std::unique_ptr<Ops> make_ops_euler3_p4f(const RefElem& re) {
  return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 4, 0, float>>(re));
}

}  // namespace cw
