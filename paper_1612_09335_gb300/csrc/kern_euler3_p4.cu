// Kernel instantiations: dimension 3, Euler, M = 4 (fifth order), FP64.  The
// FP32-mixed instance is in kern_euler3_p4f.cu, so that the two largest
// instances compile in parallel.
#include "kernels.cuh"

namespace cw {

std::unique_ptr<Ops> make_ops_euler3_p4f(const RefElem& re);

std::unique_ptr<Ops> make_ops_euler3_p4(int fp32, const RefElem& re) {
  if (fp32) return make_ops_euler3_p4f(re);
  return std::unique_ptr<Ops>(new OpsImpl<Cfg<3, 4, 0, double>>(re));
}

}  // namespace cw
