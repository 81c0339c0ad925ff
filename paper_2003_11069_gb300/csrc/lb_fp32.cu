// lb_fp32.cu -- FP32 instantiation of the step kernels (storage and arithmetic in FP32).
#include "lb_instantiate.cuh"

namespace lbnci {
const Launchers* launchers_fp32(int lattice) {
  return lattice == 0 ? table<0, float>() : table<1, float>();
}
}  // namespace lbnci
