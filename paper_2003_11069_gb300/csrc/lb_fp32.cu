// lb_fp32.cu -- FP32 populations and arithmetic.
#include "lb_instantiate.cuh"

namespace lbnci {
const Launchers* launchers_fp32(int lattice) {
  return lattice == 0 ? table<0, Plain<0, float>>() : table<1, Plain<1, float>>();
}
}  // namespace lbnci
