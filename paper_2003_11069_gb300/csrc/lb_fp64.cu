// lb_fp64.cu -- FP64 instantiation of the step kernels. Built with --fmad=false so
// that no multiply-add is contracted: the arithmetic then rounds exactly as the
// written expressions do, which is what per-step parity at 1e-12 relies on.
#include "lb_instantiate.cuh"

namespace lbnci {
const Launchers* launchers_fp64(int lattice) {
  return lattice == 0 ? table<0, double>() : table<1, double>();
}
}  // namespace lbnci
