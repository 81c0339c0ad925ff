// lb_fp64.cu -- FP64 populations and arithmetic. Built with --fmad=false so that no
// multiply-add is contracted: the arithmetic then rounds exactly as the written
// expressions do, which is what per-step parity with the FP64 oracle relies on.
#include "lb_instantiate.cuh"

namespace lbnci {
const Launchers* launchers_fp64(int lattice) {
  return lattice == 0 ? table<0, Plain<0, double>>() : table<1, Plain<1, double>>();
}
}  // namespace lbnci
