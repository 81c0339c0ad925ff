// lb_fp16.cu -- populations stored as FP16 deviations from the lattice-weight
// equilibrium at rest (plus FP32 reference densities), arithmetic in FP32.
#include "lb_instantiate.cuh"

namespace lbnci {
const Launchers* launchers_fp16dev(int lattice) {
  return lattice == 0 ? table<0, HalfDev<0>>() : table<1, HalfDev<1>>();
}
}  // namespace lbnci
