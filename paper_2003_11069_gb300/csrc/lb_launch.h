// lb_launch.h -- internal launch table between the C ABI (lb_api.cu) and the
// per-precision kernel instantiations (lb_fp64.cu, lb_fp32.cu).
#pragma once

#include <cuda_runtime.h>

#include "lb_lattice.cuh"

namespace lbnci {

struct Launchers {
  size_t elem;  // bytes per stored population
  cudaError_t (*init)(void* f, const double* rho1, const double* rho2, const double* u,
                      long long N, cudaStream_t s);
  cudaError_t (*moments)(const void* f, void* psi, const StepParams& p, cudaStream_t s);
  cudaError_t (*collide)(const void* f, void* fout, const void* psi, const StepParams& p,
                         cudaStream_t s);
  cudaError_t (*fields)(const void* f, const void* psi, const StepParams& p, const FieldOut& fo,
                        cudaStream_t s);
  cudaError_t (*to_f64)(const void* src, double* dst, long long n, cudaStream_t s);
  cudaError_t (*from_f64)(const double* src, void* dst, long long n, cudaStream_t s);
};

const Launchers* launchers_fp64(int lattice);
const Launchers* launchers_fp32(int lattice);

// Number of thread blocks of the tiled kernels (= partial-sum slots of the fields kernel).
long long tiled_blocks(int lattice, const StepParams& p);
cudaError_t reduce_partials(const double* partials, long long nblocks, double* out, cudaStream_t s);

}  // namespace lbnci
