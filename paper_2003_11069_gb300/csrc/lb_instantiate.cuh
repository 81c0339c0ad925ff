// lb_instantiate.cuh -- launch wrappers for one storage type T; included once per
// precision translation unit.
#pragma once

#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbnci {
namespace {

template <int LAT>
dim3 tiled_grid(const StepParams& p) {
  return dim3((p.nx + Tile<LAT>::X - 1) / Tile<LAT>::X, (p.ny + Tile<LAT>::Y - 1) / Tile<LAT>::Y,
              (p.nz + Tile<LAT>::Z - 1) / Tile<LAT>::Z);
}
template <int LAT> dim3 tiled_block() { return dim3(Tile<LAT>::X, Tile<LAT>::Y, Tile<LAT>::Z); }

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <int LAT, typename T>
cudaError_t l_init(void* f, const double* r1, const double* r2, const double* u, long long N,
                   cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  init_kernel<LAT, T><<<blocks_for(N, 256), 256, 0, s>>>((T*)f, r1, r2, u, N);
  return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t l_moments(const void* f, void* psi, const StepParams& p, cudaStream_t s) {
  moments_kernel<LAT, T><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, (T*)psi, p);
  return cudaGetLastError();
}

template <int LAT, typename T, bool FIELDS>
cudaError_t set_smem(size_t bytes) {
  static size_t configured = 0;
  if (bytes <= 48 * 1024 || bytes <= configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(collide_kernel<LAT, T, FIELDS>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) configured = bytes;
  return e;
}

template <int LAT, typename T>
cudaError_t l_collide(const void* f, void* fout, const void* psi, const StepParams& p, cudaStream_t s) {
  const size_t sm = collide_smem_bytes<LAT, T>(p.smax);
  cudaError_t e = set_smem<LAT, T, false>(sm);
  if (e != cudaSuccess) return e;
  FieldOut fo{};
  collide_kernel<LAT, T, false><<<tiled_grid<LAT>(p), tiled_block<LAT>(), sm, s>>>(
      (const T*)f, (T*)fout, (const T*)psi, p, fo);
  return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t l_fields(const void* f, const void* psi, const StepParams& p, const FieldOut& fo,
                     cudaStream_t s) {
  const size_t sm = collide_smem_bytes<LAT, T>(p.smax);
  cudaError_t e = set_smem<LAT, T, true>(sm);
  if (e != cudaSuccess) return e;
  collide_kernel<LAT, T, true><<<tiled_grid<LAT>(p), tiled_block<LAT>(), sm, s>>>(
      (const T*)f, nullptr, (const T*)psi, p, fo);
  return cudaGetLastError();
}

template <typename T>
cudaError_t l_to_f64(const void* src, double* dst, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  convert_kernel<T, double><<<blocks_for(n, 256), 256, 0, s>>>((const T*)src, dst, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t l_from_f64(const double* src, void* dst, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  convert_kernel<double, T><<<blocks_for(n, 256), 256, 0, s>>>(src, (T*)dst, n);
  return cudaGetLastError();
}

template <int LAT, typename T>
const Launchers* table() {
  static const Launchers L = {sizeof(T), l_init<LAT, T>, l_moments<LAT, T>, l_collide<LAT, T>,
                              l_fields<LAT, T>, l_to_f64<T>, l_from_f64<T>};
  return &L;
}

}  // namespace
}  // namespace lbnci
