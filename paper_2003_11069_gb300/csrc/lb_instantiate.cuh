// lb_instantiate.cuh -- launch wrappers for one storage type T; included once per
// precision translation unit.
#pragma once

#include "lb_fused2d.cuh"
#include "lb_kernels.cuh"
#include "lb_launch.h"

namespace lbnci {
namespace {

template <typename T>
StepT<T> convert(const HostParams& h) {
  StepT<T> p;
  p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.wall_y = h.wall_y; p.wall_z = h.wall_z;
  p.N = h.N; p.smax = h.smax;
  // Derived constants computed in T exactly as the per-site formulas would.
  p.omega = T(1) / T(h.tau);
  p.guo = T(1) - T(0.5) * p.omega;
  p.pamp = T(2) * (T(0.5) * T(h.A_s));
  p.beta = T(h.beta);
  p.g_th = T(h.g_th);
  for (int a = 0; a < 3; ++a) p.G[a] = T(h.G[a]);
  // A_h(h): A for h <= h_min, A (h_min/h)^3 for h_min < h <= h_max, 0 beyond (Eq. near_c).
  for (int k = 0; k < 8; ++k) {
    const T hd = T(k), hmin = T(h.h_min), hmax = T(h.h_max), A = T(h.A_h);
    if (k == 0) p.Ah[k] = T(0);
    else if (hd <= hmin) p.Ah[k] = A;
    else if (hd <= hmax) { const T r = hmin / hd; p.Ah[k] = A * (r * r * r); }
    else p.Ah[k] = T(0);
  }
  return p;
}

template <int LAT>
dim3 tiled_grid(const HostParams& p) {
  return dim3((p.nx + Tile<LAT>::X - 1) / Tile<LAT>::X, (p.ny + Tile<LAT>::Y - 1) / Tile<LAT>::Y,
              (p.nz + Tile<LAT>::Z - 1) / Tile<LAT>::Z);
}
template <int LAT> dim3 tiled_block() { return dim3(Tile<LAT>::X, Tile<LAT>::Y, Tile<LAT>::Z); }

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes, size_t* configured) {
  if (bytes <= 48 * 1024 || bytes <= *configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *configured = bytes;
  return e;
}

// Sites per thread of the fused D2Q9 kernel (2: 32x16 tiles, 4: 32x32 tiles).
template <typename T, int SPT>
cudaError_t launch_fused2d(const void* fa, void* fb, const StepT<T>& p, cudaStream_t s) {
  static size_t configured = 0;
  const size_t sm = fused2d_smem_bytes<T>(p.smax, SPT);
  cudaError_t e = allow_smem(fused2d_kernel<T, SPT>, sm, &configured);
  if (e != cudaSuccess) return e;
  const dim3 grid((p.nx + kFusedTX - 1) / kFusedTX, (p.ny + kFusedThreadsY * SPT - 1) / (kFusedThreadsY * SPT), 1);
  fused2d_kernel<T, SPT><<<grid, dim3(kFusedTX, kFusedThreadsY, 1), sm, s>>>((const T*)fa, (T*)fb, p);
  return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t l_init(void* f, const double* r1, const double* r2, const double* u, const HostParams& p,
                   cudaStream_t s) {
  if (p.N == 0) return cudaSuccess;
  init_kernel<LAT, T><<<blocks_for(p.N, 256), 256, 0, s>>>((T*)f, r1, r2, u, p.N);
  return cudaGetLastError();
}

template <int LAT, typename T, bool FIELDS>
cudaError_t launch_tiled(const void* f, void* fout, const void* psi, const StepT<T>& p, const FieldOut& fo,
                         cudaStream_t s) {
  static size_t configured = 0;
  const size_t sm = tiled_smem_bytes<LAT, T>(p.smax);
  cudaError_t e = allow_smem(tiled_kernel<LAT, T, FIELDS>, sm, &configured);
  if (e != cudaSuccess) return e;
  HostParams hp{};
  hp.nx = p.nx; hp.ny = p.ny; hp.nz = p.nz;
  tiled_kernel<LAT, T, FIELDS><<<tiled_grid<LAT>(hp), tiled_block<LAT>(), sm, s>>>(
      (const T*)f, (T*)fout, (const T*)psi, p, fo);
  return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t l_step(const void* fa, void* fb, void* psi, const HostParams& h, cudaStream_t s, int* nk) {
  const StepT<T> p = convert<T>(h);
  if (LAT == 0) {
    *nk = 1;
    return h.spt == 4 ? launch_fused2d<T, 4>(fa, fb, p, s) : launch_fused2d<T, 2>(fa, fb, p, s);
  }
  moments_kernel<LAT, T><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)fa, (T*)psi, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *nk = 2;
  return launch_tiled<LAT, T, false>(fa, fb, psi, p, FieldOut{}, s);
}

template <int LAT, typename T>
cudaError_t l_fields(const void* f, void* psi, const HostParams& h, const FieldOut& fo, cudaStream_t s, int* nk) {
  const StepT<T> p = convert<T>(h);
  moments_kernel<LAT, T><<<blocks_for(p.N, 256), 256, 0, s>>>((const T*)f, (T*)psi, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *nk = 2;
  return launch_tiled<LAT, T, true>(f, nullptr, psi, p, fo, s);
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
  static const Launchers L = {sizeof(T), l_init<LAT, T>, l_step<LAT, T>, l_fields<LAT, T>, l_to_f64<T>,
                              l_from_f64<T>};
  return &L;
}

}  // namespace
}  // namespace lbnci
