// lb_instantiate.cuh -- launch wrappers for one storage layout; included once per
// storage translation unit.
#pragma once

#include "lb_fused2d.cuh"
#include "lb_march3d.cuh"
#include "lb_kernels.cuh"
#include "lb_launch.h"

#include <cstring>

namespace lbnci {
namespace {

template <typename T>
StepT<T> convert(const HostParams& h) {
  StepT<T> p;
  p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.wall_y = h.wall_y; p.wall_z = h.wall_z;
  p.N = h.N; p.smax = h.smax;
  p.edm = h.forcing == 1;
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
  p.seedw = h.seedw;
  p.parity = h.parity;
  return p;
}

template <int LAT>
dim3 tiled_grid(const HostParams& p) {
  return dim3((p.nx + Tile<LAT>::X - 1) / Tile<LAT>::X, (p.ny + Tile<LAT>::Y - 1) / Tile<LAT>::Y,
              (p.nz + Tile<LAT>::Z - 1) / Tile<LAT>::Z);
}
template <int LAT> dim3 tiled_block() { return dim3(Tile<LAT>::X, Tile<LAT>::Y, Tile<LAT>::Z); }

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }


// Sites per thread of the fused D2Q9 kernel (2: 32x16 tiles, 4: 32x32 tiles).
// FP32 kernels come in a Guo and an EDM build; FP64 has one (it checks p.edm itself).
template <typename ST>
constexpr bool edm_build_exists() { return !std::is_same<typename ST::Compute, double>::value; }

template <typename ST, int SPT, bool EDM>
cudaError_t launch_fused2d_v(const void* fa, void* fb, const StepT<typename ST::Compute>& p, cudaStream_t s) {
  using T = typename ST::Compute;
  static SmemAllowance configured;
  const size_t sm = fused2d_smem_bytes<T>(p.smax, SPT);
  cudaError_t e = allow_smem(fused2d_kernel<ST, SPT, EDM>, sm, configured);
  if (e != cudaSuccess) return e;
  const dim3 grid((p.nx + kFusedTX - 1) / kFusedTX, (p.ny + kFusedThreadsY * SPT - 1) / (kFusedThreadsY * SPT), 1);
  fused2d_kernel<ST, SPT, EDM><<<grid, dim3(kFusedTX, kFusedThreadsY, 1), sm, s>>>(
      ST::reader(fa, (unsigned)p.N), ST::writer(fb, (unsigned)p.N), p);
  return cudaGetLastError();
}

template <typename ST, int SPT>
cudaError_t launch_fused2d(const void* fa, void* fb, const StepT<typename ST::Compute>& p, cudaStream_t s) {
  if constexpr (edm_build_exists<ST>()) {
    if (p.edm) return launch_fused2d_v<ST, SPT, true>(fa, fb, p, s);
  }
  return launch_fused2d_v<ST, SPT, false>(fa, fb, p, s);
}

template <int LAT, typename ST>
cudaError_t l_init(void* f, const double* r1, const double* r2, const double* u, const HostParams& p,
                   cudaStream_t s) {
  if (p.N == 0) return cudaSuccess;
  init_kernel<LAT, ST><<<blocks_for(p.N, 256), 256, 0, s>>>(ST::writer(f, (unsigned)p.N), r1, r2, u, p.N);
  return cudaGetLastError();
}

template <int LAT, typename ST, bool FIELDS, bool EDM = false>
cudaError_t launch_tiled_v(const void* f, void* fout, const void* psi, const HostParams& h,
                           const StepT<typename ST::Compute>& p, const FieldOut& fo, cudaStream_t s) {
  using T = typename ST::Compute;
  static SmemAllowance configured;
  const size_t sm = tiled_smem_bytes<LAT, T>(p.smax);
  cudaError_t e = allow_smem(tiled_kernel<LAT, ST, FIELDS, EDM>, sm, configured);
  if (e != cudaSuccess) return e;
  typename ST::Writer w = FIELDS ? typename ST::Writer{} : ST::writer(fout, (unsigned)p.N);
  tiled_kernel<LAT, ST, FIELDS, EDM><<<tiled_grid<LAT>(h), tiled_block<LAT>(), sm, s>>>(
      ST::reader(f, (unsigned)p.N), w, (const T*)psi, p, fo);
  return cudaGetLastError();
}

template <int LAT, typename ST, bool FIELDS>
cudaError_t launch_tiled(const void* f, void* fout, const void* psi, const HostParams& h,
                         const StepT<typename ST::Compute>& p, const FieldOut& fo, cudaStream_t s) {
  if constexpr (!FIELDS && edm_build_exists<ST>()) {
    if (p.edm) return launch_tiled_v<LAT, ST, false, true>(f, fout, psi, h, p, fo, s);
  }
  return launch_tiled_v<LAT, ST, FIELDS, false>(f, fout, psi, h, p, fo, s);
}

// D3Q27 collision marching along z (after moments_kernel has written psi), built for
// each number of probe steps S = smax.
template <typename ST, bool EDM, int S>
cudaError_t launch_march3d_v(const void* fa, void* fb, const void* psi, const HostParams& h,
                             const StepT<typename ST::Compute>& p, cudaStream_t s) {
  using T = typename ST::Compute;
  static SmemAllowance configured;
  const size_t sm = march3d_smem_bytes<T>(S);
  cudaError_t e = allow_smem(march3d_kernel<ST, EDM, S>, sm, configured);
  if (e != cudaSuccess) return e;
  constexpr int TX = MarchTile<T>::TX, TY = MarchTile<T>::TY;
  const int bx = (p.nx + TX - 1) / TX, by = (p.ny + TY - 1) / TY;
  // one CTA per SM (the rings fill its shared memory), each with an equal share of the
  // columns' planes (a grid of bx by z-segment blocks left a partial second wave)
  const long long work = (long long)bx * by * p.nz;
  long long grid = (long long)h.num_sms;
  if (grid > work) grid = work;
  march3d_kernel<ST, EDM, S><<<(unsigned)grid, dim3(TX, TY, 1), sm, s>>>(
      ST::reader(fa, (unsigned)p.N), ST::writer(fb, (unsigned)p.N), (const T*)psi, p, bx, work);
  return cudaGetLastError();
}

template <typename ST, bool EDM>
cudaError_t launch_march3d_s(const void* fa, void* fb, const void* psi, const HostParams& h,
                             const StepT<typename ST::Compute>& p, cudaStream_t s) {
  static_assert(kMaxProbe == 4, "one build per probe count");
  switch (p.smax) {
    case 0: return launch_march3d_v<ST, EDM, 0>(fa, fb, psi, h, p, s);
    case 1: return launch_march3d_v<ST, EDM, 1>(fa, fb, psi, h, p, s);
    case 2: return launch_march3d_v<ST, EDM, 2>(fa, fb, psi, h, p, s);
    case 3: return launch_march3d_v<ST, EDM, 3>(fa, fb, psi, h, p, s);
    default: return launch_march3d_v<ST, EDM, 4>(fa, fb, psi, h, p, s);
  }
}

template <typename ST>
cudaError_t launch_march3d(const void* fa, void* fb, const void* psi, const HostParams& h,
                           const StepT<typename ST::Compute>& p, cudaStream_t s) {
  if constexpr (edm_build_exists<ST>()) {
    if (p.edm) return launch_march3d_s<ST, true>(fa, fb, psi, h, p, s);
  }
  return launch_march3d_s<ST, false>(fa, fb, psi, h, p, s);
}

template <int LAT, typename ST>
cudaError_t l_step(const void* fa, void* fb, void* psi, const HostParams& h, cudaStream_t s, int* nk) {
  using T = typename ST::Compute;
  const StepT<T> p = convert<T>(h);
  if constexpr (LAT == 0) {
    *nk = 1;
    return h.spt == 4 ? launch_fused2d<ST, 4>(fa, fb, p, s) : launch_fused2d<ST, 2>(fa, fb, p, s);
  } else {
    moments_kernel<LAT, ST><<<blocks_for(p.N, 256), 256, 0, s>>>(ST::reader(fa, (unsigned)p.N), (T*)psi, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *nk = 2;
    if (h.d3_kernel == 1) return launch_tiled<LAT, ST, false>(fa, fb, psi, h, p, FieldOut{}, s);
    return launch_march3d<ST>(fa, fb, psi, h, p, s);
  }
}

template <int LAT, typename ST>
cudaError_t l_fields(const void* f, void* psi, const HostParams& h, const FieldOut& fo, cudaStream_t s, int* nk) {
  using T = typename ST::Compute;
  const StepT<T> p = convert<T>(h);
  moments_kernel<LAT, ST><<<blocks_for(p.N, 256), 256, 0, s>>>(ST::reader(f, (unsigned)p.N), (T*)psi, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *nk = 2;
  return launch_tiled<LAT, ST, true>(f, nullptr, psi, h, p, fo, s);
}

template <int LAT, typename ST>
cudaError_t l_decode(const void* f, double* out, int s0, int count, long long pitch, int N, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  decode_kernel<LAT, ST><<<blocks_for(count, 256), 256, 0, s>>>(ST::reader(f, (unsigned)N), out, s0, count, pitch);
  return cudaGetLastError();
}

template <int LAT, typename ST>
cudaError_t l_encode(const double* in, void* f, int s0, int count, long long pitch, int N, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  encode_kernel<LAT, ST><<<blocks_for(count, 256), 256, 0, s>>>(in, ST::writer(f, (unsigned)N), s0, count, pitch);
  return cudaGetLastError();
}

template <typename ST>
void l_batch_fill(void* dst, const HostParams& h, const void* buf0, const void* buf1) {
  BatchMember<typename ST::Compute> m;
  m.p = convert<typename ST::Compute>(h);
  m.buf[0] = buf0;
  m.buf[1] = buf1;
  m.ntx = (h.nx + kFusedTX - 1) / kFusedTX;
  memcpy(dst, &m, sizeof(m));
}

int l_batch_tiles(const HostParams& h, int spt) {
  const int ty = kFusedThreadsY * spt;
  return ((h.nx + kFusedTX - 1) / kFusedTX) * ((h.ny + ty - 1) / ty);
}

template <typename ST, int SPT, bool EDM>
cudaError_t launch_batch_v(const void* members, const int* tile0, int n, int total_tiles, int parity,
                           int smax_max, cudaStream_t s) {
  static SmemAllowance configured;
  const size_t sm = fused2d_smem_bytes<typename ST::Compute>(smax_max, SPT);
  cudaError_t e = allow_smem(fused2d_batch_kernel<ST, SPT, EDM>, sm, configured);
  if (e != cudaSuccess) return e;
  fused2d_batch_kernel<ST, SPT, EDM><<<total_tiles, dim3(kFusedTX, kFusedThreadsY, 1), sm, s>>>(
      (const BatchMember<typename ST::Compute>*)members, tile0, n, parity);
  return cudaGetLastError();
}

// All members of an ensemble share the forcing scheme (checked at creation).
template <typename ST, int SPT>
cudaError_t launch_batch(const void* members, const int* tile0, int n, int total_tiles, int parity, int smax_max,
                         int edm, cudaStream_t s) {
  if constexpr (edm_build_exists<ST>()) {
    if (edm) return launch_batch_v<ST, SPT, true>(members, tile0, n, total_tiles, parity, smax_max, s);
  }
  return launch_batch_v<ST, SPT, false>(members, tile0, n, total_tiles, parity, smax_max, s);
}

template <int LAT, typename ST>
cudaError_t l_batch_step(const void* members, const int* tile0, int n, int total_tiles, int parity, int spt,
                         int smax_max, int edm, cudaStream_t s) {
  if constexpr (LAT != 0) {
    return cudaErrorNotSupported;
  } else {
    return spt == 4 ? launch_batch<ST, 4>(members, tile0, n, total_tiles, parity, smax_max, edm, s)
                    : launch_batch<ST, 2>(members, tile0, n, total_tiles, parity, smax_max, edm, s);
  }
}

template <int LAT, typename ST>
const Launchers* table() {
  static const Launchers L = {ST::bytes, sizeof(typename ST::Compute), l_init<LAT, ST>, l_step<LAT, ST>,
                              l_fields<LAT, ST>, l_decode<LAT, ST>, l_encode<LAT, ST>,
                              sizeof(BatchMember<typename ST::Compute>), l_batch_fill<ST>, l_batch_tiles,
                              l_batch_step<LAT, ST>};
  return &L;
}

}  // namespace
}  // namespace lbnci
