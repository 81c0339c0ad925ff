// lb_storage.cuh -- how a population state is laid out in device memory.
//
// Every kernel reads populations through Storage::Reader::get<i>(site) and writes them
// through Storage::Writer::put<i>(site, ...), so one kernel source serves each layout:
//
//   Plain<LAT, T>   f[k][i][site] in T (FP64 or FP32): 2 Q planes.
//   HalfDev<LAT>    deviations from the lattice-weight equilibrium at rest,
//                   delta_i^k = f_i^k - w_i rho_ref^k, stored as FP16 pairs
//                   (component 1, component 2) in Q half2 planes, plus one float2 plane
//                   of the reference densities rho_ref = (rho_1, rho_2) of each site
//                   (the collision keeps rho_k per site, so this is also the density
//                   the stored populations sum to). Arithmetic is FP32. A pulled
//                   population is decoded with the reference density of the site it
//                   came from: f_i(y) = w_i rho_ref(y - c_i) + delta_i(y - c_i).
#pragma once

#include <cuda_fp16.h>

#include "lb_lattice.cuh"

namespace lbnci {

template <int LAT, typename T>
struct Plain {
  using Compute = T;
  static constexpr int Q = Lattice<LAT>::Q;
  static constexpr bool kHalf = false;
  static size_t bytes(size_t N) { return 2 * (size_t)Q * N * sizeof(T); }

  struct Reader {
    const T* __restrict__ f;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void get(unsigned site, T& a, T& b) const {
      a = f[(unsigned)I * N + site];
      b = f[(unsigned)(Q + I) * N + site];
    }
  };
  struct Writer {
    T* __restrict__ f;
    unsigned N;
    // (r1, r2): the densities of the site, unused by this layout
    template <int I>
    __device__ __forceinline__ void put(unsigned site, T a, T b, T, T) const {
      f[(unsigned)I * N + site] = a;
      f[(unsigned)(Q + I) * N + site] = b;
    }
    __device__ __forceinline__ void put_rho(unsigned, T, T) const {}
  };
  __host__ __device__ static Reader reader(const void* base, unsigned N) { return Reader{(const T*)base, N}; }
  __host__ __device__ static Writer writer(void* base, unsigned N) { return Writer{(T*)base, N}; }
};

template <int LAT>
struct HalfDev {
  using Compute = float;
  static constexpr int Q = Lattice<LAT>::Q;
  static constexpr bool kHalf = true;
  __host__ __device__ static size_t rho_offset(size_t N) { return ((size_t)Q * N * sizeof(__half2) + 255) & ~(size_t)255; }
  static size_t bytes(size_t N) { return rho_offset(N) + N * sizeof(float2); }

  struct Reader {
    const __half2* __restrict__ d;
    const float2* __restrict__ rho;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void get(unsigned site, float& a, float& b) const {
      constexpr float w = float(Lattice<LAT>::w(I));
      const float2 r = rho[site];
      const float2 v = __half22float2(d[(unsigned)I * N + site]);
      a = fmaf(w, r.x, v.x);
      b = fmaf(w, r.y, v.y);
    }
  };
  struct Writer {
    __half2* __restrict__ d;
    float2* __restrict__ rho;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void put(unsigned site, float a, float b, float r1, float r2) const {
      constexpr float w = float(Lattice<LAT>::w(I));
      d[(unsigned)I * N + site] = __floats2half2_rn(fmaf(-w, r1, a), fmaf(-w, r2, b));
    }
    __device__ __forceinline__ void put_rho(unsigned site, float r1, float r2) const {
      rho[site] = make_float2(r1, r2);
    }
  };
  __host__ __device__ static Reader reader(const void* base, unsigned N) {
    return Reader{(const __half2*)base, (const float2*)((const char*)base + rho_offset(N)), N};
  }
  __host__ __device__ static Writer writer(void* base, unsigned N) {
    return Writer{(__half2*)base, (float2*)((char*)base + rho_offset(N)), N};
  }
};

}  // namespace lbnci
