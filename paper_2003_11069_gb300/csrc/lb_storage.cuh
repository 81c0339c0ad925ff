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
//
// A step stores through put_step, which HalfDev rounds stochastically: a deviation
// goes to one of its two neighbouring FP16 values with probabilities in proportion to
// its distance from the other (cvt.rs, fed 32 random bits per pair), so the rounding is
// unbiased. Rounding to nearest is not: near a steady flow a site computes nearly the
// same value every step, so it rounds the same way every step, and the body force's
// share of a step (w_i 3 c_i.G, of the order of one FP16 unit of the velocity part of
// the deviation in a Poiseuille channel, G W^2 / nu ~ u) is lost or doubled coherently;
// measured with rounding to nearest, the flow rate of a 256-wide channel ended 4% low.
// The random bits are a hash of the site and a per-step seed the step kernel reads from
// the sim (StepT::seedw), so runs are reproducible and a member of an ensemble rounds
// exactly as the same lattice stepped alone. Initial states (put) round to nearest.
#pragma once

#include <cuda_fp16.h>

#include "lb_lattice.cuh"

namespace lbnci {

// Random bits of a site for one step: the 32-bit finaliser of MurmurHash3 (Appleby) of
// site + seed * 0x9E3779B9 (consecutive seeds move every site's input by the 32-bit
// golden-ratio constant, so a site sees a new input at every step).
__device__ __forceinline__ unsigned dither_bits(unsigned site, unsigned seed) {
  unsigned h = site + seed * 0x9E3779B9u;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// The seed of this launch's stochastic rounding; one thread of the launch (lead) moves
// the sim's other word on, for the next step.
template <typename T>
__device__ __forceinline__ unsigned step_seed(const StepT<T>& p, int parity, bool lead) {
  if (!p.seedw) return 0u;
  const unsigned s = p.seedw[parity];
  if (lead) p.seedw[parity ^ 1] = s + 1u;
  return s;
}

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
    unsigned seed;  // unused by this layout
    // (r1, r2): the densities of the site, unused by this layout
    template <int I>
    __device__ __forceinline__ void put(unsigned site, T a, T b, T, T) const {
      f[(unsigned)I * N + site] = a;
      f[(unsigned)(Q + I) * N + site] = b;
    }
    __device__ __forceinline__ unsigned site_bits(unsigned) const { return 0u; }
    template <int I>
    __device__ __forceinline__ void put_step(unsigned site, T a, T b, T r1, T r2, unsigned) const {
      put<I>(site, a, b, r1, r2);
    }
    __device__ __forceinline__ void put_rho(unsigned, T, T) const {}
  };
  __host__ __device__ static Reader reader(const void* base, unsigned N) { return Reader{(const T*)base, N}; }
  __host__ __device__ static Writer writer(void* base, unsigned N) { return Writer{(T*)base, N}; }
};

// (lo, hi) rounded stochastically to a half2 word (lo in the low half, as
// __floats2half2_rn places its first argument). cvt.rs.f16x2.f32 takes its second
// source to the low half and its first to the high half, drawing the random bits of
// the high half from the word's upper 16 bits and those of the low half from its lower
// 16 (measured on GB300). Direction I uses the site's bits rotated by 7 I.
template <int I>
__device__ __forceinline__ unsigned half2_stochastic(float lo, float hi, unsigned h) {
  const unsigned r = __funnelshift_l(h, h, (7 * I) & 31);
  unsigned v;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(v) : "f"(hi), "f"(lo), "r"(r));
  return v;
}

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
    unsigned seed;  // this step's dither seed (step_seed)
    // rounded to nearest (initial states)
    template <int I>
    __device__ __forceinline__ void put(unsigned site, float a, float b, float r1, float r2) const {
      constexpr float w = float(Lattice<LAT>::w(I));
      d[(unsigned)I * N + site] = __floats2half2_rn(fmaf(-w, r1, a), fmaf(-w, r2, b));
    }
    __device__ __forceinline__ unsigned site_bits(unsigned site) const { return dither_bits(site, seed); }
    // rounded stochastically with the site's bits h (a step's output)
    template <int I>
    __device__ __forceinline__ void put_step(unsigned site, float a, float b, float r1, float r2,
                                             unsigned h) const {
      constexpr float w = float(Lattice<LAT>::w(I));
      reinterpret_cast<unsigned*>(d)[(unsigned)I * N + site] = half2_stochastic<I>(fmaf(-w, r1, a), fmaf(-w, r2, b), h);
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
