// lb_lattice.cuh -- D2Q9 / D3Q27 velocity sets as compile-time functions of the
// direction index, and the kernel parameter block.
//
// Direction i has c_i given by the base-3 digits of i (x lowest, then y, then z),
// digit d -> {0,+1,-1}[d]; weights by |c_i|^2 are the standard D2Q9 (4/9, 1/9, 1/36)
// and D3Q27 (8/27, 2/27, 1/54, 1/216) ones, c_s^2 = 1/3 (arXiv:2003.11069 names the
// D3Q27 lattice in "Materials and Methods"; D2Q9 is its two-dimensional analogue).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbnci {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1, so that every
// per-direction constant below is a constant expression (folded by the compiler,
// never evaluated at run time in FP64).
template <typename F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int digit_c(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }
__host__ __device__ constexpr int pow3(int a) { return a == 0 ? 1 : 3 * pow3(a - 1); }
// Component a (0 = x, 1 = y, 2 = z) of velocity i.
__host__ __device__ constexpr int cc(int i, int a) { return digit_c((i / pow3(a)) % 3); }
__host__ __device__ constexpr int speed2(int i) {
  return cc(i, 0) * cc(i, 0) + cc(i, 1) * cc(i, 1) + cc(i, 2) * cc(i, 2);
}
// Opposite direction: swap digits 1 <-> 2 in every position.
__host__ __device__ constexpr int flip_digit(int d) { return d == 0 ? 0 : 3 - d; }
__host__ __device__ constexpr int opposite(int i) {
  return flip_digit(i % 3) + 3 * flip_digit((i / 3) % 3) + 9 * flip_digit(i / 9);
}

template <int LAT> struct Lattice;

template <> struct Lattice<0> {  // D2Q9
  static constexpr int D = 2, Q = 9;
  __host__ __device__ static constexpr double w(int i) {
    return speed2(i) == 0 ? 4.0 / 9.0 : (speed2(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <> struct Lattice<1> {  // D3Q27
  static constexpr int D = 3, Q = 27;
  __host__ __device__ static constexpr double w(int i) {
    return speed2(i) == 0 ? 8.0 / 27.0
         : (speed2(i) == 1 ? 2.0 / 27.0 : (speed2(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
};

// Parameters of one step in the arithmetic type T of the kernels (converted once on
// the host, so an FP32 kernel never touches FP64).
template <typename T>
struct StepT {
  int nx, ny, nz;
  int wall_y, wall_z;
  int N;        // nx*ny*nz (< 2^31)
  int smax;     // probe steps of the NCI ray search (0 = NCI off)
  int edm;      // 1: exact difference method, NCI force on the dispersed phase only
  T omega;      // 1/tau
  T guo;        // 1 - omega/2 (Guo source prefactor)
  T pamp;       // 2 * (A_s/2): perturbation amplitude summed over both components
  T beta;       // recolouring segregation
  T g_th;       // interface threshold on |grad psi|
  T G[3];       // body force
  T Ah[8];      // A_h(h) for integer probe distance h (0 unused): A for h <= h_min,
                // A (h_min/h)^3 for h_min < h <= h_max, 0 beyond
  unsigned* seedw;  // FP16-deviation storage: the sim's two dither-seed words (or null);
  int parity;       // the launch reads seedw[parity] and sets seedw[parity ^ 1] to it + 1
};

// Largest number of NCI probe steps the kernels support (h_max < kMaxProbe + 1).
constexpr int kMaxProbe = 4;

// Optional per-site outputs of the fields kernel (device pointers, FP64).
struct FieldOut {
  double* rho1;
  double* rho2;
  double* psi;
  double* grad;  // [3][N]
  double* frep;  // [3][N]
  int* hit;
  double* u;     // [3][N]
  double* partials;  // [blocks][kRedSlots] reductions
};

constexpr int kRedSlots = 10;  // mass1, mass2, P_x, P_y, P_z, flux, flux_disp, n_if, n_nci, n_bad

// Thread-block tile of the tiled (fields and 3D step) kernels.
template <int LAT> struct Tile;
template <> struct Tile<0> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<1> { static constexpr int X = 32, Y = 4, Z = 2; };

// Fused D2Q9 step kernel: 32 x (8*SPT) sites per 256-thread block.
constexpr int kFusedTX = 32, kFusedThreadsY = 8;

}  // namespace lbnci
