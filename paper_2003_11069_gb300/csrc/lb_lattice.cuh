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

namespace lbnci {

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

// Parameters of one step, passed by value to every kernel.
struct StepParams {
  int nx, ny, nz;
  int wall_y, wall_z;
  long long N;        // nx*ny*nz
  double tau, A_s, beta, A_h, h_min, h_max, g_th;
  double G[3];
  int smax;           // probe steps of the NCI ray search (0 = NCI off)
};

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

// Thread-block tile of the tiled kernels.
template <int LAT> struct Tile;
template <> struct Tile<0> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<1> { static constexpr int X = 32, Y = 4, Z = 2; };

}  // namespace lbnci
