// lb_kernels.cuh -- CUDA kernels of one colour-gradient NCI lattice Boltzmann step
// (arXiv:2003.11069, "Materials and Methods"), templated on the lattice and on the
// storage/compute type T (double or float). Instantiated by lb_fp64.cu (compiled
// without multiply-add contraction: the parity path) and lb_fp32.cu.
//
// Per-site stages, in the paper's order:
//   pull-stream with halfway bounce-back             Eq. (CGLBE)
//   rho_k = sum_i f_i^k, psi = (rho1-rho2)/(rho1+rho2)
//   isotropic gradient of psi, n = -grad psi/|grad psi|, delta_I = |grad psi|/2
//   NCI ray search, F_rep = -A_h(h) n delta_I         Eq. (near_c)
//   Guo velocity, BGK + Guo source + perturbation, recolouring (Omega^(3)[Omega^(1)+Omega^(2)])
//
// Kernels:
//   fused2d_kernel  : the D2Q9 step in one pass (lb_fused2d.cuh)
//   moments_kernel  : psi of the streamed state (3D step and the fields path)
//   tiled_kernel    : gradient + NCI + collision from a psi array staged in shared
//                     memory; FIELDS variant writes macroscopic fields and partial sums
#pragma once

#include "lb_lattice.cuh"
#include "lb_storage.cuh"

namespace lbnci {

// FP64: IEEE operations only (round exactly as the oracle's C does).
// FP32: fast intrinsics where the result feeds no bit-exact comparison.
template <typename T> struct M;
template <> struct M<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  // |g| and the unit vector -g/|g| (0 when g = 0)
  static __device__ __forceinline__ double unit(const double g[3], double n[3]) {
    const double gn = ::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn > 0.0) { n[0] = -g[0] / gn; n[1] = -g[1] / gn; n[2] = -g[2] / gn; }
    else { n[0] = 0.0; n[1] = 0.0; n[2] = 0.0; }
    return gn;
  }
};
template <> struct M<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float unit(const float g[3], float n[3]) {
    const float g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (g2 > 0.0f) {
      const float inv = rsqrtf(g2);
      n[0] = -g[0] * inv; n[1] = -g[1] * inv; n[2] = -g[2] * inv;
      return g2 * inv;
    }
    n[0] = 0.0f; n[1] = 0.0f; n[2] = 0.0f;
    return 0.0f;
  }
};

// Round half away from zero by comparisons only (no float-to-int conversion): the
// probe offset round(s n_a) of the NCI ray search at step s. |n_a| <= 1 bounds
// |s n_a| by s, so only the half-integers below s need testing.
template <int S, typename T>
__device__ __forceinline__ int round_probe(T v) {
  const T a = v < T(0) ? -v : v;
  int m = a >= T(0.5);
  if constexpr (S >= 2) m += a >= T(1.5);
  if constexpr (S >= 3) m += a >= T(2.5);
  if constexpr (S >= 4) m += a >= T(3.5);
  return v < T(0) ? -m : m;
}

// Wrap a coordinate into [0, n) (a few periods at most; no integer division).
__device__ __forceinline__ int wrapn(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// Visit the cells c = tid, tid + NT, ... of an RX x RY x RZ region together with
// their coordinates (lx, ly, lz), stepping the coordinates incrementally so that the
// loop itself needs no integer division.
template <typename F>
__device__ __forceinline__ void for_region(int tid, int NT, int RX, int RY, int RZ, F&& fn) {
  const int total = RX * RY * RZ;
  int lx = tid % RX, ly = (tid / RX) % RY, lz = tid / (RX * RY);
  const int sx = NT % RX, sy = (NT / RX) % RY, sz = NT / (RX * RY);
  for (int c = tid; c < total; c += NT) {
    fn(c, lx, ly, lz);
    lx += sx; ly += sy; lz += sz;
    if (lx >= RX) { lx -= RX; ++ly; }
    if (ly >= RY) { ly -= RY; ++lz; }
  }
}

// Pull the 2Q populations of site (x,y,z) from the post-collision state: from the
// upstream site x - c_i, or, when that lies beyond a wall, the opposite population
// of the site itself (halfway bounce-back).
template <int LAT, typename T, typename RD>
__device__ __forceinline__ void pull_site(const RD& f, int x, int y, int z, const StepT<T>& p,
                                          T out[2][Lattice<LAT>::Q]) {
  constexpr int Q = Lattice<LAT>::Q;
  constexpr bool D3 = Lattice<LAT>::D == 3;
  const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
  int ym, yp, zm = 0, zp = 0;
  bool bym = false, byp = false, bzm = false, bzp = false;
  if (p.wall_y) { ym = y - 1; yp = y + 1; bym = y == 0; byp = y == p.ny - 1; }
  else { ym = y == 0 ? p.ny - 1 : y - 1; yp = y == p.ny - 1 ? 0 : y + 1; }
  if (D3) {
    if (p.wall_z) { zm = z - 1; zp = z + 1; bzm = z == 0; bzp = z == p.nz - 1; }
    else { zm = z == 0 ? p.nz - 1 : z - 1; zp = z == p.nz - 1 ? 0 : z + 1; }
  }
  const int idx = x + p.nx * (y + p.ny * z);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = cc(i, 0), cy = cc(i, 1), cz = cc(i, 2);
    bool bounce = (cy == 1 && bym) || (cy == -1 && byp);
    if (D3) bounce = bounce || (cz == 1 && bzm) || (cz == -1 && bzp);
    const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
    const int sy = cy == 1 ? ym : (cy == -1 ? yp : y);
    const int sz = D3 ? (cz == 1 ? zm : (cz == -1 ? zp : z)) : 0;
    const int src = sx + p.nx * (sy + p.ny * sz);
    if (bounce) f.template get<opposite(i)>((unsigned)idx, out[0][i], out[1][i]);
    else f.template get<i>((unsigned)src, out[0][i], out[1][i]);
  });
}

// pull_site for a site whose upstream neighbours are all interior (no wrap, no wall):
// every population comes from a fixed offset idx - c_i.(1, nx, nx ny).
template <int LAT, typename T, typename RD>
__device__ __forceinline__ void pull_interior(const RD& f, int idx, const StepT<T>& p,
                                              T out[2][Lattice<LAT>::Q]) {
  constexpr int Q = Lattice<LAT>::Q;
  const int sy = p.nx, sz = p.nx * p.ny;
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int src = idx - cc(i, 0) - sy * cc(i, 1) - sz * cc(i, 2);
    f.template get<i>((unsigned)src, out[0][i], out[1][i]);
  });
}

// True when site (x,y,z) can use pull_interior.
template <int LAT, typename T>
__device__ __forceinline__ bool is_interior(int x, int y, int z, const StepT<T>& p) {
  bool in = x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1;
  if (Lattice<LAT>::D == 3) in = in && z > 0 && z < p.nz - 1;
  return in;
}

template <int LAT, typename T, typename RD>
__device__ __forceinline__ void pull_any(const RD& f, int x, int y, int z, const StepT<T>& p,
                                         T out[2][Lattice<LAT>::Q]) {
  if (is_interior<LAT, T>(x, y, z, p)) pull_interior<LAT, T, RD>(f, x + p.nx * (y + p.ny * z), p, out);
  else pull_site<LAT, T, RD>(f, x, y, z, p, out);
}

// psi = (rho1 - rho2)/(rho1 + rho2) of pulled populations (sums in direction order).
template <int Q, typename T>
__device__ __forceinline__ T psi_of(const T fin[2][Q], T* r1out = nullptr, T* r2out = nullptr) {
  T r1 = T(0), r2 = T(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) r1 += fin[0][i];
#pragma unroll
  for (int i = 0; i < Q; ++i) r2 += fin[1][i];
  if (r1out) *r1out = r1;
  if (r2out) *r2out = r2;
  return M<T>::div(r1 - r2, r1 + r2);
}

// Isotropic gradient (1/c_s^2) sum_i w_i c_i psi(x + c_i) from a shared-memory psi
// region with strides (1, RX, RXY). Cells beyond a wall hold the psi of their mirror
// image across the wall plane (the clamped coordinate), which is what the stencil of a
// site next to a wall reads: neutral wetting.
template <int LAT, typename T>
__device__ __forceinline__ void grad_smem(const T* __restrict__ sp, int RX, int RXY, int c, T g[3]) {
  constexpr int Q = Lattice<LAT>::Q;
  constexpr bool D3 = Lattice<LAT>::D == 3;
  g[0] = T(0); g[1] = T(0); g[2] = T(0);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i > 0) {
      constexpr T wx = T(Lattice<LAT>::w(i) * cc(i, 0));
      constexpr T wy = T(Lattice<LAT>::w(i) * cc(i, 1));
      constexpr T wz = T(Lattice<LAT>::w(i) * cc(i, 2));
      const T v = sp[c + cc(i, 0) + RX * cc(i, 1) + RXY * cc(i, 2)];
      if constexpr (cc(i, 0) != 0) g[0] += wx * v;
      if constexpr (cc(i, 1) != 0) g[1] += wy * v;
      if constexpr (D3 && cc(i, 2) != 0) g[2] += wz * v;
    }
  });
  g[0] = T(3) * g[0];
  g[1] = T(3) * g[1];
  g[2] = T(3) * g[2];
}

// Clamp a coordinate into [0, n): the mirror image of the first cell beyond a wall.
__device__ __forceinline__ int clampc(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Guo velocity u = (j + F/2)/rho with j = sum_k sum_i f_i^k c_i.
template <int LAT, typename T>
__device__ __forceinline__ void momentum(const T fin[2][Lattice<LAT>::Q], T j[3]) {
  constexpr int Q = Lattice<LAT>::Q;
  j[0] = T(0); j[1] = T(0); j[2] = T(0);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const T fi = fin[0][i] + fin[1][i];
    if constexpr (cc(i, 0) != 0) j[0] += cc(i, 0) > 0 ? fi : -fi;
    if constexpr (cc(i, 1) != 0) j[1] += cc(i, 1) > 0 ? fi : -fi;
    if constexpr (Lattice<LAT>::D == 3 && cc(i, 2) != 0) j[2] += cc(i, 2) > 0 ? fi : -fi;
  });
}

// f_eq of the second-order lattice BGK model, c_s^2 = 1/3, for direction i.
template <int LAT, int I, typename T>
__device__ __forceinline__ T feq_dir(T rho, const T v[3]) {
  constexpr T w = T(Lattice<LAT>::w(I));
  constexpr T cx = T(cc(I, 0)), cy = T(cc(I, 1)), cz = T(cc(I, 2));
  const T cu = cx * v[0] + cy * v[1] + cz * v[2];
  const T uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  return w * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
}

// The collision written term by term as in the oracle (FP64 rounds exactly like it):
// Guo forcing, or, with p.edm, relaxation towards f_eq(rho, j/rho) and the exact
// difference method after recolouring, component k gaining
// f_eq(rho_k, u + dU_k) - f_eq(rho_k, u), dU_k = F_k/rho_k, F_1 = G rho_1/rho + F_rep,
// F_2 = G rho_2/rho (the near-contact force acts on the dispersed phase only).
template <int LAT, typename T, typename WR>
__device__ __forceinline__ void collide_exact(const T fin[2][Lattice<LAT>::Q], T rho1, T rho2, const T j[3],
                                              const T u[3], const T F[3], T g, const T m[3], const StepT<T>& p,
                                              const WR& fout, int idx) {
  constexpr int Q = Lattice<LAT>::Q;
  const T rho = rho1 + rho2;
  const bool edm = p.edm != 0;
  T ueq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) ueq[a] = edm ? M<T>::div(j[a], rho) : u[a];
  T u1[3], u2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T d1 = T(0), d2 = T(0);
    if (edm) {
      const T G = p.G[a], Frep = F[a] - p.G[a];
      if (rho1 > T(0)) d1 = M<T>::div(M<T>::div(G * rho1, rho) + Frep, rho1);
      if (rho2 > T(0)) d2 = M<T>::div(M<T>::div(G * rho2, rho), rho2);
    }
    u1[a] = ueq[a] + d1;
    u2[a] = ueq[a] + d2;
  }
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const T seg = M<T>::div(p.beta * rho1 * rho2, rho);
  const T pamp = p.pamp * g;
  const T c1 = M<T>::div(rho1, rho), c2 = M<T>::div(rho2, rho);
  const unsigned hb = fout.site_bits((unsigned)idx);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr T w = T(Lattice<LAT>::w(i));
    constexpr T cx = T(cc(i, 0)), cy = T(cc(i, 1)), cz = T(cc(i, 2));
    constexpr T w3 = w / T(3);
    constexpr T inv_len = speed2(i) == 0 ? T(0)
                        : T(1) / (speed2(i) == 1 ? T(1) : (speed2(i) == 2 ? T(1.4142135623730951)
                                                                           : T(1.7320508075688772)));
    const T fi = fin[0][i] + fin[1][i];
    const T cm = cx * m[0] + cy * m[1] + cz * m[2];
    T fs;
    if (!edm) {
      const T cu = cx * u[0] + cy * u[1] + cz * u[2];
      const T cF = cx * F[0] + cy * F[1] + cz * F[2];
      const T S = p.guo * w * (T(3) * (cF - uF) + T(9) * cu * cF);
      fs = fi - p.omega * (fi - feq_dir<LAT, i, T>(rho, u)) + S;
    } else {
      fs = fi - p.omega * (fi - feq_dir<LAT, i, T>(rho, ueq));
    }
    fs += pamp * (w * cm * cm - w3);
    const T rc = seg * w * (cm * inv_len);
    T o1 = c1 * fs + rc;
    T o2 = c2 * fs - rc;
    if (edm) {
      o1 += feq_dir<LAT, i, T>(rho1, u1) - feq_dir<LAT, i, T>(rho1, ueq);
      o2 += feq_dir<LAT, i, T>(rho2, u2) - feq_dir<LAT, i, T>(rho2, ueq);
    }
    fout.template put_step<i>((unsigned)idx, o1, o2, rho1, rho2, hb);
  });
  fout.put_rho((unsigned)idx, rho1, rho2);
}

// BGK relaxation towards f_eq(rho, u) with the Guo source, plus the perturbation
// (A_s/2)|grad psi| [w_i (c_i.m)^2 - w_i/3] of each component, on the total
// population; then recolouring f^1 = (rho1/rho) f* + beta rho1 rho2/rho w_i cos(theta_i),
// f^2 = (rho2/rho) f* - same, cos(theta_i) = c_i.m/|c_i|. m = grad psi/|grad psi|.
// EDM: the kernel variant built for the exact-difference-method forcing. FP64 always
// takes the term-by-term path (which checks p.edm itself); FP32 kernels are built twice,
// so the common Guo path keeps its register budget.
template <int LAT, typename T, typename WR, bool EDM = false>
__device__ __forceinline__ void collide_store(const T fin[2][Lattice<LAT>::Q], T rho1, T rho2, const T j[3],
                                              const T u[3], const T F[3], T g, const T m[3], const StepT<T>& p,
                                              const WR& fout, int idx) {
  constexpr int Q = Lattice<LAT>::Q;
  if constexpr (std::is_same<T, double>::value || EDM) {
    collide_exact<LAT, T, WR>(fin, rho1, rho2, j, u, F, g, m, p, fout, idx);
    return;
  }
  const T rho = rho1 + rho2;
  constexpr bool D3 = Lattice<LAT>::D == 3;  // D2Q9: u and F have no z component
  const T uF = u[0] * F[0] + u[1] * F[1] + (D3 ? u[2] * F[2] : T(0));
  const T uu = u[0] * u[0] + u[1] * u[1] + (D3 ? u[2] * u[2] : T(0));
  const T seg = M<T>::div(p.beta * rho1 * rho2, rho);
  const T pamp = p.pamp * g;
  const T c1 = M<T>::div(rho1, rho);
  // FP32: the same operator regrouped per site,
  //   f*_i = (1 - omega) f_i + w_i B_i,
  //   B_i = K0 + c.u (omega rho (3 + 4.5 c.u) + 9 guo c.F) + 3 guo c.F + pamp (c.m)^2,
  //   K0 = omega rho (1 - 1.5 u.u) - 3 guo u.F - pamp/3,
  // evaluated per pair of opposite directions (i, opposite(i)): c.u, c.F and c.m change
  // sign between the two, so B splits into a part even in c,
  //   E = K0 + 4.5 omega rho (c.u)^2 + 9 guo (c.u)(c.F) + pamp (c.m)^2,
  // and an odd part O = 3 omega rho c.u + 3 guo c.F (B = E + O and E - O), and the
  // recolouring term changes sign; the pair shares those products. The rest population
  // of each component is set to rho_k minus the others (its exact value), so per-site
  // mass is kept to the rounding of one sum instead of drifting with the coherent
  // rounding of K0.
  const T orho = p.omega * rho;
  const T K0 = orho * (T(1) - T(1.5) * uu) - T(3) * p.guo * uF - pamp * T(1.0 / 3.0);
  const T a3 = T(3) * orho, a45 = T(4.5) * orho, g3 = T(3) * p.guo, g9 = T(9) * p.guo;
  const T om1 = T(1) - p.omega;
  const unsigned hb = fout.site_bits((unsigned)idx);
  T s1 = T(0), s2 = T(0);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int o = opposite(i);
    if constexpr (i > 0 && i < o) {
      constexpr T w = T(Lattice<LAT>::w(i));
      constexpr int ix = cc(i, 0), iy = cc(i, 1), iz = cc(i, 2);
      constexpr T wl = T(Lattice<LAT>::w(i) / (speed2(i) == 1 ? 1.0 : (speed2(i) == 2 ? 1.4142135623730951
                                                                                       : 1.7320508075688772)));
      auto dotc = [&](const T v[3]) {
        T r = T(0);
        if constexpr (ix == 1) r += v[0]; else if constexpr (ix == -1) r -= v[0];
        if constexpr (iy == 1) r += v[1]; else if constexpr (iy == -1) r -= v[1];
        if constexpr (iz == 1) r += v[2]; else if constexpr (iz == -1) r -= v[2];
        return r;
      };
      const T cu = dotc(u), cF = dotc(F), cm = dotc(m);
      const T E = fmaf(pamp, cm * cm, fmaf(g9, cu * cF, fmaf(a45, cu * cu, K0)));
      const T O = fmaf(g3, cF, a3 * cu);
      const T fsp = fmaf(w, E + O, om1 * (fin[0][i] + fin[1][i]));
      const T fsm = fmaf(w, E - O, om1 * (fin[0][o] + fin[1][o]));
      const T rc = (seg * wl) * cm;
      const T o1p = fmaf(c1, fsp, rc), o1m = fmaf(c1, fsm, -rc);
      const T o2p = fsp - o1p, o2m = fsm - o1m;
      s1 += o1p + o1m;
      s2 += o2p + o2m;
      fout.template put_step<i>((unsigned)idx, o1p, o2p, rho1, rho2, hb);
      fout.template put_step<o>((unsigned)idx, o1m, o2m, rho1, rho2, hb);
    }
  });
  fout.template put_step<0>((unsigned)idx, rho1 - s1, rho2 - s2, rho1, rho2, hb);
  fout.put_rho((unsigned)idx, rho1, rho2);
}

// ---------------------------------------------------------------------------- moments
template <int LAT, typename ST>
__global__ void __launch_bounds__(256) moments_kernel(typename ST::Reader f, typename ST::Compute* __restrict__ psi,
                                                      StepT<typename ST::Compute> p) {
  using T = typename ST::Compute;
  constexpr int Q = Lattice<LAT>::Q;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.N) return;
  const int x = idx % p.nx;
  const int y = (idx / p.nx) % p.ny;
  const int z = idx / (p.nx * p.ny);
  T fin[2][Q];
  pull_any<LAT, T>(f, x, y, z, p, fin);
  psi[idx] = psi_of<Q, T>(fin);
}

// ---------------------------------------------------------------------------- tiled
template <int LAT> __host__ __device__ constexpr int region_rz(int R) {
  return Lattice<LAT>::D == 3 ? Tile<LAT>::Z + 2 * R : 1;
}

template <int LAT, typename T>
size_t tiled_smem_bytes(int smax) {
  const int R = smax + 1;
  return sizeof(T) * (size_t)(Tile<LAT>::X + 2 * R) * (Tile<LAT>::Y + 2 * R) * region_rz<LAT>(R);
}

// Gradient, NCI and collision from a psi array: the psi tile and its halo of radius
// smax+1 are staged in shared memory; probes recompute the gradient there.
template <int LAT, typename ST, bool FIELDS, bool EDM = false>
__global__ void __launch_bounds__(256)
tiled_kernel(typename ST::Reader f, typename ST::Writer fout, const typename ST::Compute* __restrict__ psi,
             StepT<typename ST::Compute> p, FieldOut fo) {
  using T = typename ST::Compute;
  constexpr int D = Lattice<LAT>::D;
  constexpr int Q = Lattice<LAT>::Q;
  constexpr int TX = Tile<LAT>::X, TY = Tile<LAT>::Y, TZ = Tile<LAT>::Z;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sp = reinterpret_cast<T*>(smem_raw);

  const int R = p.smax + 1;
  const int RX = TX + 2 * R, RY = TY + 2 * R, RZ = region_rz<LAT>(R);
  const int RXY = RX * RY;
  const int RZoff = D == 3 ? R : 0;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
  if constexpr (ST::kHalf && !FIELDS)
    fout.seed = step_seed(p, p.parity, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0);

  for_region(tid, TX * TY * TZ, RX, RY, RZ, [&](int t, int lx, int ly, int lz) {
    const int gx = wrapn(x0 - R + lx, p.nx);
    int gy = y0 - R + ly;
    int gz = D == 3 ? z0 - RZoff + lz : 0;
    gy = p.wall_y ? clampc(gy, p.ny) : wrapn(gy, p.ny);
    if (D == 3) gz = p.wall_z ? clampc(gz, p.nz) : wrapn(gz, p.nz);
    sp[t] = psi[gx + p.nx * (gy + p.ny * gz)];
  });
  __syncthreads();

  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < p.nx && y < p.ny && z < p.nz;

  double red[kRedSlots];
  if (FIELDS) for (int q = 0; q < kRedSlots; ++q) red[q] = 0.0;

  if (active) {
    const int idx = x + p.nx * (y + p.ny * z);
    const unsigned N = (unsigned)p.N;
    T fin[2][Q];
    pull_any<LAT, T>(f, x, y, z, p, fin);
    T rho1, rho2;
    const T psi_own = psi_of<Q, T>(fin, &rho1, &rho2);
    const T rho = rho1 + rho2;
    T j[3];
    momentum<LAT, T>(fin, j);
    const int c0 = (threadIdx.x + R) + RX * (threadIdx.y + R) + RXY * (threadIdx.z + RZoff);
    T grad[3], n[3];
    grad_smem<LAT, T>(sp, RX, RXY, c0, grad);
    const T g = M<T>::unit(grad, n);
    T frep[3] = {T(0), T(0), T(0)};
    int hit = 0;
    const bool iface = g > p.g_th;
    if (p.smax > 0 && iface) {
      static_for<kMaxProbe>([&](auto I) {
        constexpr int s = decltype(I)::value + 1;
        if (hit < 0 || hit > 0 || s > p.smax) return;  // stopped, found, or past h_max
        const int dx = round_probe<s, T>(T(s) * n[0]);
        const int dy = round_probe<s, T>(T(s) * n[1]);
        const int dz = D == 3 ? round_probe<s, T>(T(s) * n[2]) : 0;
        const int py = y + dy, pz = z + dz;
        if ((p.wall_y && (py < 0 || py >= p.ny)) || (D == 3 && p.wall_z && (pz < 0 || pz >= p.nz))) {
          hit = -1;  // the ray left the fluid through a wall: no facing interface
          return;
        }
        T gp[3], np_[3];
        grad_smem<LAT, T>(sp, RX, RXY, c0 + dx + RX * dy + RXY * dz, gp);
        const T gpn = M<T>::unit(gp, np_);
        if (!(gpn > p.g_th)) return;
        T dot = np_[0] * n[0] + np_[1] * n[1];
        if (D == 3) dot += np_[2] * n[2];
        if (dot < T(0)) hit = s;
      });
      if (hit < 0) hit = 0;
      if (hit) {
        const T A = p.Ah[hit];
        const T deltaI = T(0.5) * g;
        frep[0] = -A * n[0] * deltaI;
        frep[1] = -A * n[1] * deltaI;
        frep[2] = -A * n[2] * deltaI;
      }
    }
    T F[3], u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = p.G[a] + frep[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = M<T>::div(j[a] + T(0.5) * F[a], rho);

    if constexpr (FIELDS) {
      if (fo.rho1) fo.rho1[idx] = (double)rho1;
      if (fo.rho2) fo.rho2[idx] = (double)rho2;
      if (fo.psi) fo.psi[idx] = (double)psi_own;
      for (int a = 0; a < 3; ++a) {
        if (fo.grad) fo.grad[a * N + idx] = (double)grad[a];
        if (fo.frep) fo.frep[a * N + idx] = (double)frep[a];
        if (fo.u) fo.u[a * N + idx] = (double)u[a];
      }
      if (fo.hit) fo.hit[idx] = hit;
      const double r1 = rho1, r2 = rho2, rr = rho;
      red[0] = r1;
      red[1] = r2;
      red[2] = rr * (double)u[0];
      red[3] = rr * (double)u[1];
      red[4] = rr * (double)u[2];
      red[5] = rr * (double)u[0];
      red[6] = r1 * (double)u[0];
      red[7] = iface ? 1.0 : 0.0;
      red[8] = hit ? 1.0 : 0.0;
      const bool bad = !(isfinite(r1) && isfinite(r2) && rr > 0.0) ||
                       !(isfinite((double)u[0]) && isfinite((double)u[1]) && isfinite((double)u[2]));
      red[9] = bad ? 1.0 : 0.0;
    } else {
      const T m[3] = {-n[0], -n[1], -n[2]};
      collide_store<LAT, T, typename ST::Writer, EDM>(fin, rho1, rho2, j, u, F, g, m, p, fout, idx);
    }
  }

  if (FIELDS) {
    // Block reduction in FP64: warp shuffles, then one warp over the warp sums.
    __shared__ double wsum[8][kRedSlots];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < kRedSlots; ++q) {
      double v = red[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[warp][q] = v;
    }
    __syncthreads();
    if (warp == 0) {
      const int nw = (TX * TY * TZ) / 32;
#pragma unroll
      for (int q = 0; q < kRedSlots; ++q) {
        double v = lane < nw ? wsum[lane][q] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
          const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
          fo.partials[b * kRedSlots + q] = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------- setup
template <int LAT, typename ST>
__global__ void __launch_bounds__(256) init_kernel(typename ST::Writer f, const double* __restrict__ rho1,
                                                   const double* __restrict__ rho2,
                                                   const double* __restrict__ u, int N) {
  using T = typename ST::Compute;
  constexpr int Q = Lattice<LAT>::Q;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const size_t n = (size_t)N;
  T us[3] = {T(0), T(0), T(0)};
  if (u) { us[0] = T(u[idx]); us[1] = T(u[n + idx]); us[2] = T(u[2 * n + idx]); }
  const T uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  const T r[2] = {T(rho1[idx]), T(rho2[idx])};
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr T w = T(Lattice<LAT>::w(i));
    const T cu = T(cc(i, 0)) * us[0] + T(cc(i, 1)) * us[1] + T(cc(i, 2)) * us[2];
    const T e1 = w * r[0] * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
    const T e2 = w * r[1] * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
    f.template put<i>((unsigned)idx, e1, e2, r[0], r[1]);
  });
  f.put_rho((unsigned)idx, r[0], r[1]);
}

// FP64 [2][Q][pitch] copies of sites [s0, s0 + count) of a state and back: the site
// range lets the host move a state through a bounded staging buffer.
template <int LAT, typename ST>
__global__ void __launch_bounds__(256) decode_kernel(typename ST::Reader f, double* __restrict__ out, int s0,
                                                     int count, long long pitch) {
  using T = typename ST::Compute;
  constexpr int Q = Lattice<LAT>::Q;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    T a, b;
    f.template get<i>((unsigned)(s0 + j), a, b);
    out[(long long)i * pitch + j] = (double)a;
    out[(long long)(Q + i) * pitch + j] = (double)b;
  });
}

template <int LAT, typename ST>
__global__ void __launch_bounds__(256) encode_kernel(const double* __restrict__ in, typename ST::Writer f, int s0,
                                                     int count, long long pitch) {
  using T = typename ST::Compute;
  constexpr int Q = Lattice<LAT>::Q;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  T v[2][Q];
  T r1 = T(0), r2 = T(0);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    v[0][i] = T(in[(long long)i * pitch + j]);
    v[1][i] = T(in[(long long)(Q + i) * pitch + j]);
    r1 += v[0][i];
    r2 += v[1][i];
  });
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f.template put<i>((unsigned)(s0 + j), v[0][i], v[1][i], r1, r2);
  });
  f.put_rho((unsigned)(s0 + j), r1, r2);
}


}  // namespace lbnci
