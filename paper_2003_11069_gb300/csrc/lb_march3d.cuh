// lb_march3d.cuh -- the collision half of the D3Q27 step, marching along z.
//
// A block walks columns of 64 x 8 sites (FP32 arithmetic: 512 threads, one CTA per SM;
// FP64: 32 x 8, 256 threads) through z segments: the launch has one CTA per resident
// slot and splits all columns' planes evenly between them. A column twice as wide as a
// 128-byte line halves the share of a warp's shifted pulls that reach into the
// neighbouring column's lines, which that column's CTA, at another z, has already let
// go from L2 (32 x 8 columns read the state 1.75 times from DRAM). Shared memory holds
// two rings of planes:
//   psi ring     3 planes of psi on the column plus a halo of smax + 1 (from the psi
//                array written by moments_kernel; the plane beyond a z wall holds the
//                mirror of the wall plane);
//   (n, g) ring  2 smax + 1 planes of the unit normal n = -grad psi/|grad psi| and
//                |grad psi| on the column plus a halo of smax, each computed once.
// Iteration q computes (n, g) of plane q - 1 and collides plane q - smax - 1, whose NCI
// rays find every probe's (n, g) in the ring; the loads of psi plane q + 1 are issued
// at the start of iteration q and stored into the ring at its end, so their latency
// overlaps the iteration's arithmetic. The psi array is
// read about three times per site instead of once per halo cell of a 3-D tile, and no
// gradient is recomputed along a ray. Arithmetic is that of the other step kernels
// (same helpers and expression order), so FP64 rounds like the oracle.
#pragma once

#include "lb_kernels.cuh"

namespace lbnci {

// Column of a block: 64 x 8 sites for 4-byte arithmetic (the rings take 182 KB for
// smax = 4), 32 x 8 for FP64 (202 KB).
template <typename T>
struct MarchTile {
  static constexpr int TX = sizeof(T) == 4 ? 64 : 32, TY = 8, NT = TX * TY;
};

template <typename T>
size_t march3d_smem_bytes(int smax) {
  constexpr int TX = MarchTile<T>::TX, TY = MarchTile<T>::TY;
  const int R = smax + 1;
  const size_t psi = 3 * (size_t)(TX + 2 * R) * (TY + 2 * R);
  const size_t ng = (size_t)(2 * smax + 1) * 4 * (TX + 2 * smax) * (TY + 2 * smax);
  return sizeof(T) * (psi + ng);
}

// Isotropic D3Q27 gradient of the cell c of a psi plane, with the planes below and
// above it in separate buffers (same direction order as grad_smem).
template <typename T>
__device__ __forceinline__ void grad_ring(const T* __restrict__ pm, const T* __restrict__ p0,
                                          const T* __restrict__ pp, int RX, int c, T g[3]) {
  g[0] = T(0); g[1] = T(0); g[2] = T(0);
  static_for<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i > 0) {
      constexpr T wx = T(Lattice<1>::w(i) * cc(i, 0));
      constexpr T wy = T(Lattice<1>::w(i) * cc(i, 1));
      constexpr T wz = T(Lattice<1>::w(i) * cc(i, 2));
      const T* pl = cc(i, 2) < 0 ? pm : (cc(i, 2) > 0 ? pp : p0);
      const T v = pl[c + cc(i, 0) + RX * cc(i, 1)];
      if constexpr (cc(i, 0) != 0) g[0] += wx * v;
      if constexpr (cc(i, 1) != 0) g[1] += wy * v;
      if constexpr (cc(i, 2) != 0) g[2] += wz * v;
    }
  });
  g[0] = T(3) * g[0];
  g[1] = T(3) * g[1];
  g[2] = T(3) * g[2];
}

// S = smax (number of NCI probe steps) is a template parameter: every extent of the
// rings, the plane ring's modulus and the probe loop are compile-time constants.
template <typename ST, bool EDM, int S>
__global__ void __launch_bounds__(MarchTile<typename ST::Compute>::NT, 1)
march3d_kernel(typename ST::Reader f, typename ST::Writer fout, const typename ST::Compute* __restrict__ psi,
               StepT<typename ST::Compute> p, int ncol_x, long long work) {
  using T = typename ST::Compute;
  constexpr int Q = 27, TX = MarchTile<T>::TX, TY = MarchTile<T>::TY, NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = S + 1, W = 2 * S + 1;
  constexpr int RX = TX + 2 * R, RY = TY + 2 * R, RXY = RX * RY;
  constexpr int GX = TX + 2 * S, GY = TY + 2 * S, GXY = GX * GY;
  T* s_psi = reinterpret_cast<T*>(smem_raw);  // [3][RXY]
  T* s_ng = s_psi + 3 * RXY;                   // [W][4][GXY]: n_x, n_y, n_z, |grad psi|
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  if constexpr (ST::kHalf) fout.seed = step_seed(p, p.parity, blockIdx.x == 0 && tid == 0);
  // ring slots of plane q >= -(2 S + 1) (the first psi plane and the lowest probe plane)
  auto ring3 = [](int q) { return (int)((unsigned)(q + 3 * W) % 3u); };
  auto ringW = [](int q) { return (int)((unsigned)(q + 2 * W) % (unsigned)W); };

  // The work is every column's nz planes, numbered column by column; each of the
  // gridDim.x CTAs (the resident ones) takes an equal share and marches through the
  // column segments in it, filling its rings afresh at each segment's start.
  const long long w0 = work * blockIdx.x / gridDim.x, w1 = work * (blockIdx.x + 1) / gridDim.x;
  for (long long w = w0; w < w1;) {
  const int col = (int)(w / p.nz);
  const int zs = (int)(w - (long long)col * p.nz);
  const int ze = (int)min((long long)p.nz, zs + (w1 - w));
  w += ze - zs;
  const int x0 = (col % ncol_x) * TX, y0 = (col / ncol_x) * TY;
  const int x = x0 + tx, y = y0 + ty;
  const bool col_active = x < p.nx && y < p.ny;

  // psi plane q (beyond a z wall only the first plane is read: the mirror of the wall
  // plane): this thread's cells c = tid + k NT, loaded into registers, then stored.
  constexpr int kPsiPer = (RXY + NT - 1) / NT;  // cells of a psi plane per thread
  auto psi_load = [&](int q, T v[kPsiPer]) {
    if (p.wall_z && (q < -1 || q > p.nz)) return;
    const int gz = p.wall_z ? clampc(q, p.nz) : wrapn(q, p.nz);
#pragma unroll
    for (int k = 0; k < kPsiPer; ++k) {
      const int c = tid + k * NT;
      if (c < RXY) {
        const int ly = c / RX, lx = c - ly * RX;
        const int gx = wrapn(x0 - R + lx, p.nx);
        const int gy = p.wall_y ? clampc(y0 - R + ly, p.ny) : wrapn(y0 - R + ly, p.ny);
        v[k] = psi[gx + p.nx * (gy + p.ny * gz)];
      }
    }
  };
  auto psi_store = [&](int q, const T v[kPsiPer]) {
    if (p.wall_z && (q < -1 || q > p.nz)) return;
    T* dst = s_psi + ring3(q) * RXY;
#pragma unroll
    for (int k = 0; k < kPsiPer; ++k) {
      const int c = tid + k * NT;
      if (c < RXY) dst[c] = v[k];
    }
  };
  {
    T v[kPsiPer];
    psi_load(zs - R, v);
    psi_store(zs - R, v);
  }
  __syncthreads();

  for (int q = zs - R; q < ze + R; ++q) {
    T vnext[kPsiPer];
    const bool more = q + 1 < ze + R;
    if (more) psi_load(q + 1, vnext);
    // (n, |grad psi|) of plane q - 1 on the column and a halo of smax
    const int qg = q - 1;
    if (qg >= zs - S && qg < ze + S && (!p.wall_z || (qg >= 0 && qg < p.nz))) {
      const T* pm = s_psi + ring3(qg - 1) * RXY;
      const T* p0 = s_psi + ring3(qg) * RXY;
      const T* pp = s_psi + ring3(qg + 1) * RXY;
      T* dst = s_ng + ringW(qg) * 4 * GXY;
      for_region(tid, NT, GX, GY, 1, [&](int c, int lx, int ly, int) {
        T grad[3], n[3];
        grad_ring<T>(pm, p0, pp, RX, (lx + 1) + RX * (ly + 1), grad);
        const T gn = M<T>::unit(grad, n);
        dst[c] = n[0];
        dst[GXY + c] = n[1];
        dst[2 * GXY + c] = n[2];
        dst[3 * GXY + c] = gn;
      });
    }
    __syncthreads();
    // collide plane z = q - R
    const int z = q - R;
    if (z >= zs && col_active) {
      const int idx = x + p.nx * (y + p.ny * z);
      T fin[2][Q];
      pull_any<1, T>(f, x, y, z, p, fin);
      T rho1, rho2;
      psi_of<Q, T>(fin, &rho1, &rho2);
      const T rho = rho1 + rho2;
      T j[3];
      momentum<1, T>(fin, j);
      const int c = (tx + S) + GX * (ty + S);
      const T* own = s_ng + ringW(z) * 4 * GXY;
      const T n0 = own[c], n1 = own[GXY + c], n2 = own[2 * GXY + c], g = own[3 * GXY + c];
      T frep[3] = {T(0), T(0), T(0)};
      if (S > 0 && g > p.g_th) {
        int hit = 0;
        T A = T(0);  // A_h(h) of the hit (indexed at compile time: no local copy of p)
        static_for<kMaxProbe>([&](auto I) {
          constexpr int st = decltype(I)::value + 1;
          if (hit != 0 || st > S) return;  // found, stopped at a wall, or past h_max
          const int dx = round_probe<st, T>(T(st) * n0);
          const int dy = round_probe<st, T>(T(st) * n1);
          const int dz = round_probe<st, T>(T(st) * n2);
          const int py = y + dy, pz = z + dz;
          if ((p.wall_y && (py < 0 || py >= p.ny)) || (p.wall_z && (pz < 0 || pz >= p.nz))) {
            hit = -1;
            return;
          }
          const T* pl = s_ng + ringW(pz) * 4 * GXY;
          const int cp = c + dx + GX * dy;
          if (!(pl[3 * GXY + cp] > p.g_th)) return;
          T dot = pl[cp] * n0 + pl[GXY + cp] * n1;
          dot += pl[2 * GXY + cp] * n2;
          if (dot < T(0)) { hit = st; A = p.Ah[st]; }
        });
        if (hit > 0) {
          const T deltaI = T(0.5) * g;
          frep[0] = -A * n0 * deltaI;
          frep[1] = -A * n1 * deltaI;
          frep[2] = -A * n2 * deltaI;
        }
      }
      T F[3], u[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) F[a] = p.G[a] + frep[a];
#pragma unroll
      for (int a = 0; a < 3; ++a) u[a] = M<T>::div(j[a] + T(0.5) * F[a], rho);
      const T m[3] = {-n0, -n1, -n2};
      collide_store<1, T, typename ST::Writer, EDM>(fin, rho1, rho2, j, u, F, g, m, p, fout, idx);
    }
    // plane q + 1 replaces plane q - 2, whose last reader was the (n, g) pass above
    if (more) psi_store(q + 1, vnext);
    __syncthreads();
  }
  }  // column segments
}

}  // namespace lbnci
