// lb_fused2d.cuh -- the whole D2Q9 step in one pass over the populations.
//
// A 256-thread block owns a 32 x (8*SPT) tile; each thread owns SPT sites of one
// column and keeps their 18 pulled populations in registers from the first phase to
// the collision, so each population is read from memory once for the collision.
//   phase 1: pull own sites (registers) and the psi halo of radius smax+1 (the halo's
//            populations are pulled, reduced to psi and dropped; neighbouring blocks
//            read the same lines, which L2 serves);
//   phase 2: unit normal n = -grad psi/|grad psi| and |grad psi| for the tile and a
//            halo of radius smax, once per cell, into shared memory;
//   phase 3: NCI ray search over the shared (n, |grad psi|) cells, Guo velocity,
//            BGK + source + perturbation, recolouring, store.
// Arithmetic is expression-for-expression that of the tiled kernel, so the FP64
// instantiation rounds like the oracle.
#pragma once

#include "lb_kernels.cuh"

namespace lbnci {

template <typename T>
size_t fused2d_smem_bytes(int smax, int spt) {
  const int R = smax + 1;
  const int TY = kFusedThreadsY * spt;
  const size_t psi = (size_t)(kFusedTX + 2 * R) * (TY + 2 * R);
  const size_t ng = 3 * (size_t)(kFusedTX + 2 * smax) * (TY + 2 * smax);
  return sizeof(T) * (psi + ng);
}

// Resident blocks per SM the fused kernels are built for (their register budget).
template <typename ST, int SPT>
constexpr int fused2d_min_blocks() {
  return SPT <= 2 ? (sizeof(typename ST::Compute) == 4 && !ST::kHalf ? 3 : 2) : 1;
}

// One 32 x (8*SPT) tile with origin (x0, y0) of a lattice; the whole block calls it.
template <typename ST, int SPT, bool EDM>
__device__ __forceinline__ void fused2d_tile(const typename ST::Reader& f, const typename ST::Writer& fout,
                                             const StepT<typename ST::Compute>& p, int x0, int y0,
                                             unsigned char* smem_raw) {
  using T = typename ST::Compute;
  constexpr int Q = 9, TX = kFusedTX, TYT = kFusedThreadsY, TY = TYT * SPT;
  constexpr int NT = TX * TYT;
  const int S = p.smax, R = S + 1;
  const int RX = TX + 2 * R, RY = TY + 2 * R;
  const int GX = TX + 2 * S, GY = TY + 2 * S, GXY = GX * GY;
  T* s_psi = reinterpret_cast<T*>(smem_raw);
  T* s_ng = s_psi + RX * RY;  // [3][GXY]: n_x, n_y, |grad psi|
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;

  // phase 1: own sites into registers, their psi into shared memory; an own position
  // beyond a ragged lattice edge holds the psi of the site it wraps to
  T fin[SPT][2][Q];
  bool act[SPT];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    const int x = x0 + tx, y = y0 + ty + s * TYT;
    act[s] = x < p.nx && y < p.ny;
    const int c = (tx + R) + RX * (ty + s * TYT + R);
    if (act[s]) {
      pull_any<0, T>(f, x, y, 0, p, fin[s]);
      s_psi[c] = psi_of<Q, T>(fin[s]);
    } else {
      const int gx = wrapn(x, p.nx);
      const int gy = p.wall_y ? clampc(y, p.ny) : wrapn(y, p.ny);
      T h[2][Q];
      pull_site<0, T>(f, gx, gy, 0, p, h);
      s_psi[c] = psi_of<Q, T>(h);
    }
  }
  // the halo ring of width R, enumerated compactly: two bands of R full rows, then
  // the R-wide left and right sides of the tile rows
  {
    const unsigned mRX = 0xFFFFFFFFu / (unsigned)RX + 1u;       // h / RX == umulhi(h, mRX)
    const unsigned m2R = 0xFFFFFFFFu / (unsigned)(2 * R) + 1u;  // exact for h < 2^16
    const int nband = R * RX, nside = 2 * R * TY;
    for (int h = tid; h < 2 * nband + nside; h += NT) {
      int lx, ly;
      if (h < 2 * nband) {
        const int hb = h < nband ? h : h - nband;
        const int row = (int)__umulhi((unsigned)hb, mRX);
        lx = hb - row * RX;
        ly = h < nband ? row : R + TY + row;
      } else {
        const int hs = h - 2 * nband;
        const int row = (int)__umulhi((unsigned)hs, m2R);
        const int col = hs - row * 2 * R;
        lx = col < R ? col : col + TX;
        ly = R + row;
      }
      // beyond a wall only the first row is read (as the mirror of the wall row)
      int gy = y0 - R + ly;
      if (p.wall_y && (gy < -1 || gy > p.ny)) continue;
      const int gx = wrapn(x0 - R + lx, p.nx);
      gy = p.wall_y ? clampc(gy, p.ny) : wrapn(gy, p.ny);
      T hf[2][Q];
      pull_any<0, T>(f, gx, gy, 0, p, hf);
      s_psi[lx + RX * ly] = psi_of<Q, T>(hf);
    }
  }
  __syncthreads();

  // phase 2: n and |grad psi| of every cell within smax of the tile
  for_region(tid, NT, GX, GY, 1, [&](int c, int lx, int ly, int) {
    int gy = y0 - S + ly;
    if (p.wall_y) { if (gy < 0 || gy >= p.ny) return; } else gy = wrapn(gy, p.ny);
    T grad[3], n[3];
    grad_smem<0, T>(s_psi, RX, 0, (lx + 1) + RX * (ly + 1), grad);
    const T g = M<T>::unit(grad, n);
    s_ng[c] = n[0];
    s_ng[GXY + c] = n[1];
    s_ng[2 * GXY + c] = g;
  });
  __syncthreads();

  // phase 3: NCI, forcing, collision, recolouring, store
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    if (!act[s]) continue;
    const int x = x0 + tx, y = y0 + ty + s * TYT;
    const int idx = x + p.nx * y;
    const int c = (tx + S) + GX * (ty + s * TYT + S);
    const T n0 = s_ng[c], n1 = s_ng[GXY + c], g = s_ng[2 * GXY + c];
    T rho1, rho2;
    psi_of<Q, T>(fin[s], &rho1, &rho2);
    const T rho = rho1 + rho2;
    T j[3];
    momentum<0, T>(fin[s], j);
    T frep[3] = {T(0), T(0), T(0)};
    if (S > 0 && g > p.g_th) {
      int hit = 0;
      static_for<kMaxProbe>([&](auto I) {
        constexpr int st = decltype(I)::value + 1;
        if (hit != 0 || st > S) return;  // found, stopped at a wall, or past h_max
        const int dx = round_probe<st, T>(T(st) * n0);
        const int dy = round_probe<st, T>(T(st) * n1);
        const int py = y + dy;
        if (p.wall_y && (py < 0 || py >= p.ny)) { hit = -1; return; }
        const int cp = c + dx + GX * dy;
        if (!(s_ng[2 * GXY + cp] > p.g_th)) return;
        const T dot = s_ng[cp] * n0 + s_ng[GXY + cp] * n1;
        if (dot < T(0)) hit = st;
      });
      if (hit < 0) hit = 0;
      if (hit) {
        const T A = p.Ah[hit];
        const T deltaI = T(0.5) * g;
        frep[0] = -A * n0 * deltaI;
        frep[1] = -A * n1 * deltaI;
      }
    }
    T F[3], u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = p.G[a] + frep[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = M<T>::div(j[a] + T(0.5) * F[a], rho);
    const T m[3] = {-n0, -n1, T(0)};
    collide_store<0, T, typename ST::Writer, EDM>(fin[s], rho1, rho2, j, u, F, g, m, p, fout, idx);
  }
}

template <typename ST, int SPT, bool EDM>
__global__ void __launch_bounds__(256, (fused2d_min_blocks<ST, SPT>()))
fused2d_kernel(typename ST::Reader f, typename ST::Writer fout, StepT<typename ST::Compute> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename ST::Writer w = fout;
  if constexpr (ST::kHalf)
    w.seed = step_seed(p, p.parity, blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0);
  fused2d_tile<ST, SPT, EDM>(f, w, p, blockIdx.x * kFusedTX, blockIdx.y * (kFusedThreadsY * SPT), smem_raw);
}

// One lattice of an ensemble: its step parameters, its two state buffers and the
// number of its tile columns; tiles of member m are blocks [tile0[m], tile0[m+1]).
template <typename T>
struct BatchMember {
  StepT<T> p;
  const void* buf[2];
  int ntx;
};

// The D2Q9 step of every member of an ensemble in one launch: block b finds its member
// by binary search over the tile offsets, then steps one tile of it with the member's
// own parameters, reading buf[parity] and writing buf[1 - parity].
template <typename ST, int SPT, bool EDM>
__global__ void __launch_bounds__(256, (fused2d_min_blocks<ST, SPT>()))
fused2d_batch_kernel(const BatchMember<typename ST::Compute>* __restrict__ members, const int* __restrict__ tile0,
                     int nmembers, int parity) {
  using T = typename ST::Compute;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  int lo = 0, hi = nmembers - 1;
  while (lo < hi) {  // last member whose first tile is <= b
    const int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= b) lo = mid; else hi = mid - 1;
  }
  const BatchMember<T>& mb = members[lo];
  const StepT<T> p = mb.p;
  const int t = b - tile0[lo];
  const int by = t / mb.ntx, bx = t - by * mb.ntx;
  const unsigned N = (unsigned)p.N;
  typename ST::Writer w = ST::writer(const_cast<void*>(mb.buf[1 - parity]), N);
  if constexpr (ST::kHalf)  // the member's first tile moves its seed on
    w.seed = step_seed(p, parity, t == 0 && threadIdx.x == 0 && threadIdx.y == 0);
  fused2d_tile<ST, SPT, EDM>(ST::reader(mb.buf[parity], N), w, p, bx * kFusedTX, by * (kFusedThreadsY * SPT),
                             smem_raw);
}

}  // namespace lbnci
