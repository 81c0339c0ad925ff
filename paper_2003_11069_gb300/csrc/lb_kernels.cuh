// lb_kernels.cuh -- CUDA kernels of one colour-gradient NCI lattice Boltzmann step
// (arXiv:2003.11069, "Materials and Methods"), templated on the lattice and on the
// storage/compute type T (double or float). Instantiated by lb_fp64.cu (compiled
// without multiply-add contraction, the parity path) and lb_fp32.cu.
//
// Step = two launches:
//   moments_kernel : pull-stream the post-collision state, rho_k = sum_i f_i^k,
//                    psi = (rho1 - rho2)/(rho1 + rho2)  -> psi[N]
//   collide_kernel : stage the psi tile + halo of radius smax+1 in shared memory,
//                    gradient (isotropic, 2nd order), NCI ray search and F_rep,
//                    Guo velocity, BGK + Guo source + perturbation, recolouring,
//                    write f* to the other buffer.
// The fields variant of collide_kernel writes the macroscopic fields and block
// partial sums instead of populations.
#pragma once

#include "lb_lattice.cuh"

namespace lbnci {

template <typename T> __device__ __forceinline__ T tround(T v);
template <> __device__ __forceinline__ double tround<double>(double v) { return round(v); }
template <> __device__ __forceinline__ float tround<float>(float v) { return roundf(v); }
template <typename T> __device__ __forceinline__ T tsqrt(T v);
template <> __device__ __forceinline__ double tsqrt<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float tsqrt<float>(float v) { return sqrtf(v); }

// Wrap a coordinate that is at most one period out of range.
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
// Wrap any coordinate into [0, n).
__device__ __forceinline__ int wrapn(int v, int n) { int r = v % n; return r < 0 ? r + n : r; }

// Pull population i of component k into site (x,y,z): from the upstream site, or,
// when that lies beyond a wall, the opposite population of the site itself
// (halfway bounce-back).
template <int LAT, typename T>
__device__ __forceinline__ T pull(const T* __restrict__ f, int k, int i, int x, int y, int z,
                                  long long idx, const StepParams& p) {
  constexpr int Q = Lattice<LAT>::Q;
  const int sx = wrap1(x - cc(i, 0), p.nx);
  int sy = y - cc(i, 1);
  int sz = z - cc(i, 2);
  bool wall = false;
  if (p.wall_y) wall |= (sy < 0 || sy >= p.ny); else sy = wrap1(sy, p.ny);
  if (Lattice<LAT>::D == 3) {
    if (p.wall_z) wall |= (sz < 0 || sz >= p.nz); else sz = wrap1(sz, p.nz);
  } else {
    sz = 0;
  }
  const size_t N = (size_t)p.N;
  if (wall) return f[(size_t)(k * Q + opposite(i)) * N + (size_t)idx];
  const long long src = (long long)sx + (long long)p.nx * ((long long)sy + (long long)p.ny * sz);
  return f[(size_t)(k * Q + i) * N + (size_t)src];
}

template <int LAT, typename T>
__global__ void __launch_bounds__(256) moments_kernel(const T* __restrict__ f, T* __restrict__ psi,
                                                      StepParams p) {
  constexpr int Q = Lattice<LAT>::Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.N) return;
  const int x = (int)(idx % p.nx);
  const int y = (int)((idx / p.nx) % p.ny);
  const int z = (int)(idx / ((long long)p.nx * p.ny));
  T r[2] = {T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
#pragma unroll
    for (int i = 0; i < Q; ++i) r[k] += pull<LAT, T>(f, k, i, x, y, z, idx, p);
  }
  psi[idx] = (r[0] - r[1]) / (r[0] + r[1]);
}

// Isotropic gradient (1/c_s^2) sum_i w_i c_i psi(x + c_i) from the shared-memory
// region; a neighbour beyond a wall is replaced by its mirror image across the wall
// plane (the crossing velocity components are dropped). (lx,ly,lz): region
// coordinates, (gy,gz): global coordinates for the wall test.
template <int LAT, typename T>
__device__ __forceinline__ void grad_at(const T* __restrict__ sp, int RX, int RY, int lx, int ly,
                                        int lz, int gy, int gz, const StepParams& p, T g[3]) {
  constexpr int Q = Lattice<LAT>::Q;
  g[0] = T(0); g[1] = T(0); g[2] = T(0);
  const bool ylo = p.wall_y && gy == 0, yhi = p.wall_y && gy == p.ny - 1;
  const bool zlo = Lattice<LAT>::D == 3 && p.wall_z && gz == 0;
  const bool zhi = Lattice<LAT>::D == 3 && p.wall_z && gz == p.nz - 1;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int dy = cc(i, 1), dz = cc(i, 2);
    if ((dy < 0 && ylo) || (dy > 0 && yhi)) dy = 0;
    if ((dz < 0 && zlo) || (dz > 0 && zhi)) dz = 0;
    const T v = sp[(lx + cc(i, 0)) + RX * ((ly + dy) + RY * (lz + dz))];
    if (cc(i, 0) != 0) g[0] += T(Lattice<LAT>::w(i) * cc(i, 0)) * v;
    if (cc(i, 1) != 0) g[1] += T(Lattice<LAT>::w(i) * cc(i, 1)) * v;
    if (Lattice<LAT>::D == 3 && cc(i, 2) != 0) g[2] += T(Lattice<LAT>::w(i) * cc(i, 2)) * v;
  }
  g[0] = T(3) * g[0];
  g[1] = T(3) * g[1];
  g[2] = T(3) * g[2];
}

template <typename T>
__device__ __forceinline__ T norm3(const T g[3]) {
  return tsqrt<T>(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

// A_h(h): A for h <= h_min, A (h_min/h)^3 for h_min < h <= h_max, 0 beyond (Eq. near_c).
template <typename T>
__device__ __forceinline__ T nci_strength(int h, const StepParams& p) {
  const T hd = T(h);
  if (hd <= T(p.h_min)) return T(p.A_h);
  if (hd <= T(p.h_max)) {
    const T r = T(p.h_min) / hd;
    return T(p.A_h) * (r * r * r);
  }
  return T(0);
}

template <int LAT> __host__ __device__ constexpr int region_rz(int R) {
  return Lattice<LAT>::D == 3 ? Tile<LAT>::Z + 2 * R : 1;
}

template <int LAT, typename T>
size_t collide_smem_bytes(int smax) {
  const int R = smax + 1;
  return sizeof(T) * (size_t)(Tile<LAT>::X + 2 * R) * (Tile<LAT>::Y + 2 * R) * region_rz<LAT>(R);
}

template <int LAT, typename T, bool FIELDS>
__global__ void __launch_bounds__(256)
collide_kernel(const T* __restrict__ f, T* __restrict__ fout, const T* __restrict__ psi,
               StepParams p, FieldOut fo) {
  constexpr int D = Lattice<LAT>::D;
  constexpr int Q = Lattice<LAT>::Q;
  constexpr int TX = Tile<LAT>::X, TY = Tile<LAT>::Y, TZ = Tile<LAT>::Z;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sp = reinterpret_cast<T*>(smem_raw);

  const int R = p.smax + 1;
  const int RX = TX + 2 * R, RY = TY + 2 * R, RZ = region_rz<LAT>(R);
  const int RZoff = D == 3 ? R : 0;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);

  // Stage psi of the tile and its halo (periodic wrap; cells beyond a wall are never read).
  const int ncell = RX * RY * RZ;
  for (int t = tid; t < ncell; t += TX * TY * TZ) {
    const int lx = t % RX, ly = (t / RX) % RY, lz = t / (RX * RY);
    const int gx = wrapn(x0 - R + lx, p.nx);
    int gy = y0 - R + ly;
    int gz = D == 3 ? z0 - RZoff + lz : 0;
    bool out = false;
    if (p.wall_y) out |= (gy < 0 || gy >= p.ny); else gy = wrapn(gy, p.ny);
    if (D == 3) { if (p.wall_z) out |= (gz < 0 || gz >= p.nz); else gz = wrapn(gz, p.nz); }
    sp[t] = out ? T(0) : psi[(long long)gx + (long long)p.nx * ((long long)gy + (long long)p.ny * gz)];
  }
  __syncthreads();

  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
  const bool active = x < p.nx && y < p.ny && z < p.nz;

  double red[kRedSlots];
  if (FIELDS) for (int q = 0; q < kRedSlots; ++q) red[q] = 0.0;

  if (active) {
    const long long idx = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
    const size_t N = (size_t)p.N;
    // 1. pull
    T fin[2][Q];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int i = 0; i < Q; ++i) fin[k][i] = pull<LAT, T>(f, k, i, x, y, z, idx, p);
    // 2. moments
    T rho1 = T(0), rho2 = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) rho1 += fin[0][i];
#pragma unroll
    for (int i = 0; i < Q; ++i) rho2 += fin[1][i];
    const T rho = rho1 + rho2;
    T j[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const T fi = fin[0][i] + fin[1][i];
      if (cc(i, 0) != 0) j[0] += cc(i, 0) > 0 ? fi : -fi;
      if (cc(i, 1) != 0) j[1] += cc(i, 1) > 0 ? fi : -fi;
      if (D == 3 && cc(i, 2) != 0) j[2] += cc(i, 2) > 0 ? fi : -fi;
    }
    // 3. gradient, normal
    const int lx = threadIdx.x + R, ly = threadIdx.y + R, lz = threadIdx.z + RZoff;
    T grad[3];
    grad_at<LAT, T>(sp, RX, RY, lx, ly, lz, y, z, p, grad);
    const T g = norm3<T>(grad);
    // 4. NCI ray search along n = -grad psi/|grad psi|
    T frep[3] = {T(0), T(0), T(0)};
    int hit = 0;
    const bool iface = g > T(p.g_th);
    if (p.smax > 0 && iface) {
      T n[3];
      n[0] = -grad[0] / g;
      n[1] = -grad[1] / g;
      n[2] = D == 3 ? -grad[2] / g : T(0);
      for (int s = 1; s <= p.smax; ++s) {
        const int dx = (int)tround<T>(T(s) * n[0]);
        const int dy = (int)tround<T>(T(s) * n[1]);
        const int dz = D == 3 ? (int)tround<T>(T(s) * n[2]) : 0;
        const int py = y + dy, pz = z + dz;
        if (p.wall_y && (py < 0 || py >= p.ny)) break;
        if (D == 3 && p.wall_z && (pz < 0 || pz >= p.nz)) break;
        T gp[3];
        grad_at<LAT, T>(sp, RX, RY, lx + dx, ly + dy, lz + dz, py, pz, p, gp);
        const T gpn = norm3<T>(gp);
        if (!(gpn > T(p.g_th))) continue;
        T dot = (-gp[0] / gpn) * n[0] + (-gp[1] / gpn) * n[1];
        if (D == 3) dot += (-gp[2] / gpn) * n[2];
        if (dot < T(0)) { hit = s; break; }
      }
      if (hit) {
        const T A = nci_strength<T>(hit, p);
        const T deltaI = T(0.5) * g;
        frep[0] = -A * n[0] * deltaI;
        frep[1] = -A * n[1] * deltaI;
        frep[2] = -A * n[2] * deltaI;
      }
    }
    // 5. force and Guo velocity
    T F[3], u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = T(p.G[a]) + frep[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + T(0.5) * F[a]) / rho;

    if (FIELDS) {
      if (fo.rho1) fo.rho1[idx] = (double)rho1;
      if (fo.rho2) fo.rho2[idx] = (double)rho2;
      if (fo.psi) fo.psi[idx] = (double)((rho1 - rho2) / rho);
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
      // 6. BGK + Guo source + perturbation on the total population; 7. recolouring.
      T m[3] = {T(0), T(0), T(0)};
      if (g > T(0)) { m[0] = grad[0] / g; m[1] = grad[1] / g; m[2] = grad[2] / g; }
      const T omega = T(1) / T(p.tau);
      const T guo = T(1) - T(0.5) * omega;
      const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
      const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      const T seg = T(p.beta) * rho1 * rho2 / rho;
      const T pamp = T(2) * (T(0.5) * T(p.A_s)) * g;
      const T c1 = rho1 / rho, c2 = rho2 / rho;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const T w = T(Lattice<LAT>::w(i));
        const T fi = fin[0][i] + fin[1][i];
        const T cu = T(cc(i, 0)) * u[0] + T(cc(i, 1)) * u[1] + T(cc(i, 2)) * u[2];
        const T cF = T(cc(i, 0)) * F[0] + T(cc(i, 1)) * F[1] + T(cc(i, 2)) * F[2];
        const T cm = T(cc(i, 0)) * m[0] + T(cc(i, 1)) * m[1] + T(cc(i, 2)) * m[2];
        const T S = guo * w * (T(3) * (cF - uF) + T(9) * cu * cF);
        const T feq = w * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        T fs = fi - omega * (fi - feq) + S;
        fs += pamp * (w * cm * cm - w / T(3));
        const T inv_len = speed2(i) == 0 ? T(0) : T(1) / tsqrt<T>(T(speed2(i)));
        const T rc = seg * w * (cm * inv_len);
        fout[(size_t)i * N + idx] = c1 * fs + rc;
        fout[(size_t)(Q + i) * N + idx] = c2 * fs - rc;
      }
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

// Sum the per-block partials in a fixed order (deterministic) into out[kRedSlots].
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double* __restrict__ partials,
                                                              long long nblocks, double* __restrict__ out);

template <int LAT, typename T>
__global__ void __launch_bounds__(256) init_kernel(T* __restrict__ f, const double* __restrict__ rho1,
                                                   const double* __restrict__ rho2,
                                                   const double* __restrict__ u, long long N) {
  constexpr int Q = Lattice<LAT>::Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const size_t n = (size_t)N;
  T us[3] = {T(0), T(0), T(0)};
  if (u) { us[0] = T(u[idx]); us[1] = T(u[n + idx]); us[2] = T(u[2 * n + idx]); }
  const T uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  const T r[2] = {T(rho1[idx]), T(rho2[idx])};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const T cu = T(cc(i, 0)) * us[0] + T(cc(i, 1)) * us[1] + T(cc(i, 2)) * us[2];
    const T w = T(Lattice<LAT>::w(i));
#pragma unroll
    for (int k = 0; k < 2; ++k)
      f[(size_t)(k * Q + i) * n + idx] = w * r[k] * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
  }
}

template <typename S, typename D>
__global__ void __launch_bounds__(256) convert_kernel(const S* __restrict__ src, D* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = D(src[i]);
}

}  // namespace lbnci
