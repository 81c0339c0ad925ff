// lb_carry3d.cuh -- D3Q27 steps on lattices of whole 32 x 8 columns for FP32 and FP16-dev
// storage (arXiv:2003.11069, "Materials and Methods": Eq. (CGLBE), the colour gradient,
// the near-contact force of Eq. (near_c) and Omega = Omega^(3)[Omega^(1) + Omega^(2)]):
// the single-read step described first, and, at the end of the file, the streaming step
// (normals3d_kernel, collide3d_kernel after moments_kernel), the default, with the total +
// recolouring form of the state (TotalRecol, collide3t_kernel) that its FP32 steps under
// Guo forcing store.
//
// Single-read step: every population is read once.
//
// The colour gradient at a site needs psi, hence the densities rho_k, of its 26
// neighbours, and rho_k(y) at the start of a step sums the populations streamed into y:
// rho_k(y) = sum_i f*_i^k(y - c_i). Instead of re-reading the state for them, the
// collision of the previous step produces them ("density carry"): every site's 27 new
// populations are summed into the densities of the sites they stream into.
//
// Three kernels per step:
//   interface3d_kernel  (columns of 32 x 8 sites marching along z) rho_k of each site =
//                       its column's carried part + the parts the neighbouring columns
//                       exported into it; psi; isotropic gradient; writes
//                       (n, |grad psi|) per site (16 bytes).
//   nci3d_kernel        the near-contact ray of every interface site over those normals
//                       (probes read through L2); writes the distance h (0..4) per site
//                       (1 byte). A kernel of its own so that the probes' dependent
//                       loads are hidden by many resident warps.
//   carry3d_kernel      per plane of a 32 x 8 column marching along z through a segment of
//                       zseg planes (items (segment, column), taken segment by segment by
//                       two persistent CTAs per SM): TMA copies bring,
//                       for each of the 54 population planes, exactly the 36 x 8 window
//                       its direction pulls from (x0-4.. or x0.., rows y0-c_y..) into
//                       shared memory; pull, Guo forcing with the NCI force, BGK +
//                       perturbation + recolouring, coalesced stores of the 54 new
//                       populations; then the carry of the new populations: summed
//                       along x by warp shuffles, along y through shared memory, along z
//                       in registers as the column marches, into the next step's
//                       densities of the column's sites and of the 84-cell ring just
//                       outside it (exported, one writer per slot: deterministic). The
//                       parts a segment sends into the plane below its first and above
//                       its last plane (34 x 10 cells each: the column and its ring) are
//                       exported as ghost planes.
// A population whose target lies beyond a wall bounces back into its own site (halfway
// bounce-back), so it is carried into its own site's density.
//
// Every wait on the copy's mbarrier is bounded (about a second); on expiry the kernel
// sets bit 0 of the error word, waits (bounded) for its copy in flight and returns; a
// shared-memory base that is not 1024-byte aligned sets bit 1 before anything is copied.
#pragma once

#include "lb_kernels.cuh"
#include "lb_march3d.cuh"
#include "lb_tma.cuh"

namespace lbnci {

// Columns: 32 x 8 sites, one thread per site.
constexpr int kC3X = 32, kC3Y = 8, kC3T = kC3X * kC3Y;
// The ring of a column (per plane): the cells just outside it that its new populations
// stream into. Records of kRing float2 (rho1, rho2): x0-1 for rows y0-1..y0+8 (XL),
// x0+32 for the same rows (XR), row y0-1 for x0..x0+31 (YB), row y0+8 (YT).
constexpr int kRingXL = 0, kRingXR = kC3Y + 2, kRingYB = 2 * (kC3Y + 2), kRingYT = kRingYB + kC3X;
constexpr int kRing = kRingYT + kC3X;  // 84

struct CarryGrid {
  int nx, ny, nz;
  int ncx, ncy;  // columns along x and y (nx / 32, ny / 8)
  int wall_y, wall_z;
  int zseg, nseg;  // planes per z segment of the collision kernel, number of segments
};

__host__ __device__ __forceinline__ size_t ring_base(int col, int z, int nz) {
  return ((size_t)col * nz + z) * kRing;
}

// Ghost planes: per (column, segment, side) the 34 x 10 cells (x0-1..x0+32, y0-1..y0+8)
// of the plane below the segment's first plane (side 0) or above its last (side 1).
constexpr int kGhostX = kC3X + 2, kGhostCells = kGhostX * (kC3Y + 2);  // 340
__host__ __device__ __forceinline__ size_t ghost_base(int col, int seg, int side, int nseg) {
  return (((size_t)col * nseg + seg) * 2 + side) * kGhostCells;
}

// (rho1, rho2) of site (x, y, z): its column's carried part; what the x-side, the
// y-side and the diagonal neighbouring columns exported into it (ring records of plane
// z); then, on a segment's first plane, the up-ghosts of the segment below (own, x-side,
// y-side, diagonal column) and, on a segment's last plane, the down-ghosts of the
// segment above (this order).
__device__ __forceinline__ float2 carry_density(const float2* __restrict__ carry, const float2* __restrict__ ring,
                                                const float2* __restrict__ ghost, const CarryGrid& g, int x, int y,
                                                int z) {
  float2 r = carry[x + g.nx * (y + g.ny * z)];
  const int cx = x >> 5, lx = x & (kC3X - 1), cy = y >> 3, ly = y & (kC3Y - 1);
  int cxn = -1, xs = 0, cyn = -1, ys = 0;
  if (lx == 0) { cxn = cx == 0 ? g.ncx - 1 : cx - 1; xs = kRingXR; }
  else if (lx == kC3X - 1) { cxn = cx == g.ncx - 1 ? 0 : cx + 1; xs = kRingXL; }
  if (ly == 0) { cyn = cy > 0 ? cy - 1 : (g.wall_y ? -1 : g.ncy - 1); ys = kRingYT; }
  else if (ly == kC3Y - 1) { cyn = cy < g.ncy - 1 ? cy + 1 : (g.wall_y ? -1 : 0); ys = kRingYB; }
  auto add = [&](float2 e) {
    r.x += e.x;
    r.y += e.y;
  };
  if (cxn >= 0) add(ring[ring_base(cxn + g.ncx * cy, z, g.nz) + xs + ly + 1]);
  if (cyn >= 0) add(ring[ring_base(cx + g.ncx * cyn, z, g.nz) + ys + lx]);
  if (cxn >= 0 && cyn >= 0)  // the diagonal column's x-side record: its row y0+8 or y0-1
    add(ring[ring_base(cxn + g.ncx * cyn, z, g.nz) + xs + (ly == 0 ? kC3Y + 1 : 0)]);
  // the cell in the ghost planes of this column and of the neighbours that hold it
  const int gx_own = lx + 1, gy_own = ly + 1;
  const int gx_x = lx == 0 ? kC3X + 1 : 0;       // in the x-side neighbour's ghost plane
  const int gy_y = ly == 0 ? kC3Y + 1 : 0;       // in the y-side neighbour's ghost plane
  const int seg = z / g.zseg;
  const int zf = seg * g.zseg, zl = min(zf + g.zseg, g.nz) - 1;
  auto ghosts = [&](int sg, int side) {
    add(ghost[ghost_base(cx + g.ncx * cy, sg, side, g.nseg) + gy_own * kGhostX + gx_own]);
    if (cxn >= 0) add(ghost[ghost_base(cxn + g.ncx * cy, sg, side, g.nseg) + gy_own * kGhostX + gx_x]);
    if (cyn >= 0) add(ghost[ghost_base(cx + g.ncx * cyn, sg, side, g.nseg) + gy_y * kGhostX + gx_own]);
    if (cxn >= 0 && cyn >= 0) add(ghost[ghost_base(cxn + g.ncx * cyn, sg, side, g.nseg) + gy_y * kGhostX + gx_x]);
  };
  if (z == zf) {  // the segment below sends its up-ghost (periodic z: the last segment)
    const int sb = seg > 0 ? seg - 1 : (g.wall_z ? -1 : g.nseg - 1);
    if (sb >= 0) ghosts(sb, 1);
  }
  if (z == zl) {  // the segment above sends its down-ghost (periodic z: the first segment)
    const int sa = seg < g.nseg - 1 ? seg + 1 : (g.wall_z ? -1 : 0);
    if (sa >= 0) ghosts(sa, 0);
  }
  return r;
}

// ------------------------------------------------------------------ densities from a state
// The carry of a state that no step produced (after lb_init_fields / lb_set_populations):
// the pulled densities of every site, complete, so the rings are zero.
template <typename ST>
__global__ void __launch_bounds__(256) carry_init_kernel(typename ST::Reader f, float2* __restrict__ carry,
                                                         StepT<float> p) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.N) return;
  const int x = idx % p.nx, y = (idx / p.nx) % p.ny, z = idx / (p.nx * p.ny);
  float fin[2][27];
  pull_any<1, float>(f, x, y, z, p, fin);
  float r1, r2;
  psi_of<27, float>(fin, &r1, &r2);
  carry[idx] = make_float2(r1, r2);
}

// ------------------------------------------------------------------ interface pass
// Blocks of 32 x 8 x kI3Z sites (one column, kI3Z planes; 256 threads, kI3Z sites each):
// psi of the block and its one-cell ring (34 x 10 x (kI3Z + 2) cells; beyond a wall the
// mirror cell, along periodic axes the image) from the carried densities, one barrier,
// then each site's isotropic gradient: n = -grad psi/|grad psi| and |grad psi|.
constexpr int kI3Z = 8;
__global__ void __launch_bounds__(kC3T) interface3d_kernel(const float2* __restrict__ carry,
                                                           const float2* __restrict__ ring,
                                                           const float2* __restrict__ ghost,
                                                           float4* __restrict__ ng, CarryGrid g) {
  constexpr int RX = kC3X + 2, RY = kC3Y + 2, RXY = RX * RY, RZ = kI3Z + 2, NR = RXY * RZ;
  __shared__ float s_psi[NR];
  const int col = blockIdx.x, cx = col % g.ncx, cy = col / g.ncx;
  const int x0 = cx * kC3X, y0 = cy * kC3Y, z0 = blockIdx.y * kI3Z;
  const int tid = threadIdx.x, tx = tid & (kC3X - 1), ty = tid >> 5;
  for (int c = tid; c < NR; c += kC3T) {
    const int rz = c / RXY, rxy = c - rz * RXY, ry = rxy / RX, rx = rxy - ry * RX;
    const int gx = wrapn(x0 - 1 + rx, g.nx);
    const int gy = g.wall_y ? clampc(y0 - 1 + ry, g.ny) : wrapn(y0 - 1 + ry, g.ny);
    const int gz = g.wall_z ? clampc(z0 - 1 + rz, g.nz) : wrapn(z0 - 1 + rz, g.nz);
    const float2 r = carry_density(carry, ring, ghost, g, gx, gy, gz);
    s_psi[c] = M<float>::div(r.x - r.y, r.x + r.y);
  }
  __syncthreads();
  const int nz_here = min(kI3Z, g.nz - z0);
  const size_t nxy = (size_t)g.nx * g.ny;
  const size_t site_xy = (size_t)(x0 + tx) + (size_t)g.nx * (y0 + ty);
  for (int k = 0; k < nz_here; ++k) {
    float grad[3], n[3];
    const float* p0 = s_psi + (k + 1) * RXY;
    grad_ring<float>(p0 - RXY, p0, p0 + RXY, RX, (tx + 1) + RX * (ty + 1), grad);
    const float gg = M<float>::unit(grad, n);
    ng[site_xy + nxy * (z0 + k)] = make_float4(n[0], n[1], n[2], gg);
  }
}

// ------------------------------------------------------------------ NCI ray
// h(x) of every site from the interface pass's (n, |grad psi|): x is an interface site
// when |grad psi| > g_th; probes y_s = x + round(s n), s = 1..smax (half away from zero
// per component); a probe beyond a wall ends the search; the first probe that is an
// interface site facing x (n(y).n(x) < 0) gives h = s. Blocks of 32 x 8 sites, one plane.
__device__ __forceinline__ int nci_ray(const float4* __restrict__ ng, const float4 v, int x, int y, int z,
                                       const StepT<float>& p) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  int h = 0;
  if (v.w > p.g_th) {
    const float n0 = v.x, n1 = v.y, n2 = v.z;
    float4 q[kMaxProbe];
    int stop = kMaxProbe + 1;
    // probes in two batches (s = 1, 2, then 3, 4 when still needed): each batch's loads
    // are issued together, then decided in order
    auto load = [&](auto I) {
      constexpr int s = decltype(I)::value + 1;
      q[s - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s > p.smax || s >= stop) return;
      const int dx = round_probe<s, float>(float(s) * n0);
      const int dy = round_probe<s, float>(float(s) * n1);
      const int dz = round_probe<s, float>(float(s) * n2);
      int px = x + dx, py = y + dy, pz = z + dz;
      if ((p.wall_y && (py < 0 || py >= ny)) || (p.wall_z && (pz < 0 || pz >= nz))) {
        stop = s;  // the ray leaves the fluid through a wall: no facing interface
        return;
      }
      px = px < 0 ? px + nx : (px >= nx ? px - nx : px);
      if (!p.wall_y) py = wrapn(py, ny);
      if (!p.wall_z) pz = wrapn(pz, nz);
      q[s - 1] = ng[(unsigned)px + (unsigned)nx * ((unsigned)py + (unsigned)ny * (unsigned)pz)];
    };
    auto decide = [&](auto I) {
      constexpr int s = decltype(I)::value + 1;
      if (h != 0 || s > p.smax || s >= stop) return;
      const float4 w = q[s - 1];
      if (!(w.w > p.g_th)) return;
      float dot = w.x * n0 + w.y * n1;
      dot += w.z * n2;
      if (dot < 0.f) h = s;
    };
    static_assert(kMaxProbe == 4, "two batches of two probes");
    load(std::integral_constant<int, 0>{});
    load(std::integral_constant<int, 1>{});
    decide(std::integral_constant<int, 0>{});
    decide(std::integral_constant<int, 1>{});
    if (h == 0 && stop > 2 && p.smax > 2) {
      load(std::integral_constant<int, 2>{});
      load(std::integral_constant<int, 3>{});
      decide(std::integral_constant<int, 2>{});
      decide(std::integral_constant<int, 3>{});
    }
  }
  return h;
}

__global__ void __launch_bounds__(256) nci3d_kernel(const float4* __restrict__ ng, unsigned char* __restrict__ hit,
                                                    StepT<float> p) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  const unsigned site = (unsigned)x + (unsigned)p.nx * ((unsigned)y + (unsigned)p.ny * (unsigned)z);
  hit[site] = (unsigned char)nci_ray(ng, ng[site], x, y, z, p);
}

// ------------------------------------------------------------------ collision + carry
// Shared-memory stage of one plane: for each class of directions (c_y, c_z) and
// component k, one 40 x 8 x 3 window: columns x0-4..x0+35, rows y0-c_y..y0+7-c_y of the
// source plane z - c_z, for the class's three population planes c_x = 0, +1, -1 (digit
// order; one TMA copy). FP16-dev: the nine classes' half2 deviation windows, then the
// reference densities of the three source planes (40 x 10 cells from x0-4, y0-1).
constexpr int kW3X = 40, kW3Y = kC3Y, kW3Cells = kW3X * kW3Y;
constexpr unsigned kW3Bytes = 3 * kW3Cells * 4;  // 3,840: one class window (a multiple of 128)
constexpr int kR3X = 40, kR3Y = kC3Y + 2, kR3Cells = kR3X * kR3Y;
constexpr unsigned kR3Bytes = kR3Cells * 8;  // 3,200
static_assert(kW3Bytes % 128 == 0 && kR3Bytes % 128 == 0, "TMA destinations stay 128-byte aligned");

// Direction i's float within its class window, relative to the thread's cell ty*40 + tx:
// population plane (digit of c_x) and the column of the source site x - c_x.
__host__ __device__ constexpr int win_off(int i) { return (i % 3) * kW3Cells + 4 - cc(i, 0); }

// Every stage also holds the plane's (n, |grad psi|) (32 x 8 float4) and NCI distances
// (32 x 8 bytes), copied with the populations.
constexpr unsigned kNgBytes = kC3T * 16, kHitBytes = kC3T;
template <typename ST> struct C3Stage;
template <> struct C3Stage<Plain<1, float>> {  // window of (k, class c) at (9 k + c) kW3Bytes
  static constexpr int kNgOff = 18 * (int)kW3Bytes;
  static constexpr int kHitOff = kNgOff + (int)kNgBytes;
  static constexpr unsigned kTx = 18 * kW3Bytes + kNgBytes + kHitBytes;
  static constexpr int kSize = kHitOff + (int)kHitBytes;
};
template <> struct C3Stage<HalfDev<1>> {  // deviation window of class c at c kW3Bytes, then densities
  static constexpr int kRhoOff = 9 * (int)kW3Bytes;
  static constexpr int kNgOff = kRhoOff + 3 * (int)kR3Bytes;
  static constexpr int kHitOff = kNgOff + (int)kNgBytes;
  static constexpr unsigned kTx = 9 * kW3Bytes + 3 * kR3Bytes + kNgBytes + kHitBytes;
  static constexpr int kSize = kHitOff + (int)kHitBytes;
};

// Shared memory of carry3d_kernel (bytes from a 1024-aligned base): the stage, two
// buffers (alternate planes) of the y-exchange of the x-summed carry (classes c_y = +1,
// -1, 0 x c_z digit x 8 rows x 34 cells, float2), the ring cells' running sums, the
// "full" mbarrier (the stage's copies landed), the "empty" one (every warp has pulled
// from the stage), a counter of the warps done pulling, an abort flag.
constexpr int kC3ACols = kC3X + 2;
constexpr int kC3AFloats2 = 3 * 3 * kC3Y * kC3ACols;
constexpr int kC3ABytes = 2 * kC3AFloats2 * 8;  // 39,168
constexpr int kC3Warps = kC3T / 32;
struct RingAcc {
  float2 acc, bp;
};
template <typename ST> struct C3Smem {
  static constexpr int kOffA = (C3Stage<ST>::kSize + 1023) / 1024 * 1024;
  static constexpr int kOffRing = kOffA + kC3ABytes;
  static constexpr int kOffBar = kOffRing + kRing * (int)sizeof(RingAcc);  // full, empty, count, abort
  static constexpr int kBytes = kOffBar + 64;
};
static_assert(2 * (C3Smem<Plain<1, float>>::kBytes + 1024) <= 228 * 1024, "two CTAs per SM");

// The collision's writer: stores the new populations and keeps each one as the next
// step will pull it (FP16-dev: decoded from its stored deviation) for the carry.
template <typename ST> struct C3Writer;
template <> struct C3Writer<Plain<1, float>> {
  float* __restrict__ f;
  unsigned N;
  float (*o)[27];
  template <int I>
  __device__ __forceinline__ void put_step(unsigned site, float a, float b, float, float, unsigned) const {
    (f + (size_t)I * N)[site] = a;
    (f + (size_t)(27 + I) * N)[site] = b;
    o[0][I] = a;
    o[1][I] = b;
  }
  __device__ __forceinline__ unsigned site_bits(unsigned) const { return 0u; }
  __device__ __forceinline__ void put_rho(unsigned, float, float) const {}
};
template <> struct C3Writer<HalfDev<1>> {
  __half2* __restrict__ d;
  float2* __restrict__ rho;
  unsigned N;
  unsigned seed;
  float (*o)[27];
  __device__ __forceinline__ unsigned site_bits(unsigned site) const { return dither_bits(site, seed); }
  template <int I>
  __device__ __forceinline__ void put_step(unsigned site, float a, float b, float r1, float r2, unsigned hb) const {
    constexpr float w = float(Lattice<1>::w(I));
    const unsigned v = half2_stochastic<I>(fmaf(-w, r1, a), fmaf(-w, r2, b), hb);
    reinterpret_cast<unsigned*>(d)[(size_t)I * N + site] = v;
    const float2 fv = __half22float2(*reinterpret_cast<const __half2*>(&v));
    o[0][I] = fmaf(w, r1, fv.x);
    o[1][I] = fmaf(w, r2, fv.y);
  }
  __device__ __forceinline__ void put_rho(unsigned site, float r1, float r2) const {
    rho[site] = make_float2(r1, r2);
  }
};

// Pull of direction I from the stage; t = ty * 36 + tx (the thread's window cell before
// the direction's column offset), c = its cell in the 40 x 10 density box.
template <typename ST> struct C3Pull;
template <> struct C3Pull<Plain<1, float>> {
  template <int I>
  static __device__ __forceinline__ void get(const unsigned char* sm, int t, int, float& a, float& b) {
    const float* w0 = reinterpret_cast<const float*>(sm + (I / 3) * kW3Bytes);
    const float* w1 = reinterpret_cast<const float*>(sm + (9 + I / 3) * kW3Bytes);
    a = w0[t + win_off(I)];
    b = w1[t + win_off(I)];
  }
};
template <> struct C3Pull<HalfDev<1>> {
  template <int I>
  static __device__ __forceinline__ void get(const unsigned char* sm, int t, int c, float& a, float& b) {
    constexpr int gz = I / 9;
    constexpr float w = float(Lattice<1>::w(I));
    const __half2* dv = reinterpret_cast<const __half2*>(sm + (I / 3) * kW3Bytes);
    const float2* rr = reinterpret_cast<const float2*>(sm + C3Stage<HalfDev<1>>::kRhoOff + gz * (int)kR3Bytes);
    const float2 v = __half22float2(dv[t + win_off(I)]);
    const float2 r = rr[c - cc(I, 1) * kR3X - cc(I, 0)];
    a = fmaf(w, r.x, v.x);
    b = fmaf(w, r.y, v.y);
  }
};

struct Carry3dArgs {
  const float4* ng;          // (n, |grad psi|) per site, from interface3d_kernel
  const unsigned char* hit;  // NCI distance h per site, from nci3d_kernel
  float2* carry;             // out: next step's densities, column part
  float2* ring;              // out: next step's densities, ring exports
  float2* ghost;             // out: next step's densities, ghost planes of the segments
  int* err;                  // bit 0: a copy's wait expired; bit 1: misaligned shared memory
  int ncx, ncol;
  int zseg, nseg, nitems;    // items: segment-major, item k = (segment k / ncol, column k % ncol)
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Running z-sum of one cell's carry through a segment [zs, ze): final(z) =
// (b(z; 0) + b(z-1; +1)) + b(z+1; -1), where b(z; c) sums the populations of plane z moving
// by c along z. The segment's first plane lacks b(zs-1; +1) and its last b(ze; -1): they
// come from the neighbouring segments' ghosts, to which this segment sends b(zs; -1)
// (down) and b(ze-1; +1) (up).
using RingAccZ = RingAcc;
template <typename Out, typename Ghost>
__device__ __forceinline__ void zsum(RingAccZ& A, float2 b0, float2 bp, float2 bm, int z, int zs, Out&& out,
                                     Ghost&& down) {
  if (z > zs) {
    out(z - 1, f2add(A.acc, bm));
    A.acc = f2add(b0, A.bp);
  } else {
    down(bm);
    A.acc = b0;
  }
  A.bp = bp;
}
template <typename Out, typename Ghost>
__device__ __forceinline__ void zsum_end(const RingAccZ& A, int ze, Out&& out, Ghost&& up) {
  out(ze - 1, A.acc);
  up(A.bp);
}

template <typename ST, bool EDM>
__global__ void __launch_bounds__(kC3T, 2)
carry3d_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
               const __grid_constant__ CUtensorMap map_ng, const __grid_constant__ CUtensorMap map_hit,
               typename ST::Reader f, typename ST::Writer fw, StepT<float> p, Carry3dArgs a) {
  constexpr bool HALF = ST::kHalf;
  using SM = C3Smem<ST>;
  extern __shared__ __align__(1024) unsigned char sm[];
  float2* const s_a0 = reinterpret_cast<float2*>(sm + SM::kOffA);  // [2][cls 3][czd 3][row 8][34]
  RingAcc* s_ring = reinterpret_cast<RingAcc*>(sm + SM::kOffRing);
  unsigned long long* bar_full = reinterpret_cast<unsigned long long*>(sm + SM::kOffBar);
  unsigned long long* bar_empty = bar_full + 1;
  int* s_cnt = reinterpret_cast<int*>(sm + SM::kOffBar + 16);
  volatile int* s_abort = s_cnt + 1;

  const int tid = threadIdx.x, tx = tid & (kC3X - 1), ty = tid >> 5;
  if (smem_u32(sm) & 1023u) {
    if (tid == 0) atomicOr(a.err, 2);
    return;
  }
  if (tid == 0) {
    mbar_init(bar_full, 1);
    mbar_init(bar_empty, kC3Warps);
    *s_cnt = 0;
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_a)) : "memory");
    if (HALF) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_b)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_ng)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_hit)) : "memory");
  }
  __syncthreads();

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  unsigned seed = 0u;  // dither seed of the FP16 stores
  if constexpr (HALF) seed = step_seed(p, p.parity, blockIdx.x == 0 && tid == 0);
  // One warp: the copies of plane z of a column, lane w < 18 the class window w (FP32:
  // class w % 9 of component w / 9; FP16-dev: lanes < 9), lanes 27..29 the density
  // boxes (FP16-dev), lanes 30, 31 the plane's (n, |grad psi|) and NCI distances.
  auto issue = [&](int item, int z) {
    const int col = item % a.ncol;
    const int x0 = (col % a.ncx) * kC3X, y0 = (col / a.ncx) * kC3Y;
    if (tx == 0) mbar_expect_tx(bar_full, C3Stage<ST>::kTx);
    __syncwarp();
    if (tx < (HALF ? 9 : 18)) {
      const int c = tx % 9, k = tx / 9;  // class (digits of c_y, c_z) and component
      const int cy = digit_c(c % 3), cz = digit_c(c / 3);
      int zs = z - cz;  // source plane (beyond a z wall: zero fill, never read)
      if (!p.wall_z) zs = wrapn(zs, nz);
      if constexpr (HALF) tma_load_4d(sm + c * kW3Bytes, &map_a, x0 - 4, y0 - cy, zs, 3 * c, bar_full);
      else tma_load_5d(sm + tx * kW3Bytes, &map_a, x0 - 4, y0 - cy, zs, 0, c + 9 * k, bar_full);
    } else if (tx == 30) {
      tma_load_3d(sm + C3Stage<ST>::kNgOff, &map_ng, 4 * x0, y0, z, bar_full);
    } else if (tx == 31) {
      tma_load_3d(sm + C3Stage<ST>::kHitOff, &map_hit, x0, y0, z, bar_full);
    } else if constexpr (HALF) {
      if (tx >= 27 && tx < 30) {  // the density boxes of source planes z, z - 1, z + 1
        const int gz = tx - 27;
        int zs = z - (gz == 0 ? 0 : (gz == 1 ? 1 : -1));
        if (!p.wall_z) zs = wrapn(zs, nz);
        tma_load_3d(sm + C3Stage<ST>::kRhoOff + gz * kR3Bytes, &map_b, 2 * (x0 - 4), y0 - 1, zs, bar_full);
      }
    }
  };

  unsigned ph_full = 0, ph_empty = 0, it = 0;
  int item = blockIdx.x;
  auto seg_of = [&](int k, int& zs, int& ze) {
    const int sg = k / a.ncol;
    zs = sg * a.zseg;
    ze = min(zs + a.zseg, nz);
  };
  if (item < a.nitems && ty == 0) {
    int zs, ze;
    seg_of(item, zs, ze);
    issue(item, zs);
  }
  // The ring cells this thread owns (their running sums live in shared memory): the
  // x-side cell of its row (lanes 0, 31), a corner (lanes 0, 31 of rows 0, 7), the
  // y-side cell of its column (rows 0, 7); -1 = none.
  int rid[3] = {-1, -1, -1};
  if (tx == 0 || tx == kC3X - 1) {
    const int base = tx == 0 ? kRingXL : kRingXR;
    rid[0] = base + ty + 1;
    if (ty == 0) rid[1] = base;
    if (ty == kC3Y - 1) rid[1] = base + kC3Y + 1;
  }
  if (ty == 0) rid[2] = kRingYB + tx;
  if (ty == kC3Y - 1) rid[2] = kRingYT + tx;
  // a ring cell's place in the ghost planes (34 x 10)
  auto ring_ghost = [](int id) {
    if (id < kRingXR) return (id - kRingXL) * kGhostX;
    if (id < kRingYB) return (id - kRingXR) * kGhostX + kC3X + 1;
    if (id < kRingYT) return 1 + (id - kRingYB);
    return (kC3Y + 1) * kGhostX + 1 + (id - kRingYT);
  };

  while (item < a.nitems) {
    const int col = item % a.ncol, seg = item / a.ncol;
    int zs, ze;
    seg_of(item, zs, ze);
    const int x0 = (col % a.ncx) * kC3X, y0 = (col / a.ncx) * kC3Y;
    const int x = x0 + tx, y = y0 + ty;
    const unsigned site_xy = (unsigned)x + (unsigned)nx * (unsigned)y;
    // patches: window cells beyond the lattice along a periodic axis arrive as zeros
    const bool patch = x0 == 0 || x0 + kC3X == nx || (!p.wall_y && (y0 == 0 || y0 + kC3Y == ny));
    RingAcc own{};
    float2* const gdown = a.ghost + ghost_base(col, seg, 0, a.nseg);
    float2* const gup = a.ghost + ghost_base(col, seg, 1, a.nseg);
    const int own_g = (ty + 1) * kGhostX + tx + 1;
    const bool bym = p.wall_y && y == 0, byp = p.wall_y && y == ny - 1;
    for (int z = zs; z < ze; ++z, ++it) {
      const unsigned site = site_xy + nxy * (unsigned)z;
      float2* const s_a = s_a0 + (it & 1u) * kC3AFloats2;
      auto A_at = [&](int cls, int czd, int row, int c) -> float2& {
        return s_a[((cls * 3 + czd) * kC3Y + row) * kC3ACols + c];
      };
      // ---- the plane's populations, normals and NCI distances (each thread waits for
      // the copies itself)
      const bool ok = mbar_wait(bar_full, ph_full);
      if (!ok) *s_abort = 1;  // acted on at the next barrier, where every thread meets
      ph_full ^= 1u;
      const float4 ngv = reinterpret_cast<const float4*>(sm + C3Stage<ST>::kNgOff)[tid];
      const int hv = sm[C3Stage<ST>::kHitOff + tid];
      if (patch) {
        // window cells outside the lattice along a periodic axis: for each direction the
        // column of 8 cells beyond x (c_x != 0) and the row of 32 cells beyond y (c_y != 0)
        for (int e = tid; e < 27 * 40; e += kC3T) {
          const int i = e / 40, q = e - 40 * (e / 40);
          const int cx = digit_c(i % 3), cy = digit_c((i / 3) % 3), cz = digit_c(i / 9);
          int col_w, row;
          if (q < kC3Y) {
            if (cx == 0) continue;
            row = q;
            col_w = cx > 0 ? 3 : 4 + kC3X;  // source x0 - 1 (c_x = +1) or x0 + 32 (c_x = -1)
          } else {
            if (cy == 0) continue;
            row = cy > 0 ? 0 : kC3Y - 1;  // source y0 - 1 or y0 + 8
            col_w = 4 - cx + (q - kC3Y);
          }
          const int gx = x0 - 4 + col_w, gy = y0 - cy + row;
          int zs = z - cz;
          if (p.wall_z && (zs < 0 || zs >= nz)) continue;
          if (p.wall_y && (gy < 0 || gy >= ny)) continue;  // beyond a wall: never read
          if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
          zs = wrapn(zs, nz);
          const unsigned src = (unsigned)wrapn(gx, nx) + (unsigned)nx * ((unsigned)wrapn(gy, ny) + (unsigned)ny * zs);
          const int c = (i % 3) * kW3Cells + row * kW3X + col_w;
          if constexpr (HALF) {
            reinterpret_cast<unsigned*>(sm + (i / 3) * kW3Bytes)[c] =
                __ldg(reinterpret_cast<const unsigned*>(f.d) + (size_t)i * f.N + src);
          } else {
            const float v0 = __ldg(f.f + (size_t)i * f.N + src), v1 = __ldg(f.f + (size_t)(27 + i) * f.N + src);
            reinterpret_cast<float*>(sm + (i / 3) * kW3Bytes)[c] = v0;
            reinterpret_cast<float*>(sm + (9 + i / 3) * kW3Bytes)[c] = v1;
          }
        }
        if constexpr (HALF) {  // border cells of the three 40 x 10 density boxes
          for (int e = tid; e < 3 * kRing; e += kC3T) {
            const int cell = e / 3, gz = e - 3 * (e / 3);
            int bc, br;
            if (cell < 2 * (kC3Y + 2)) { bc = cell < kC3Y + 2 ? 3 : 4 + kC3X; br = cell % (kC3Y + 2); }
            else { bc = 4 + (cell - 2 * (kC3Y + 2)) % kC3X; br = cell < kRingYT ? 0 : kR3Y - 1; }
            const int gx = x0 - 4 + bc, gy = y0 - 1 + br;
            int zs = z - (gz == 0 ? 0 : (gz == 1 ? 1 : -1));
            if (p.wall_z && (zs < 0 || zs >= nz)) continue;
            if (p.wall_y && (gy < 0 || gy >= ny)) continue;
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
            zs = wrapn(zs, nz);
            const unsigned src = (unsigned)wrapn(gx, nx) + (unsigned)nx * ((unsigned)wrapn(gy, ny) + (unsigned)ny * zs);
            reinterpret_cast<float2*>(sm + C3Stage<ST>::kRhoOff + gz * kR3Bytes)[br * kR3X + bc] = __ldg(f.rho + src);
          }
        }
        fence_async_smem();  // these generic writes precede the next copy into the stage
        __syncthreads();
      }
      const bool bzm = p.wall_z && z == 0, bzp = p.wall_z && z == nz - 1;
      const bool wall_site = bym || byp || bzm || bzp;
      float fin[2][27];
      const int t0 = ty * kW3X + tx;  // the thread's cell in a class window
      const int c0 = (ty + 1) * kR3X + tx + 4;
      if (!wall_site) {
        static_for<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          C3Pull<ST>::template get<i>(sm, t0, c0, fin[0][i], fin[1][i]);
        });
      } else {  // halfway bounce-back: from the site's own opposite population
        static_for<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int cy = cc(i, 1), cz = cc(i, 2);
          const bool bounce = (cy == 1 && bym) || (cy == -1 && byp) || (cz == 1 && bzm) || (cz == -1 && bzp);
          if (bounce) f.template get<opposite(i)>(site, fin[0][i], fin[1][i]);
          else C3Pull<ST>::template get<i>(sm, t0, c0, fin[0][i], fin[1][i]);
        });
      }
      // ---- the NCI force of the distance the ray pass found
      const float n0 = ngv.x, n1 = ngv.y, n2 = ngv.z, gg = ngv.w;
      float frep0 = 0.f, frep1 = 0.f, frep2 = 0.f;
      if (hv > 0) {
        const float A = hv == 1 ? p.Ah[1] : (hv == 2 ? p.Ah[2] : (hv == 3 ? p.Ah[3] : p.Ah[4]));
        const float deltaI = 0.5f * gg;
        frep0 = -A * n0 * deltaI;
        frep1 = -A * n1 * deltaI;
        frep2 = -A * n2 * deltaI;
      }
      // ---- release the stage: every warp arrives on the empty barrier; the last warp
      // to get here refills the stage with the next plane (it waits, bounded, for the
      // barrier's phase so that every warp's reads are ordered before the copies)
      int nitem = item, nzn = z + 1;
      if (nzn == ze) {
        nitem = item + (int)gridDim.x;
        int zs2, ze2;
        seg_of(nitem, zs2, ze2);
        nzn = zs2;
      }
      const bool more = nitem < a.nitems;
      __syncwarp();
      int last = 0;
      if (tx == 0) {
        mbar_arrive(bar_empty);
        last = atomicAdd(s_cnt, 1) == kC3Warps - 1;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        const bool ok_e = mbar_wait(bar_empty, ph_empty);
        if (tx == 0) *s_cnt = 0;
        if (!ok_e) *s_abort = 1;
        if (more && !*s_abort) issue(nitem, nzn);
      }
      ph_empty ^= 1u;

      // ---- collision
      float o[2][27];
      // densities and momentum, summed in three partial sums (by c_z) so that the
      // additions form short independent chains
      float r1g[3] = {0.f, 0.f, 0.f}, r2g[3] = {0.f, 0.f, 0.f}, jg[3][3] = {};
      static_for<27>([&](auto I) {
        constexpr int i = decltype(I)::value, gz = i / 9;
        r1g[gz] += fin[0][i];
        r2g[gz] += fin[1][i];
        const float t = fin[0][i] + fin[1][i];
        if constexpr (cc(i, 0) != 0) jg[gz][0] += cc(i, 0) > 0 ? t : -t;
        if constexpr (cc(i, 1) != 0) jg[gz][1] += cc(i, 1) > 0 ? t : -t;
        if constexpr (cc(i, 2) != 0) jg[gz][2] += cc(i, 2) > 0 ? t : -t;
      });
      const float rho1 = (r1g[0] + r1g[1]) + r1g[2], rho2 = (r2g[0] + r2g[1]) + r2g[2];
      const float rho = rho1 + rho2;
      float j[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) j[c] = (jg[0][c] + jg[1][c]) + jg[2][c];
      const float F[3] = {p.G[0] + frep0, p.G[1] + frep1, p.G[2] + frep2};
      float u[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c] = __fdividef(j[c] + 0.5f * F[c], rho);
      const float m[3] = {-n0, -n1, -n2};
      C3Writer<ST> wr;
      if constexpr (HALF) { wr.d = fw.d; wr.rho = fw.rho; wr.seed = seed; }
      else { wr.f = fw.f; }
      wr.N = fw.N;
      wr.o = o;
      collide_store<1, float, C3Writer<ST>, EDM>(fin, rho1, rho2, j, u, F, gg, m, p, wr, site);

      // ---- carry: where the new populations stream to
      float2 self = make_float2(0.f, 0.f);
      if (wall_site) {  // a population whose target lies beyond a wall bounces back here
        static_for<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int cy = cc(i, 1), cz = cc(i, 2);
          const bool cross = (cy == -1 && bym) || (cy == 1 && byp) || (cz == -1 && bzm) || (cz == 1 && bzp);
          if (cross) {
            self.x += o[0][i];
            self.y += o[1][i];
            o[0][i] = 0.f;
            o[1][i] = 0.f;
          }
        });
      }
      // along x: warp shuffles within the row; lane 0's c_x = -1 and lane 31's c_x = +1
      // populations leave the column (ring cells x0-1 and x0+32)
      float2 a_own[3];
      static_for<9>([&](auto C) {
        constexpr int cls = decltype(C)::value;
        constexpr int cyd = cls % 3, czd = cls / 3;
        constexpr int i0 = 3 * cyd + 9 * czd, ip = i0 + 1, im = i0 + 2;  // c_x = 0, +1, -1
        float2 sv;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float up = __shfl_up_sync(0xffffffffu, o[k][ip], 1);
          const float dn = __shfl_down_sync(0xffffffffu, o[k][im], 1);
          float v = o[k][i0];
          if (tx > 0) v += up;
          if (tx < kC3X - 1) v += dn;
          if (k == 0) sv.x = v; else sv.y = v;
        }
        const float2 eL = make_float2(o[0][im], o[1][im]), eR = make_float2(o[0][ip], o[1][ip]);
        constexpr int sc = cyd == 0 ? 2 : (cyd == 1 ? 0 : 1);  // exchange class: c_y = +1, -1, 0
        if (cyd == 0) a_own[czd] = sv;
        else A_at(sc, czd, ty, tx + 1) = sv;
        if (tx == 0) A_at(sc, czd, ty, 0) = eL;
        if (tx == kC3X - 1) A_at(sc, czd, ty, kC3X + 1) = eR;
      });
      __syncthreads();
      if (*s_abort) {  // a wait ran out: leave together, after the copy in flight (bounded)
        if (tid == 0) atomicOr(a.err, 1);
        if (!ok) mbar_wait(bar_full, ph_full ^ 1u);
        return;
      }
      // along y (rows through shared memory) and z (running sums as the column marches)
      float2 b[3];
#pragma unroll
      for (int czd = 0; czd < 3; ++czd) {
        float2 v = a_own[czd];
        if (ty > 0) v = f2add(v, A_at(0, czd, ty - 1, tx + 1));
        if (ty < kC3Y - 1) v = f2add(v, A_at(1, czd, ty + 1, tx + 1));
        b[czd] = v;
      }
      b[0] = f2add(b[0], self);
      zsum(own, b[0], b[1], b[2], z, zs, [&](int zz, float2 v) { a.carry[site_xy + nxy * (unsigned)zz] = v; },
           [&](float2 v) { gdown[own_g] = v; });
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int id = rid[r];
        if (id < 0) continue;
        int cx_, ry;  // the ring cell in exchange coordinates: column 0..33, row -1..8
        if (id < kRingYB) { cx_ = id < kRingXR ? 0 : kC3X + 1; ry = (id - (id < kRingXR ? kRingXL : kRingXR)) - 1; }
        else { cx_ = 1 + (id - (id < kRingYT ? kRingYB : kRingYT)); ry = id < kRingYT ? -1 : kC3Y; }
        float2 rb[3];
#pragma unroll
        for (int czd = 0; czd < 3; ++czd) {
          float2 v = make_float2(0.f, 0.f);
          if (ry >= 0 && ry < kC3Y) v = A_at(2, czd, ry, cx_);
          if (ry - 1 >= 0 && ry - 1 < kC3Y) v = f2add(v, A_at(0, czd, ry - 1, cx_));
          if (ry + 1 >= 0 && ry + 1 < kC3Y) v = f2add(v, A_at(1, czd, ry + 1, cx_));
          rb[czd] = v;
        }
        RingAcc acc = s_ring[id];
        zsum(acc, rb[0], rb[1], rb[2], z, zs, [&](int zz, float2 v) { a.ring[ring_base(col, zz, nz) + id] = v; },
             [&](float2 v) { gdown[ring_ghost(id)] = v; });
        s_ring[id] = acc;
      }
    }
    zsum_end(own, ze, [&](int zz, float2 v) { a.carry[site_xy + nxy * (unsigned)zz] = v; },
             [&](float2 v) { gup[own_g] = v; });
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int id = rid[r];
      if (id < 0) continue;
      zsum_end(s_ring[id], ze, [&](int zz, float2 v) { a.ring[ring_base(col, zz, nz) + id] = v; },
               [&](float2 v) { gup[ring_ghost(id)] = v; });
    }
    item += gridDim.x;
  }
}

// ---------------------------------------------------------------------------------
// The streaming D3Q27 step (FP32 and FP16-dev storage; lattices of whole 32 x 8 columns):
// a moments pass writes psi (and, for a step that stores the total + recolouring form,
// (rho_1, rho_2)); normals3d_kernel the per-site (n, |grad psi|); the collision
// (collide3d_kernel for two populations per direction, collide3t_kernel for the total form,
// at the end of the file) then runs the near-contact ray of its site over those normals
// (probes through L2), pulls, collides and stores, with no shared memory and no barrier, its
// block's neighbours reading the same planes at the same time from L2.

// (n, |grad psi|) of a 32 x 8 column's sites on kN3Z consecutive planes from the psi
// array: the block keeps psi of its 34 x 10 cells (beyond a wall the mirror cell, along
// periodic axes the image) in a shared-memory ring of four planes; the loads of plane z + 2
// are issued before plane z is computed and stored after it, into the slot plane z - 2
// held, so their latency overlaps the arithmetic and one barrier per plane suffices (62 us
// per duct step against 65 us with three slots and two barriers). Every site sums its 26
// neighbours in direction order.
constexpr int kN3Z = 16;
__global__ void __launch_bounds__(256) normals3d_kernel(const float* __restrict__ psi, float4* __restrict__ ng,
                                                        StepT<float> p) {
  constexpr int RX = 34, RXY = RX * 10, PER = (RXY + 255) / 256;
  __shared__ float s_psi[4 * RXY];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, z0 = blockIdx.z * kN3Z;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int z1 = min(nz, z0 + kN3Z);
  auto load = [&](int q, float v[PER]) {  // plane q (wrapped or mirrored) into registers
    const int gz = p.wall_z ? clampc(q, nz) : wrapn(q, nz);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int c = tid + 256 * k;
      if (c < RXY) {
        const int ly = c / RX, lx = c - ly * RX;
        const int gx = wrapn(x0 - 1 + lx, nx);
        const int gy = p.wall_y ? clampc(y0 - 1 + ly, ny) : wrapn(y0 - 1 + ly, ny);
        v[k] = psi[(unsigned)gx + (unsigned)nx * ((unsigned)gy + (unsigned)ny * (unsigned)gz)];
      }
    }
  };
  auto store = [&](int q, const float v[PER]) {  // into ring slot q mod 4
    float* dst = s_psi + ((q + 4) & 3) * RXY;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int c = tid + 256 * k;
      if (c < RXY) dst[c] = v[k];
    }
  };
  {
    float v[PER];
    load(z0 - 1, v);
    store(z0 - 1, v);
    load(z0, v);
    store(z0, v);
    load(z0 + 1, v);
    store(z0 + 1, v);
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const int cxy = (threadIdx.x + 1) + RX * (threadIdx.y + 1);
  for (int z = z0; z < z1; ++z) {
    float vn[PER];
    const bool more = z + 1 < z1;  // plane z + 2 is needed by the next iteration
    if (more) load(z + 2, vn);
    const float* pm = s_psi + ((z + 3) & 3) * RXY;
    const float* p0 = s_psi + (z & 3) * RXY;
    const float* pp = s_psi + ((z + 1) & 3) * RXY;
    float g[3];
    grad_ring<float>(pm, p0, pp, RX, cxy, g);
    float n[3];
    const float gn = M<float>::unit(g, n);
    ng[(unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z)] = make_float4(n[0], n[1], n[2], gn);
    // plane z + 2 goes to the fourth slot, the one plane z - 2 held: every thread finished
    // reading it before the barrier that ended the previous plane
    if (more) store(z + 2, vn);
    __syncthreads();
  }
}

// psi of every site, in 32 x 8 blocks of one plane (the streaming step's moments pass for
// FP16-dev storage): a block's sources lie within 3 planes of 34 x 10 cells, so the
// reference densities each pulled population is decoded with are reused from L1 by the
// block's other sites.
template <typename ST>
__global__ void __launch_bounds__(256) moments3_kernel(typename ST::Reader f, float* __restrict__ psi,
                                                       float2* __restrict__ rho12, StepT<float> p) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  const int site = x + p.nx * (y + p.ny * z);
  float fin[2][27];
  pull_any<1, float>(f, x, y, z, p, fin);
  float r1, r2;
  psi[site] = psi_of<27, float>(fin, &r1, &r2);
  // the collision storing a total form takes (rho_1, rho_2) from here: the component sums
  // the fields kernel also forms, so the two count each component's mass alike
  if (rho12) rho12[site] = make_float2(r1, r2);
}

template <typename ST, bool EDM>
__global__ void __launch_bounds__(256) collide3d_kernel(typename ST::Reader f, typename ST::Writer fout,
                                                        const float4* __restrict__ ng, StepT<float> p) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if constexpr (ST::kHalf)
    fout.seed = step_seed(p, p.parity, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
                                           threadIdx.y == 0);
  const int site = x + p.nx * (y + p.ny * z);
  // FP32: the pulls first, so that their loads are in flight while the ray's dependent
  // probes resolve (2.5% faster); FP16-dev: the ray first (pulls first raised its
  // registers from 80 to 103, two blocks per SM instead of three: 11% slower)
  float fin[2][27];
  float4 v;
  int h;
  if constexpr (!ST::kHalf) {
    pull_any<1, float>(f, x, y, z, p, fin);
    v = ng[site];
    h = p.smax > 0 ? nci_ray(ng, v, x, y, z, p) : 0;
  } else {
    v = ng[site];
    h = p.smax > 0 ? nci_ray(ng, v, x, y, z, p) : 0;
    pull_any<1, float>(f, x, y, z, p, fin);
  }
  float rho1, rho2;
  psi_of<27, float>(fin, &rho1, &rho2);
  const float rho = rho1 + rho2;
  float j[3];
  momentum<1, float>(fin, j);
  float A = 0.f;  // A_h(h), indexed at compile time
  static_for<kMaxProbe>([&](auto I) {
    constexpr int s = decltype(I)::value + 1;
    if (h == s) A = p.Ah[s];
  });
  const float deltaI = 0.5f * v.w;
  const float F[3] = {p.G[0] - A * v.x * deltaI, p.G[1] - A * v.y * deltaI, p.G[2] - A * v.z * deltaI};
  float u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = M<float>::div(j[a] + 0.5f * F[a], rho);
  const float m[3] = {-v.x, -v.y, -v.z};
  collide_store<1, float, typename ST::Writer, EDM>(fin, rho1, rho2, j, u, F, v.w, m, p, fout, site);
}

// ------------------------------------------------------------------ total + recolouring form
// With Guo forcing the collision's output at a site is fixed by the total post-collision
// populations f*_i = f_i^1 + f_i^2 and the recolouring Omega^(3): for a moving direction
//   f_i^1 = phi_1 f*_i + (w_i/|c_i|) c_i.s,   f_i^2 = f*_i - f_i^1,
// phi_1 = rho_1/rho, s = beta (rho_1 rho_2/rho) m (the recolouring term written with the
// vector s instead of the angle to m). A state in this form holds the 26 moving totals, the
// rest population of each component and one float4 (phi_1, s) per site. The rest
// populations stay per component: rho_k minus phi_k times the sum S of the stored moving
// totals (the moving populations of component 1 sum to phi_1 S, since the recolouring
// terms of opposite directions cancel exactly), so each site's component masses are kept
// to the rounding of the sums, as in the two-population collision. The exact-difference
// forcing adds a term per component after the recolouring; its steps keep the
// two-population form.
//
//   TotalRecol      FP32 totals: plane 0 f_0^1, planes 1..26 f*_i, plane 27 f_0^2 (planes
//                   0 and 27 are also where the two-population layout keeps the rest
//                   populations), then the coefficient plane: 128 bytes per site. The
//                   collision sums S with Kahan's compensation (collide_totals).
//   TotalRecolHalf  FP16 totals, as deviations from the lattice-weight equilibrium of one
//                   reference density rho_0 of the sim (f*_i = w_i rho_0 + d_i; the total
//                   density of the model's two fluids stays close to its mean, so d_i is of
//                   the order of w_i (|rho - rho_0| + 3 |c_i.u|)): 26 half planes, then the
//                   two FP32 rest planes and the coefficient plane: 76 bytes per site. A
//                   step rounds d_i stochastically (half2_stochastic, the site's dither
//                   bits); the rest populations use the rounded totals.
//                   The reference is held as w_i rho_0 = (216 w_i) r with 216 w_i in
//                   {64, 16, 4, 1} and r = rho_0/216 rounded to a multiple of 2^-24 (the
//                   host's rho_unit): every decoded total is then a multiple of 2^-24 and,
//                   below 1, exact in FP32, and so is the collision's sum of a site's
//                   totals. With w_i rho_0 rounded instead, the totals' low bits were the
//                   same at every site and that sum's one rounding went the same way nearly
//                   everywhere: the rest populations made 7.5e-9 of the mass per site and
//                   step.
//
// Both offer the two-population reader interface (get<I>: both components of direction I),
// through which the moments pass, the fields kernel and population copies read them; the
// collision, which needs no split, reads TotalRecol's Totals (get<I>: the total alone) or
// TotalRecolHalf's Devs (the deviations d_i: it works on them, collide_totals_dev).

// (w_i/|c_i|) c_i.s of moving direction I, s = (c.y, c.z, c.w), summed over the nonzero
// components of c_i in x, y, z order for I < opposite(I), and exactly the negative of its
// opposite's for the others: every reader evaluates it with these same operations, and the
// terms of a pair of opposite directions cancel exactly (the collision's rest populations
// rely on it).
template <int I>
__device__ __forceinline__ float recolour_term(const float4 c) {
  if constexpr (I > opposite(I)) return -recolour_term<opposite(I)>(c);
  constexpr int ix = cc(I, 0), iy = cc(I, 1), iz = cc(I, 2);
  constexpr float wl = float(Lattice<1>::w(I) / (speed2(I) == 1 ? 1.0
                                                 : (speed2(I) == 2 ? 1.4142135623730951 : 1.7320508075688772)));
  float r = 0.f;
  if constexpr (ix == 1) r += c.y; else if constexpr (ix == -1) r -= c.y;
  if constexpr (iy == 1) r += c.z; else if constexpr (iy == -1) r -= c.z;
  if constexpr (iz == 1) r += c.w; else if constexpr (iz == -1) r -= c.w;
  return wl * r;
}

// Component 1 and 2 of a moving direction from its total t and the coefficients c.
template <int I>
__device__ __forceinline__ void split_total(float t, const float4 c, float& a, float& b) {
  a = fmaf(c.x, t, recolour_term<I>(c));
  b = t - a;
}

struct TotalRecol {
  using Compute = float;
  static constexpr int Q = 27;
  static constexpr bool kHalf = false;
  __host__ __device__ static size_t coef_offset(size_t N) { return (28 * N * sizeof(float) + 255) & ~(size_t)255; }
  static size_t bytes(size_t N) { return coef_offset(N) + N * sizeof(float4); }

  struct Reader {
    const float* __restrict__ f;
    const float4* __restrict__ coef;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void get(unsigned site, float& a, float& b) const {
      if constexpr (I == 0) {
        a = f[site];
        b = f[27u * N + site];
      } else {
        split_total<I>(f[(unsigned)I * N + site], coef[site], a, b);
      }
    }
  };
  struct Totals {
    const float* __restrict__ f;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void get(unsigned site, float& a, float& b) const {
      if constexpr (I == 0) a = f[site] + f[27u * N + site];
      else a = f[(unsigned)I * N + site];
      b = 0.f;
    }
  };
  struct Writer {
    float* __restrict__ f;
    float4* __restrict__ coef;
    unsigned N;
    unsigned seed;  // unused by this form
    __device__ __forceinline__ bool compensate() const { return true; }  // the collision's sum of the totals
    __device__ __forceinline__ unsigned site_bits(unsigned) const { return 0u; }
    // the totals of directions I and its opposite O; (tp, tm) = the stored values
    template <int I, int O>
    __device__ __forceinline__ void put_pair(unsigned site, float fp, float fm, unsigned, float& tp, float& tm) const {
      f[(unsigned)I * N + site] = fp;
      f[(unsigned)O * N + site] = fm;
      tp = fp;
      tm = fm;
    }
    __device__ __forceinline__ void put_rest(unsigned site, float r1, float r2, float4 c) const {
      f[site] = r1;
      f[27u * N + site] = r2;
      coef[site] = c;
    }
  };
  __host__ __device__ static Reader reader(const void* base, unsigned N, float = 0.f) {
    return Reader{(const float*)base, (const float4*)((const char*)base + coef_offset(N)), N};
  }
  __host__ __device__ static Totals totals(const void* base, unsigned N, float = 0.f) {
    return Totals{(const float*)base, N};
  }
  __host__ __device__ static Writer writer(void* base, unsigned N, float = 0.f) {
    return Writer{(float*)base, (float4*)((char*)base + coef_offset(N)), N, 0u};
  }
};

struct TotalRecolHalf {
  using Compute = float;
  static constexpr int Q = 27;
  static constexpr bool kHalf = true;
  __host__ __device__ static size_t rest_offset(size_t N) { return (26 * N * sizeof(__half) + 255) & ~(size_t)255; }
  __host__ __device__ static size_t coef_offset(size_t N) {
    return (rest_offset(N) + 2 * N * sizeof(float) + 255) & ~(size_t)255;
  }
  static size_t bytes(size_t N) { return coef_offset(N) + N * sizeof(float4); }

  // 216 w_I: 64, 16, 4 or 1 (exact)
  template <int I>
  __host__ __device__ static constexpr float k216() { return float(216.0 * Lattice<1>::w(I)); }
  // f*_i = (216 w_i) r + d_i, one expression for every reader and the writer
  template <int I>
  __device__ __forceinline__ static float total(const __half* d, unsigned N, unsigned site, float r) {
    return fmaf(k216<I>(), r, __half2float(d[(unsigned)(I - 1) * N + site]));
  }

  struct Reader {
    const __half* __restrict__ d;
    const float* __restrict__ r;
    const float4* __restrict__ coef;
    unsigned N;
    float r0;  // rho_0/216 on the 2^-24 grid (the host's rho_unit)
    template <int I>
    __device__ __forceinline__ void get(unsigned site, float& a, float& b) const {
      if constexpr (I == 0) {
        a = r[site];
        b = r[N + site];
      } else {
        split_total<I>(total<I>(d, N, site, r0), coef[site], a, b);
      }
    }
  };
  // The deviations d_i alone, as pairs (d_i, 0) (0 for the rest direction, which the
  // collision does not pull): the collision of a step that reads this form works on them.
  struct Devs {
    const __half* __restrict__ d;
    unsigned N;
    template <int I>
    __device__ __forceinline__ void get(unsigned site, float& a, float& b) const {
      if constexpr (I == 0) a = 0.f;
      else a = __half2float(d[(unsigned)(I - 1) * N + site]);
      b = 0.f;
    }
  };
  struct Writer {
    __half* __restrict__ d;
    float* __restrict__ r;
    float4* __restrict__ coef;
    unsigned N;
    float r0;  // rho_0/216 on the 2^-24 grid (the host's rho_unit)
    unsigned seed;  // this step's dither seed (step_seed)
    // the collision's sum of the totals: exact while the totals and their sums stay below 1
    // (multiples of 2^-24), that is for rho_0 up to about 1.25; compensated above
    __device__ __forceinline__ bool compensate() const { return r0 > 1.25f / 216.f; }
    __device__ __forceinline__ unsigned site_bits(unsigned site) const { return dither_bits(site, seed); }
    // d_I and d_O rounded stochastically as one half2 (I low, O high) with the site's bits h;
    // (tp, tm) = the totals a reader will see
    template <int I, int O>
    __device__ __forceinline__ void put_pair(unsigned site, float fp, float fm, unsigned h, float& tp,
                                             float& tm) const {
      constexpr float w = k216<I>();
      const unsigned v = half2_stochastic<I>(fmaf(-w, r0, fp), fmaf(-w, r0, fm), h);
      const unsigned short lo = (unsigned short)(v & 0xFFFFu), hi = (unsigned short)(v >> 16);
      unsigned short* du = reinterpret_cast<unsigned short*>(d);
      du[(unsigned)(I - 1) * N + site] = lo;
      du[(unsigned)(O - 1) * N + site] = hi;
      tp = fmaf(w, r0, __half2float(__ushort_as_half(lo)));
      tm = fmaf(w, r0, __half2float(__ushort_as_half(hi)));
    }
    // deviations already relative to the reference, rounded stochastically; (qp, qm) = the
    // stored values
    template <int I, int O>
    __device__ __forceinline__ void put_pair_dev(unsigned site, float dp, float dm, unsigned h, float& qp,
                                                 float& qm) const {
      const unsigned v = half2_stochastic<I>(dp, dm, h);
      const unsigned short lo = (unsigned short)(v & 0xFFFFu), hi = (unsigned short)(v >> 16);
      unsigned short* du = reinterpret_cast<unsigned short*>(d);
      du[(unsigned)(I - 1) * N + site] = lo;
      du[(unsigned)(O - 1) * N + site] = hi;
      qp = __half2float(__ushort_as_half(lo));
      qm = __half2float(__ushort_as_half(hi));
    }
    __device__ __forceinline__ void put_rest(unsigned site, float r1, float r2, float4 c) const {
      r[site] = r1;
      r[N + site] = r2;
      coef[site] = c;
    }
  };
  __host__ __device__ static Devs devs(const void* base, unsigned N) { return Devs{(const __half*)base, N}; }
  __host__ __device__ static Reader reader(const void* base, unsigned N, float r0) {
    const char* b = (const char*)base;
    return Reader{(const __half*)b, (const float*)(b + rest_offset(N)), (const float4*)(b + coef_offset(N)), N, r0};
  }
  __host__ __device__ static Writer writer(void* base, unsigned N, float r0) {
    char* b = (char*)base;
    return Writer{(__half*)b, (float*)(b + rest_offset(N)), (float4*)(b + coef_offset(N)), N, r0, 0u};
  }
};

// The FP32 operator of collide_store (BGK with the Guo source and the perturbation per
// pair of opposite directions) on the totals t, stored in a total + recolouring form.
template <typename WR>
__device__ __forceinline__ void collide_totals(const float t[27], float rho1, float rho2, float rho, const float u[3],
                                               const float F[3], float g, const float m[3], const StepT<float>& p,
                                               const WR& fout, unsigned site) {
  const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float seg = M<float>::div(p.beta * rho1 * rho2, rho);
  const float pamp = p.pamp * g;
  const float c1 = M<float>::div(rho1, rho);
  const float orho = p.omega * rho;
  const float K0 = orho * (1.f - 1.5f * uu) - 3.f * p.guo * uF - pamp * (1.0f / 3.0f);
  const float a3 = 3.f * orho, a45 = 4.5f * orho, g3 = 3.f * p.guo, g9 = 9.f * p.guo;
  const float om1 = 1.f - p.omega;
  const float4 cf = make_float4(c1, seg * m[0], seg * m[1], seg * m[2]);
  const unsigned hb = fout.site_bits(site);
  // S: the sum of the stored moving totals, which the rest populations below complete to
  // rho_k. Its rounding becomes mass: a plain running sum of populations of nearly the same
  // sizes at every site rounds the same way nearly everywhere (measured: the FP16 form lost
  // 2.2e-8 of each component's mass per step, FP32 gained 1.9e-9). FP32 sums them with
  // Kahan's compensation, which leaves one rounding of the exact sum; the FP16 totals are
  // multiples of 2^-24 below 1 (TotalRecolHalf), so their plain sum is exact (for rho_0 up
  // to about 1.25; compensated above).
  const bool kahan = fout.compensate();  // the same for every thread of the launch
  float S = 0.f, cS = 0.f;
  auto add = [&](float v) {
    if (kahan) {
      const float y = v - cS;
      const float t2 = S + y;
      cS = (t2 - S) - y;
      S = t2;
    } else {
      S += v;
    }
  };
  static_for<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int o = opposite(i);
    if constexpr (i > 0 && i < o) {
      constexpr float w = float(Lattice<1>::w(i));
      constexpr int ix = cc(i, 0), iy = cc(i, 1), iz = cc(i, 2);
      auto dotc = [&](const float v[3]) {
        float r = 0.f;
        if constexpr (ix == 1) r += v[0]; else if constexpr (ix == -1) r -= v[0];
        if constexpr (iy == 1) r += v[1]; else if constexpr (iy == -1) r -= v[1];
        if constexpr (iz == 1) r += v[2]; else if constexpr (iz == -1) r -= v[2];
        return r;
      };
      const float cu = dotc(u), cF = dotc(F), cm = dotc(m);
      const float E = fmaf(pamp, cm * cm, fmaf(g9, cu * cF, fmaf(a45, cu * cu, K0)));
      const float O = fmaf(g3, cF, a3 * cu);
      const float fsp = fmaf(w, E + O, om1 * t[i]);
      const float fsm = fmaf(w, E - O, om1 * t[o]);
      float tp, tm;
      fout.template put_pair<i, o>(site, fsp, fsm, hb, tp, tm);
      add(tp);
      add(tm);
    }
  });
  // Component 1 of the moving populations sums to phi_1 S (a pair's recolouring terms are
  // exact negatives of each other), component 2 to S - phi_1 S: the rest populations make
  // each component's total rho_k, to the rounding of the sums.
  const float s1 = c1 * S;
  fout.put_rest(site, rho1 - s1, rho2 - (S - s1), cf);
}

// collide_totals for a step that reads and stores the FP16 form, on the deviations
// d_i = f*_i - (216 w_i) r0 themselves: the references carry no momentum (sum_i c_i w_i = 0),
// so j is the deviations' momentum, and the collision's output deviation is
//   (1 - omega) d_i + w_i (E_i +/- O_i - 216 omega r0),
// formed without the totals: the offset enters K0 through rho - 216 r0, exact for rho within
// a factor of two of the reference, so the deviations keep their own precision. The sum of
// the stored totals is S = 152 r0 + sum of the stored deviations (152 = 216 (1 - w_0)).
__device__ __forceinline__ void collide_totals_dev(const float d[27], float rho1, float rho2, float rho,
                                                   const float u[3], const float F[3], float g, const float m[3],
                                                   const StepT<float>& p, const TotalRecolHalf::Writer& fout,
                                                   unsigned site) {
  const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float seg = M<float>::div(p.beta * rho1 * rho2, rho);
  const float pamp = p.pamp * g;
  const float c1 = M<float>::div(rho1, rho);
  const float r0 = fout.r0;
  const float K0d = p.omega * ((rho - 216.f * r0) - 1.5f * rho * uu) - 3.f * p.guo * uF - pamp * (1.0f / 3.0f);
  const float orho = p.omega * rho;
  const float a3 = 3.f * orho, a45 = 4.5f * orho, g3 = 3.f * p.guo, g9 = 9.f * p.guo;
  const float om1 = 1.f - p.omega;
  const float4 cf = make_float4(c1, seg * m[0], seg * m[1], seg * m[2]);
  const unsigned hb = fout.site_bits(site);
  const bool kahan = fout.compensate();  // the same for every thread of the launch
  float S = 0.f, cS = 0.f;               // the stored deviations (see collide_totals)
  auto add = [&](float v) {
    if (kahan) {
      const float y = v - cS;
      const float t2 = S + y;
      cS = (t2 - S) - y;
      S = t2;
    } else {
      S += v;
    }
  };
  static_for<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int o = opposite(i);
    if constexpr (i > 0 && i < o) {
      constexpr float w = float(Lattice<1>::w(i));
      constexpr int ix = cc(i, 0), iy = cc(i, 1), iz = cc(i, 2);
      auto dotc = [&](const float v[3]) {
        float r = 0.f;
        if constexpr (ix == 1) r += v[0]; else if constexpr (ix == -1) r -= v[0];
        if constexpr (iy == 1) r += v[1]; else if constexpr (iy == -1) r -= v[1];
        if constexpr (iz == 1) r += v[2]; else if constexpr (iz == -1) r -= v[2];
        return r;
      };
      const float cu = dotc(u), cF = dotc(F), cm = dotc(m);
      const float E = fmaf(pamp, cm * cm, fmaf(g9, cu * cF, fmaf(a45, cu * cu, K0d)));
      const float O = fmaf(g3, cF, a3 * cu);
      float qp, qm;
      fout.template put_pair_dev<i, o>(site, fmaf(w, E + O, om1 * d[i]), fmaf(w, E - O, om1 * d[o]), hb, qp, qm);
      add(qp);
      add(qm);
    }
  });
  const float St = fmaf(152.f, r0, S);
  const float s1 = c1 * St;
  fout.put_rest(site, rho1 - s1, rho2 - (St - s1), cf);
}

// The streaming collision storing a total + recolouring form (WR), from a state in that
// form (RD TotalRecol::Totals or TotalRecolHalf::Devs, TOTALS) or in the two-population
// layout of the precision (RD the
// Plain or HalfDev reader: the first step after a state was set). (rho_1, rho_2) of the
// site come from the moments pass (rho12), rho = rho_1 + rho_2; the totals give j. Capped at
// 64 registers (four blocks per SM, no spills reading the form): 395 us per FP32 duct step
// against 441 us at 80 registers and three blocks when measured, the kernel waiting on its
// loads.
template <typename RD, bool TOTALS, typename WR>
__global__ void __launch_bounds__(256, 4) collide3t_kernel(RD f, WR fout, const float2* __restrict__ rho12,
                                                           const float4* __restrict__ ng, StepT<float> p) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  const unsigned site = (unsigned)x + (unsigned)p.nx * ((unsigned)y + (unsigned)p.ny * (unsigned)z);
  if constexpr (std::is_same<WR, TotalRecolHalf::Writer>::value)
    fout.seed = step_seed(p, p.parity, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
                                           threadIdx.y == 0);
  float fin[2][27];
  pull_any<1, float>(f, x, y, z, p, fin);  // the pulls' loads in flight while the ray resolves
  const float4 v = ng[site];
  const int h = p.smax > 0 ? nci_ray(ng, v, x, y, z, p) : 0;
  if constexpr (!TOTALS) {
#pragma unroll
    for (int i = 0; i < 27; ++i) fin[0][i] += fin[1][i];
  }
  const float* t = fin[0];
  float j[3] = {0.f, 0.f, 0.f};
  static_for<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (cc(i, 0) != 0) j[0] += cc(i, 0) > 0 ? t[i] : -t[i];
    if constexpr (cc(i, 1) != 0) j[1] += cc(i, 1) > 0 ? t[i] : -t[i];
    if constexpr (cc(i, 2) != 0) j[2] += cc(i, 2) > 0 ? t[i] : -t[i];
  });
  const float2 r12 = rho12[site];
  const float rho1 = r12.x, rho2 = r12.y;
  const float rho = rho1 + rho2;
  float A = 0.f;  // A_h(h), indexed at compile time
  static_for<kMaxProbe>([&](auto I) {
    constexpr int s = decltype(I)::value + 1;
    if (h == s) A = p.Ah[s];
  });
  const float deltaI = 0.5f * v.w;
  const float F[3] = {p.G[0] - A * v.x * deltaI, p.G[1] - A * v.y * deltaI, p.G[2] - A * v.z * deltaI};
  float u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = M<float>::div(j[a] + 0.5f * F[a], rho);
  const float m[3] = {-v.x, -v.y, -v.z};
  if constexpr (std::is_same<RD, TotalRecolHalf::Devs>::value)
    collide_totals_dev(t, rho1, rho2, rho, u, F, v.w, m, p, fout, site);  // t: the deviations
  else
    collide_totals<WR>(t, rho1, rho2, rho, u, F, v.w, m, p, fout, site);
}

}  // namespace lbnci
