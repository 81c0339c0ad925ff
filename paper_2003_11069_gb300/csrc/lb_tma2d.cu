// lb_tma2d.cu -- persistent, TMA-fed D2Q9 step for FP32 populations
// (arXiv:2003.11069, "Materials and Methods": the colour-gradient step
// Omega = Omega^(3)[Omega^(1) + Omega^(2)] with the near-contact force of Eq. (near_c);
// the per-site arithmetic is that of lb_kernels.cuh).
//
// Persistent CTAs of 512 threads (two per SM) walk 32 x 16 tiles, one thread per site:
// tiles blockIdx.x and blockIdx.x + gridDim.x first, then tiles from an atomic counter.
// The gradient of psi and the NCI ray search at a site read psi
// up to R = smax + 1 = 5 sites away, and psi at a site is a sum of the 18 populations
// streamed into it, so a tile needs the populations of its 48 x 28 neighbourhood
// (x0-8..x0+39, y0-6..y0+21; the x range is widened to keep TMA coordinates 16-byte
// aligned). One elected thread loads that box, all 18 population planes, with a
// single TMA copy into the CTA's shared-memory stage; two CTAs share an SM, and a CTA
// issues its next tile's copy as soon as this tile has read the stage, so copies
// overlap the other CTA's arithmetic and cost no load instructions. After its first two
// tiles a CTA takes tiles from an atomic counter, which evens out tiles of uneven cost
// (interface density, periodic edges) across CTAs. Box cells
// beyond the lattice along a periodic axis arrive as zeros and are replaced by their
// periodic images with plain loads (first and last tile columns, and the first and
// last tile rows without walls). Everything the step reads then comes from shared
// memory:
//   phase 1: pull the own site (kept in registers) and every halo cell from the box,
//            psi into shared memory;
//   phase 2: unit normal and |grad psi| of the own site (registers) and of the ring of
//            width smax around the tile, stored as probe normals (zero where
//            |grad psi| <= g_th, so a probe needs one load and one sign test);
//   phase 3: NCI ray search, Guo velocity, BGK + source + perturbation, recolouring,
//            coalesced stores of the 18 new populations.
// Ragged tiles use the same path: an own position beyond the lattice holds the psi of
// its periodic image (or, beyond a wall, of its mirror) and stores nothing.
//
// Consecutive steps overlap through programmatic dependent launch: a CTA lets the next
// step's grid be scheduled as soon as it starts; that grid's CTAs take the slots this
// grid's CTAs leave, initialise their mbarrier and wait for this grid to complete
// before they read the state or touch the tile counters.
//
// Every wait on an mbarrier is bounded (about one second); on expiry the kernel
// records a flag (bit 0) that the host reports, waits (bounded again) for its own
// copies in flight, and returns. A shared-memory base that is not 1024-byte aligned
// sets bit 1 before any copy is issued.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "lb_kernels.cuh"
#include "lb_launch.h"
#include "lb_tma.cuh"

namespace lbnci {
namespace {

constexpr int TX = kTmaTX, TY = kTmaTY, NT = TX * TY;  // 32 x 16 tile, one thread per site
constexpr int kQ = 9;
// population box: 18 planes x 28 rows (y0-6..y0+21) x 48 columns (x0-8..x0+39)
constexpr int kBX = 48, kBY = 28, kBOX = 8, kBOY = 6, kBPlane = kBX * kBY;
constexpr int kBoxFloats = 2 * kQ * kBPlane;
constexpr unsigned kBoxBytes = kBoxFloats * 4;
constexpr int kBoxStride = (kBoxBytes + 1023) / 1024 * 1024;
// FP16-deviation storage: 9 planes of half2 deviations (one 32-bit word per cell), then
// the reference densities (float2 per cell) of the same 48 x 28 cells.
constexpr unsigned kHalfDevBytes = kQ * kBPlane * 4, kHalfRhoBytes = kBPlane * 8;
constexpr int kHalfRhoOff = (kHalfDevBytes + 1023) / 1024 * 1024;
static_assert(kHalfRhoOff + (int)kHalfRhoBytes <= kBoxStride, "half boxes fit the stage");

// Shared-memory layout (bytes from a 1024-aligned base): the population box, psi of
// the tile and its halo, probe normals, the mbarrier and the next tile's index.
constexpr int kRmax = kMaxProbe + 1;
constexpr int kPsiBytes = (TX + 2 * kRmax) * (TY + 2 * kRmax) * 4;           // (32+10) x (16+10) floats
constexpr int kPBytes = (TX + 2 * kMaxProbe) * (TY + 2 * kMaxProbe) * 8;     // (32+8) x (16+8) float2
constexpr int kOffPsi = kBoxStride;
constexpr int kOffP = kOffPsi + kPsiBytes;
constexpr int kOffBar = kOffP + kPBytes;
constexpr int kSmemBytes = kOffBar + 256;  // mbarrier, next tile (4 ints), 2 x StepT<float>
static_assert(2 * (kSmemBytes + 1024) <= 228 * 1024, "shared memory: two CTAs per SM (1 KB reserved each)");
static_assert(32 + 2 * sizeof(StepT<float>) <= 256, "mbarrier, next tile and two parameter slots");

// Probe offset of the NCI ray: round(s n_a) to the nearest integer (ties to even),
// returned as the float's bit pattern b with round(s n_a) = b - kMagicBits; adding
// 1.5 2^23 leaves the integer in the low mantissa bits (|s n_a| <= 4 here). The FP64
// kernels round half away from zero; the two differ only when s n_a is exactly a
// half-integer, a tie at which the FP32 path may take either side.
constexpr float kMagic = 12582912.0f;
constexpr unsigned kMagicBits = 0x4B400000u;
__device__ __forceinline__ unsigned probe_bits(float s, float v) { return __float_as_uint(fmaf(s, v, kMagic)); }


// Halo cell h of a ring of width W around the 32 x 16 tile, in region coordinates
// (region = (32 + 2W) x (16 + 2W)): two bands of W full rows, then the W-wide sides.
template <int W>
__device__ __forceinline__ void ring_cell(int h, int& lx, int& ly) {
  constexpr int RX = TX + 2 * W, nband = W * RX;
  if (h < 2 * nband) {
    const int hb = h < nband ? h : h - nband;
    const int row = hb / RX;
    lx = hb - row * RX;
    ly = h < nband ? row : W + TY + row;
  } else {
    const int hs = h - 2 * nband;
    const int row = hs / (2 * W);
    const int col = hs - row * (2 * W);
    lx = col < W ? col : col + TX;
    ly = W + row;
  }
}

// Pull the 2 Q populations of the site at box position c (plane offsets kBPlane);
// bounce-back at walls from the site itself.
__device__ __forceinline__ void pull_box(const float* __restrict__ bx, int c, bool bym, bool byp,
                                         float fin[2][kQ]) {
  if (!(bym || byp)) {
    static_for<kQ>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int off = -cc(i, 1) * kBX - cc(i, 0);
      fin[0][i] = bx[i * kBPlane + c + off];
      fin[1][i] = bx[(kQ + i) * kBPlane + c + off];
    });
  } else {
    static_for<kQ>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cy = cc(i, 1);
      constexpr int off = -cy * kBX - cc(i, 0);
      const bool bounce = (cy == 1 && bym) || (cy == -1 && byp);
      fin[0][i] = bounce ? bx[opposite(i) * kBPlane + c] : bx[i * kBPlane + c + off];
      fin[1][i] = bounce ? bx[(kQ + opposite(i)) * kBPlane + c] : bx[(kQ + i) * kBPlane + c + off];
    });
  }
}

// Stores the collision's populations plane by plane: each plane's base address is
// the same for all threads, so a store needs only the site's offset.
struct PlaneWriter {
  float* __restrict__ f;
  unsigned N;
  template <int I>
  __device__ __forceinline__ void put_step(unsigned site, float a, float b, float, float, unsigned) const {
    (f + (size_t)I * N)[site] = a;
    (f + (size_t)(kQ + I) * N)[site] = b;
  }
  __device__ __forceinline__ unsigned site_bits(unsigned) const { return 0u; }
  __device__ __forceinline__ void put_rho(unsigned, float, float) const {}
};

// One lattice of a batched step (device memory): its tensor maps, step parameters, the
// two state buffers and its tiles' place in the batch. (Aligned as CUtensorMap is.)
struct TmaMember {
  CUtensorMap map[4];  // plain: box of buffer 0, 1; FP16-dev: deviations 0, 1, densities 0, 1
  StepT<float> p;
  float* buf[2];
  int ntx, ntiles, tile0;
};

// pull_box for FP16-deviation storage: f_i^k = w_i rho_ref^k(src) + delta_i^k(src), the
// reference densities of the cell the population comes from.
__device__ __forceinline__ void pull_box_half(const unsigned char* __restrict__ bxb, int c, bool bym, bool byp,
                                              float fin[2][kQ]) {
  const __half2* dv = reinterpret_cast<const __half2*>(bxb);
  const float2* rr = reinterpret_cast<const float2*>(bxb + kHalfRhoOff);
  static_for<kQ>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cy = cc(i, 1);
    constexpr int off = -cy * kBX - cc(i, 0);
    constexpr float w = float(Lattice<0>::w(i));
    const bool bounce = (cy == 1 && bym) || (cy == -1 && byp);
    const int src = bounce ? c : c + off;
    const int pl = bounce ? opposite(i) : i;
    const float2 d = __half22float2(dv[pl * kBPlane + src]);
    const float2 r = rr[src];
    fin[0][i] = fmaf(w, r.x, d.x);
    fin[1][i] = fmaf(w, r.y, d.y);
  });
}

struct TmaArgs {
  int* err;      // bit 0: a TMA wait expired; bit 1: misaligned shared memory
  int* counter;  // two tile counters, used by alternate launches (zero before first use)
  int parity;    // this launch uses counter[parity] and zeroes counter[parity ^ 1]
  int ntx, ntiles;
  const TmaMember* members;  // batched step: the member table
  const int4* index;         // batched step: per member {first tile, tile columns, tiles, 0}
  int nmem;
  int state;     // batched step: members read buf[state] and write buf[state ^ 1]
  unsigned stall_bytes;  // failure-path test only: bytes expected on top of the first copy
  int nstatic;   // tiles each CTA takes statically (blockIdx.x + k gridDim.x, k < nstatic)
                 // before it takes tiles from the counter
};

// Tile t of a lattice with ntx tile columns and ntiles tiles -> its origin. Numbering:
// the tiles of the first and last tile columns (whose boxes need periodic images
// patched in, the slowest tiles) come first, two per tile row, then the others row by
// row. The first tiles are the CTAs' static ones, so the counter's tiles even out the
// extra cost.
__device__ __forceinline__ void tile_origin(int t, int ntx, int ntiles, int& x0, int& y0) {
  const int nty = ntiles / ntx;
  const int nedge = ntx > 2 ? 2 * nty : 0;
  int bxx, byy;
  if (t < nedge) {
    byy = t >> 1;
    bxx = (t & 1) ? ntx - 1 : 0;
  } else {
    // u / rowlen by a float reciprocal, corrected to the exact quotient (u < 2^22)
    const int rowlen = nedge > 0 ? ntx - 2 : ntx;
    const int u = t - nedge;
    byy = (int)((float)u * __frcp_rn((float)rowlen));
    if (byy * rowlen > u) --byy;
    else if ((byy + 1) * rowlen <= u) ++byy;
    bxx = (nedge > 0 ? 1 : 0) + (u - byy * rowlen);
  }
  x0 = bxx * TX;
  y0 = byy * TY;
}

// A tile's lattice (member of a batch; 0 for a single lattice) and origin.
struct TileLoc {
  int m, x0, y0;
};

// Two CTAs per SM (64 registers a thread). BATCH: tiles of all members of a batch,
// each member's parameters copied into shared memory for its tiles. ST: the storage
// layout, Plain<0, float> (FP32) or HalfDev<0> (FP16 deviations, FP32 arithmetic);
// map_rho is the reference-density map of the latter.
template <int S, bool EDM, bool BATCH, typename ST>
__global__ void __launch_bounds__(NT, 2)
tma2d_kernel(const __grid_constant__ CUtensorMap map_pop, const __grid_constant__ CUtensorMap map_rho,
             typename ST::Reader f_one, typename ST::Writer fout_one, StepT<float> p_one, TmaArgs a) {
  constexpr bool HALF = ST::kHalf;
  constexpr int R = S + 1;  // psi halo
  constexpr int RX = TX + 2 * R, RY = TY + 2 * R;
  constexpr int GX = TX + 2 * S, GY = TY + 2 * S;
  constexpr int NHALO = RX * RY - NT, NRING = GX * GY - NT;
  // The dynamic shared memory starts the CTA's shared window (no static shared
  // memory here), so it is 1024-byte aligned; checked below. Indexing it directly
  // keeps every access a shared-memory access with 32-bit addresses.
  extern __shared__ __align__(1024) unsigned char sm[];
  float* const bx = reinterpret_cast<float*>(sm);
  float* s_psi = reinterpret_cast<float*>(sm + kOffPsi);
  float2* s_P = reinterpret_cast<float2*>(sm + kOffP);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + kOffBar);
  int* s_next = reinterpret_cast<int*>(sm + kOffBar + 8);  // next tile, its member and origin
  StepT<float>* s_p = reinterpret_cast<StepT<float>*>(sm + kOffBar + 32);  // [2], BATCH

  const int tid = threadIdx.x;
  const int tx = tid & (TX - 1), ty = tid >> 5;

  if (smem_u32(sm) & 1023u) {  // TMA destinations need the alignment: report, do nothing
    if (tid == 0) atomicOr(a.err, 2);
    return;
  }
  // Programmatic dependent launch: the next step's grid may be scheduled now; its CTAs
  // take the slots this grid's CTAs leave and run their prologue meanwhile.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!BATCH)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&map_pop)) : "memory");
  }
  __syncthreads();

  auto locate = [&](int t) {
    TileLoc l{0, 0, 0};
    if constexpr (BATCH) {
      // last member whose first tile is <= t, searched in the compact index (16 bytes a
      // member: its lines stay in L1, where the full records, one line apart, do not)
      int lo = 0, hi = a.nmem - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.index[mid].x <= t) lo = mid; else hi = mid - 1;
      }
      l.m = lo;
      const int4 e = a.index[lo];
      tile_origin(t - e.x, e.y, e.z, l.x0, l.y0);
    } else {
      tile_origin(t, a.ntx, a.ntiles, l.x0, l.y0);
    }
    return l;
  };
  unsigned extra = a.stall_bytes;  // nonzero only in the failure-path test: the wait runs out
  auto issue = [&](const TileLoc& l) {  // one thread: TMA load of a tile's box into the stage
    const CUtensorMap* map = BATCH ? &a.members[l.m].map[a.state] : &map_pop;
    if constexpr (HALF) {
      const CUtensorMap* mr = BATCH ? &a.members[l.m].map[2 + a.state] : &map_rho;
      mbar_expect_tx(&bar[0], kHalfDevBytes + kHalfRhoBytes + extra);
      tma_load_3d(bx, map, l.x0 - kBOX, l.y0 - kBOY, 0, &bar[0]);
      tma_load_2d(sm + kHalfRhoOff, mr, 2 * (l.x0 - kBOX), l.y0 - kBOY, &bar[0]);
    } else {
      mbar_expect_tx(&bar[0], kBoxBytes + extra);
      tma_load_3d(bx, map, l.x0 - kBOX, l.y0 - kBOY, 0, &bar[0]);
    }
    extra = 0;
  };
  auto pull = [&](int c, bool bym, bool byp, float out[2][kQ]) {
    if constexpr (HALF) pull_box_half(sm, c, bym, byp, out);
    else pull_box(bx, c, bym, byp, out);
  };

  // Up to here only shared memory was touched, so this may have run while the previous
  // step's grid was finishing. Wait for that grid to complete (its writes visible)
  // before reading its state or touching the tile counters; then the first copy is
  // issued and the per-thread offsets below are computed while it is in flight.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid == 0 && blockIdx.x == 0) a.counter[a.parity ^ 1] = 0;  // the next launch's counter
  unsigned seed_one = 0u;  // dither seed of a single lattice's stochastic rounding
  if constexpr (HALF && !BATCH) seed_one = step_seed(p_one, a.parity, tid == 0 && blockIdx.x == 0);

  unsigned phase = 0;    // parity of the next completion of the mbarrier
  bool pending = false;  // a TMA load into the stage is in flight
  int tile = blockIdx.x;
  TileLoc cur = locate(tile < a.ntiles ? tile : 0);
  if (tile < a.ntiles) {
    if (tid == 0) issue(cur);
    pending = true;
  }

  // This thread's halo cells (tid, tid + NT) and ring cell (tid) are the same in every
  // tile. Each is packed once into one word: offset in the psi region (or, for the
  // ring cell, in the probe region) | offset in the population box (or psi region) << 11
  // | (row relative to the tile + 8) << 22.
  static_assert(RX * RY <= 2048 && kBPlane <= 2048 && GX * GY <= 2048, "packed offsets");
  unsigned hcell[2] = {0u, 0u};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = tid + q * NT;
    if (h < NHALO) {
      int lx, ly;
      ring_cell<R>(h, lx, ly);
      hcell[q] = (unsigned)(lx + RX * ly) | ((unsigned)((ly - R + kBOY) * kBX + (lx - R + kBOX)) << 11) |
                 ((unsigned)(ly - R + 8) << 22);
    }
  }
  unsigned rcell = 0u;
  if constexpr (S > 0) {
    if (tid < NRING) {
      int lx, ly;
      ring_cell<S>(tid, lx, ly);
      rcell = (unsigned)(lx + GX * ly) | ((unsigned)((lx + 1) + RX * (ly + 1)) << 11) | ((unsigned)(ly - S + 8) << 22);
    }
  }
  auto lo11 = [](unsigned v) { return (int)(v & 2047u); };
  auto mid11 = [](unsigned v) { return (int)((v >> 11) & 2047u); };
  auto row8 = [](unsigned v) { return (int)(v >> 22) - 8; };

  // Thread 0 reserves tiles one iteration ahead, so the counter's round trip is never
  // waited for: at each tile it publishes the tile reserved before (read by all after
  // phase 1) and reserves the one after it. The first nstatic tiles of a CTA are
  // blockIdx.x + k gridDim.x; the counter hands out tiles from nstatic gridDim.x on.
  const int nstatic = a.nstatic > 0 ? a.nstatic : 1;
  int nres = 1;  // static tiles reserved so far (the current one included)
  auto next_tile = [&]() {
    if (nres < nstatic) return (int)blockIdx.x + (nres++) * (int)gridDim.x;
    return nstatic * (int)gridDim.x + atomicAdd(&a.counter[a.parity], 1);
  };
  int reserved = tid == 0 ? next_tile() : 0;
  int k = 0;
  while (tile < a.ntiles) {
    if (tid == 0) {
      s_next[0] = reserved;
      if (reserved < a.ntiles) {
        const TileLoc l = locate(reserved);
        s_next[1] = l.m;
        s_next[2] = l.x0;
        s_next[3] = l.y0;
      }
      reserved = next_tile();
    }
    const int slot = k & 1;
    if constexpr (BATCH) {  // this tile's member parameters (read after the next barrier)
      static_assert(sizeof(StepT<float>) % 4 == 0 && sizeof(StepT<float>) / 4 <= NT, "parameter copy");
      if (tid < (int)(sizeof(StepT<float>) / 4))
        reinterpret_cast<int*>(&s_p[slot])[tid] = reinterpret_cast<const int*>(&a.members[cur.m].p)[tid];
    }
    const int x0 = cur.x0, y0 = cur.y0;
    float fin[2][kQ];
    float rho1 = 0.f, rho2 = 0.f;

    // ---- phase 1: own populations (registers) and psi of the tile and its halo
    const bool ok = mbar_wait(&bar[0], phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.err, 1);
      if (pending) mbar_wait(&bar[0], phase);  // wait (bounded) for the copy still in flight
      return;
    }
    phase ^= 1u;
    pending = false;
    const StepT<float>& p = BATCH ? s_p[slot] : p_one;
    typename ST::Reader f = f_one;
    typename ST::Writer fout = fout_one;
    if constexpr (BATCH) {
      f = ST::reader(a.members[cur.m].buf[a.state], (unsigned)p.N);
      fout = ST::writer(a.members[cur.m].buf[a.state ^ 1], (unsigned)p.N);
    }
    if constexpr (HALF) {  // a member's seed is moved on by the CTA that takes its tile at (0, 0)
      if constexpr (BATCH) fout.seed = step_seed(p, a.state, tid == 0 && x0 == 0 && y0 == 0);
      else fout.seed = seed_one;
    }
    const bool walls = p.wall_y != 0;
    const int nx = p.nx, ny = p.ny;
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;

    // Box cells beyond the lattice along a periodic axis (always x; y without walls)
    // arrive from the copy as zeros and are overwritten with their periodic images
    // (plain loads, all 18 planes of a cell in flight together): out-of-range columns
    // [0, cl) and [cr, kBX) (all rows), then out-of-range rows [0, rt) and [rb, kBY)
    // (in-range columns). Beyond a wall nothing is read (bounce-back).
    const int cl = x0 < kBOX ? kBOX - x0 : 0, cr = min(kBX, nx - x0 + kBOX);
    const int rt = !walls && y0 < kBOY ? kBOY - y0 : 0, rb = walls ? kBY : min(kBY, ny - y0 + kBOY);
    const int ncol = cl + (kBX - cr);
    const int nfix = ncol * kBY + (rt + (kBY - rb)) * (cr - cl);
    if (nfix > 0) {
      for (int e = tid; e < nfix; e += NT) {
        int c, r;  // row-major: neighbouring threads, neighbouring columns
        if (e < ncol * kBY) {
          r = e / ncol;
          const int j = e - r * ncol;
          c = j < cl ? j : cr + (j - cl);
        } else {
          const int e2 = e - ncol * kBY, w = cr - cl;
          const int j = e2 / w;
          c = cl + (e2 - j * w);
          r = j < rt ? j : rb + (j - rt);
        }
        const unsigned src = (unsigned)(wrapn(x0 - kBOX + c, nx) + nx * wrapn(y0 - kBOY + r, ny));
        if constexpr (HALF) {  // the cell's 9 deviation words and its reference densities
          unsigned v[kQ];
          const unsigned* dg = reinterpret_cast<const unsigned*>(f.d);
          static_for<kQ>([&](auto I) {
            constexpr int pl = decltype(I)::value;
            v[pl] = __ldg(dg + (size_t)pl * f.N + src);
          });
          const float2 rv = __ldg(f.rho + src);
          unsigned* db = reinterpret_cast<unsigned*>(sm);
          static_for<kQ>([&](auto I) {
            constexpr int pl = decltype(I)::value;
            db[pl * kBPlane + r * kBX + c] = v[pl];
          });
          reinterpret_cast<float2*>(sm + kHalfRhoOff)[r * kBX + c] = rv;
        } else {
          float v[2 * kQ];
          static_for<2 * kQ>([&](auto I) {
            constexpr int pl = decltype(I)::value;
            v[pl] = __ldg(f.f + (size_t)pl * f.N + src);
          });
          static_for<2 * kQ>([&](auto I) {
            constexpr int pl = decltype(I)::value;
            bx[pl * kBPlane + r * kBX + c] = v[pl];
          });
        }
      }
      fence_async_smem();  // these generic writes precede the next TMA write of the stage
      __syncthreads();
    }
    {  // an own position beyond a ragged edge holds the psi of the site it wraps to (x,
       // periodic y: the box holds the image) or of its mirror across the wall
      const int gy = walls ? clampc(y, ny) : y;
      pull((gy - y0 + kBOY) * kBX + (tx + kBOX), walls && gy == 0, walls && gy == ny - 1, fin);
      s_psi[(tx + R) + RX * (ty + R)] = psi_of<kQ, float>(fin, &rho1, &rho2);
    }
    // the halo reaches a wall (or the mirror row beyond it) only in the first and last
    // tile rows of a walled channel
    const bool wall_halo = walls && (y0 < R + 1 || y0 + TY + R + 1 > ny);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (tid + q * NT >= NHALO) continue;
      int bo = mid11(hcell[q]);
      bool bym = false, byp = false;
      if (wall_halo) {
        const int gy = y0 + row8(hcell[q]);
        if (gy < -1 || gy > ny) continue;  // beyond a wall only the mirror row is read
        const int gyc = clampc(gy, ny);
        bo += (gyc - gy) * kBX;
        bym = gyc == 0;
        byp = gyc == ny - 1;
      }
      float hf[2][kQ];
      pull(bo, bym, byp, hf);
      s_psi[lo11(hcell[q])] = psi_of<kQ, float>(hf);
    }
    __syncthreads();
    const int next = s_next[0];
    TileLoc nloc{0, 0, 0};
    if (next < a.ntiles) {  // the stage has been read: load the next tile into it
      nloc = TileLoc{s_next[1], s_next[2], s_next[3]};
      if (tid == 0) issue(nloc);
      pending = true;
    }

    // ---- phase 2: unit normal and |grad psi|; own site in registers, every cell
    // within S of the tile as a probe normal (zero where |grad psi| <= g_th)
    float n0, n1, g;
    {
      float grad[3], n[3];
      grad_smem<0, float>(s_psi, RX, 0, (tx + R) + RX * (ty + R), grad);
      g = M<float>::unit(grad, n);
      n0 = n[0];
      n1 = n[1];
      if constexpr (S > 0) s_P[(tx + S) + GX * (ty + S)] = g > p.g_th ? make_float2(n0, n1) : make_float2(0.f, 0.f);
    }
    if constexpr (S > 0) {
      const int gy = y0 + row8(rcell);
      if (tid < NRING && !(walls && (gy < 0 || gy >= ny))) {  // probes stop at walls
        float grad[3], n[3];
        grad_smem<0, float>(s_psi, RX, 0, mid11(rcell), grad);
        const float gg = M<float>::unit(grad, n);
        s_P[lo11(rcell)] = gg > p.g_th ? make_float2(n[0], n[1]) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();

    // ---- phase 3: NCI ray search, forcing, collision, recolouring, store
    if (act) {
      const float rho = rho1 + rho2;
      float j[3];
      momentum<0, float>(fin, j);
      float frep0 = 0.f, frep1 = 0.f;
      if (S > 0 && g > p.g_th) {
        // g > g_th > = 0 implies a finite normal with |n_a| <= 1, so |probe offset| <= s
        const bool near_wall = walls && (y0 < S || y0 + TY + S > ny);
        int hit = 0;
        float A = 0.f;  // A_h(h) of the hit (indexed at compile time: no local copy of p)
        const float2* Pc = s_P + (tx + S) + GX * (ty + S);
        static_for<(S > 0 ? S : 1)>([&](auto I) {
          constexpr int st = decltype(I)::value + 1;
          if (hit != 0 || st > p.smax) return;
          const unsigned bxu = probe_bits(float(st), n0), byu = probe_bits(float(st), n1);
          if (near_wall) {
            const int py = y + (int)(byu - kMagicBits);
            if (py < 0 || py >= ny) { hit = -1; return; }
          }
          const int off = (int)(bxu + (unsigned)GX * byu - (unsigned)(GX + 1) * kMagicBits);
          const float2 q = Pc[off];
          if (q.x * n0 + q.y * n1 < 0.f) { hit = st; A = p.Ah[st]; }
        });
        if (hit > 0) {
          const float deltaI = 0.5f * g;
          frep0 = -A * n0 * deltaI;
          frep1 = -A * n1 * deltaI;
        }
      }
      const float F[3] = {p.G[0] + frep0, p.G[1] + frep1, p.G[2]};
      float u[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c] = __fdividef(j[c] + 0.5f * F[c], rho);
      const float m[3] = {-n0, -n1, 0.f};
      if constexpr (HALF)
        collide_store<0, float, typename ST::Writer, EDM>(fin, rho1, rho2, j, u, F, g, m, p, fout, x + nx * y);
      else
        collide_store<0, float, PlaneWriter, EDM>(fin, rho1, rho2, j, u, F, g, m, p, PlaneWriter{fout.f, fout.N},
                                                   x + nx * y);
    }
    tile = next;
    cur = nloc;
    ++k;
  }
}

StepT<float> to_step(const HostParams& h) {
  StepT<float> p;
  p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.wall_y = h.wall_y; p.wall_z = h.wall_z;
  p.N = h.N; p.smax = h.smax;
  p.edm = h.forcing == 1;
  p.omega = 1.0f / float(h.tau);
  p.guo = 1.0f - 0.5f * p.omega;
  p.pamp = 2.0f * (0.5f * float(h.A_s));
  p.beta = float(h.beta);
  p.g_th = float(h.g_th);
  for (int a = 0; a < 3; ++a) p.G[a] = float(h.G[a]);
  for (int k = 0; k < 8; ++k) {
    const float hd = float(k), hmin = float(h.h_min), hmax = float(h.h_max), A = float(h.A_h);
    if (k == 0) p.Ah[k] = 0.0f;
    else if (hd <= hmin) p.Ah[k] = A;
    else if (hd <= hmax) { const float r = hmin / hd; p.Ah[k] = A * (r * r * r); }
    else p.Ah[k] = 0.0f;
  }
  p.seedw = h.seedw;
  p.parity = h.parity;
  return p;
}

// Populations of one state as a 3-D tensor (x, y, plane) of 32-bit words, box 48 x 28 x
// planes: 18 float planes (FP32) or 9 half2 deviation planes (FP16-dev). L2 fetches of the
// box rows (192 bytes) are promoted to 128-byte lines (256-byte promotion measured 3% slower
// on back-to-back 2048 x 256 steps).
CUtensorMapL2promotion promotion_of(int bytes) {
  return bytes <= 0 ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                    : (bytes <= 64 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
                                   : (bytes <= 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                   : CU_TENSOR_MAP_L2_PROMOTION_L2_256B));
}

bool encode_pop(CUtensorMap* m, const void* base, const HostParams& h, unsigned planes = 2 * kQ, int promo = 128) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)h.nx, (cuuint64_t)h.ny, planes};
  const cuuint64_t strides[2] = {(cuuint64_t)h.nx * 4, (cuuint64_t)h.N * 4};
  const cuuint32_t box[3] = {kBX, kBY, planes};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promotion_of(promo),
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Reference densities of an FP16-dev state as a 2-D tensor (2 nx floats, ny), box 96 x 28.
bool encode_rho(CUtensorMap* m, const void* base, const HostParams& h, int promo = 128) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)h.nx * 2, (cuuint64_t)h.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)h.nx * 8};
  const cuuint32_t box[2] = {2 * kBX, kBY};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promotion_of(promo),
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, bool EDM, bool BATCH, typename ST>
cudaError_t launch_v(const CUtensorMap& map, const CUtensorMap& map_rho, const void* fa, void* fb,
                     const StepT<float>& p, TmaArgs a, int num_sms, cudaStream_t s) {
  static SmemAllowance configured;
  cudaError_t e = allow_smem(tma2d_kernel<S, EDM, BATCH, ST>, kSmemBytes, configured);
  if (e != cudaSuccess) return e;
  if (a.ntiles <= 0) return cudaSuccess;
  const int slots = 2 * num_sms;  // resident CTAs
  const int grid = a.ntiles < slots ? a.ntiles : slots;
  // programmatic stream serialisation: the launch may begin while the previous kernel on
  // the stream finishes; the kernel waits for it (griddepcontrol.wait) before any
  // global access
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tma2d_kernel<S, EDM, BATCH, ST>, map, map_rho, ST::reader(fa, (unsigned)p.N),
                            ST::writer(fb, (unsigned)p.N), p, a);
}

template <bool BATCH, typename ST>
cudaError_t launch_st(const CUtensorMap& map, const CUtensorMap& map_rho, const void* fa, void* fb,
                      const StepT<float>& p, const TmaArgs& a, int smax, bool edm, int num_sms, cudaStream_t s) {
  if (smax == 0)
    return edm ? launch_v<0, true, BATCH, ST>(map, map_rho, fa, fb, p, a, num_sms, s)
               : launch_v<0, false, BATCH, ST>(map, map_rho, fa, fb, p, a, num_sms, s);
  return edm ? launch_v<kMaxProbe, true, BATCH, ST>(map, map_rho, fa, fb, p, a, num_sms, s)
             : launch_v<kMaxProbe, false, BATCH, ST>(map, map_rho, fa, fb, p, a, num_sms, s);
}

template <bool BATCH>
cudaError_t launch_any(const CUtensorMap& map, const CUtensorMap& map_rho, const void* fa, void* fb,
                       const StepT<float>& p, const TmaArgs& a, int smax, bool edm, bool half, int num_sms,
                       cudaStream_t s) {
  return half ? launch_st<BATCH, HalfDev<0>>(map, map_rho, fa, fb, p, a, smax, edm, num_sms, s)
              : launch_st<BATCH, Plain<0, float>>(map, map_rho, fa, fb, p, a, smax, edm, num_sms, s);
}

}  // namespace

bool tma2d_supported(const HostParams& h) { return h.nx % 4 == 0 && h.nz == 1 && encode_fn() != nullptr; }

cudaError_t tma2d_prepare(TmaMaps* m, const void* fa, const void* fb, const HostParams& h, int promo) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(m->bytes);
  std::memset(m->bytes, 0, sizeof(m->bytes));
  if (!h.half)
    return encode_pop(&maps[0], fa, h, 2 * kQ, promo) && encode_pop(&maps[1], fb, h, 2 * kQ, promo)
               ? cudaSuccess
               : cudaErrorInvalidValue;
  const size_t ro = HalfDev<0>::rho_offset((size_t)h.N);
  const bool ok = encode_pop(&maps[0], fa, h, kQ, promo) && encode_pop(&maps[1], fb, h, kQ, promo) &&
                  encode_rho(&maps[2], (const char*)fa + ro, h, promo) &&
                  encode_rho(&maps[3], (const char*)fb + ro, h, promo);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tma2d_step(const TmaMaps& m, int from, const void* fa, void* fb, int* err, int* counter,
                       const HostParams& h, cudaStream_t s) {
  const StepT<float> p = to_step(h);
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(m.bytes);
  const CUtensorMap& map = maps[from];
  const CUtensorMap& map_rho = maps[h.half ? 2 + from : from];
  TmaArgs a{};
  a.stall_bytes = h.tma_stall_test ? 16u : 0u;
  a.err = err;
  a.counter = counter;
  a.parity = from & 1;  // the state alternates with every step, and so do the counters
  a.ntx = (p.nx + TX - 1) / TX;
  a.ntiles = a.ntx * ((p.ny + TY - 1) / TY);
  a.nstatic = 2;
  return launch_any<false>(map, map_rho, fa, fb, p, a, h.smax, h.forcing == 1, h.half != 0, h.num_sms, s);
}

static_assert(sizeof(TmaMember) % 64 == 0, "member records keep the tensor maps 64-byte aligned and the index 16");
size_t tma2d_table_bytes(int nmem) { return (size_t)nmem * (sizeof(TmaMember) + sizeof(int4)); }

int tma2d_member_fill(void* table, int k, int nmem, const TmaMaps& m, const HostParams& h, void* buf0, void* buf1,
                      int tile0) {
  static_assert(sizeof(TmaMember::map) <= sizeof(TmaMaps::bytes), "member maps: the first four of the sim's maps");
  TmaMember mb;
  std::memset(&mb, 0, sizeof(mb));
  std::memcpy(mb.map, m.bytes, sizeof(mb.map));
  mb.p = to_step(h);
  mb.buf[0] = (float*)buf0;
  mb.buf[1] = (float*)buf1;
  mb.ntx = (h.nx + TX - 1) / TX;
  mb.ntiles = mb.ntx * ((h.ny + TY - 1) / TY);
  mb.tile0 = tile0;
  std::memcpy((unsigned char*)table + (size_t)k * sizeof(TmaMember), &mb, sizeof(mb));
  const int4 e = make_int4(tile0, mb.ntx, mb.ntiles, 0);
  std::memcpy((unsigned char*)table + (size_t)nmem * sizeof(TmaMember) + (size_t)k * sizeof(int4), &e, sizeof(e));
  return mb.ntiles;
}

cudaError_t tma2d_batch_step(const void* members, int nmem, int total_tiles, int state, int* err, int* counter,
                             int smax_max, int edm, int half, int num_sms, int nstatic, cudaStream_t s) {
  TmaArgs a{};
  a.nstatic = nstatic;
  a.err = err;
  a.counter = counter;
  a.parity = state & 1;
  a.ntx = 1;
  a.ntiles = total_tiles;
  a.members = (const TmaMember*)members;
  a.index = (const int4*)((const unsigned char*)members + (size_t)nmem * sizeof(TmaMember));
  a.nmem = nmem;
  a.state = state & 1;
  StepT<float> none;
  std::memset(&none, 0, sizeof(none));
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  return launch_any<true>(unused, unused, nullptr, nullptr, none, a, smax_max, edm != 0, half != 0, num_sms, s);
}

}  // namespace lbnci
