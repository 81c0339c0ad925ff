// lb_launch.h -- internal launch table between the C ABI (lb_api.cu) and the
// per-storage kernel instantiations (lb_fp64.cu, lb_fp32.cu, lb_fp16.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "lb_lattice.cuh"

namespace lbnci {

// The largest dynamic shared memory each device has been told a kernel may use.
// cudaFuncSetAttribute applies to the current device only, so a process that launches
// on several devices needs one record per device; two threads that race here may both
// set the attribute, which is harmless.
constexpr int kMaxDevices = 64;
struct SmemAllowance {
  std::atomic<size_t> bytes[kMaxDevices];
};

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes, SmemAllowance& a) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kMaxDevices;
  if (tracked && a.bytes[dev].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && tracked) {
    size_t cur = a.bytes[dev].load(std::memory_order_acquire);
    while (cur < bytes && !a.bytes[dev].compare_exchange_weak(cur, bytes, std::memory_order_acq_rel)) {
    }
  }
  return e;
}

// Everything a launcher needs, in FP64; each instantiation converts it to its own
// arithmetic type once per call.
struct HostParams {
  int nx, ny, nz, wall_y, wall_z, N, smax;
  int spt;      // sites per thread of the fused D2Q9 kernel (2 or 4)
  int num_sms;  // multiprocessors of the device
  int forcing;  // 0: Guo, 1: exact difference method on the dispersed phase
  int d3_kernel;  // D3Q27 collision: 0 marching along z (default), 1 tiled
  int tma;        // 1: D2Q9 FP32 / FP16-dev steps run the persistent TMA-fed kernel
  int half;       // FP16-deviation storage
  int tma_stall_test;  // 1: its first copy is expected to bring 16 more bytes than it does,
                       // so its bounded wait runs out (test of the failure path only)
  int carry3d;    // 1: D3Q27 FP32 / FP16-dev steps run the single-read carry kernels
  int c3_zseg;    // planes per z segment of their collision kernel
  int stream3d;   // 1: D3Q27 steps run moments, normals and a streaming collision
  int totals;     // 1: streaming steps with Guo forcing store the total + recolouring form
  float rho_ref;  // reference density rho_0 of the FP16 totals (f*_i = w_i rho_0 + d_i)
  unsigned* seedw;  // device: two dither-seed words of the FP16-deviation stores
  int parity;       // state buffer the next step reads (0: the one the sim was created with)
  double tau, A_s, beta, A_h, h_min, h_max, g_th, G[3];
};

struct Launchers {
  size_t (*state_bytes)(size_t N);  // bytes of one population state
  size_t compute_elem;              // bytes of the arithmetic type (psi scratch elements)
  cudaError_t (*init)(void* f, const double* rho1, const double* rho2, const double* u,
                      const HostParams& p, cudaStream_t s);
  // One full step fa -> fb (psi: scratch of N compute elements). Kernels launched -> *nk.
  cudaError_t (*step)(const void* fa, void* fb, void* psi, const HostParams& p, cudaStream_t s, int* nk);
  cudaError_t (*fields)(const void* f, void* psi, const HostParams& p, const FieldOut& fo,
                        cudaStream_t s, int* nk);
  // FP64 [2][Q][pitch] copies of sites [s0, s0 + count) of a state, and back.
  cudaError_t (*decode)(const void* f, double* out, int s0, int count, long long pitch, int N, cudaStream_t s);
  cudaError_t (*encode)(const double* in, void* f, int s0, int count, long long pitch, int N, cudaStream_t s);
  // Ensembles of D2Q9 lattices: bytes of one member record, filling one on the host,
  // tile counts per member for a tile shape, and the batched step over all members.
  size_t batch_member_bytes;
  void (*batch_fill)(void* dst, const HostParams& p, const void* buf0, const void* buf1);
  int (*batch_tiles)(const HostParams& p, int spt);
  cudaError_t (*batch_step)(const void* members, const int* tile0, int n, int total_tiles, int parity, int spt,
                            int smax_max, int edm, cudaStream_t s);
};

// Persistent TMA-fed D2Q9 step (lb_tma2d.cu) for FP32 and FP16-dev storage, tiles of
// kTmaTX x kTmaTY sites.
constexpr int kTmaTX = 32, kTmaTY = 16;
struct TmaMaps {
  // tensor maps: FP32: box of state buffer A, B; FP16-dev: deviations of A, B, then the
  // reference densities of A, B; the single-read D3Q27 step adds its per-site
  // (n, |grad psi|) and NCI distances (slots 4, 5)
  alignas(64) unsigned char bytes[6 * 128];
};
bool tma2d_supported(const HostParams& h);
// promo: L2 promotion of the copies' fetches in bytes (0, 64, 128 or 256; 128 by default)
cudaError_t tma2d_prepare(TmaMaps* m, const void* fa, const void* fb, const HostParams& h, int promo = 128);
// One step from state `from` (0: buffer A, 1: buffer B) into the other buffer. counter:
// two device ints, zero at first use, reserved for this sim's steps (alternate states
// use alternate counters).
cudaError_t tma2d_step(const TmaMaps& m, int from, const void* fa, void* fb, int* err, int* counter,
                       const HostParams& h, cudaStream_t s);
// Batched TMA step over the members of an ensemble: a device table of tma2d_table_bytes
// (nmem) bytes, filled on the host by tma2d_member_fill for k = 0 .. nmem - 1 (member
// records, then a compact index of the members' first tiles and tile grids that the
// kernel searches; returns the member's tile count; tile0 = tiles of the members before
// it). Members read their buffer `state` and write the other; counter as for tma2d_step,
// reserved for the batch.
size_t tma2d_table_bytes(int nmem);
int tma2d_member_fill(void* table, int k, int nmem, const TmaMaps& m, const HostParams& h, void* buf0, void* buf1,
                      int tile0);
// nstatic: tiles each CTA takes statically before it takes tiles from the counter.
cudaError_t tma2d_batch_step(const void* members, int nmem, int total_tiles, int state, int* err, int* counter,
                             int smax_max, int edm, int half, int num_sms, int nstatic, cudaStream_t s);

// Single-read D3Q27 step (lb_carry3d.cu) for FP32 and FP16-dev storage on lattices with
// nx % 32 == 0 and ny % 8 == 0: an interface pass (psi, gradient, normal from the
// carried densities) and a TMA-fed collision that also produces the next step's
// densities. Device buffers: carry (N float2), ring (carry3d_ring_bytes), ghost
// (carry3d_ghost_bytes), ng (N float4), hit (N bytes).
bool carry3d_supported(const HostParams& h);
size_t carry3d_ring_bytes(const HostParams& h);
size_t carry3d_ghost_bytes(const HostParams& h);
// tensor maps of both state buffers (FP32: populations of A, B; FP16-dev: deviations of
// A, B, then reference densities of A, B)
cudaError_t carry3d_prepare(TmaMaps* m, const void* fa, const void* fb, const void* ng, const void* hit,
                            const HostParams& h);
// the carried densities of a state no step produced (pulled from it; rings zeroed)
cudaError_t carry3d_init(const void* f, void* carry, void* ring, void* ghost, const HostParams& h, cudaStream_t s);
// one step from state `from` (0: buffer A, 1: buffer B) into the other; *nk = launches
// Streaming D3Q27 step (lb_carry3d.cu) for FP32 and FP16-dev storage on lattices of whole
// 32 x 8 columns: moments (psi), normals3d ((n, |grad psi|) into ng, N float4), collide3d
// (near-contact ray, pull, collision: fa -> fb). Kernels launched -> *nk.
// With h.totals, steps under Guo forcing store the total + recolouring form of the
// precision (TotalRecol / TotalRecolHalf in lb_carry3d.cuh: the total populations, the rest
// population of each component and (rho_1/rho, beta rho_1 rho_2/rho m) per site; FP16 totals
// as deviations from w_i h.rho_ref); totals_in says that fa holds that form; rho12 (N float2)
// carries (rho_1, rho_2) from the moments pass to the collision.
bool stream3d_supported(const HostParams& h);
bool stream3d_stores_totals(const HostParams& h);
cudaError_t stream3d_step(const void* fa, void* fb, void* psi, void* ng, void* rho12, int totals_in,
                          const HostParams& h, cudaStream_t s, int* nk);
// fields and population copies of a state in the total + recolouring form (the
// Launchers::fields / decode of the other states)
cudaError_t stream3d_form_fields(const void* f, void* psi, const HostParams& h, const FieldOut& fo, cudaStream_t s,
                                 int* nk);
cudaError_t stream3d_form_decode(const void* f, double* out, int s0, int count, long long pitch, const HostParams& h,
                                 cudaStream_t s);
size_t stream3d_totals_bytes(size_t N, int half);
cudaError_t carry3d_step(const TmaMaps& m, int from, const void* fa, void* fb, void* carry, void* ring, void* ghost,
                         void* ng, void* hit, int* err, const HostParams& h, cudaStream_t s, int* nk);

const Launchers* launchers_fp64(int lattice);
const Launchers* launchers_fp32(int lattice);
const Launchers* launchers_fp16dev(int lattice);

// Number of thread blocks of the tiled kernels (= partial-sum slots of the fields kernel).
long long tiled_blocks(int lattice, const HostParams& p);
cudaError_t reduce_partials(const double* partials, long long nblocks, double* out, cudaStream_t s);

}  // namespace lbnci
