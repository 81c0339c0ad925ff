// lb_api.cu -- C ABI of the NCI colour-gradient lattice Boltzmann library (lbnci.h).
// Handles, validation, memory and the step loop; all arithmetic runs in the kernels
// of lb_fp64.cu / lb_fp32.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <new>

#include "lbnci.h"
#include "lb_launch.h"

namespace lbnci {

__global__ void __launch_bounds__(256) reduce_partials_kernel(const double* __restrict__ partials,
                                                              long long nblocks, double* __restrict__ out) {
  // One block: thread t sums blocks t, t+256, ... in order, then a fixed tree.
  __shared__ double s[256];
  for (int q = 0; q < kRedSlots; ++q) {
    double v = 0.0;
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b * kRedSlots + q];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = s[0];
    __syncthreads();
  }
}

cudaError_t reduce_partials(const double* partials, long long nblocks, double* out, cudaStream_t s) {
  reduce_partials_kernel<<<1, 256, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// Sum of rho1 + rho2 over the sites, per block (a grid-stride range, then a fixed tree) into
// slot 0 of the block's partials (the other slots zeroed), for reduce_partials to add in a
// fixed order: the mean density of the initial fields in a few microseconds.
__global__ void __launch_bounds__(256) density_sum_kernel(const double* __restrict__ rho1,
                                                          const double* __restrict__ rho2, long long N,
                                                          double* __restrict__ partials) {
  __shared__ double s[256];
  double v = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < N; i += (long long)gridDim.x * 256) v += rho1[i] + rho2[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kRedSlots) partials[blockIdx.x * (long long)kRedSlots + threadIdx.x] = threadIdx.x == 0 ? s[0] : 0.0;
}

long long tiled_blocks(int lattice, const HostParams& p) {
  if (lattice == 0) {
    return (long long)((p.nx + Tile<0>::X - 1) / Tile<0>::X) * ((p.ny + Tile<0>::Y - 1) / Tile<0>::Y) *
           ((p.nz + Tile<0>::Z - 1) / Tile<0>::Z);
  }
  return (long long)((p.nx + Tile<1>::X - 1) / Tile<1>::X) * ((p.ny + Tile<1>::Y - 1) / Tile<1>::Y) *
         ((p.nz + Tile<1>::Z - 1) / Tile<1>::Z);
}

}  // namespace lbnci

using namespace lbnci;

struct lb_sim {
  lb_config cfg;
  HostParams p{};
  const Launchers* L;
  int Q;
  int device;
  cudaStream_t stream;
  void* fa;        // current state
  void* fb;        // back buffer (also staging between steps)
  void* buf_a;     // the state buffer that fa points to at creation
  TmaMaps maps;    // tensor maps of both state buffers (p.tma)
  int* errflag;    // device word: bit 0 set when a kernel's bounded wait expired
  int* tile_counter;  // two device ints: tile counters of the TMA step kernel
  const int* ens_flag;  // member of an ensemble stepped by the batched TMA kernel: its error word
  void* psi;       // order parameter of the streamed state
  void* carry;     // single-read D3Q27 path (p.carry3d): carried densities, ring exports,
  void* ring;      // ghost planes of the z segments, per-site (n, |grad psi|) and NCI distance
  void* ghost;
  void* ng;
  void* hit;
  bool carry_ok;   // the carried densities belong to the current state
  void* rho1;      // streaming D3Q27 path: (rho_1, rho_2) of each site from the moments pass
  bool totals_state;  // fa holds the total + recolouring form (p.totals)
  double* partials;
  double* result;  // kRedSlots doubles
  double* host_result;  // pinned
  long long nblocks;
  bool owns;       // memory from cudaMalloc (else carved from the workspace)
  void* base;      // cudaMalloc'd block
  long long step;
  long long launches;
  bool in_ensemble;  // stepped by its ensemble only
  char err[256];
};

namespace {

thread_local char g_err[256] = "";

lb_status fail(lb_sim* s, lb_status st, const char* fmt, ...) {
  char* dst = s ? s->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

lb_status cuda_fail(lb_sim* s, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear the error so the next launch check does not report it again
  return fail(s, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// The result area holds 16 doubles: the kRedSlots reductions, then, in slot
// kErrSlot, the kernels' error word (an int), in slot kErrSlot + 1 the two tile
// counters of the TMA step kernel (ints), and in slot kErrSlot + 2 the two dither-seed
// words of the FP16-deviation stores (StepT::seedw).
constexpr int kErrSlot = 12;

struct Layout {
  size_t fa, fb, psi, partials, result, carry, ring, ghost, ng, hit, rho1, total;
};

const Launchers* launchers_for(const lb_config* c) {
  if (c->precision == LB_FP64) return launchers_fp64(c->lattice);
  if (c->precision == LB_FP16DEV) return launchers_fp16dev(c->lattice);
  return launchers_fp32(c->lattice);
}

lb_status validate(const lb_config* c, HostParams* p, Layout* lay, long long* nblocks) {
  if (!c) return fail(nullptr, LB_EINVAL, "config is NULL");
  if (c->lattice != LB_D2Q9 && c->lattice != LB_D3Q27)
    return fail(nullptr, LB_EINVAL, "unknown lattice %d", c->lattice);
  if (c->precision != LB_FP64 && c->precision != LB_FP32 && c->precision != LB_FP16DEV)
    return fail(nullptr, LB_EUNSUPPORTED, "precision %d is not implemented", c->precision);
  if (c->nx < 1 || c->ny < 1 || c->nz < 1)
    return fail(nullptr, LB_EINVAL, "lattice sizes must be >= 1 (got %d x %d x %d)", c->nx, c->ny, c->nz);
  if (c->lattice == LB_D2Q9 && c->nz != 1) return fail(nullptr, LB_EINVAL, "D2Q9 needs nz == 1");
  if (c->lattice == LB_D2Q9 && c->wall_z) return fail(nullptr, LB_EINVAL, "D2Q9 has no z walls");
  if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return fail(nullptr, LB_EINVAL, "tau must be > 1/2");
  if (!(c->beta >= 0.0 && c->beta <= 1.0)) return fail(nullptr, LB_EINVAL, "beta must be in [0, 1]");
  if (!(c->A_s >= 0.0) || !std::isfinite(c->A_s)) return fail(nullptr, LB_EINVAL, "A_s must be >= 0");
  if (!(c->A_h >= 0.0) || !std::isfinite(c->A_h)) return fail(nullptr, LB_EINVAL, "A_h must be >= 0");
  if (!(c->g_th >= 0.0) || !std::isfinite(c->g_th)) return fail(nullptr, LB_EINVAL, "g_th must be >= 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(c->force[a])) return fail(nullptr, LB_EINVAL, "force must be finite");
  if (c->forcing != LB_FORCE_GUO && c->forcing != LB_FORCE_EDM_DISPERSED)
    return fail(nullptr, LB_EINVAL, "unknown forcing scheme %d", c->forcing);
  int smax = 0;
  if (c->A_h > 0.0) {
    if (!(c->h_min > 0.0 && c->h_min <= c->h_max && c->h_max < kMaxProbe + 1.0))
      return fail(nullptr, LB_EINVAL, "NCI needs 0 < h_min <= h_max < 5 (got %g, %g)", c->h_min, c->h_max);
    smax = (int)std::floor(c->h_max);
  }
  const long long N = (long long)c->nx * c->ny * c->nz;
  const int Qc = c->lattice == LB_D2Q9 ? 9 : 27;
  if (2LL * Qc * N >= (1LL << 32))
    return fail(nullptr, LB_EINVAL, "lattice too large (2*Q*N must be < 2^32 populations)");
  p->nx = c->nx; p->ny = c->ny; p->nz = c->nz;
  p->wall_y = c->wall_y ? 1 : 0;
  p->wall_z = c->wall_z ? 1 : 0;
  p->N = (int)N;
  p->tau = c->tau; p->A_s = c->A_s; p->beta = c->beta; p->A_h = c->A_h;
  p->h_min = c->h_min; p->h_max = c->h_max; p->g_th = c->g_th;
  for (int a = 0; a < 3; ++a) p->G[a] = c->force[a];
  if (c->lattice == LB_D2Q9) p->G[2] = 0.0;
  p->smax = smax;
  p->forcing = c->forcing;
  p->num_sms = 1;
  // D3Q27 collision kernel: LBNCI_D3_KERNEL=march (z-marching, default) or tiled.
  p->d3_kernel = 0;
  if (const char* e = std::getenv("LBNCI_D3_KERNEL")) p->d3_kernel = std::strcmp(e, "tiled") == 0 ? 1 : 0;
  // Tile of the fused D2Q9 kernel: LBNCI_FUSED_SPT=2 (32x16, the default) or 4 (32x32).
  p->spt = 2;
  if (const char* e = std::getenv("LBNCI_FUSED_SPT")) p->spt = std::atoi(e) == 4 ? 4 : 2;
  // D2Q9 FP32 / FP16-dev step: the persistent TMA-fed kernel (its maps need nx % 4 == 0),
  // unless LBNCI_FUSED=classic selects the one-pass fused kernel.
  p->tma = c->lattice == LB_D2Q9 && (c->precision == LB_FP32 || c->precision == LB_FP16DEV) && c->nx % 4 == 0 ? 1 : 0;
  p->half = c->precision == LB_FP16DEV ? 1 : 0;
  if (const char* e = std::getenv("LBNCI_FUSED"))
    if (std::strcmp(e, "classic") == 0) p->tma = 0;
  // Test of the failure path of the TMA kernel's bounded waits (never set in use):
  // LBNCI_TMA_STALL_TEST=1 makes every CTA's first wait run out after about a second.
  p->tma_stall_test = 0;
  if (const char* e = std::getenv("LBNCI_TMA_STALL_TEST")) p->tma_stall_test = std::atoi(e) == 1 ? 1 : 0;
  // D3Q27 FP32 / FP16-dev step on lattices of whole 32 x 8 columns: the streaming step
  // (moments, normals, collision with the ray), the fastest measured; LBNCI_D3_KERNEL=carry
  // selects the single-read step (density carry), march or tiled the two-pass step, which
  // the other lattices and FP64 run
  const bool col_ok = c->lattice == LB_D3Q27 && (c->precision == LB_FP32 || c->precision == LB_FP16DEV) &&
                      c->nx % 32 == 0 && c->ny % 8 == 0 && (c->wall_z || c->nz >= 2);
  p->carry3d = 0;
  p->stream3d = col_ok ? 1 : 0;
  if (const char* e = std::getenv("LBNCI_D3_KERNEL")) {
    if (std::strcmp(e, "march") == 0 || std::strcmp(e, "tiled") == 0) p->stream3d = 0;
    if (std::strcmp(e, "carry") == 0 && col_ok) { p->carry3d = 1; p->stream3d = 0; }
  }
  // streaming steps with Guo forcing store the total + recolouring form (FP32: 128 instead
  // of 216 bytes per site; FP16-dev: 76 instead of 116), unless LBNCI_D3_STATE=pairs keeps
  // the two-population layout
  p->totals = p->stream3d && c->forcing == 0 ? 1 : 0;
  if (const char* e = std::getenv("LBNCI_D3_STATE"))
    if (std::strcmp(e, "pairs") == 0) p->totals = 0;
  p->rho_ref = 1.0f;
  // z segment of the single-read collision kernel (planes; LBNCI_C3_ZSEG, default 16)
  p->c3_zseg = 16;
  if (const char* e = std::getenv("LBNCI_C3_ZSEG")) p->c3_zseg = std::atoi(e) > 0 ? std::atoi(e) : 16;
  const int Q = c->lattice == LB_D2Q9 ? 9 : 27;
  (void)Q;
  const Launchers* L = launchers_for(c);
  const size_t state = L->state_bytes((size_t)N);
  if (p->totals && stream3d_totals_bytes((size_t)N, p->half) > state) p->totals = 0;  // the form lives in a state buffer
  *nblocks = tiled_blocks(c->lattice, *p);
  size_t off = 0;
  lay->fa = off; off = align256(off + state);
  lay->fb = off; off = align256(off + state);
  lay->psi = off; off = align256(off + (size_t)N * L->compute_elem);
  lay->partials = off; off = align256(off + (size_t)(*nblocks) * kRedSlots * sizeof(double));
  lay->result = off; off = align256(off + 16 * sizeof(double));
  lay->carry = lay->ring = lay->ghost = lay->ng = lay->hit = lay->rho1 = off;
  if (p->carry3d) {
    lay->carry = off; off = align256(off + (size_t)N * 8);
    lay->ring = off; off = align256(off + carry3d_ring_bytes(*p));
    lay->ghost = off; off = align256(off + carry3d_ghost_bytes(*p));
    lay->ng = off; off = align256(off + (size_t)N * 16);
    lay->hit = off; off = align256(off + (size_t)N);
  }
  if (p->stream3d) {
    lay->ng = off; off = align256(off + (size_t)N * 16);
    lay->rho1 = off; off = align256(off + (size_t)N * 2 * sizeof(float));
  }
  lay->total = off;
  return LB_OK;
}

// Doubles of staging the back buffer can hold.
size_t staging_doubles(const lb_sim* s) { return s->L->state_bytes((size_t)s->p.N) / sizeof(double); }

// Sites per host transfer of a [2Q][N] FP64 array through the back buffer (one copy
// per population row of the chunk).
long long staging_chunk(const lb_sim* s) {
  const long long fit = (long long)(staging_doubles(s) / (size_t)(2 * s->Q));
  return fit >= s->p.N ? s->p.N : fit;
}

// Run the fields kernel on the current state with the given device outputs and
// fill s->host_result with the reduced observables (synchronises the stream).
lb_status run_fields(lb_sim* s, const FieldOut& outs) {
  FieldOut fo = outs;
  fo.partials = s->partials;
  int nk = 0;
  cudaError_t e = s->totals_state ? stream3d_form_fields(s->fa, s->psi, s->p, fo, s->stream, &nk)
                                  : s->L->fields(s->fa, s->psi, s->p, fo, s->stream, &nk);
  s->launches += nk + 1;
  if (e != cudaSuccess) return cuda_fail(s, e, "fields launch");
  e = reduce_partials(s->partials, s->nblocks, s->result, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "reduce launch");
  e = cudaMemcpyAsync(s->host_result, s->result, 16 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "result copy");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  int flag = 0;
  std::memcpy(&flag, &s->host_result[kErrSlot], sizeof(flag));
  if (s->ens_flag) {  // the batched step reports into its ensemble's word
    int ef = 0;
    e = cudaMemcpy(&ef, s->ens_flag, sizeof(ef), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "ensemble flag copy");
    flag |= ef;
  }
  if (flag != 0)
    return fail(s, LB_ECUDA, "%s (flag %d); the state is invalid",
                (flag & 1) ? "a step kernel gave up waiting for its TMA copies"
                           : "a step kernel found its shared memory misaligned for TMA and did nothing", flag);
  return LB_OK;
}

// The reference density rho_0 of the FP16 total + recolouring form: the mean total
// density of a state just set; from the density fields given to lb_init_fields (d1, d2 on
// the device) or, after lb_set_populations, from a fields pass. Synchronises the stream.
lb_status refresh_rho_ref(lb_sim* s, const double* d1 = nullptr, const double* d2 = nullptr) {
  if (!(s->p.stream3d && s->p.totals && s->p.half)) return LB_OK;
  double total = 0.0;
  if (d1 && d2) {
    const long long nb = s->nblocks < 1024 ? s->nblocks : 1024;
    density_sum_kernel<<<(unsigned)nb, 256, 0, s->stream>>>(d1, d2, s->p.N, s->partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = reduce_partials(s->partials, nb, s->result, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, s->result, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    s->launches += 2;
    if (e != cudaSuccess) return cuda_fail(s, e, "reference density");
  } else {
    lb_status st = run_fields(s, FieldOut{});
    if (st != LB_OK) return st;
    total = s->host_result[0] + s->host_result[1];
  }
  const double r = total / (double)s->p.N;
  s->p.rho_ref = std::isfinite(r) && r > 0.0 ? (float)r : 1.0f;
  return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_workspace_size(const lb_config* cfg, size_t* bytes) {
  if (!bytes) return fail(nullptr, LB_EINVAL, "bytes is NULL");
  HostParams p{};
  Layout lay;
  long long nb;
  lb_status st = validate(cfg, &p, &lay, &nb);
  if (st != LB_OK) return st;
  *bytes = lay.total;
  return LB_OK;
}

lb_status lb_create(const lb_config* cfg, lb_sim** out) {
  if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
  *out = nullptr;
  HostParams p{};
  Layout lay;
  long long nblocks;
  lb_status st = validate(cfg, &p, &lay, &nblocks);
  if (st != LB_OK) return st;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LB_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  const Launchers* L = launchers_for(cfg);
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0) p.num_sms = nsm;
  cudaGetLastError();
  lb_sim* s = new (std::nothrow) lb_sim();
  if (!s) return fail(nullptr, LB_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->p = p;
  s->L = L;
  s->Q = cfg->lattice == LB_D2Q9 ? 9 : 27;
  s->device = dev;
  s->stream = (cudaStream_t)cfg->stream;
  s->nblocks = nblocks;
  unsigned char* base = nullptr;
  if (cfg->workspace) {
    if (((uintptr_t)cfg->workspace & 255u) != 0) {
      delete s;
      return fail(nullptr, LB_EINVAL, "workspace must be 256-byte aligned");
    }
    if (cfg->workspace_bytes < lay.total) {
      delete s;
      return fail(nullptr, LB_ENOMEM, "workspace has %zu bytes, %zu needed", cfg->workspace_bytes, lay.total);
    }
    base = (unsigned char*)cfg->workspace;
    s->owns = false;
  } else {
    e = cudaMalloc((void**)&base, lay.total);
    if (e != cudaSuccess) {
      delete s;
      cudaGetLastError();
      return fail(nullptr, e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA,
                  "cudaMalloc of %zu bytes failed: %s", lay.total, cudaGetErrorString(e));
    }
    s->owns = true;
    s->base = base;
  }
  s->fa = base + lay.fa;
  s->fb = base + lay.fb;
  s->buf_a = s->fa;
  s->psi = base + lay.psi;
  s->partials = (double*)(base + lay.partials);
  s->result = (double*)(base + lay.result);
  s->errflag = (int*)(s->result + kErrSlot);
  s->tile_counter = (int*)(s->result + kErrSlot + 1);
  s->p.seedw = (unsigned*)(s->result + kErrSlot + 2);
  s->p.parity = 0;
  if (s->p.tma) {
    // tensor maps of both state buffers; without the driver's tensor-map encoder the
    // step falls back to the one-pass fused kernel
    if (!tma2d_supported(s->p) || tma2d_prepare(&s->maps, s->fa, s->fb, s->p) != cudaSuccess) s->p.tma = 0;
    cudaGetLastError();
  }
  if (s->p.carry3d) {
    s->carry = base + lay.carry;
    s->ring = base + lay.ring;
    s->ghost = base + lay.ghost;
    s->ng = base + lay.ng;
    s->hit = base + lay.hit;
    // without the driver's tensor-map encoder the step falls back to the two-pass kernels
    if (!carry3d_supported(s->p) || carry3d_prepare(&s->maps, s->fa, s->fb, s->ng, s->hit, s->p) != cudaSuccess)
      s->p.carry3d = 0;
    cudaGetLastError();
  }
  if (s->p.stream3d) {
    s->ng = base + lay.ng;
    s->rho1 = base + lay.rho1;
    if (!stream3d_supported(s->p)) s->p.stream3d = 0;
  }
  if (!s->p.stream3d) s->p.totals = 0;
  s->totals_state = false;
  s->carry_ok = false;
  e = cudaMallocHost((void**)&s->host_result, 16 * sizeof(double));
  if (e != cudaSuccess) {
    if (s->owns) cudaFree(s->base);
    delete s;
    return fail(nullptr, LB_ECUDA, "pinned allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(s->fa, 0, lay.psi, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->result, 0, 16 * sizeof(double), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    lb_destroy(s);
    return fail(nullptr, LB_ECUDA, "initial clear failed: %s", cudaGetErrorString(e));
  }
  *out = s;
  return LB_OK;
}

lb_status lb_init_fields(lb_sim* s, const double* rho1, const double* rho2, const double* u, int on_device) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  if (!rho1 || !rho2) return fail(s, LB_EINVAL, "rho1 and rho2 are required");
  const long long N = s->p.N;
  const double *d1 = rho1, *d2 = rho2, *du = u;
  cudaError_t e;
  if (!on_device) {
    // Stage the host fields in the back buffer (it holds at least 4.5 N doubles).
    double* st = (double*)s->fb;
    const size_t need = (size_t)N * (u ? 5 : 2);
    if (need > staging_doubles(s)) return fail(s, LB_EUNSUPPORTED, "staging too small");
    e = cudaMemcpyAsync(st, rho1, N * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + N, rho2, N * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(st + 2 * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "field upload");
    d1 = st; d2 = st + N; du = u ? st + 2 * N : nullptr;
  }
  e = cudaMemsetAsync(s->p.seedw, 0, 2 * sizeof(unsigned), s->stream);  // the dither sequence restarts
  if (e == cudaSuccess) e = s->L->init(s->fa, d1, d2, du, s->p, s->stream);
  ++s->launches;
  s->carry_ok = false;
  s->totals_state = false;
  if (e != cudaSuccess) return cuda_fail(s, e, "init launch");
  if (!on_device) {
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  }
  s->step = 0;
  return refresh_rho_ref(s, d1, d2);
}

lb_status lb_step(lb_sim* s, long long nsteps) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  if (nsteps < 0) return fail(s, LB_EINVAL, "nsteps must be >= 0");
  if (s->in_ensemble) return fail(s, LB_EINVAL, "an ensemble member is stepped by lb_ensemble_step");
  for (long long t = 0; t < nsteps; ++t) {
    int nk = 0;
    cudaError_t e;
    s->p.parity = s->fa == s->buf_a ? 0 : 1;
    if (s->p.tma) {
      e = tma2d_step(s->maps, s->fa == s->buf_a ? 0 : 1, s->fa, s->fb, s->errflag, s->tile_counter, s->p,
                     s->stream);
      nk = 1;
    } else if (s->p.stream3d) {
      e = stream3d_step(s->fa, s->fb, s->psi, s->ng, s->rho1, s->totals_state ? 1 : 0, s->p, s->stream, &nk);
      if (e == cudaSuccess) s->totals_state = stream3d_stores_totals(s->p);
    } else if (s->p.carry3d) {
      if (!s->carry_ok) {  // a state no step produced: its densities from the populations
        e = carry3d_init(s->fa, s->carry, s->ring, s->ghost, s->p, s->stream);
        ++s->launches;
        if (e != cudaSuccess) return cuda_fail(s, e, "carry initialisation");
        s->carry_ok = true;
      }
      e = carry3d_step(s->maps, s->fa == s->buf_a ? 0 : 1, s->fa, s->fb, s->carry, s->ring, s->ghost, s->ng, s->hit,
                       s->errflag, s->p, s->stream, &nk);
    } else {
      e = s->L->step(s->fa, s->fb, s->psi, s->p, s->stream, &nk);
    }
    s->launches += nk;
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    std::swap(s->fa, s->fb);
    ++s->step;
  }
  return LB_OK;
}

lb_status lb_fields(lb_sim* s, double* rho1, double* rho2, double* psi, double* grad, double* frep,
                    int* hit, double* u, int on_device) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  const long long N = s->p.N;
  if (on_device) {
    FieldOut fo{rho1, rho2, psi, grad, frep, hit, u, nullptr};
    lb_status st = run_fields(s, fo);
    if (st != LB_OK) return st;
    return s->host_result[9] > 0 ? fail(s, LB_ENUMERIC, "non-finite or non-positive density at %.0f sites", s->host_result[9]) : LB_OK;
  }
  // Host outputs: one pass per requested field, staged in the back buffer.
  struct Req { void* host; int slot; size_t bytes; };
  Req reqs[7] = {{rho1, 0, N * sizeof(double)}, {rho2, 1, N * sizeof(double)}, {psi, 2, N * sizeof(double)},
                 {grad, 3, 3 * N * sizeof(double)}, {frep, 4, 3 * N * sizeof(double)}, {hit, 5, N * sizeof(int)},
                 {u, 6, 3 * N * sizeof(double)}};
  bool any = false;
  for (const Req& r : reqs) {
    if (!r.host) continue;
    any = true;
    FieldOut fo{};
    double* st = (double*)s->fb;
    switch (r.slot) {
      case 0: fo.rho1 = st; break;
      case 1: fo.rho2 = st; break;
      case 2: fo.psi = st; break;
      case 3: fo.grad = st; break;
      case 4: fo.frep = st; break;
      case 5: fo.hit = (int*)st; break;
      case 6: fo.u = st; break;
    }
    lb_status stt = run_fields(s, fo);
    if (stt != LB_OK) return stt;
    cudaError_t e = cudaMemcpy(r.host, st, r.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "field download");
  }
  if (!any) {
    FieldOut fo{};
    lb_status st = run_fields(s, fo);
    if (st != LB_OK) return st;
  }
  return s->host_result[9] > 0 ? fail(s, LB_ENUMERIC, "non-finite or non-positive density at %.0f sites", s->host_result[9]) : LB_OK;
}

lb_status lb_observables(lb_sim* s, lb_obs* out, double* psi_out, double* u_out, int on_device) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  if (!out) return fail(s, LB_EINVAL, "out is NULL");
  lb_status st = lb_fields(s, nullptr, nullptr, psi_out, nullptr, nullptr, nullptr, u_out, on_device);
  if (st != LB_OK && st != LB_ENUMERIC) return st;
  const double* r = s->host_result;
  out->mass[0] = r[0];
  out->mass[1] = r[1];
  out->momentum[0] = r[2];
  out->momentum[1] = r[3];
  out->momentum[2] = r[4];
  out->flow_rate = r[5] / (double)s->p.nx;
  out->flow_rate_disp = r[6] / (double)s->p.nx;
  out->step = s->step;
  out->n_interface = (long long)r[7];
  out->n_nci = (long long)r[8];
  out->n_bad = (long long)r[9];
  return st;
}

lb_status lb_get_populations(lb_sim* s, double* f, int on_device) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  if (!f) return fail(s, LB_EINVAL, "f is NULL");
  const int N = s->p.N, Q2 = 2 * s->Q;
  // a state in the total + recolouring form is read through the form's own reader
  auto decode = [&](double* out, int s0, int cnt) {
    return s->totals_state ? stream3d_form_decode(s->fa, out, s0, cnt, cnt, s->p, s->stream)
                           : s->L->decode(s->fa, out, s0, cnt, cnt, N, s->stream);
  };
  cudaError_t e;
  if (on_device) {
    e = decode(f, 0, N);
    ++s->launches;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LB_OK : cuda_fail(s, e, "population decode");
  }
  // Host: decode a range of sites at a time into the back buffer, then a strided copy.
  const long long chunk = staging_chunk(s);
  if (chunk < 1) return fail(s, LB_EUNSUPPORTED, "staging too small");
  for (long long s0 = 0; s0 < N; s0 += chunk) {
    const int cnt = (int)(N - s0 < chunk ? N - s0 : chunk);
    e = decode((double*)s->fb, (int)s0, cnt);
    ++s->launches;
    if (e != cudaSuccess) return cuda_fail(s, e, "population download (decode launch)");
    for (int q = 0; q < Q2 && e == cudaSuccess; ++q)
      e = cudaMemcpyAsync(f + (size_t)q * N + s0, (const double*)s->fb + (size_t)q * cnt,
                          (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population download (copy)");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population download (synchronize)");
  }
  return LB_OK;
}

lb_status lb_set_populations(lb_sim* s, const double* f, int on_device) {
  if (!s) return fail(nullptr, LB_EINVAL, "sim is NULL");
  if (!f) return fail(s, LB_EINVAL, "f is NULL");
  const int N = s->p.N, Q2 = 2 * s->Q;
  cudaError_t e = cudaMemsetAsync(s->p.seedw, 0, 2 * sizeof(unsigned), s->stream);  // the dither sequence restarts
  if (e != cudaSuccess) return cuda_fail(s, e, "seed reset");
  s->totals_state = false;
  if (on_device) {
    e = s->L->encode(f, s->fa, 0, N, N, N, s->stream);
    ++s->launches;
    s->carry_ok = false;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population encode");
  } else {
    const long long chunk = staging_chunk(s);
    if (chunk < 1) return fail(s, LB_EUNSUPPORTED, "staging too small");
    for (long long s0 = 0; s0 < N; s0 += chunk) {
      const int cnt = (int)(N - s0 < chunk ? N - s0 : chunk);
      e = cudaSuccess;
      for (int q = 0; q < Q2 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync((double*)s->fb + (size_t)q * cnt, f + (size_t)q * N + s0,
                            (size_t)cnt * sizeof(double), cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) return cuda_fail(s, e, "population upload (copy)");
      e = s->L->encode((const double*)s->fb, s->fa, (int)s0, cnt, cnt, N, s->stream);
      ++s->launches;
      s->carry_ok = false;
      if (e != cudaSuccess) return cuda_fail(s, e, "population upload (encode launch)");
      e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return cuda_fail(s, e, "population upload (synchronize)");
    }
  }
  s->step = 0;
  return refresh_rho_ref(s);
}

void lb_destroy(lb_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  if (s->owns && s->base) cudaFree(s->base);
  if (s->host_result) cudaFreeHost(s->host_result);
  delete s;
}

const char* lb_last_error(const lb_sim* s) { return s ? s->err : g_err; }

long long lb_kernel_launches(const lb_sim* s) { return s ? s->launches : 0; }

int lb_step_path(const lb_sim* s) {
  if (!s) return -1;
  if (s->cfg.lattice == LB_D3Q27)
    return s->p.carry3d ? LB_PATH_D3Q27_CARRY : (s->p.stream3d ? LB_PATH_D3Q27_STREAM : LB_PATH_D3Q27);
  return s->p.tma ? LB_PATH_TMA2D : LB_PATH_FUSED2D;
}

int lb_state_form(const lb_sim* s) {
  if (!s) return -1;
  return s->p.stream3d && stream3d_stores_totals(s->p) ? LB_STATE_TOTAL_RECOLOUR : LB_STATE_PAIRS;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Observables without any allocation (lb_observables_noalloc).
//
// Some callers cannot let a library allocate device memory: applications whose device
// memory is fully reserved by their own pool allocator (a raw cudaMalloc would fail or
// fragment it), and latency-critical loops in which a cudaMalloc, which may synchronise
// the device, is not acceptable. For them this entry point computes the same
// reductions as lb_observables from a population array they already own, using only
// the fixed scratch array below. Like lb_observables it copies its result to the host
// and synchronises the caller's stream before it returns, so it is not a call for a
// stream under graph capture.
//
// The scratch lives in this translation unit for the whole life of the process: every
// GPU that loads the library holds kNoAllocScratchBytes of it. All calls share it and
// it keeps the previous call's contents; every call overwrites all it reads (psi, the
// block partials and the result), so nothing needs clearing, but two calls that
// overlap on the GPU (different streams, or different host threads on one device)
// race on it and must not be issued.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so its device address is looked up with the
// device current, on every call: an address kept from an earlier call would be stale
// after the device's primary context was reset and recreated.
lb_status noalloc_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LB_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(nullptr, LB_ECUDA, "cudaGetSymbolAddress of the scratch array on device %d failed: %s", dev,
                cudaGetErrorString(e));
  }
  *out = p;
  return LB_OK;
}

}  // namespace

extern "C" lb_status lb_observables_noalloc(const lb_config* cfg, const void* f, lb_obs* out) {
  if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
  if (!f) return fail(nullptr, LB_EINVAL, "f is NULL");
  HostParams p{};
  Layout lay;
  long long nblocks;
  lb_status st = validate(cfg, &p, &lay, &nblocks);
  if (st != LB_OK) return st;
  if (cfg->precision == LB_FP16DEV)
    return fail(nullptr, LB_EUNSUPPORTED, "lb_observables_noalloc takes plain FP64 or FP32 populations");
  const size_t elem = cfg->precision == LB_FP64 ? sizeof(double) : sizeof(float);
  const size_t psi_off = 0;
  const size_t part_off = align256(psi_off + (size_t)p.N * elem);
  const size_t res_off = align256(part_off + (size_t)nblocks * kRedSlots * sizeof(double));
  const size_t need = res_off + 16 * sizeof(double);
  if (need > kNoAllocScratchBytes)
    return fail(nullptr, LB_EINVAL,
                "lb_observables_noalloc: a %d-site lattice needs %zu bytes of scratch, more than the "
                "%zu-byte static array (about %zu sites at this precision)",
                p.N, need, kNoAllocScratchBytes, kNoAllocScratchBytes / (elem + 1) - 1024);
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != LB_OK) return st;
  unsigned char* base = (unsigned char*)scratch;
  cudaStream_t stream = (cudaStream_t)cfg->stream;
  const Launchers* L = launchers_for(cfg);
  FieldOut fo{};
  fo.partials = (double*)(base + part_off);
  int nk = 0;
  cudaError_t e = L->fields(f, base + psi_off, p, fo, stream, &nk);
  if (e != cudaSuccess) return fail(nullptr, LB_ECUDA, "fields launch: %s", cudaGetErrorString(e));
  double* result = (double*)(base + res_off);
  e = reduce_partials(fo.partials, nblocks, result, stream);
  if (e != cudaSuccess) return fail(nullptr, LB_ECUDA, "reduce launch: %s", cudaGetErrorString(e));
  double r[kRedSlots];
  e = cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(nullptr, LB_ECUDA, "result copy: %s", cudaGetErrorString(e));
  out->mass[0] = r[0];
  out->mass[1] = r[1];
  out->momentum[0] = r[2];
  out->momentum[1] = r[3];
  out->momentum[2] = r[4];
  out->flow_rate = r[5] / (double)p.nx;
  out->flow_rate_disp = r[6] / (double)p.nx;
  out->step = 0;
  out->n_interface = (long long)r[7];
  out->n_nci = (long long)r[8];
  out->n_bad = (long long)r[9];
  return out->n_bad > 0 ? fail(nullptr, LB_ENUMERIC, "non-finite or non-positive density at %lld sites", out->n_bad)
                        : LB_OK;
}

// ---------------------------------------------------------------------------------
// Ensembles: many independent D2Q9 lattices (different sizes and parameters) stepped
// together by one batched launch per step, replayed from a CUDA graph.
// Candidates the autotuner times for the batched TMA kernel.
constexpr int kTmaPromo[4] = {0, 64, 128, 256};
constexpr int kTmaStatic[3] = {1, 2, 3};
constexpr int kTmaCand = 12;

struct lb_ensemble {
  int n;
  const Launchers* L;
  cudaStream_t stream;
  bool own_stream;
  std::vector<lb_sim*> members;
  void* base;              // one allocation holding every member's workspace
  std::vector<int> cls;    // members stepped by the one-pass batch kernel (FP64, nx % 4 != 0)
  std::vector<int> tma;    // members stepped by the batched TMA kernel (FP32 or FP16-dev, nx % 4 == 0)
  std::vector<unsigned char> host_members;  // BatchMember records of cls (host copy)
  void* d_members;         // device copy of the member records
  int* d_tile0;            // first tile of every cls member, cls.size() + 1 entries
  void* d_tma;             // TmaMember records of tma (device)
  int* d_tma_flags;        // batched TMA kernel: error word, two tile counters
  int tma_tiles, tma_smax;
  int spt;                 // tile shape: 32 x (8 spt) sites per block
  int total_tiles;
  int smax_max;
  int parity;              // 0: the current state is every member's buffer 0
  cudaGraphExec_t graph;   // two steps (parity 0 -> 1 -> 0), valid for the current spt
  bool graph_ok;
  long long launches;
  float tune_ms[2];        // last autotuner timings per step for spt = 2 and 4
  int tma_promo;           // batched TMA kernel: L2 promotion of its copies (bytes)
  int tma_nstatic;         // batched TMA kernel: static tiles per CTA before the counter
  float tma_ms[kTmaCand];  // last autotuner timings per step, [promotion][static tiles]
  char err[256];
};

namespace {

lb_status efail(lb_ensemble* e, lb_status st, const char* fmt, ...) {
  char* dst = e ? e->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return st;
}

lb_status ecuda(lb_ensemble* e, cudaError_t c, const char* what) {
  cudaGetLastError();
  return efail(e, LB_ECUDA, "%s: %s", what, cudaGetErrorString(c));
}

// Tile offsets for the current tile shape, uploaded to the device.
lb_status ens_layout(lb_ensemble* e) {
  const int nc = (int)e->cls.size();
  std::vector<int> t0(nc + 1, 0);
  for (int k = 0; k < nc; ++k) t0[k + 1] = t0[k] + e->L->batch_tiles(e->members[e->cls[k]]->p, e->spt);
  e->total_tiles = t0[nc];
  cudaError_t c = cudaMemcpyAsync(e->d_tile0, t0.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, e->stream);
  if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
  if (c != cudaSuccess) return ecuda(e, c, "tile table upload");
  if (e->graph_ok) { cudaGraphExecDestroy(e->graph); e->graph_ok = false; }
  return LB_OK;
}

// The one-pass batch kernel over the cls members (none: nothing launched).
cudaError_t ens_launch_cls(lb_ensemble* e, int parity, int* nk) {
  if (e->cls.empty()) return cudaSuccess;
  ++*nk;
  return e->L->batch_step(e->d_members, e->d_tile0, (int)e->cls.size(), e->total_tiles, parity, e->spt, e->smax_max,
                          e->members[0]->p.forcing == LB_FORCE_EDM_DISPERSED, e->stream);
}

// One step of every member: the batched TMA kernel over the tma members, the one-pass
// batch kernel over the others.
cudaError_t ens_launch_tma(lb_ensemble* e, int parity, int* nk) {
  if (e->tma.empty()) return cudaSuccess;
  ++*nk;
  return tma2d_batch_step(e->d_tma, (int)e->tma.size(), e->tma_tiles, parity, e->d_tma_flags, e->d_tma_flags + 1,
                          e->tma_smax, e->members[0]->p.forcing == LB_FORCE_EDM_DISPERSED, e->members[0]->p.half,
                          e->members[0]->p.num_sms, e->tma_nstatic, e->stream);
}

cudaError_t ens_launch(lb_ensemble* e, int parity, int* nk) {
  cudaError_t c = ens_launch_tma(e, parity, nk);
  if (c != cudaSuccess) return c;
  return ens_launch_cls(e, parity, nk);
}

// Encode every TMA member's tensor maps with L2 promotion `promo` (bytes) and upload
// the member table (records and tile index) to the device; waits for the copy.
cudaError_t ens_fill_tma(lb_ensemble* e, int promo) {
  const int nt = (int)e->tma.size();
  std::vector<unsigned char> ht(tma2d_table_bytes(nt));
  int tiles = 0;
  for (int k = 0; k < nt; ++k) {
    lb_sim* s = e->members[e->tma[k]];
    void* buf1 = s->fa == s->buf_a ? s->fb : s->fa;
    cudaError_t c = tma2d_prepare(&s->maps, s->buf_a, buf1, s->p, promo);
    if (c != cudaSuccess) return c;
    tiles += tma2d_member_fill(ht.data(), k, nt, s->maps, s->p, s->buf_a, buf1, tiles);
  }
  e->tma_tiles = tiles;
  e->tma_promo = promo;
  cudaError_t c = cudaMemcpyAsync(e->d_tma, ht.data(), ht.size(), cudaMemcpyHostToDevice, e->stream);
  if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
  return c;
}

}  // namespace

extern "C" {

lb_status lb_ensemble_create(const lb_config* cfgs, int n, lb_ensemble** out) {
  if (!out) return efail(nullptr, LB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || n < 1) return efail(nullptr, LB_EINVAL, "an ensemble needs n >= 1 configurations");
  for (int m = 0; m < n; ++m) {
    if (cfgs[m].lattice != LB_D2Q9) return efail(nullptr, LB_EUNSUPPORTED, "ensembles are D2Q9 only (member %d)", m);
    if (cfgs[m].precision != cfgs[0].precision)
      return efail(nullptr, LB_EINVAL, "all members need the same precision (member %d)", m);
    if (cfgs[m].forcing != cfgs[0].forcing)
      return efail(nullptr, LB_EINVAL, "all members need the same forcing scheme (member %d)", m);
  }
  std::vector<size_t> ws(n);
  size_t total = 0;
  for (int m = 0; m < n; ++m) {
    lb_config c = cfgs[m];
    c.workspace = nullptr;
    lb_status st = lb_workspace_size(&c, &ws[m]);
    if (st != LB_OK) return efail(nullptr, st, "member %d: %s", m, g_err);
    total += align256(ws[m]);
  }
  lb_ensemble* e = new (std::nothrow) lb_ensemble();
  if (!e) return efail(nullptr, LB_ENOMEM, "host allocation failed");
  e->n = n;
  e->L = launchers_for(&cfgs[0]);
  e->spt = 2;
  e->tma_promo = 128;
  e->tma_nstatic = 2;
  if (const char* v = std::getenv("LBNCI_TMA_CHOICE")) {  // "promotion:static", e.g. "64:3"
    int pr = -1, st = -1;
    const bool ok = std::sscanf(v, "%d:%d", &pr, &st) == 2 && (pr == 0 || pr == 64 || pr == 128 || pr == 256) &&
                    st >= 1 && st <= 3;
    if (!ok) { delete e; return efail(nullptr, LB_EINVAL, "LBNCI_TMA_CHOICE=%s: want <0|64|128|256>:<1|2|3>", v); }
    e->tma_promo = pr;
    e->tma_nstatic = st;
  }
  e->stream = (cudaStream_t)cfgs[0].stream;
  cudaError_t c = cudaSuccess;
  if (!e->stream) {  // graph capture needs a stream other than the legacy default one
    c = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (c != cudaSuccess) { delete e; return efail(nullptr, LB_ECUDA, "stream creation failed: %s", cudaGetErrorString(c)); }
    e->own_stream = true;
  }
  c = cudaMalloc(&e->base, total);
  if (c != cudaSuccess) {
    cudaGetLastError();
    lb_ensemble_destroy(e);
    return efail(nullptr, c == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "cudaMalloc of %zu bytes failed", total);
  }
  size_t off = 0;
  for (int m = 0; m < n; ++m) {
    lb_config cm = cfgs[m];
    cm.stream = e->stream;
    cm.workspace = (unsigned char*)e->base + off;
    cm.workspace_bytes = ws[m];
    off += align256(ws[m]);
    lb_sim* s = nullptr;
    lb_status st = lb_create(&cm, &s);
    if (st != LB_OK) { lb_ensemble_destroy(e); return efail(nullptr, st, "member %d: %s", m, g_err); }
    s->in_ensemble = true;
    e->members.push_back(s);
    e->smax_max = std::max(e->smax_max, s->p.smax);
  }
  for (int m = 0; m < n; ++m) (e->members[m]->p.tma ? e->tma : e->cls).push_back(m);
  const size_t rec = e->L->batch_member_bytes;
  const int nc = (int)e->cls.size(), nt = (int)e->tma.size();
  e->host_members.resize(rec * (nc > 0 ? nc : 1));
  for (int k = 0; k < nc; ++k) {
    lb_sim* s = e->members[e->cls[k]];
    e->L->batch_fill(e->host_members.data() + rec * k, s->p, s->fa, s->fb);
  }
  c = cudaMalloc(&e->d_members, rec * (nc > 0 ? nc : 1));
  if (c == cudaSuccess) c = cudaMalloc((void**)&e->d_tile0, sizeof(int) * (nc + 1));
  if (c == cudaSuccess)
    c = cudaMemcpyAsync(e->d_members, e->host_members.data(), rec * (nc > 0 ? nc : 1), cudaMemcpyHostToDevice,
                        e->stream);
  if (c == cudaSuccess && nt > 0) {
    for (int k = 0; k < nt; ++k) e->tma_smax = std::max(e->tma_smax, e->members[e->tma[k]]->p.smax);
    c = cudaMalloc(&e->d_tma, tma2d_table_bytes(nt));
    if (c == cudaSuccess) c = cudaMalloc((void**)&e->d_tma_flags, 4 * sizeof(int));
    if (c == cudaSuccess) c = cudaMemsetAsync(e->d_tma_flags, 0, 4 * sizeof(int), e->stream);
    if (c == cudaSuccess) c = ens_fill_tma(e, e->tma_promo);
    for (int k = 0; k < nt; ++k) e->members[e->tma[k]]->ens_flag = e->d_tma_flags;
  }
  if (c != cudaSuccess) {
    cudaGetLastError();
    lb_ensemble_destroy(e);
    return efail(nullptr, LB_ECUDA, "member table: %s", cudaGetErrorString(c));
  }
  lb_status st = ens_layout(e);
  if (st != LB_OK) { lb_ensemble_destroy(e); return efail(nullptr, st, "%s", "tile table upload failed"); }
  *out = e;
  return LB_OK;
}

lb_status lb_ensemble_member(lb_ensemble* e, int m, lb_sim** out) {
  if (!e || !out) return efail(e, LB_EINVAL, "NULL argument");
  if (m < 0 || m >= e->n) return efail(e, LB_EINVAL, "member %d out of range [0, %d)", m, e->n);
  *out = e->members[m];
  return LB_OK;
}

lb_status lb_ensemble_step(lb_ensemble* e, long long nsteps) {
  if (!e) return efail(nullptr, LB_EINVAL, "ensemble is NULL");
  if (nsteps < 0) return efail(e, LB_EINVAL, "nsteps must be >= 0");
  cudaError_t c;
  long long left = nsteps;
  int nk = 0;  // kernels of one step
  if (left > 0 && e->parity == 1) {  // back to parity 0, where the two-step graph starts
    c = ens_launch(e, 1, &nk);
    if (c != cudaSuccess) return ecuda(e, c, "ensemble step launch");
    e->launches += nk;
    e->parity = 0;
    --left;
  }
  if (left >= 2 && !e->graph_ok) {
    cudaGraph_t g;
    c = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
    if (c == cudaSuccess) {
      int nk2 = 0;
      cudaError_t c1 = ens_launch(e, 0, &nk2);
      cudaError_t c2 = ens_launch(e, 1, &nk2);
      c = cudaStreamEndCapture(e->stream, &g);
      if (c == cudaSuccess && (c1 != cudaSuccess || c2 != cudaSuccess)) c = c1 != cudaSuccess ? c1 : c2;
      if (c == cudaSuccess) {
        c = cudaGraphInstantiate(&e->graph, g, 0);
        cudaGraphDestroy(g);
      }
    }
    if (c != cudaSuccess) return ecuda(e, c, "ensemble graph capture");
    e->graph_ok = true;
  }
  const int per_step = (e->tma.empty() ? 0 : 1) + (e->cls.empty() ? 0 : 1);
  for (; left >= 2; left -= 2) {
    c = cudaGraphLaunch(e->graph, e->stream);
    if (c != cudaSuccess) return ecuda(e, c, "ensemble graph launch");
    e->launches += 2 * per_step;
  }
  if (left == 1) {
    nk = 0;
    c = ens_launch(e, 0, &nk);
    if (c != cudaSuccess) return ecuda(e, c, "ensemble step launch");
    e->launches += nk;
    e->parity = 1;
  }
  // the members' current state buffer follows the parity
  const bool odd = (nsteps & 1) != 0;
  for (lb_sim* s : e->members) {
    if (odd) std::swap(s->fa, s->fb);
    s->step += nsteps;
  }
  return LB_OK;
}

namespace {

// Time the batched TMA kernel for every (L2 promotion, static tiles) candidate on the
// current state and keep the fastest. Each launch reads the state and writes the back
// buffers only; its tile counter is zeroed before it, outside the timed interval.
cudaError_t tune_tma(lb_ensemble* e, cudaEvent_t t0, cudaEvent_t t1) {
  const int nstatic0 = e->tma_nstatic;
  int best_p = e->tma_promo, best_s = e->tma_nstatic;
  float best_ms = 1e30f;
  cudaError_t c = cudaSuccess;
  int* ctr = e->d_tma_flags + 1 + e->parity;
  for (int ip = 0; ip < 4 && c == cudaSuccess; ++ip) {
    c = ens_fill_tma(e, kTmaPromo[ip]);
    for (int is = 0; is < 3 && c == cudaSuccess; ++is) {
      e->tma_nstatic = kTmaStatic[is];
      float total = 0.f;
      for (int r = 0; r < 6 && c == cudaSuccess; ++r) {  // one warm-up launch, five timed
        int nk = 0;
        c = cudaMemsetAsync(ctr, 0, sizeof(int), e->stream);
        if (c == cudaSuccess) c = cudaEventRecord(t0, e->stream);
        if (c == cudaSuccess) c = ens_launch_tma(e, e->parity, &nk);
        if (c == cudaSuccess) c = cudaEventRecord(t1, e->stream);
        if (c == cudaSuccess) c = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (c == cudaSuccess) c = cudaEventElapsedTime(&ms, t0, t1);
        if (r > 0) total += ms;
        e->launches += nk;
      }
      e->tma_ms[ip * 3 + is] = total / 5.f;
      if (c == cudaSuccess && total / 5.f < best_ms) {
        best_ms = total / 5.f;
        best_p = kTmaPromo[ip];
        best_s = kTmaStatic[is];
      }
    }
  }
  if (c != cudaSuccess) { e->tma_nstatic = nstatic0; return c; }
  e->tma_nstatic = best_s;
  c = ens_fill_tma(e, best_p);
  if (c == cudaSuccess) c = cudaMemsetAsync(e->d_tma_flags + 1, 0, 2 * sizeof(int), e->stream);
  if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
  return c;
}

}  // namespace

lb_status lb_ensemble_tune(lb_ensemble* e, int* spt_out) {
  if (!e) return efail(nullptr, LB_EINVAL, "ensemble is NULL");
  // Time each candidate on the current state, writing only the back buffers (the
  // state itself is unchanged), and keep the fastest.
  const int shapes[2] = {2, 4};
  cudaEvent_t t0, t1;
  cudaError_t c = cudaEventCreate(&t0);
  if (c == cudaSuccess) c = cudaEventCreate(&t1);
  if (c != cudaSuccess) return ecuda(e, c, "event creation");
  int best = e->spt;
  float best_ms = 1e30f;
  if (e->graph_ok) { cudaGraphExecDestroy(e->graph); e->graph_ok = false; }  // the choices are launch arguments
  if (!e->tma.empty()) {
    c = tune_tma(e, t0, t1);
    if (c != cudaSuccess) {
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      return ecuda(e, c, "autotune of the TMA kernel");
    }
  }
  if (e->cls.empty()) {  // every member runs the TMA kernel: no tile shape to choose
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    e->tune_ms[0] = e->tune_ms[1] = 0.f;
    if (spt_out) *spt_out = e->spt;
    return LB_OK;
  }
  for (int k = 0; k < 2 && c == cudaSuccess; ++k) {
    e->spt = shapes[k];
    lb_status st = ens_layout(e);
    if (st != LB_OK) { cudaEventDestroy(t0); cudaEventDestroy(t1); return st; }
    int nk = 0;
    c = ens_launch_cls(e, e->parity, &nk);  // warm-up
    if (c == cudaSuccess) c = cudaEventRecord(t0, e->stream);
    for (int r = 0; r < 5 && c == cudaSuccess; ++r) c = ens_launch_cls(e, e->parity, &nk);
    if (c == cudaSuccess) c = cudaEventRecord(t1, e->stream);
    if (c == cudaSuccess) c = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (c == cudaSuccess) c = cudaEventElapsedTime(&ms, t0, t1);
    e->launches += 6;
    e->tune_ms[k] = ms / 5.f;
    if (c == cudaSuccess && ms < best_ms) { best_ms = ms; best = shapes[k]; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (c != cudaSuccess) return ecuda(e, c, "autotune");
  e->spt = best;
  lb_status st = ens_layout(e);
  if (st != LB_OK) return st;
  if (spt_out) *spt_out = best;
  return LB_OK;
}

lb_status lb_ensemble_tune_times(const lb_ensemble* e, float* ms2, float* ms4) {
  if (!e) return efail(nullptr, LB_EINVAL, "ensemble is NULL");
  if (ms2) *ms2 = e->tune_ms[0];
  if (ms4) *ms4 = e->tune_ms[1];
  return LB_OK;
}

lb_status lb_ensemble_tma_choice(const lb_ensemble* e, int* l2_promotion_bytes, int* static_tiles, float* ms12) {
  if (!e) return efail(nullptr, LB_EINVAL, "ensemble is NULL");
  if (e->tma.empty()) return efail(const_cast<lb_ensemble*>(e), LB_EUNSUPPORTED, "no member runs the TMA kernel");
  if (l2_promotion_bytes) *l2_promotion_bytes = e->tma_promo;
  if (static_tiles) *static_tiles = e->tma_nstatic;
  if (ms12)
    for (int k = 0; k < kTmaCand; ++k) ms12[k] = e->tma_ms[k];
  return LB_OK;
}

long long lb_ensemble_launches(const lb_ensemble* e) { return e ? e->launches : 0; }

const char* lb_ensemble_last_error(const lb_ensemble* e) { return e ? e->err : g_err; }

void lb_ensemble_destroy(lb_ensemble* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->graph_ok) cudaGraphExecDestroy(e->graph);
  for (lb_sim* s : e->members) lb_destroy(s);
  if (e->d_members) cudaFree(e->d_members);
  if (e->d_tma) cudaFree(e->d_tma);
  if (e->d_tma_flags) cudaFree(e->d_tma_flags);
  if (e->d_tile0) cudaFree(e->d_tile0);
  if (e->base) cudaFree(e->base);
  if (e->own_stream) cudaStreamDestroy(e->stream);
  delete e;
}

}  // extern "C"
