// lb_carry3d.cu -- launchers of the D3Q27 steps of lb_carry3d.cuh for FP32 and
// FP16-deviation storage: the single-read step (with its tensor maps) and the streaming
// step.
#include <cmath>
#include <cstring>

#include "lb_carry3d.cuh"
#include "lb_launch.h"

namespace lbnci {
namespace {

StepT<float> to_step3(const HostParams& h) {
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
  // A_h(h): A for h <= h_min, A (h_min/h)^3 for h_min < h <= h_max, 0 beyond (Eq. near_c)
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

CarryGrid grid_of(const HostParams& h) {
  CarryGrid g;
  g.nx = h.nx; g.ny = h.ny; g.nz = h.nz;
  g.ncx = h.nx / kC3X; g.ncy = h.ny / kC3Y;
  g.wall_y = h.wall_y; g.wall_z = h.wall_z;
  g.zseg = h.c3_zseg > 0 ? (h.c3_zseg < h.nz ? h.c3_zseg : h.nz) : h.nz;
  g.nseg = (h.nz + g.zseg - 1) / g.zseg;
  return g;
}

// FP32 population planes of one state as a 5-D tensor (x, y, z, d, e) with population
// plane d + 3 e (d = digit of c_x, e = class + 9 k); box 40 x 8 x 1 x 3 x 1: one class
// window. FP16-dev half2 deviation planes as a 4-D tensor (x, y, z, plane); box
// 40 x 8 x 1 x 3.
bool encode_planes(CUtensorMap* m, const void* base, const HostParams& h, bool half) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  if (half) {
    const cuuint64_t dims[4] = {(cuuint64_t)h.nx, (cuuint64_t)h.ny, (cuuint64_t)h.nz, 27};
    const cuuint64_t strides[3] = {(cuuint64_t)h.nx * 4, (cuuint64_t)h.nx * h.ny * 4, (cuuint64_t)h.N * 4};
    const cuuint32_t box[4] = {kW3X, kW3Y, 1, 3};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const cuuint64_t dims[5] = {(cuuint64_t)h.nx, (cuuint64_t)h.ny, (cuuint64_t)h.nz, 3, 18};
  const cuuint64_t strides[4] = {(cuuint64_t)h.nx * 4, (cuuint64_t)h.nx * h.ny * 4, (cuuint64_t)h.N * 4,
                                 (cuuint64_t)h.N * 12};
  const cuuint32_t box[5] = {kW3X, kW3Y, 1, 3, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-site (n, |grad psi|) as a 3-D tensor (4 nx floats, y, z), box 128 x 8 x 1 (a column
// plane); NCI distances as a 3-D tensor of bytes (nx, y, z), box 32 x 8 x 1.
bool encode_ng(CUtensorMap* m, const void* base, const HostParams& h) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)h.nx * 4, (cuuint64_t)h.ny, (cuuint64_t)h.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)h.nx * 16, (cuuint64_t)h.nx * h.ny * 16};
  const cuuint32_t box[3] = {4 * kC3X, kC3Y, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool encode_hit(CUtensorMap* m, const void* base, const HostParams& h) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)h.nx, (cuuint64_t)h.ny, (cuuint64_t)h.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)h.nx, (cuuint64_t)h.nx * h.ny};
  const cuuint32_t box[3] = {kC3X, kC3Y, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Reference densities of an FP16-dev state as a 3-D tensor (2 nx floats, y, z), box 80 x 10 x 1.
bool encode_rho3(CUtensorMap* m, const void* base, const HostParams& h) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)h.nx * 2, (cuuint64_t)h.ny, (cuuint64_t)h.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)h.nx * 8, (cuuint64_t)h.nx * h.ny * 8};
  const cuuint32_t box[3] = {2 * kR3X, kR3Y, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename ST, bool EDM>
cudaError_t launch_c3(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mng, const CUtensorMap& mhit,
                      const void* fa, void* fb, const StepT<float>& p, const Carry3dArgs& a, int num_sms,
                      cudaStream_t s) {
  static SmemAllowance configured;
  constexpr int smem = C3Smem<ST>::kBytes;
  cudaError_t e = allow_smem(carry3d_kernel<ST, EDM>, smem, configured);
  if (e != cudaSuccess) return e;
  // two persistent CTAs per SM take the items segment by segment
  const int slots = 2 * num_sms;
  const int grid = a.nitems < slots ? a.nitems : slots;
  carry3d_kernel<ST, EDM><<<grid, kC3T, smem, s>>>(ma, mb, mng, mhit, ST::reader(fa, (unsigned)p.N),
                                                    ST::writer(fb, (unsigned)p.N), p, a);
  return cudaGetLastError();
}

template <typename ST>
cudaError_t launch_c3_any(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mng,
                          const CUtensorMap& mhit, const void* fa, void* fb, const StepT<float>& p,
                          const Carry3dArgs& a, int num_sms, cudaStream_t s) {
  return p.edm ? launch_c3<ST, true>(ma, mb, mng, mhit, fa, fb, p, a, num_sms, s)
               : launch_c3<ST, false>(ma, mb, mng, mhit, fa, fb, p, a, num_sms, s);
}

}  // namespace

bool carry3d_supported(const HostParams& h) {
  return h.nx % kC3X == 0 && h.ny % kC3Y == 0 && (h.wall_z || h.nz >= 2) && encode_fn() != nullptr;
}

size_t carry3d_ring_bytes(const HostParams& h) {
  return (size_t)(h.nx / kC3X) * (h.ny / kC3Y) * h.nz * kRing * sizeof(float2);
}

size_t carry3d_ghost_bytes(const HostParams& h) {
  const CarryGrid g = grid_of(h);
  return (size_t)g.ncx * g.ncy * g.nseg * 2 * kGhostCells * sizeof(float2);
}

cudaError_t carry3d_prepare(TmaMaps* m, const void* fa, const void* fb, const void* ng, const void* hit,
                            const HostParams& h) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(m->bytes);
  std::memset(m->bytes, 0, sizeof(m->bytes));
  if (!encode_ng(&maps[4], ng, h) || !encode_hit(&maps[5], hit, h)) return cudaErrorInvalidValue;
  if (!h.half)
    return encode_planes(&maps[0], fa, h, false) && encode_planes(&maps[1], fb, h, false) ? cudaSuccess
                                                                                            : cudaErrorInvalidValue;
  const size_t ro = HalfDev<1>::rho_offset((size_t)h.N);
  const bool ok = encode_planes(&maps[0], fa, h, true) && encode_planes(&maps[1], fb, h, true) &&
                  encode_rho3(&maps[2], (const char*)fa + ro, h) && encode_rho3(&maps[3], (const char*)fb + ro, h);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t carry3d_init(const void* f, void* carry, void* ring, void* ghost, const HostParams& h, cudaStream_t s) {
  const StepT<float> p = to_step3(h);
  const unsigned blocks = (unsigned)((p.N + 255) / 256);
  if (h.half)
    carry_init_kernel<HalfDev<1>><<<blocks, 256, 0, s>>>(HalfDev<1>::reader(f, (unsigned)p.N), (float2*)carry, p);
  else
    carry_init_kernel<Plain<1, float>><<<blocks, 256, 0, s>>>(Plain<1, float>::reader(f, (unsigned)p.N),
                                                              (float2*)carry, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ring, 0, carry3d_ring_bytes(h), s);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(ghost, 0, carry3d_ghost_bytes(h), s);
}

cudaError_t carry3d_step(const TmaMaps& m, int from, const void* fa, void* fb, void* carry, void* ring, void* ghost,
                         void* ng, void* hit, int* err, const HostParams& h, cudaStream_t s, int* nk) {
  const StepT<float> p = to_step3(h);
  const CarryGrid g = grid_of(h);
  const int ncol = g.ncx * g.ncy;
  *nk = 0;
  interface3d_kernel<<<dim3((unsigned)ncol, (unsigned)((g.nz + kI3Z - 1) / kI3Z)), kC3T, 0, s>>>(
      (const float2*)carry, (const float2*)ring, (const float2*)ghost, (float4*)ng, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nk;
  if (p.smax > 0) {
    nci3d_kernel<<<dim3((unsigned)(g.nx / 32), (unsigned)(g.ny / 8), (unsigned)g.nz), dim3(32, 8), 0, s>>>(
        (const float4*)ng, (unsigned char*)hit, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*nk;
  } else {  // no near-contact force: every distance is 0
    e = cudaMemsetAsync(hit, 0, (size_t)p.N, s);
    if (e != cudaSuccess) return e;
  }
  Carry3dArgs a;
  a.ng = (const float4*)ng;
  a.hit = (const unsigned char*)hit;
  a.carry = (float2*)carry;
  a.ring = (float2*)ring;
  a.ghost = (float2*)ghost;
  a.err = err;
  a.ncx = g.ncx;
  a.ncol = ncol;
  a.zseg = g.zseg;
  a.nseg = g.nseg;
  a.nitems = ncol * g.nseg;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(m.bytes);
  const CUtensorMap& ma = maps[from];
  const CUtensorMap& mb = maps[h.half ? 2 + from : from];
  e = h.half ? launch_c3_any<HalfDev<1>>(ma, mb, maps[4], maps[5], fa, fb, p, a, h.num_sms, s)
             : launch_c3_any<Plain<1, float>>(ma, mb, maps[4], maps[5], fa, fb, p, a, h.num_sms, s);
  if (e == cudaSuccess) ++*nk;
  return e;
}

namespace {
template <typename ST>
cudaError_t launch_collide3d(const void* fa, void* fb, const float4* ng, const StepT<float>& p, dim3 grid,
                             cudaStream_t s) {
  if (p.edm)
    collide3d_kernel<ST, true><<<grid, dim3(32, 8), 0, s>>>(ST::reader(fa, (unsigned)p.N),
                                                            ST::writer(fb, (unsigned)p.N), ng, p);
  else
    collide3d_kernel<ST, false><<<grid, dim3(32, 8), 0, s>>>(ST::reader(fa, (unsigned)p.N),
                                                             ST::writer(fb, (unsigned)p.N), ng, p);
  return cudaGetLastError();
}
}  // namespace

bool stream3d_supported(const HostParams& h) { return h.nx % 32 == 0 && h.ny % 8 == 0; }

bool stream3d_stores_totals(const HostParams& h) { return h.totals && h.forcing != 1; }

namespace {
// rho_0/216 rounded to a multiple of 2^-24: the unit of the FP16 totals' reference (216 w_i) r
float rho_unit(const HostParams& h) {
  return float(std::rint(double(h.rho_ref) / 216.0 * 16777216.0) / 16777216.0);
}
}  // namespace

namespace {
// the collision storing the total + recolouring form of the precision
template <typename RD, bool TOTALS, typename WR>
cudaError_t launch_collide3t(RD rd, WR wr, const void* rho12, const void* ng, const StepT<float>& p, dim3 grid,
                             cudaStream_t s) {
  collide3t_kernel<RD, TOTALS, WR><<<grid, dim3(32, 8), 0, s>>>(rd, wr, (const float2*)rho12, (const float4*)ng, p);
  return cudaGetLastError();
}
}  // namespace

cudaError_t stream3d_step(const void* fa, void* fb, void* psi, void* ng, void* rho12, int totals_in,
                          const HostParams& h, cudaStream_t s, int* nk) {
  const StepT<float> p = to_step3(h);
  *nk = 0;
  const bool totals_out = stream3d_stores_totals(h);
  if (totals_in && !totals_out) return cudaErrorInvalidValue;  // no step reads that form into pairs
  const dim3 grid((unsigned)(h.nx / 32), (unsigned)(h.ny / 8), (unsigned)h.nz);
  const unsigned N = (unsigned)p.N;
  const float r0 = rho_unit(h);
  float2* r12 = totals_out ? (float2*)rho12 : nullptr;
  // 32 x 8 blocks where the sources carry per-site data that repeats within the block
  // (FP16-dev pairs: the reference densities, 0.85 ms per duct step against 0.95 ms with
  // blocks of 256 consecutive sites; the total forms: the recolouring coefficients, about
  // two thirds of whose sectors hit L1); the two-population FP32 state has none and keeps
  // the flat kernel (the same time)
  if (totals_in && h.half) {
    moments3_kernel<TotalRecolHalf><<<grid, dim3(32, 8), 0, s>>>(TotalRecolHalf::reader(fa, N, r0), (float*)psi,
                                                                 r12, p);
  } else if (totals_in) {
    moments3_kernel<TotalRecol><<<grid, dim3(32, 8), 0, s>>>(TotalRecol::reader(fa, N), (float*)psi, r12, p);
  } else if (h.half) {
    moments3_kernel<HalfDev<1>><<<grid, dim3(32, 8), 0, s>>>(HalfDev<1>::reader(fa, N), (float*)psi, r12, p);
  } else if (totals_out) {
    moments3_kernel<Plain<1, float>><<<grid, dim3(32, 8), 0, s>>>(Plain<1, float>::reader(fa, N), (float*)psi, r12,
                                                                  p);
  } else {
    const unsigned nb = (unsigned)((p.N + 255) / 256);
    moments_kernel<1, Plain<1, float>><<<nb, 256, 0, s>>>(Plain<1, float>::reader(fa, N), (float*)psi, p);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nk;
  const dim3 gridn((unsigned)(h.nx / 32), (unsigned)(h.ny / 8), (unsigned)((h.nz + kN3Z - 1) / kN3Z));
  normals3d_kernel<<<gridn, dim3(32, 8), 0, s>>>((const float*)psi, (float4*)ng, p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nk;
  if (totals_out && h.half) {
    const TotalRecolHalf::Writer wr = TotalRecolHalf::writer(fb, N, r0);
    e = totals_in ? launch_collide3t<TotalRecolHalf::Devs, true>(TotalRecolHalf::devs(fa, N), wr, rho12, ng, p,
                                                                 grid, s)
                  : launch_collide3t<HalfDev<1>::Reader, false>(HalfDev<1>::reader(fa, N), wr, rho12, ng, p, grid, s);
  } else if (totals_out) {
    const TotalRecol::Writer wr = TotalRecol::writer(fb, N);
    e = totals_in ? launch_collide3t<TotalRecol::Totals, true>(TotalRecol::totals(fa, N), wr, rho12, ng, p, grid, s)
                  : launch_collide3t<Plain<1, float>::Reader, false>(Plain<1, float>::reader(fa, N), wr, rho12, ng, p,
                                                                      grid, s);
  } else {
    e = h.half ? launch_collide3d<HalfDev<1>>(fa, fb, (const float4*)ng, p, grid, s)
               : launch_collide3d<Plain<1, float>>(fa, fb, (const float4*)ng, p, grid, s);
  }
  if (e == cudaSuccess) ++*nk;
  return e;
}

namespace {
// The fields kernel (and its moments pass) on a state in a total + recolouring form, read
// through the form's two-population reader; the same grid as the other precisions' fields
// launches (tiled_blocks), so the host reduces the same partials.
template <typename FORM>
cudaError_t form_fields(typename FORM::Reader rd, void* psi, const HostParams& h, const FieldOut& fo, cudaStream_t s,
                        int* nk) {
  const StepT<float> p = to_step3(h);
  moments_kernel<1, FORM><<<(unsigned)((p.N + 255) / 256), 256, 0, s>>>(rd, (float*)psi, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static SmemAllowance configured;
  const size_t sm = tiled_smem_bytes<1, float>(p.smax);
  e = allow_smem(tiled_kernel<1, FORM, true, false>, sm, configured);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((h.nx + Tile<1>::X - 1) / Tile<1>::X), (unsigned)((h.ny + Tile<1>::Y - 1) / Tile<1>::Y),
                  (unsigned)((h.nz + Tile<1>::Z - 1) / Tile<1>::Z));
  tiled_kernel<1, FORM, true, false><<<grid, dim3(Tile<1>::X, Tile<1>::Y, Tile<1>::Z), sm, s>>>(
      rd, typename FORM::Writer{}, (const float*)psi, p, fo);
  *nk = 2;
  return cudaGetLastError();
}
}  // namespace

cudaError_t stream3d_form_fields(const void* f, void* psi, const HostParams& h, const FieldOut& fo, cudaStream_t s,
                                 int* nk) {
  if (h.half) return form_fields<TotalRecolHalf>(TotalRecolHalf::reader(f, (unsigned)h.N, rho_unit(h)), psi, h, fo, s, nk);
  return form_fields<TotalRecol>(TotalRecol::reader(f, (unsigned)h.N), psi, h, fo, s, nk);
}

cudaError_t stream3d_form_decode(const void* f, double* out, int s0, int count, long long pitch, const HostParams& h,
                                 cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned nb = (unsigned)((count + 255) / 256);
  if (h.half)
    decode_kernel<1, TotalRecolHalf><<<nb, 256, 0, s>>>(TotalRecolHalf::reader(f, (unsigned)h.N, rho_unit(h)), out, s0,
                                                        count, pitch);
  else
    decode_kernel<1, TotalRecol><<<nb, 256, 0, s>>>(TotalRecol::reader(f, (unsigned)h.N), out, s0, count, pitch);
  return cudaGetLastError();
}

size_t stream3d_totals_bytes(size_t N, int half) { return half ? TotalRecolHalf::bytes(N) : TotalRecol::bytes(N); }

}  // namespace lbnci
