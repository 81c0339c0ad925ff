// unet_tc.cuh -- the U-Net's 3x3 convolution (forward and data gradient) on the
// fifth-generation tensor cores: tcgen05.mma with the accumulator in tensor memory.
//
// Implicit GEMM as in conv3x3_kernel (unet_kernels.cuh): D[m][n] = sum_k A[m][k] B[n][k]
// with m a pixel (128 per CTA), n an output channel (BN = 32, 64 or 128 per CTA) and
// k = (tap, input channel) in chunks of BK = 32 channels of one tap. Per chunk, all 256
// threads copy the A rows (the tap-shifted pixels' BK channels, zero rows beyond the first
// and last image row, periodic columns) and the B rows (the weights) with cp.async into a
// ring of four stages, in the tensor cores' K-major layout without swizzle: 8 x 16-byte
// core matrices of 128 contiguous bytes, core matrices adjacent along K 128 bytes apart
// (leading byte offset), 8-row groups BK x 16 bytes apart (stride byte offset). One thread
// issues BK/16 tcgen05.mma (K = 16 each) per chunk, accumulating in BN columns of tensor
// memory, and commits them to the stage's mbarrier; chunks are copied two stages ahead of
// the MMAs, so a stage is refilled once the mbarrier says the MMAs of two chunks back,
// which read it, are done. The epilogue reads the accumulator with tcgen05.ld (warp w:
// lanes 32 (w % 4) .., i.e. pixels 32 (w % 4) .., columns of half w / 4), adds the bias,
// applies ReLU or the ReLU-derivative mask and stores BF16.
//
// Every mbarrier wait is bounded (about a second of %globaltimer); on expiry the kernel
// sets its error word, waits (bounded) for the MMAs it issued, releases its tensor memory
// and returns without writing the output.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "lb_tma.cuh"
#include "unet_kernels.cuh"

namespace lbu {
namespace tc {

// Shared-memory matrix descriptor: K-major, no swizzle (layout type 0), version 1 (bits
// 46-47), start address, leading and stride byte offsets in 16-byte units.
__device__ __forceinline__ unsigned long long smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits
// 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(unsigned* s_addr, unsigned ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_addr)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tensor memory) = A B^T (+ D when accumulate)
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive 32-bit columns of this thread's lane (shape 32x32b: lane = warp's base + lane id)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kBM = 128;
template <int BN, int BK>
struct Smem {
  static constexpr int kStages = 4;                           // ring of chunk stages
  static constexpr int kAhead = kStages - 2;                  // chunks copied ahead of the MMAs
  static constexpr int kABytes = kBM * BK * 2;
  static constexpr int kBBytes = BN * BK * 2;
  static constexpr int kStage = kABytes + kBBytes;
  static constexpr int kOffBar = kStages * kStage;            // kStages mbarriers
  static constexpr int kBytes = kOffBar + 8 * kStages + 16;   // + tensor-memory address, padding
  static constexpr unsigned kCols = BN < 32 ? 32u : (unsigned)BN;
  static constexpr unsigned kSBO = BK * 16;                   // bytes between 8-row groups
};

// Byte offset of 16-byte chunk v (channels 8 v .. 8 v + 7) of row r in the K-major,
// non-swizzled layout of a BK-channel chunk.
template <int BK>
__device__ __forceinline__ unsigned core_off(int r, int v) {
  return (unsigned)((r >> 3) * (BK * 16) + v * 128 + (r & 7) * 16);
}

}  // namespace tc

constexpr int kTcThreads = 256;

template <int BN, int BK>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_kernel(ConvFwd a, int* err) {
  using S = tc::Smem<BN, BK>;
  constexpr int BM = tc::kBM, ST = S::kStages, AH = S::kAhead, NTH = kTcThreads;
  constexpr int NV = BK / 8;  // 16-byte chunks per row
  constexpr unsigned IDESC = tc::idesc_bf16(BM, BN);
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + S::kOffBar);
  unsigned* s_tmem = reinterpret_cast<unsigned*>(sm + S::kOffBar + 8 * ST);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = a.B * a.H * a.W;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int cpt = a.Cin / BK, nk = 9 * cpt;
  const int Hi = a.H >> a.up, Wi = a.W >> a.up;
  // A copies: thread tid takes 16-byte chunk v of rows r0 + RS j
  constexpr int TPR = NV, RS = NTH / TPR, NJ = BM / RS;
  const int v = tid % TPR, r0 = tid / TPR;
  int pb[NJ], py[NJ], px[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int m = m0 + r0 + RS * j;
    if (m < M) {
      px[j] = m % a.W;
      const int t = m / a.W;
      py[j] = t % a.H;
      pb[j] = t / a.H;
    } else {
      pb[j] = -1;
      py[j] = 0;
      px[j] = 0;
    }
  }
  auto stage_a = [&](int s) { return sm + s * S::kStage; };
  auto stage_b = [&](int s) { return sm + s * S::kStage + S::kABytes; };
  auto load = [&](int s, int kc) {
    const int tap = kc / cpt, c0 = (kc - tap * cpt) * BK;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    unsigned char* sa = stage_a(s);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int yy = py[j] + dy, xx = wrap(px[j] + dx, a.W);
      const bool ok = pb[j] >= 0 && yy >= 0 && yy < a.H;
      const bf16* src = a.x;
      if (ok) src = a.x + ((size_t)(pb[j] * Hi + (yy >> a.up)) * Wi + (xx >> a.up)) * a.xs + c0 + v * 8;
      cp_async16(sa + tc::core_off<BK>(r0 + RS * j, v), src, ok);
    }
    unsigned char* sb = stage_b(s);
#pragma unroll
    for (int i = tid; i < BN * NV; i += NTH) {
      const int n = i / NV, vv = i % NV;
      cp_async16(sb + tc::core_off<BK>(n, vv), a.w + ((size_t)(n0 + n) * 9 + tap) * a.Cin + c0 + vv * 8, true);
    }
  };

  if (warp == 0) tc::tmem_alloc(s_tmem, S::kCols);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < ST; ++s) lbnci::mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tmem = *s_tmem;

  // chunks 0 .. AH-1 in flight before the first MMA; chunk kc + AH is copied while the
  // MMAs of chunks kc - 1 and kc may still run (its stage was read by chunk kc + AH - ST)
#pragma unroll
  for (int s = 0; s < AH; ++s) {
    if (s < nk) load(s, s);
    cp_commit();
  }
  bool good = true;
  int last = -1;  // last chunk whose MMAs were issued (the same in every thread)
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc % ST;
    cp_wait<AH - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // this thread's copies -> tensor core reads
    if (!__syncthreads_and(good)) break;
    if (tid == 0) {
      tc::fence_after_sync();
      const unsigned sa = smem_u32(stage_a(s)), sb = smem_u32(stage_b(s));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)  // K = 16 per MMA: two core matrices along K, 256 bytes
        tc::mma_bf16(tmem, tc::smem_desc(sa + 256u * kk, 128u, S::kSBO), tc::smem_desc(sb + 256u * kk, 128u, S::kSBO),
                     IDESC, (kc > 0 || kk > 0) ? 1u : 0u);
      tc::mma_commit(&bar[s]);
    }
    last = kc;
    const int kn = kc + AH;
    if (kn < nk) {
      const int kp = kn - ST;  // the chunk whose MMAs last read stage kn % ST
      if (kp >= 0) good = lbnci::mbar_wait(&bar[kp % ST], (unsigned)((kp / ST) & 1));
      if (good) load(kn % ST, kn);
    }
    cp_commit();
  }
  cp_wait<0>();
  // the MMAs of the last issued chunk complete after all earlier ones
  const bool done = last >= 0 && lbnci::mbar_wait(&bar[last % ST], (unsigned)((last / ST) & 1));
  const bool ok_all = __syncthreads_and(good && done);
  tc::fence_after_sync();
  if (ok_all) {
    // warp w reads lanes 32 (w % 4) .. (its quarter of the pixels), columns of half w / 4
    const int q = warp & 3, half = warp >> 2;
    const int row = m0 + q * 32 + lane;
    const unsigned taddr = tmem + ((unsigned)(q * 32) << 16);
#pragma unroll
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
      float acc[16];
      tc::tmem_ld16(taddr + (unsigned)c0, acc);  // every lane takes part (aligned), rows beyond M included
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int col = n0 + c0 + j;
          float v0 = acc[j] + (a.bias ? a.bias[col] : 0.f), v1 = acc[j + 1] + (a.bias ? a.bias[col + 1] : 0.f);
          if (a.relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          if (a.mask) {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + (size_t)row * a.ms + col);
            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
          }
          *reinterpret_cast<__nv_bfloat162*>(a.y + (size_t)row * a.ys + col) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, S::kCols);
}

}  // namespace lbu
