// unet_kernels.cuh -- kernels of the warm-start U-Net: BF16 operands, FP32 accumulation.
//
// Convolutions are implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16 in, FP32
// accumulate), fed by cp.async into a three-stage shared-memory ring and ldmatrix:
//   forward / data gradient   M = pixels, N = output channels, K = 9 taps x input channels;
//   weight gradient           M = output channels, N = input channels of one tap,
//                             K = pixels, split over blocks, partial sums reduced in a
//                             fixed order (deterministic).
// The data gradient of a 3x3 convolution is the same kernel run on the weights flipped in
// (dy, dx) and transposed in (C_out, C_in). Activations are NHWC BF16 with an explicit
// pixel stride, so a layer can read or write one channel slice of a concatenation buffer.
// Padding: zero rows beyond the first and last image row, periodic columns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbu {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16-byte global -> shared copy; pred = false writes zeros and reads nothing
__device__ __forceinline__ void cp_async16(void* s, const void* g, bool pred) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(s)), "l"(g), "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// ------------------------------------------------------------------ 3x3 convolution
struct ConvFwd {
  const bf16* x;
  int xs;               // input pixel stride (elements)
  int B, H, W;          // output image; the input is (H >> up) x (W >> up)
  int Cin, up;
  const bf16* w;        // [Cout][9][Cin]
  const float* bias;    // [Cout] or null
  int relu;
  bf16* y;
  int ys;               // output pixel stride
  int Cout;
  const bf16* mask;     // optional: y = 0 where mask <= 0 (ReLU derivative), same grid as y
  int ms;
};

constexpr int kConvBM = 128, kConvBK = 32, kStages = 3;

template <int BN>
__global__ void __launch_bounds__(128) conv3x3_kernel(ConvFwd a) {
  constexpr int BM = kConvBM, BK = kConvBK, LD = BK + 8, ST = kStages;
  constexpr int WN = BN / 2, NT = WN / 8;
  __shared__ __align__(16) bf16 sA[ST][BM * LD];
  __shared__ __align__(16) bf16 sB[ST][BN * LD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int M = a.B * a.H * a.W;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int cpt = a.Cin / BK, nk = 9 * cpt;
  const int Hi = a.H >> a.up, Wi = a.W >> a.up;
  const int v = tid & 3;
  int pb[4], py[4], px[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = m0 + (tid >> 2) + 32 * j;
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
  auto load = [&](int s, int kc) {
    const int tap = kc / cpt, c0 = (kc - tap * cpt) * BK;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int yy = py[j] + dy, xx = wrap(px[j] + dx, a.W);
      const bool ok = pb[j] >= 0 && yy >= 0 && yy < a.H;
      const bf16* src = a.x;
      if (ok) src = a.x + ((size_t)(pb[j] * Hi + (yy >> a.up)) * Wi + (xx >> a.up)) * a.xs + c0 + v * 8;
      cp_async16(&sA[s][((tid >> 2) + 32 * j) * LD + v * 8], src, ok);
    }
#pragma unroll
    for (int i = tid; i < BN * 4; i += 128) {
      const int n = i >> 2, vv = i & 3;
      cp_async16(&sB[s][n * LD + vv * 8], a.w + ((size_t)(n0 + n) * 9 + tap) * a.Cin + c0 + vv * 8, true);
    }
  };

  float acc[4][NT][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

#pragma unroll
  for (int s = 0; s < ST - 1; ++s) {
    if (s < nk) load(s, s);
    cp_commit();
  }
  for (int kc = 0; kc < nk; ++kc) {
    cp_wait<ST - 2>();
    __syncthreads();
    if (kc + ST - 1 < nk) load((kc + ST - 1) % ST, kc + ST - 1);
    cp_commit();
    const bf16* As = sA[kc % ST];
    const bf16* Bs = sB[kc % ST];
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[4][4], bq[NT][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
        ldsm_x4(af[mt], As + (wm * 64 + mt * 16 + (lane & 15)) * LD + kk + (lane >> 4) * 8);
#pragma unroll
      for (int nt = 0; nt < NT; nt += 2) {
        unsigned r[4];
        ldsm_x4(r, Bs + (wn * WN + nt * 8 + (lane & 7) + ((lane >> 4) << 3)) * LD + kk + ((lane >> 3) & 1) * 8);
        bq[nt][0] = r[0];
        bq[nt][1] = r[1];
        bq[nt + 1][0] = r[2];
        bq[nt + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma16816(acc[mt][nt], af[mt], bq[nt][0], bq[nt][1]);
    }
  }
  cp_wait<0>();

  // epilogue: bias, ReLU or ReLU-derivative mask, BF16 store (pairs of channels)
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int col = n0 + wn * WN + nt * 8 + (lane & 3) * 2;
      const float b0 = a.bias ? a.bias[col] : 0.f, b1 = a.bias ? a.bias[col + 1] : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm * 64 + mt * 16 + (lane >> 2) + 8 * h;
        if (row >= M) continue;
        float v0 = acc[mt][nt][2 * h] + b0, v1 = acc[mt][nt][2 * h + 1] + b1;
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

// ------------------------------------------------------------------ weight gradient
struct ConvWgrad {
  const bf16* x;
  int xs, up;           // input view as in ConvFwd
  const bf16* dy;
  int dys;              // output-gradient view [pixel][Cout]
  int B, H, W, Cin, Cout;
  float* part;          // [nsplit][Cout][9 Cin]
  float* bpart;         // [nsplit][Cout] or null
  int pps;              // pixels per split, multiple of 32
};

template <int BM, int BN>
__global__ void __launch_bounds__(128) conv3x3_wgrad_kernel(ConvWgrad a) {
  constexpr int BK = 32, LDA = BM + 8, LDB = BN + 8, ST = kStages;
  constexpr int WM = BM / 2, WN = BN / 2, MT = WM / 16, NT = WN / 8;
  __shared__ __align__(16) bf16 sD[ST][BK * LDA];  // [pixel][co]
  __shared__ __align__(16) bf16 sX[ST][BK * LDB];  // [pixel][ci]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int co0 = blockIdx.x * BM;
  const int cblk = a.Cin / BN;
  const int tap = blockIdx.y / cblk, c0 = (blockIdx.y - tap * cblk) * BN;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int P = a.B * a.H * a.W;
  const int p0 = blockIdx.z * a.pps, p1 = min(p0 + a.pps, P);
  const int nk = (p1 - p0 + BK - 1) / BK;
  const int Hi = a.H >> a.up, Wi = a.W >> a.up;
  const bool do_bias = a.bpart != nullptr && blockIdx.y == 0;

  auto load = [&](int s, int kc) {
    const int pbase = p0 + kc * BK;
#pragma unroll
    for (int i = tid; i < BK * (BM / 8); i += 128) {
      const int r = i / (BM / 8), vv = i % (BM / 8);
      const int p = pbase + r;
      const bool ok = p < p1;
      cp_async16(&sD[s][r * LDA + vv * 8], ok ? a.dy + (size_t)p * a.dys + co0 + vv * 8 : a.dy, ok);
    }
#pragma unroll
    for (int i = tid; i < BK * (BN / 8); i += 128) {
      const int r = i / (BN / 8), vv = i % (BN / 8);
      const int p = pbase + r;
      bool ok = p < p1;
      const bf16* src = a.x;
      if (ok) {
        const int xq = p % a.W, t = p / a.W, yq = t % a.H, b = t / a.H;
        const int yy = yq + dy, xx = wrap(xq + dx, a.W);
        ok = yy >= 0 && yy < a.H;
        if (ok) src = a.x + ((size_t)(b * Hi + (yy >> a.up)) * Wi + (xx >> a.up)) * a.xs + c0 + vv * 8;
      }
      cp_async16(&sX[s][r * LDB + vv * 8], src, ok);
    }
  };

  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  float bsum = 0.f;

#pragma unroll
  for (int s = 0; s < ST - 1; ++s) {
    if (s < nk) load(s, s);
    cp_commit();
  }
  for (int kc = 0; kc < nk; ++kc) {
    cp_wait<ST - 2>();
    __syncthreads();
    if (kc + ST - 1 < nk) load((kc + ST - 1) % ST, kc + ST - 1);
    cp_commit();
    const bf16* Ds = sD[kc % ST];
    const bf16* Xs = sX[kc % ST];
    if (do_bias && tid < BM) {
#pragma unroll 8
      for (int r = 0; r < BK; ++r) bsum += __bfloat162float(Ds[r * LDA + tid]);
    }
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[MT][4], bq[NT][2];
      const int mi = lane >> 3;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        ldsm_x4_t(af[mt], Ds + (kk + ((mi >> 1) << 3) + (lane & 7)) * LDA + wm * WM + mt * 16 + ((mi & 1) << 3));
#pragma unroll
      for (int nt = 0; nt < NT; nt += 2) {
        unsigned r[4];
        ldsm_x4_t(r, Xs + (kk + ((mi & 1) << 3) + (lane & 7)) * LDB + wn * WN + nt * 8 + ((mi >> 1) << 3));
        bq[nt][0] = r[0];
        bq[nt][1] = r[1];
        bq[nt + 1][0] = r[2];
        bq[nt + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma16816(acc[mt][nt], af[mt], bq[nt][0], bq[nt][1]);
    }
  }
  cp_wait<0>();

  float* out = a.part + (size_t)blockIdx.z * a.Cout * 9 * a.Cin;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int col = tap * a.Cin + c0 + wn * WN + nt * 8 + (lane & 3) * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = co0 + wm * WM + mt * 16 + (lane >> 2) + 8 * h;
        *reinterpret_cast<float2*>(out + (size_t)row * 9 * a.Cin + col) =
            make_float2(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
      }
    }
  if (do_bias && tid < BM) a.bpart[(size_t)blockIdx.z * a.Cout + co0 + tid] = bsum;
}

// Sum the split partials in split order: dw[o][t][c] for c < cin_true (master layout
// [Cout][3][3][cin_true]) and db[o].
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ bpart, int nsplit,
                                    int Cout, int Cin, int cin_true, float* __restrict__ dw, float* __restrict__ db) {
  const int n = Cout * 9 * cin_true;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + Cout; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const int c = i % cin_true, t = (i / cin_true) % 9, o = i / (9 * cin_true);
      const float* p = part + (size_t)o * 9 * Cin + t * Cin + c;
      float s = 0.f;
      for (int z = 0; z < nsplit; ++z) s += p[(size_t)z * Cout * 9 * Cin];
      dw[i] = s;
    } else if (db) {
      const int o = i - n;
      float s = 0.f;
      for (int z = 0; z < nsplit; ++z) s += bpart[(size_t)z * Cout + o];
      db[o] = s;
    }
  }
}

// ------------------------------------------------------------------ element-wise kernels
union V8 {
  uint4 u;
  __nv_bfloat162 h[4];
};

// FP32 X[n][HW][cin] (samples idx[b], or b) -> BF16 [b][HW][cpad], zero padded
__global__ void pack_input_kernel(const float* __restrict__ X, const int* __restrict__ idx, int B, int HW, int cin,
                                  int cpad, bf16* __restrict__ out) {
  const int groups = cpad / 8;
  const long total = (long)B * HW * groups;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int g = (int)(i % groups);
    const long pix = i / groups;
    const int b = (int)(pix / HW), p = (int)(pix % HW);
    const long sb = idx ? idx[b] : b;
    const float* src = X + (sb * HW + p) * cin;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = g * 8 + k;
      v[k] = c < cin ? src[c] : 0.f;
    }
    V8 o;
#pragma unroll
    for (int k = 0; k < 4; ++k) o.h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    *reinterpret_cast<uint4*>(out + pix * cpad + g * 8) = o.u;
  }
}

// 2x2 max pool: in view [B][H][W] (stride is) -> out [B][H/2][W/2][C] contiguous.
// Ties go to the first element in window order (0,0), (0,1), (1,0), (1,1).
__global__ void maxpool_kernel(const bf16* __restrict__ in, int is, int B, int H, int W, int C,
                               bf16* __restrict__ out) {
  const int h = H / 2, w = W / 2, groups = C / 8;
  const long total = (long)B * h * w * groups;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int g = (int)(i % groups);
    const long q = i / groups;
    const int x = (int)(q % w), y = (int)((q / w) % h), b = (int)(q / ((long)w * h));
    V8 best;
    float bv[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int yy = 2 * y + (k >> 1), xx = 2 * x + (k & 1);
      V8 v;
      v.u = *reinterpret_cast<const uint4*>(in + ((size_t)(b * H + yy) * W + xx) * is + g * 8);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
        if (k == 0 || f.x > bv[2 * e]) {
          bv[2 * e] = f.x;
          best.h[e].x = v.h[e].x;
        }
        if (k == 0 || f.y > bv[2 * e + 1]) {
          bv[2 * e + 1] = f.y;
          best.h[e].y = v.h[e].y;
        }
      }
    }
    *reinterpret_cast<uint4*>(out + q * C + g * 8) = best.u;
  }
}

// Max-pool backward, in place on the skip slice of a concatenation gradient:
// g[q] = bf16(g[q] + (q is the window's argmax ? dp : 0)) where act[q] > 0, else 0.
__global__ void maxpool_bwd_kernel(const bf16* __restrict__ act, int as, const bf16* __restrict__ dp, bf16* g, int gs,
                                   int B, int H, int W, int C) {
  const int h = H / 2, w = W / 2, groups = C / 8;
  const long total = (long)B * h * w * groups;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int g8 = (int)(i % groups);
    const long q = i / groups;
    const int x = (int)(q % w), y = (int)((q / w) % h), b = (int)(q / ((long)w * h));
    float a[4][8];
    int arg[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int yy = 2 * y + (k >> 1), xx = 2 * x + (k & 1);
      V8 v;
      v.u = *reinterpret_cast<const uint4*>(act + ((size_t)(b * H + yy) * W + xx) * as + g8 * 8);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
        a[k][2 * e] = f.x;
        a[k][2 * e + 1] = f.y;
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      arg[c] = 0;
#pragma unroll
      for (int k = 1; k < 4; ++k)
        if (a[k][c] > a[arg[c]][c]) arg[c] = k;
    }
    V8 d;
    d.u = *reinterpret_cast<const uint4*>(dp + q * C + g8 * 8);
    float dv[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(d.h[e]);
      dv[2 * e] = f.x;
      dv[2 * e + 1] = f.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int yy = 2 * y + (k >> 1), xx = 2 * x + (k & 1);
      bf16* gp = g + ((size_t)(b * H + yy) * W + xx) * gs + g8 * 8;
      V8 v;
      v.u = *reinterpret_cast<const uint4*>(gp);
      float o[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
        o[2 * e] = f.x;
        o[2 * e + 1] = f.y;
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (arg[c] == k) o[c] += dv[c];
        if (!(a[k][c] > 0.f)) o[c] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) v.h[e] = __floats2bfloat162_rn(o[2 * e], o[2 * e + 1]);
      *reinterpret_cast<uint4*>(gp) = v.u;
    }
  }
}

// Gradient of nearest 2x upsampling followed by the ReLU derivative of the low-resolution
// activation: out[b][y][x][c] = bf16(sum of the 2x2 children of du) where act > 0, else 0.
// du [B][2h][2w][C], act and out [B][h][w][C], all contiguous.
__global__ void upsample_bwd_kernel(const bf16* __restrict__ du, const bf16* __restrict__ act, bf16* __restrict__ out,
                                    int B, int h, int w, int C) {
  const int groups = C / 8, H = 2 * h, W = 2 * w;
  const long total = (long)B * h * w * groups;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int g = (int)(i % groups);
    const long q = i / groups;
    const int x = (int)(q % w), y = (int)((q / w) % h), b = (int)(q / ((long)w * h));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int yy = 2 * y + (k >> 1), xx = 2 * x + (k & 1);
      V8 v;
      v.u = *reinterpret_cast<const uint4*>(du + ((size_t)(b * H + yy) * W + xx) * C + g * 8);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
        s[2 * e] += f.x;
        s[2 * e + 1] += f.y;
      }
    }
    V8 m, o;
    m.u = *reinterpret_cast<const uint4*>(act + q * C + g * 8);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(m.h[e]);
      o.h[e] = __floats2bfloat162_rn(f.x > 0.f ? s[2 * e] : 0.f, f.y > 0.f ? s[2 * e + 1] : 0.f);
    }
    *reinterpret_cast<uint4*>(out + q * C + g * 8) = o.u;
  }
}

// ------------------------------------------------------------------ head, loss
constexpr int kMaxOut = 8, kMaxHeadIn = 256;

// y[p][j] = b[j] + sum_c wh[j][c] x[p][c]; x BF16 [P][C], wh BF16 [nout][C], y FP32
__global__ void head_fwd_kernel(const bf16* __restrict__ x, int C, const bf16* __restrict__ wh,
                                const float* __restrict__ bh, int nout, int P, float* __restrict__ y) {
  __shared__ float sw[kMaxOut * kMaxHeadIn];
  for (int i = threadIdx.x; i < nout * C; i += blockDim.x) sw[i] = __bfloat162float(wh[i]);
  __syncthreads();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float acc[kMaxOut];
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j) acc[j] = j < nout ? bh[j] : 0.f;
    for (int c0 = 0; c0 < C; c0 += 8) {
      V8 v;
      v.u = *reinterpret_cast<const uint4*>(x + (size_t)p * C + c0);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j)
          if (j < nout) {
            acc[j] = fmaf(sw[j * C + c0 + 2 * e], f.x, acc[j]);
            acc[j] = fmaf(sw[j * C + c0 + 2 * e + 1], f.y, acc[j]);
          }
      }
    }
    for (int j = 0; j < nout; ++j) y[(size_t)p * nout + j] = acc[j];
  }
}

// Loss partial sums and dL/dy: d = y - t; partial[block] = sum lam_j d^2 (FP64);
// dy = 2 lam_j d / P. T is gathered by idx (per image of HW pixels).
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ T, const int* __restrict__ idx,
                           int HW, int nout, int P, float lam0, float lam1, float lam2, float lam3, float lam4,
                           float lam5, float lam6, float lam7, float* __restrict__ dy, double* __restrict__ partial) {
  const float lam[8] = {lam0, lam1, lam2, lam3, lam4, lam5, lam6, lam7};
  double s = 0.0;
  const float scale = 2.f / (float)P;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int b = p / HW, q = p % HW;
    const long sb = idx ? idx[b] : b;
    const float* t = T + (sb * HW + q) * nout;
    for (int j = 0; j < nout; ++j) {
      const float d = y[(size_t)p * nout + j] - t[j];
      s += (double)(lam[j] * d * d);
      dy[(size_t)p * nout + j] = scale * lam[j] * d;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double scale, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s * scale;
  }
}

// Head backward. dx[p][c] = bf16(sum_j dy[p][j] wh[j][c]) where x[p][c] > 0, else 0;
// per block of kHeadPix pixels the partial sums of dW[j][c] = sum_p dy[p][j] x[p][c] and
// db[j] = sum_p dy[p][j] go to part[block][nout (C + 1)].
constexpr int kHeadPix = 1024;
__global__ void head_bwd_kernel(const bf16* __restrict__ x, int C, const bf16* __restrict__ wh, int nout, int P,
                                const float* __restrict__ dy, bf16* __restrict__ dx, float* __restrict__ part) {
  __shared__ float sw[kMaxOut * kMaxHeadIn];
  for (int i = threadIdx.x; i < nout * C; i += blockDim.x) sw[i] = __bfloat162float(wh[i]);
  __syncthreads();
  const int p0 = blockIdx.x * kHeadPix, p1 = min(p0 + kHeadPix, P);
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    float d[kMaxOut];
    for (int j = 0; j < nout; ++j) d[j] = dy[(size_t)p * nout + j];
    for (int c0 = 0; c0 < C; c0 += 8) {
      V8 v, o;
      v.u = *reinterpret_cast<const uint4*>(x + (size_t)p * C + c0);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(v.h[e]);
        float s0 = 0.f, s1 = 0.f;
        for (int j = 0; j < nout; ++j) {
          s0 = fmaf(d[j], sw[j * C + c0 + 2 * e], s0);
          s1 = fmaf(d[j], sw[j * C + c0 + 2 * e + 1], s1);
        }
        o.h[e] = __floats2bfloat162_rn(f.x > 0.f ? s0 : 0.f, f.y > 0.f ? s1 : 0.f);
      }
      *reinterpret_cast<uint4*>(dx + (size_t)p * C + c0) = o.u;
    }
  }
  const int nw = nout * (C + 1);
  for (int o = threadIdx.x; o < nw; o += blockDim.x) {
    const int j = o / (C + 1), c = o % (C + 1);
    float s = 0.f;
    for (int p = p0; p < p1; ++p) {
      const float xv = c < C ? __bfloat162float(x[(size_t)p * C + c]) : 1.f;
      s = fmaf(dy[(size_t)p * nout + j], xv, s);
    }
    part[(size_t)blockIdx.x * nw + o] = s;
  }
}

// Sum head partials in block order into the master gradient: dW [nout][C] then db [nout].
__global__ void head_reduce_kernel(const float* __restrict__ part, int nblk, int nout, int C, float* __restrict__ dw,
                                   float* __restrict__ db) {
  const int nw = nout * (C + 1);
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nw; o += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nblk; ++z) s += part[(size_t)z * nw + o];
    const int j = o / (C + 1), c = o % (C + 1);
    if (c < C)
      dw[j * C + c] = s;
    else
      db[j] = s;
  }
}

// ------------------------------------------------------------------ parameters
struct LayerDev {
  long long w_off, b_off;  // master FP32 offsets (weight, bias)
  long long wb_off;        // BF16 [Cout][taps][cin_pad] (head: [Cout][cin])
  long long wt_off;        // BF16 flipped transpose [cin_pad][9][Cout], or -1
  int cout, cin, cin_pad, taps;
};

// Master FP32 weights -> BF16 kernel layouts (padded input channels are zero).
__global__ void refresh_weights_kernel(const LayerDev* __restrict__ L, const float* __restrict__ master,
                                       bf16* __restrict__ wb, bf16* __restrict__ wt) {
  const LayerDev d = L[blockIdx.y];
  const long n = (long)d.cout * d.taps * d.cin_pad;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % d.cin_pad), t = (int)((i / d.cin_pad) % d.taps), o = (int)(i / ((long)d.cin_pad * d.taps));
    const float v = c < d.cin ? master[d.w_off + ((long)o * d.taps + t) * d.cin + c] : 0.f;
    const bf16 h = __float2bfloat16_rn(v);
    wb[d.wb_off + i] = h;
    if (d.wt_off >= 0) wt[d.wt_off + ((long)c * 9 + (8 - t)) * d.cout + o] = h;
  }
}

// Adam (bias-corrected): c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t)
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

}  // namespace lbu
