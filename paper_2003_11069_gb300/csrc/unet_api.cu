// unet_api.cu -- the warm-start U-Net runtime behind include/lbnci_unet.h: layer table,
// activation and gradient buffers, the forward and backward launch sequences, Adam.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbnci_unet.h"
#include "unet_kernels.cuh"
#include "unet_tc.cuh"

// Error word of the tensor-core convolutions: bit 0 set when a bounded mbarrier wait
// expired (the launch then wrote no output). Read and cleared by the calls that
// synchronise their stream.
__device__ int g_tc_err;

using lbu::bf16;

namespace {

constexpr int kInPad = 32;  // input channels are padded to one K chunk of the convolution

struct LayerHost {
  int cout, cin, cin_pad, taps;
  long long w_off, b_off, wb_off, wt_off;
};

bool valid_config(const lbu_config* c, std::string* why) {
  if (!c) return *why = "null config", false;
  if (c->levels < 2 || c->levels > 6) return *why = "levels must be 2..6", false;
  if (c->base <= 0 || c->base % 32 != 0) return *why = "base must be a positive multiple of 32", false;
  if (c->base * (1 << (c->levels - 1)) > 1024) return *why = "widest level exceeds 1024 channels", false;
  if (c->in_ch < 1 || c->in_ch > kInPad) return *why = "in_ch must be 1..32", false;
  if (c->out_ch < 1 || c->out_ch > lbu::kMaxOut) return *why = "out_ch must be 1..8", false;
  if (c->base > lbu::kMaxHeadIn) return *why = "base exceeds the head kernel's 256 input channels", false;
  const int f = 1 << (c->levels - 1);
  if (c->H <= 0 || c->W <= 0 || c->H % f || c->W % f) return *why = "H and W must be multiples of 2^(levels-1)", false;
  if (c->max_batch <= 0) return *why = "max_batch must be positive", false;
  if ((long long)c->max_batch * c->H * c->W > (1LL << 30) / 64) return *why = "max_batch * H * W too large", false;
  return true;
}

std::vector<LayerHost> layer_table(const lbu_config* c) {
  std::vector<LayerHost> L;
  auto add = [&](int cout, int cin, int taps) {
    LayerHost l{};
    l.cout = cout;
    l.cin = cin;
    l.cin_pad = taps == 9 ? ((cin + 31) / 32) * 32 : cin;
    l.taps = taps;
    L.push_back(l);
  };
  std::vector<int> C(c->levels);
  for (int l = 0; l < c->levels; ++l) C[l] = c->base << l;
  int cin = c->in_ch;
  for (int l = 0; l < c->levels; ++l) {
    add(C[l], cin, 9);
    add(C[l], C[l], 9);
    cin = C[l];
  }
  for (int l = c->levels - 2; l >= 0; --l) {
    add(C[l], C[l + 1], 9);
    add(C[l], 2 * C[l], 9);
    add(C[l], C[l], 9);
  }
  add(c->out_ch, C[0], 1);
  long long off = 0, wb = 0, wt = 0;
  for (size_t i = 0; i < L.size(); ++i) {
    LayerHost& l = L[i];
    l.w_off = off;
    off += (long long)l.cout * l.taps * l.cin;
    l.b_off = off;
    off += l.cout;
    l.wb_off = wb;
    wb += (long long)l.cout * l.taps * l.cin_pad;
    if (l.taps == 9 && i > 0) {  // the first layer needs no data gradient
      l.wt_off = wt;
      wt += (long long)l.cout * 9 * l.cin_pad;
    } else {
      l.wt_off = -1;
    }
  }
  return L;
}

long long total_params(const std::vector<LayerHost>& L) {
  const LayerHost& b = L.back();
  return b.b_off + b.cout;
}

// wgrad partition: splits of the pixel range so that the grid has about 4 waves of blocks
struct WgradPlan {
  int BM, BN, nsplit, pps;
};
WgradPlan wgrad_plan(int P, int cin, int cout) {
  WgradPlan w;
  w.BM = cout % 64 == 0 ? 64 : 32;
  w.BN = cin % 64 == 0 ? 64 : 32;
  const int blocks_xy = (cout / w.BM) * 9 * (cin / w.BN);
  int ns = (4 * 152 + blocks_xy - 1) / blocks_xy;
  ns = std::max(1, std::min(ns, (P + 255) / 256));
  int pps = (P + ns - 1) / ns;
  pps = (pps + 31) / 32 * 32;
  w.pps = pps;
  w.nsplit = (P + pps - 1) / pps;
  return w;
}
size_t wgrad_bytes(const WgradPlan& w, int cin, int cout) {
  return ((size_t)w.nsplit * cout * 9 * cin + (size_t)w.nsplit * cout) * sizeof(float);
}

thread_local std::string g_err;

}  // namespace

struct lbu_net {
  lbu_config cfg;
  std::vector<LayerHost> L;
  long long nparams = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wb = nullptr, *wt = nullptr;
  lbu::LayerDev* Ldev = nullptr;
  // activations, per level l (image H>>l x W>>l, width C_l)
  std::vector<bf16*> ea, cat, pool, da, db, gA, gB, gCat, gU, gPool;
  bf16* x0 = nullptr;
  float *y = nullptr, *dy = nullptr, *xstage = nullptr, *ystage = nullptr;
  float* work = nullptr;
  size_t work_bytes = 0;
  double *partial = nullptr, *loss = nullptr;
  int npartial = 0;
  float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  long long t = 0;
  long long launches = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

lb_status fail(lbu_net* n, lb_status st, const std::string& msg) {
  if (n) n->err = msg; else g_err = msg;
  return st;
}
lb_status cuda_fail(lbu_net* n, cudaError_t e, const char* where) {
  (void)cudaGetLastError();
  return fail(n, LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define LBU_CUDA(n, call)                                        \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail((n), e_, #call);     \
  } while (0)

int width(const lbu_net* n, int l) { return n->cfg.base << l; }
int Hl(const lbu_net* n, int l) { return n->cfg.H >> l; }
int Wl(const lbu_net* n, int l) { return n->cfg.W >> l; }

template <typename T>
lb_status dalloc(lbu_net* n, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(n, e, "cudaMalloc");
  n->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return LB_OK;
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

template <int BN, int BK>
cudaError_t launch_conv_tc_k(const lbu::ConvFwd& a, dim3 grid, cudaStream_t s) {
  int* err = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&err, g_tc_err);
  if (e != cudaSuccess) return e;
  constexpr int smem = lbu::tc::Smem<BN, BK>::kBytes;
  e = cudaFuncSetAttribute(lbu::conv3x3_tc_kernel<BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  grid.y = a.Cout / BN;
  lbu::conv3x3_tc_kernel<BN, BK><<<grid, lbu::kTcThreads, smem, s>>>(a, err);
  return cudaGetLastError();
}
// chunks of 32 input channels (stages of 10-16 KB: three to five CTAs of 8 warps per SM)
template <int BN>
cudaError_t launch_conv_tc(const lbu::ConvFwd& a, dim3 grid, cudaStream_t s) {
  return launch_conv_tc_k<BN, 32>(a, grid, s);
}

// LBNCI_UNET_MMA=tcgen05 selects the tensor-memory convolution (unet_tc.cuh). It computes
// the same sums (equal to the mma.sync kernel's bit for bit on the measured layers) but is
// slower here: 7.1 ms against 5.5 ms per training step of batch 32 at 64 x 256; the
// mma.sync kernel stays the default.
bool conv_on_tcgen05() {
  const char* e = std::getenv("LBNCI_UNET_MMA");
  return e && std::strcmp(e, "tcgen05") == 0;
}

// Reports (and clears) an expired wait of a tensor-core convolution; call after a
// synchronisation of the stream.
lb_status check_tc(lbu_net* n) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(n, e, "error word read");
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int));
    return fail(n, LB_ECUDA, "a tensor-core convolution's mbarrier wait expired (no output written)");
  }
  return LB_OK;
}

// one 3x3 convolution launch (forward or data gradient)
lb_status conv(lbu_net* n, const bf16* x, int xs, int B, int H, int W, int cin, int up, const bf16* w,
               const float* bias, int relu, bf16* y, int ys, int cout, const bf16* mask, int ms,
               cudaStream_t s) {
  lbu::ConvFwd a{x, xs, B, H, W, cin, up, w, bias, relu, y, ys, cout, mask, ms};
  const int M = B * H * W;
  dim3 grid((M + lbu::kConvBM - 1) / lbu::kConvBM, 1);
  if (conv_on_tcgen05()) {
    cudaError_t e = cout % 128 == 0 ? launch_conv_tc<128>(a, grid, s)
                                    : (cout % 64 == 0 ? launch_conv_tc<64>(a, grid, s) : launch_conv_tc<32>(a, grid, s));
    if (n) ++n->launches;
    return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "conv3x3 (tcgen05) launch");
  }
  if (cout % 64 == 0) {
    grid.y = cout / 64;
    lbu::conv3x3_kernel<64><<<grid, 128, 0, s>>>(a);
  } else {
    grid.y = cout / 32;
    lbu::conv3x3_kernel<32><<<grid, 128, 0, s>>>(a);
  }
  if (n) ++n->launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "conv3x3 launch");
}

lb_status wgrad(lbu_net* n, const bf16* x, int xs, int up, const bf16* dy, int dys, int B, int H, int W, int cin,
                int cout, float* work, size_t work_bytes, cudaStream_t s, float* dw_master, float* db_master,
                int cin_true) {
  const WgradPlan p = wgrad_plan(B * H * W, cin, cout);
  if (wgrad_bytes(p, cin, cout) > work_bytes) return fail(n, LB_EINVAL, "wgrad scratch too small");
  float* part = work;
  float* bpart = work + (size_t)p.nsplit * cout * 9 * cin;
  lbu::ConvWgrad a{x, xs, up, dy, dys, B, H, W, cin, cout, part, db_master ? bpart : nullptr, p.pps};
  dim3 grid(cout / p.BM, 9 * (cin / p.BN), p.nsplit);
  if (p.BM == 64 && p.BN == 64) lbu::conv3x3_wgrad_kernel<64, 64><<<grid, 128, 0, s>>>(a);
  else if (p.BM == 64) lbu::conv3x3_wgrad_kernel<64, 32><<<grid, 128, 0, s>>>(a);
  else if (p.BN == 64) lbu::conv3x3_wgrad_kernel<32, 64><<<grid, 128, 0, s>>>(a);
  else lbu::conv3x3_wgrad_kernel<32, 32><<<grid, 128, 0, s>>>(a);
  const long long nout = (long long)cout * 9 * cin_true + cout;
  lbu::wgrad_reduce_kernel<<<grid_for(nout, 256), 256, 0, s>>>(part, bpart, p.nsplit, cout, cin, cin_true,
                                                                dw_master, db_master);
  if (n) n->launches += 2;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "wgrad launch");
}

#define LBU_TRY(expr)                  \
  do {                                 \
    lb_status st_ = (expr);            \
    if (st_ != LB_OK) return st_;      \
  } while (0)

const bf16* WB(const lbu_net* n, int i) { return n->wb + n->L[i].wb_off; }
const bf16* WT(const lbu_net* n, int i) { return n->wt + n->L[i].wt_off; }
const float* BIAS(const lbu_net* n, int i) { return n->params + n->L[i].b_off; }

// index helpers into the layer table
int enc_a(int l) { return 2 * l; }
int enc_b(int l) { return 2 * l + 1; }
int up_i(const lbu_net* n, int l) { return 2 * n->cfg.levels + 3 * (n->cfg.levels - 2 - l); }
int head_i(const lbu_net* n) { return (int)n->L.size() - 1; }

lb_status forward_impl(lbu_net* n, int B) {
  const int Lv = n->cfg.levels;
  cudaStream_t s = n->stream;
  const bf16* h = n->x0;
  int hs = kInPad;
  for (int l = 0; l < Lv; ++l) {
    const int C = width(n, l), H = Hl(n, l), W = Wl(n, l);
    LBU_TRY(conv(n, h, hs, B, H, W, n->L[enc_a(l)].cin_pad, 0, WB(n, enc_a(l)), BIAS(n, enc_a(l)), 1, n->ea[l], C,
                 C, nullptr, 0, s));
    if (l < Lv - 1) {
      LBU_TRY(conv(n, n->ea[l], C, B, H, W, C, 0, WB(n, enc_b(l)), BIAS(n, enc_b(l)), 1, n->cat[l] + C, 2 * C, C,
                   nullptr, 0, s));
      const long long work = (long long)B * (H / 2) * (W / 2) * (C / 8);
      lbu::maxpool_kernel<<<grid_for(work, 256), 256, 0, s>>>(n->cat[l] + C, 2 * C, B, H, W, C, n->pool[l]);
      ++n->launches;
      h = n->pool[l];
      hs = C;
    } else {
      LBU_TRY(conv(n, n->ea[l], C, B, H, W, C, 0, WB(n, enc_b(l)), BIAS(n, enc_b(l)), 1, n->db[l], C, C, nullptr,
                   0, s));
      h = n->db[l];
      hs = C;
    }
  }
  for (int l = Lv - 2; l >= 0; --l) {
    const int C = width(n, l), H = Hl(n, l), W = Wl(n, l), k = up_i(n, l);
    LBU_TRY(conv(n, h, hs, B, H, W, 2 * C, 1, WB(n, k), BIAS(n, k), 1, n->cat[l], 2 * C, C, nullptr, 0, s));
    LBU_TRY(conv(n, n->cat[l], 2 * C, B, H, W, 2 * C, 0, WB(n, k + 1), BIAS(n, k + 1), 1, n->da[l], C, C, nullptr,
                 0, s));
    LBU_TRY(conv(n, n->da[l], C, B, H, W, C, 0, WB(n, k + 2), BIAS(n, k + 2), 1, n->db[l], C, C, nullptr, 0, s));
    h = n->db[l];
    hs = C;
  }
  const int hi = head_i(n);
  const int P = B * n->cfg.H * n->cfg.W;
  lbu::head_fwd_kernel<<<grid_for(P, 256), 256, 0, s>>>(n->db[0], n->cfg.base, WB(n, hi), BIAS(n, hi),
                                                        n->cfg.out_ch, P, n->y);
  ++n->launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "forward launch");
}

lb_status backward_impl(lbu_net* n, int B) {
  const int Lv = n->cfg.levels;
  cudaStream_t s = n->stream;
  const int P = B * n->cfg.H * n->cfg.W;
  float* G = n->grads;
  auto GW = [&](int i) { return G + n->L[i].w_off; };
  auto GB = [&](int i) { return G + n->L[i].b_off; };
  // head
  {
    const int hi = head_i(n), C0 = n->cfg.base;
    const int nblk = (P + lbu::kHeadPix - 1) / lbu::kHeadPix;
    lbu::head_bwd_kernel<<<nblk, 256, 0, s>>>(n->db[0], C0, WB(n, hi), n->cfg.out_ch, P, n->dy, n->gB[0], n->work);
    lbu::head_reduce_kernel<<<1, 256, 0, s>>>(n->work, nblk, n->cfg.out_ch, C0, GW(hi), GB(hi));
    n->launches += 2;
  }
  // decoder, finest level first
  for (int l = 0; l <= Lv - 2; ++l) {
    const int C = width(n, l), H = Hl(n, l), W = Wl(n, l), k = up_i(n, l);
    const int C1 = width(n, l + 1);
    // dec_lb: input da[l], output gradient gB[l]
    LBU_TRY(wgrad(n, n->da[l], C, 0, n->gB[l], C, B, H, W, C, C, n->work, n->work_bytes, s, GW(k + 2), GB(k + 2), C));
    LBU_TRY(conv(n, n->gB[l], C, B, H, W, C, 0, WT(n, k + 2), nullptr, 0, n->gA[l], C, C, n->da[l], C, s));
    // dec_la: input cat[l]
    LBU_TRY(wgrad(n, n->cat[l], 2 * C, 0, n->gA[l], C, B, H, W, 2 * C, C, n->work, n->work_bytes, s, GW(k + 1),
                  GB(k + 1), 2 * C));
    LBU_TRY(conv(n, n->gA[l], C, B, H, W, C, 0, WT(n, k + 1), nullptr, 0, n->gCat[l], 2 * C, 2 * C, n->cat[l],
                 2 * C, s));
    // up_l: input = nearest upsampling of the level-(l+1) output
    const bf16* hin = n->db[l + 1];
    LBU_TRY(wgrad(n, hin, C1, 1, n->gCat[l], 2 * C, B, H, W, C1, C, n->work, n->work_bytes, s, GW(k), GB(k), C1));
    LBU_TRY(conv(n, n->gCat[l], 2 * C, B, H, W, C, 0, WT(n, k), nullptr, 0, n->gU[l], C1, C1, nullptr, 0, s));
    const long long work = (long long)B * Hl(n, l + 1) * Wl(n, l + 1) * (C1 / 8);
    lbu::upsample_bwd_kernel<<<grid_for(work, 256), 256, 0, s>>>(n->gU[l], hin, n->gB[l + 1], B, Hl(n, l + 1),
                                                                 Wl(n, l + 1), C1);
    ++n->launches;
  }
  // encoder, coarsest level first; gB[Lv-1] holds the bottom output's gradient
  for (int l = Lv - 1; l >= 0; --l) {
    const int C = width(n, l), H = Hl(n, l), W = Wl(n, l);
    const bf16* g;
    int gs;
    if (l == Lv - 1) {
      g = n->gB[l];
      gs = C;
    } else {
      const long long work = (long long)B * (H / 2) * (W / 2) * (C / 8);
      lbu::maxpool_bwd_kernel<<<grid_for(work, 256), 256, 0, s>>>(n->cat[l] + C, 2 * C, n->gPool[l],
                                                                  n->gCat[l] + C, 2 * C, B, H, W, C);
      ++n->launches;
      g = n->gCat[l] + C;
      gs = 2 * C;
    }
    LBU_TRY(wgrad(n, n->ea[l], C, 0, g, gs, B, H, W, C, C, n->work, n->work_bytes, s, GW(enc_b(l)), GB(enc_b(l)), C));
    LBU_TRY(conv(n, g, gs, B, H, W, C, 0, WT(n, enc_b(l)), nullptr, 0, n->gA[l], C, C, n->ea[l], C, s));
    const bf16* xin = l == 0 ? n->x0 : n->pool[l - 1];
    const int cin = n->L[enc_a(l)].cin_pad;
    LBU_TRY(wgrad(n, xin, cin, 0, n->gA[l], C, B, H, W, cin, C, n->work, n->work_bytes, s, GW(enc_a(l)),
                  GB(enc_a(l)), n->L[enc_a(l)].cin));
    if (l > 0)
      LBU_TRY(conv(n, n->gA[l], C, B, H, W, C, 0, WT(n, enc_a(l)), nullptr, 0, n->gPool[l - 1], cin, cin, nullptr,
                   0, s));
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "backward launch");
}

lb_status refresh(lbu_net* n) {
  size_t maxn = 0;
  for (auto& l : n->L) maxn = std::max(maxn, (size_t)l.cout * l.taps * l.cin_pad);
  dim3 grid((unsigned)std::min<size_t>((maxn + 255) / 256, 1024), (unsigned)n->L.size());
  lbu::refresh_weights_kernel<<<grid, 256, 0, n->stream>>>(n->Ldev, n->params, n->wb, n->wt);
  ++n->launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "refresh launch");
}

lb_status loss_impl(lbu_net* n, const float* T, const int* idx, int B, const float* lam) {
  const int HW = n->cfg.H * n->cfg.W, P = B * HW;
  float lm[8];
  for (int j = 0; j < 8; ++j) lm[j] = (lam && j < n->cfg.out_ch) ? lam[j] : 1.f;
  const int blocks = std::min(n->npartial, grid_for(P, 256));
  lbu::mse_kernel<<<blocks, 256, 0, n->stream>>>(n->y, T, idx, HW, n->cfg.out_ch, P, lm[0], lm[1], lm[2], lm[3],
                                                 lm[4], lm[5], lm[6], lm[7], n->dy, n->partial);
  lbu::sum_partials_kernel<<<1, 32, 0, n->stream>>>(n->partial, blocks, 1.0 / P, n->loss);
  n->launches += 2;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "loss launch");
}

lb_status pack(lbu_net* n, const float* X, const int* idx, int B) {
  const long long work = (long long)B * n->cfg.H * n->cfg.W * (kInPad / 8);
  lbu::pack_input_kernel<<<grid_for(work, 256), 256, 0, n->stream>>>(X, idx, B, n->cfg.H * n->cfg.W, n->cfg.in_ch,
                                                                     kInPad, n->x0);
  ++n->launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LB_OK : cuda_fail(n, e, "pack launch");
}

lb_status check_batch(lbu_net* n, int B) {
  if (B <= 0 || B > n->cfg.max_batch) return fail(n, LB_EINVAL, "batch must be 1..max_batch");
  return LB_OK;
}

}  // namespace

extern "C" {

int lbu_layer_count(const lbu_config* cfg) {
  std::string why;
  if (!valid_config(cfg, &why)) return -1;
  return (int)layer_table(cfg).size();
}

lb_status lbu_layer_shape(const lbu_config* cfg, int layer, int shape[4]) {
  std::string why;
  if (!valid_config(cfg, &why)) return fail(nullptr, LB_EINVAL, why);
  auto L = layer_table(cfg);
  if (layer < 0 || layer >= (int)L.size() || !shape) return fail(nullptr, LB_EINVAL, "bad layer index");
  const int k = L[layer].taps == 9 ? 3 : 1;
  shape[0] = L[layer].cout;
  shape[1] = k;
  shape[2] = k;
  shape[3] = L[layer].cin;
  return LB_OK;
}

lb_status lbu_param_count(const lbu_config* cfg, long long* count) {
  std::string why;
  if (!valid_config(cfg, &why)) return fail(nullptr, LB_EINVAL, why);
  if (!count) return fail(nullptr, LB_EINVAL, "null count");
  *count = total_params(layer_table(cfg));
  return LB_OK;
}

lb_status lbu_create(const lbu_config* cfg, lbu_net** out) {
  std::string why;
  if (!out) return fail(nullptr, LB_EINVAL, "null output handle");
  *out = nullptr;
  if (!valid_config(cfg, &why)) return fail(nullptr, LB_EINVAL, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return fail(nullptr, LB_ECUDA, "no CUDA device");
  }
  lbu_net* n = new (std::nothrow) lbu_net();
  if (!n) return fail(nullptr, LB_ENOMEM, "host allocation failed");
  n->cfg = *cfg;
  n->stream = (cudaStream_t)cfg->stream;
  cudaGetDevice(&n->device);
  n->L = layer_table(cfg);
  n->nparams = total_params(n->L);
  const int Lv = cfg->levels, B = cfg->max_batch;
  auto bail = [&](lb_status st) {
    g_err = n->err;
    lbu_destroy(n);
    return st;
  };
#define LBU_ALLOC(p, cnt)                          \
  do {                                             \
    lb_status st_ = dalloc(n, &(p), (cnt));        \
    if (st_ != LB_OK) return bail(st_);            \
  } while (0)
  LBU_ALLOC(n->params, n->nparams);
  LBU_ALLOC(n->grads, n->nparams);
  LBU_ALLOC(n->m, n->nparams);
  LBU_ALLOC(n->v, n->nparams);
  long long nwb = 0, nwt = 0;
  for (auto& l : n->L) {
    nwb = std::max(nwb, l.wb_off + (long long)l.cout * l.taps * l.cin_pad);
    if (l.wt_off >= 0) nwt = std::max(nwt, l.wt_off + (long long)l.cout * 9 * l.cin_pad);
  }
  LBU_ALLOC(n->wb, nwb);
  LBU_ALLOC(n->wt, nwt);
  LBU_ALLOC(n->Ldev, n->L.size());
  {
    std::vector<lbu::LayerDev> h(n->L.size());
    for (size_t i = 0; i < n->L.size(); ++i) {
      const LayerHost& l = n->L[i];
      h[i] = lbu::LayerDev{l.w_off, l.b_off, l.wb_off, l.wt_off, l.cout, l.cin, l.cin_pad, l.taps};
    }
    if (cudaMemcpy(n->Ldev, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(cuda_fail(n, cudaGetLastError(), "layer table copy"));
  }
  const size_t HW = (size_t)cfg->H * cfg->W;
  n->ea.assign(Lv, nullptr);
  n->cat.assign(Lv, nullptr);
  n->pool.assign(Lv, nullptr);
  n->da.assign(Lv, nullptr);
  n->db.assign(Lv, nullptr);
  n->gA.assign(Lv, nullptr);
  n->gB.assign(Lv, nullptr);
  n->gCat.assign(Lv, nullptr);
  n->gU.assign(Lv, nullptr);
  n->gPool.assign(Lv, nullptr);
  for (int l = 0; l < Lv; ++l) {
    const size_t pix = (size_t)B * (HW >> (2 * l));
    const int C = width(n, l);
    LBU_ALLOC(n->ea[l], pix * C);
    LBU_ALLOC(n->db[l], pix * C);
    LBU_ALLOC(n->gA[l], pix * C);
    LBU_ALLOC(n->gB[l], pix * C);
    if (l < Lv - 1) {
      LBU_ALLOC(n->cat[l], pix * 2 * C);
      LBU_ALLOC(n->gCat[l], pix * 2 * C);
      LBU_ALLOC(n->da[l], pix * C);
      LBU_ALLOC(n->pool[l], (pix / 4) * C);
      LBU_ALLOC(n->gPool[l], (pix / 4) * C);
      LBU_ALLOC(n->gU[l], pix * width(n, l + 1));
    }
  }
  LBU_ALLOC(n->x0, (size_t)B * HW * kInPad);
  LBU_ALLOC(n->y, (size_t)B * HW * cfg->out_ch);
  LBU_ALLOC(n->dy, (size_t)B * HW * cfg->out_ch);
  LBU_ALLOC(n->xstage, (size_t)B * HW * cfg->in_ch);
  LBU_ALLOC(n->ystage, (size_t)B * HW * cfg->out_ch);
  // scratch: the largest wgrad partial set and the head partials
  size_t wb = 0;
  for (int l = 0; l < Lv; ++l) {
    const int P = (int)((size_t)B * (HW >> (2 * l)));
    const int C = width(n, l);
    const int cins[4] = {l == 0 ? kInPad : width(n, l - 1), C, 2 * C, l < Lv - 1 ? width(n, l + 1) : C};
    for (int ci : cins) wb = std::max(wb, wgrad_bytes(wgrad_plan(P, ci, C), ci, C));
  }
  const size_t nblk = ((size_t)B * HW + lbu::kHeadPix - 1) / lbu::kHeadPix;
  wb = std::max(wb, nblk * cfg->out_ch * (cfg->base + 1) * sizeof(float));
  n->work_bytes = wb;
  LBU_ALLOC(n->work, wb / sizeof(float) + 1);
  n->npartial = 152 * 16;
  LBU_ALLOC(n->partial, n->npartial);
  LBU_ALLOC(n->loss, 1);
#undef LBU_ALLOC
  if (cudaMemset(n->params, 0, n->nparams * sizeof(float)) != cudaSuccess ||
      cudaMemset(n->m, 0, n->nparams * sizeof(float)) != cudaSuccess ||
      cudaMemset(n->v, 0, n->nparams * sizeof(float)) != cudaSuccess ||
      cudaMemset(n->grads, 0, n->nparams * sizeof(float)) != cudaSuccess)
    return bail(cuda_fail(n, cudaGetLastError(), "cudaMemset"));
  if (refresh(n) != LB_OK || cudaStreamSynchronize(n->stream) != cudaSuccess)
    return bail(cuda_fail(n, cudaGetLastError(), "initial weight refresh"));
  *out = n;
  return LB_OK;
}

void lbu_destroy(lbu_net* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  else cudaDeviceSynchronize();
  for (void* p : n->allocs) cudaFree(p);
  (void)cudaGetLastError();
  delete n;
}

const char* lbu_last_error(const lbu_net* n) { return n ? n->err.c_str() : g_err.c_str(); }

long long lbu_kernel_launches(const lbu_net* n) { return n ? n->launches : 0; }

lb_status lbu_set_params(lbu_net* n, const float* p, int on_device) {
  if (!n || !p) return fail(n, LB_EINVAL, "null argument");
  LBU_CUDA(n, cudaMemcpyAsync(n->params, p, n->nparams * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
  LBU_CUDA(n, cudaMemsetAsync(n->m, 0, n->nparams * sizeof(float), n->stream));
  LBU_CUDA(n, cudaMemsetAsync(n->v, 0, n->nparams * sizeof(float), n->stream));
  n->t = 0;
  LBU_TRY(refresh(n));
  LBU_CUDA(n, cudaStreamSynchronize(n->stream));
  return LB_OK;
}

lb_status lbu_get_params(lbu_net* n, float* p, int on_device) {
  if (!n || !p) return fail(n, LB_EINVAL, "null argument");
  LBU_CUDA(n, cudaMemcpyAsync(p, n->params, n->nparams * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  LBU_CUDA(n, cudaStreamSynchronize(n->stream));
  return LB_OK;
}

lb_status lbu_set_adam(lbu_net* n, float b1, float b2, float eps) {
  if (!n) return fail(n, LB_EINVAL, "null handle");
  if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps > 0.f)) return fail(n, LB_EINVAL, "bad Adam parameters");
  n->b1 = b1;
  n->b2 = b2;
  n->eps = eps;
  return LB_OK;
}

lb_status lbu_forward(lbu_net* n, const float* x, int batch, float* y, int on_device) {
  if (!n || !x || !y) return fail(n, LB_EINVAL, "null argument");
  LBU_TRY(check_batch(n, batch));
  const size_t HW = (size_t)n->cfg.H * n->cfg.W;
  const float* xd = x;
  if (!on_device) {
    LBU_CUDA(n, cudaMemcpyAsync(n->xstage, x, batch * HW * n->cfg.in_ch * sizeof(float), cudaMemcpyHostToDevice,
                                n->stream));
    xd = n->xstage;
  }
  LBU_TRY(pack(n, xd, nullptr, batch));
  LBU_TRY(forward_impl(n, batch));
  LBU_CUDA(n, cudaMemcpyAsync(y, n->y, batch * HW * n->cfg.out_ch * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  if (!on_device) {
    LBU_CUDA(n, cudaStreamSynchronize(n->stream));
    LBU_TRY(check_tc(n));
  }
  return LB_OK;
}

lb_status lbu_loss_grad(lbu_net* n, const float* X, const float* T, const int* idx, int batch, const float* lam,
                        float* loss, float* grads) {
  if (!n || !X || !T) return fail(n, LB_EINVAL, "null argument");
  LBU_TRY(check_batch(n, batch));
  LBU_TRY(pack(n, X, idx, batch));
  LBU_TRY(forward_impl(n, batch));
  LBU_TRY(loss_impl(n, T, idx, batch, lam));
  LBU_TRY(backward_impl(n, batch));
  if (grads)
    LBU_CUDA(n, cudaMemcpyAsync(grads, n->grads, n->nparams * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
  if (loss) {
    double h = 0.0;
    LBU_CUDA(n, cudaMemcpyAsync(&h, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    LBU_CUDA(n, cudaStreamSynchronize(n->stream));
    LBU_TRY(check_tc(n));
    *loss = (float)h;
  }
  return LB_OK;
}

lb_status lbu_train_step(lbu_net* n, const float* X, const float* T, const int* idx, int batch, const float* lam,
                         float lr, float* loss) {
  if (!n) return fail(n, LB_EINVAL, "null handle");
  if (!(lr > 0.f)) return fail(n, LB_EINVAL, "learning rate must be positive");
  LBU_TRY(lbu_loss_grad(n, X, T, idx, batch, lam, nullptr, nullptr));
  ++n->t;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)n->b1, (double)n->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)n->b2, (double)n->t)));
  lbu::adam_kernel<<<grid_for(n->nparams, 256), 256, 0, n->stream>>>(n->params, n->grads, n->m, n->v, n->nparams,
                                                                    lr, n->b1, n->b2, n->eps, c1, c2);
  ++n->launches;
  LBU_CUDA(n, cudaGetLastError());
  LBU_TRY(refresh(n));
  if (loss) {
    double h = 0.0;
    LBU_CUDA(n, cudaMemcpyAsync(&h, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    LBU_CUDA(n, cudaStreamSynchronize(n->stream));
    LBU_TRY(check_tc(n));
    *loss = (float)h;
  }
  return LB_OK;
}

lb_status lbu_conv3x3(const unsigned short* x, int x_stride, int batch, int h, int w, int c_in, int upsample,
                      const unsigned short* wgt, const float* bias, int relu, unsigned short* y, int y_stride,
                      int c_out, void* stream) {
  if (!x || !wgt || !y) return fail(nullptr, LB_EINVAL, "null argument");
  if (batch <= 0 || h <= 0 || w <= 0 || c_in <= 0 || c_out <= 0 || c_in % 32 || c_out % 32)
    return fail(nullptr, LB_EINVAL, "sizes: positive, channels multiples of 32");
  if (x_stride < c_in || y_stride < c_out || x_stride % 8 || y_stride % 8)
    return fail(nullptr, LB_EINVAL, "strides: at least the channel count, multiples of 8");
  if (upsample && (h % 2 || w % 2)) return fail(nullptr, LB_EINVAL, "upsampled output must have even size");
  return conv(nullptr, (const bf16*)x, x_stride, batch, h, w, c_in, upsample ? 1 : 0, (const bf16*)wgt, bias, relu,
              (bf16*)y, y_stride, c_out, nullptr, 0, (cudaStream_t)stream);
}

size_t lbu_conv3x3_wgrad_work(int batch, int h, int w, int c_in, int c_out) {
  if (batch <= 0 || h <= 0 || w <= 0 || c_in <= 0 || c_out <= 0) return 0;
  return wgrad_bytes(wgrad_plan(batch * h * w, c_in, c_out), c_in, c_out);
}

lb_status lbu_conv3x3_wgrad(const unsigned short* x, int x_stride, int batch, int h, int w, int c_in, int upsample,
                            const unsigned short* dy, int dy_stride, int c_out, float* dw, float* db, void* work,
                            size_t work_bytes, void* stream) {
  if (!x || !dy || !dw || !work) return fail(nullptr, LB_EINVAL, "null argument");
  if (batch <= 0 || h <= 0 || w <= 0 || c_in % 32 || c_out % 32 || c_in <= 0 || c_out <= 0)
    return fail(nullptr, LB_EINVAL, "sizes: positive, channels multiples of 32");
  if (x_stride < c_in || dy_stride < c_out || x_stride % 8 || dy_stride % 8)
    return fail(nullptr, LB_EINVAL, "strides: at least the channel count, multiples of 8");
  if (upsample && (h % 2 || w % 2)) return fail(nullptr, LB_EINVAL, "upsampled output must have even size");
  return wgrad(nullptr, (const bf16*)x, x_stride, upsample ? 1 : 0, (const bf16*)dy, dy_stride, batch, h, w, c_in,
               c_out, (float*)work, work_bytes, (cudaStream_t)stream, dw, db, c_in);
}

}  // extern "C"
