// Learned elimination proposal: a small CNN over the pixel grid that reads
// six per-pixel features of the sharing-ADMM state and predicts which pixels
// may be dropped early.  Architecture (fixed): five 3x3 convolutions
// (6 -> 32, then 32 -> 32, zero padding 1) each followed by GELU, a 1x1 head
// (32 -> 1) and a sigmoid.  Weights are BF16-rounded copies of FP32 master
// parameters; all sums are FP32.  Training: binary cross-entropy with a
// positive-class weight, Adam.  The paper has no counterpart (this is the
// extension that proposes drops; Algorithm 1 still runs as the fallback).
//
// Activations are NCHW float32.  Flat parameter layout (SADMM_CNN_PARAMS):
//   W1[32][6][3][3] b1[32] W2[32][32][3][3] b2[32] ... W5 b5 Wh[32] bh[1]
#include "common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace sadmm {
namespace {

constexpr int kC = 32;                 // hidden channels
constexpr int kCin0 = 6;               // input features
constexpr int kLayers = 5;
constexpr int kTileXY = 16;            // output tile 16 x 16, one thread per pixel

__host__ __device__ constexpr int conv_w_size(int cin) { return kC * cin * 9; }
__host__ __device__ constexpr int layer_offset(int l) {
  // l = 0..4 conv layers, 5 = head
  return l == 0 ? 0 : conv_w_size(kCin0) + kC + (l - 1) * (conv_w_size(kC) + kC);
}
constexpr int kHeadOffset = layer_offset(5);
constexpr int kParams = kHeadOffset + kC + 1;
static_assert(kParams == 38785, "parameter count");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// Direct 3x3 convolution, zero padding 1:
//   out[b][o][y][x] = bias[o] + sum_{c,ky,kx} w[o][c][ky][kx] in[b][c][y+ky-1][x+kx-1]
// One CTA per (image, 16x16 tile), one thread per output pixel computing all
// NOUT outputs; input channels are staged through shared memory 8 at a time
// (tile with halo + the matching weight slice).  GELU epilogue when `pre` is
// set (pre keeps the pre-activation, out the activation); plain otherwise.
// The input gradient of a convolution is the convolution of dZ with the
// kernel transposed in channels and flipped in both offsets,
// wt[ci][co][2-ky][2-kx] = w[co][ci][ky][kx] (prep_transpose_kernel), run by
// this kernel without bias or GELU.
constexpr int kCiChunk = 8;
constexpr int kOutGroup = 16;          // output channels per CTA

// Output channels are split over blockIdx.z in groups of OG (more CTAs for a
// single image); each thread forms OG outputs of one pixel.
template <int CIN, int NOUT, int OG>
__global__ void __launch_bounds__(kTileXY * kTileXY)
conv3x3_kernel(const float* __restrict__ in, const float* __restrict__ w, const float* __restrict__ bias,
               float* __restrict__ pre, float* __restrict__ out, int H, int Wd, int tiles_x) {
  static_assert(OG % 4 == 0 && NOUT % OG == 0, "output groups of whole float4s");
  __shared__ float s_in[kCiChunk][kTileXY + 2][kTileXY + 2];
  __shared__ __align__(16) float s_w[kCiChunk * 9 * OG];         // [c][k][o]: four outputs per 16-byte read
  const int b = blockIdx.y;
  const int og = blockIdx.z * OG;
  const int ty0 = (blockIdx.x / tiles_x) * kTileXY, tx0 = (blockIdx.x % tiles_x) * kTileXY;
  const int t = threadIdx.x;
  const int ly = t / kTileXY, lx = t % kTileXY;
  const int y = ty0 + ly, x = tx0 + lx;
  float acc[OG];
#pragma unroll
  for (int o = 0; o < OG; ++o) acc[o] = bias ? bias[og + o] : 0.f;
  const float* inb = in + (size_t)b * CIN * H * Wd;
  constexpr int kHalo = (kTileXY + 2) * (kTileXY + 2);
  for (int c0 = 0; c0 < CIN; c0 += kCiChunk) {
    const int nc = min(kCiChunk, CIN - c0);
    __syncthreads();
    for (int e = t; e < OG * kCiChunk * 9; e += blockDim.x) {
      const int o = e / (kCiChunk * 9), c = (e / 9) % kCiChunk, k = e % 9;
      s_w[(c * 9 + k) * OG + o] = c < nc ? w[((size_t)(og + o) * CIN + c0 + c) * 9 + k] : 0.f;
    }
    for (int e = t; e < kCiChunk * kHalo; e += blockDim.x) {
      const int c = e / kHalo, r = e % kHalo;
      const int yy = ty0 + r / (kTileXY + 2) - 1, xx = tx0 + r % (kTileXY + 2) - 1;
      float v = 0.f;
      if (c < nc && yy >= 0 && yy < H && xx >= 0 && xx < Wd) v = inb[((size_t)(c0 + c) * H + yy) * Wd + xx];
      s_in[c][r / (kTileXY + 2)][r % (kTileXY + 2)] = v;
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float v = s_in[c][ly + k / 3][lx + k % 3];
        const float4* wk = reinterpret_cast<const float4*>(s_w + (c * 9 + k) * OG);
#pragma unroll
        for (int o4 = 0; o4 < OG / 4; ++o4) {
          const float4 ww = wk[o4];
          acc[4 * o4 + 0] = fmaf(ww.x, v, acc[4 * o4 + 0]);
          acc[4 * o4 + 1] = fmaf(ww.y, v, acc[4 * o4 + 1]);
          acc[4 * o4 + 2] = fmaf(ww.z, v, acc[4 * o4 + 2]);
          acc[4 * o4 + 3] = fmaf(ww.w, v, acc[4 * o4 + 3]);
        }
      }
    }
  }
  if (y >= H || x >= Wd) return;
  const size_t base = (size_t)b * NOUT * H * Wd + (size_t)y * Wd + x;
#pragma unroll
  for (int o = 0; o < OG; ++o) {
    const size_t idx = base + (size_t)(og + o) * H * Wd;
    if (pre) {
      pre[idx] = acc[o];
      out[idx] = gelu(acc[o]);
    } else {
      out[idx] = acc[o];
    }
  }
}

// wt[ci][co][k] = w[co][ci][8 - k]  (k = 3 ky + kx; flipping both offsets)
__global__ void prep_transpose_kernel(const float* __restrict__ w, int cin, float* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kC * cin * 9) return;
  const int co = e / (cin * 9), ci = (e / 9) % cin, k = e % 9;
  wt[(ci * kC + co) * 9 + (8 - k)] = w[e];
}

// dW[co][ci][k] = sum_{b,y,x} dz[b][co][y][x] in[b][ci][y+ky-1][x+kx-1];
// db[co] = sum dz[b][co].  One CTA per (co, ci); fixed-order block reduction.
__global__ void __launch_bounds__(256)
conv3x3_bwd_w_kernel(const float* __restrict__ in, const float* __restrict__ dz, int cin, int B, int H, int Wd,
                     float* __restrict__ dw, float* __restrict__ db) {
  const int co = blockIdx.x / cin, ci = blockIdx.x % cin;
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  const int HW = H * Wd;
  for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
    const int b = e / HW, p = e % HW, y = p / Wd, x = p % Wd;
    const float g = dz[((size_t)b * kC + co) * HW + p];
    const float* ib = in + ((size_t)b * cin + ci) * HW;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
      const float v = (yy >= 0 && yy < H && xx >= 0 && xx < Wd) ? ib[yy * Wd + xx] : 0.f;
      acc[k] = fmaf(g, v, acc[k]);
    }
    acc[9] += g;
  }
  __shared__ float red[8][10];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane == 0) red[warp][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    float s = 0.f;
    for (int w8 = 0; w8 < 8; ++w8) s += red[w8][threadIdx.x];
    if (threadIdx.x < 9) dw[(co * cin + ci) * 9 + threadIdx.x] = s;
    else if (ci == 0) db[co] = s;
  }
}

// head: p = sigmoid(bh + sum_c wh[c] a[c]); optionally the BCE gradient
// dz = (p - y) * weight / count and per-block loss partials.
__global__ void head_kernel(const float* __restrict__ a, const float* __restrict__ wh, const float* __restrict__ bh,
                            int B, int HW, float* __restrict__ prob, const float* __restrict__ labels,
                            float pos_weight, float* __restrict__ dz, double* __restrict__ loss_part) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (e < B * HW) {
    const int b = e / HW, p = e % HW;
    float z = bh[0];
    for (int c = 0; c < kC; ++c) z = fmaf(wh[c], a[((size_t)b * kC + c) * HW + p], z);
    const float pr = 1.f / (1.f + expf(-z));
    if (prob) prob[e] = pr;
    if (labels) {
      const float y = labels[e];
      const float wgt = y > 0.5f ? pos_weight : 1.f;
      const double cnt = (double)B * HW;
      // loss = -w [y log p + (1-y) log(1-p)], computed from z for stability
      const double zd = z;
      const double lp = zd >= 0 ? -log1p(exp(-zd)) : zd - log1p(exp(zd));       // log p
      const double lq = zd >= 0 ? -zd - log1p(exp(-zd)) : -log1p(exp(zd));      // log (1-p)
      l = -wgt * (y * lp + (1.0 - y) * lq) / cnt;
      dz[e] = (float)(wgt * (pr - y) / cnt);
    }
  }
  if (!loss_part) return;
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) s += red[w8];
    loss_part[blockIdx.x] = s;
  }
}

// head gradients: dWh[c] = sum dz a[c], dbh = sum dz (one CTA per c, c = 32 is
// the bias); dA[c] = dz * wh[c] (elementwise kernel below).
__global__ void head_bwd_w_kernel(const float* __restrict__ a, const float* __restrict__ dz, int B, int HW,
                                  float* __restrict__ dwh, float* __restrict__ dbh) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (int e = threadIdx.x; e < B * HW; e += blockDim.x) {
    const int b = e / HW, p = e % HW;
    s = fmaf(dz[e], c < kC ? a[((size_t)b * kC + c) * HW + p] : 1.f, s);
  }
  __shared__ float red[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w8 = 0; w8 < 8; ++w8) t += red[w8];
    if (c < kC) dwh[c] = t; else dbh[0] = t;
  }
}

// dZ[b][c][p] = dA * gelu'(pre), with dA = dz[b][p] wh[c] for the last layer
// (head) or the transposed-conv output otherwise.
__global__ void gelu_bwd_kernel(const float* __restrict__ pre, const float* __restrict__ da,
                                const float* __restrict__ dz_head, const float* __restrict__ wh, int B, int HW,
                                float* __restrict__ dz) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)B * kC * HW) return;
  float g;
  if (dz_head) {
    const int c = (int)((e / HW) % kC);
    const size_t b = e / ((size_t)kC * HW);
    g = dz_head[b * HW + e % HW] * wh[c];
  } else {
    g = da[e];
  }
  dz[e] = g * gelu_grad(pre[e]);
}

__global__ void round_bf16_kernel(const float* __restrict__ master, float* __restrict__ w, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) w[e] = __bfloat162float(__float2bfloat16_rn(master[e]));
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  w[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct CnnCtx {
  int H = 0, W = 0, maxB = 0;
  std::vector<void*> owned;
  float* master = nullptr;     // FP32 parameters
  float* wq = nullptr;         // BF16-rounded parameters used by the kernels
  float* wt = nullptr;         // transposed conv weights (scratch)
  float *adam_m = nullptr, *adam_v = nullptr;
  int adam_t = 0;
  float* act[kLayers + 1] = {};   // act[0] = input copy slot unused; act[l+1] = output of layer l
  float* pre[kLayers] = {};
  float *dz = nullptr, *da = nullptr, *dzh = nullptr;
  double* loss_part = nullptr;
  void* dalloc(size_t b) {
    void* p = nullptr;
    if (cudaMalloc(&p, b ? b : 16) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  }
};

namespace {

int tiles(const CnnCtx& c) { return div_up(c.H, kTileXY) * div_up(c.W, kTileXY); }

int cnn_forward_impl(CnnCtx& c, const float* in, int B, float* prob, cudaStream_t st) {
  const int tx = div_up(c.W, kTileXY);
  const dim3 grid(tiles(c), B, kC / kOutGroup);
  const float* x = in;
  for (int l = 0; l < kLayers; ++l) {
    const float* w = c.wq + layer_offset(l);
    const float* bias = w + (l == 0 ? conv_w_size(kCin0) : conv_w_size(kC));
    if (l == 0)
      conv3x3_kernel<kCin0, kC, kOutGroup><<<grid, kTileXY * kTileXY, 0, st>>>(x, w, bias, c.pre[l], c.act[l + 1], c.H,
                                                                              c.W, tx);
    else
      conv3x3_kernel<kC, kC, kOutGroup><<<grid, kTileXY * kTileXY, 0, st>>>(x, w, bias, c.pre[l], c.act[l + 1], c.H,
                                                                           c.W, tx);
    SADMM_LAUNCH_CHECK();
    x = c.act[l + 1];
  }
  const int n = B * c.H * c.W;
  head_kernel<<<div_up(n, 256), 256, 0, st>>>(x, c.wq + kHeadOffset, c.wq + kHeadOffset + kC, B, c.H * c.W, prob,
                                              nullptr, 1.f, nullptr, nullptr);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace
}  // namespace sadmm

struct sadmm_cnn_ctx : sadmm::CnnCtx {};

extern "C" {

int sadmm_cnn_create(int H, int W, int max_batch, sadmm_cnn_t* out) {
  using namespace sadmm;
  if (!out || H < 1 || W < 1 || max_batch < 1 || (long long)H * W * max_batch > (1ll << 26)) {
    set_error("sadmm_cnn_create: bad sizes");
    return SADMM_EINVAL;
  }
  *out = nullptr;
  sadmm_cnn_ctx* c = new (std::nothrow) sadmm_cnn_ctx();
  if (!c) return SADMM_ENOMEM;
  c->H = H; c->W = W; c->maxB = max_batch;
  bool ok = true;
  auto A = [&](size_t b) { void* p = c->dalloc(b); if (!p) ok = false; return p; };
  c->master = (float*)A(kParams * 4);
  c->wq = (float*)A(kParams * 4);
  c->wt = (float*)A(conv_w_size(kC) * 4);
  c->adam_m = (float*)A(kParams * 4);
  c->adam_v = (float*)A(kParams * 4);
  const size_t plane = (size_t)max_batch * H * W;
  for (int l = 0; l < kLayers; ++l) {
    c->pre[l] = (float*)A(plane * kC * 4);
    c->act[l + 1] = (float*)A(plane * kC * 4);
  }
  c->dz = (float*)A(plane * kC * 4);
  c->da = (float*)A(plane * kC * 4);
  c->dzh = (float*)A(plane * 4);
  c->loss_part = (double*)A((size_t)div_up(plane, 256) * 8);
  if (!ok) {
    for (void* p : c->owned) cudaFree(p);
    delete c;
    set_error("sadmm_cnn_create: allocation failed");
    return SADMM_ENOMEM;
  }
  cudaMemset(c->master, 0, kParams * 4);
  cudaMemset(c->wq, 0, kParams * 4);
  cudaMemset(c->adam_m, 0, kParams * 4);
  cudaMemset(c->adam_v, 0, kParams * 4);
  *out = c;
  return SADMM_OK;
}

int sadmm_cnn_num_params(void) { return sadmm::kParams; }

int sadmm_cnn_set_params(sadmm_cnn_t c, const float* params) {
  using namespace sadmm;
  if (!c || !params) return SADMM_EINVAL;
  SADMM_CUDA_TRY(cudaMemcpy(c->master, params, kParams * 4, cudaMemcpyDefault));
  round_bf16_kernel<<<div_up(kParams, 256), 256>>>(c->master, c->wq, kParams);
  SADMM_LAUNCH_CHECK();
  SADMM_CUDA_TRY(cudaMemset(c->adam_m, 0, kParams * 4));
  SADMM_CUDA_TRY(cudaMemset(c->adam_v, 0, kParams * 4));
  c->adam_t = 0;
  SADMM_CUDA_TRY(cudaDeviceSynchronize());
  return SADMM_OK;
}

int sadmm_cnn_get_params(sadmm_cnn_t c, float* params, int rounded) {
  using namespace sadmm;
  if (!c || !params) return SADMM_EINVAL;
  SADMM_CUDA_TRY(cudaMemcpy(params, rounded ? c->wq : c->master, kParams * 4, cudaMemcpyDefault));
  return SADMM_OK;
}

int sadmm_cnn_forward(sadmm_cnn_t c, const float* in, int B, float* prob, void* stream) {
  using namespace sadmm;
  if (!c || !in || !prob || B < 1 || B > c->maxB) { set_error("sadmm_cnn_forward: bad arguments"); return SADMM_EINVAL; }
  return cnn_forward_impl(*c, in, B, prob, (cudaStream_t)stream);
}

int sadmm_cnn_backward(sadmm_cnn_t c, const float* in, const float* labels, int B, double pos_weight,
                       float* grad, double* loss, void* stream) {
  using namespace sadmm;
  if (!c || !in || !labels || !grad || B < 1 || B > c->maxB) {
    set_error("sadmm_cnn_backward: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SADMM_TRY(cnn_forward_impl(*c, in, B, nullptr, st));
  const int HW = c->H * c->W, n = B * HW;
  const int nb = div_up(n, 256);
  // head: probabilities, BCE gradient dz_head and loss partials
  head_kernel<<<nb, 256, 0, st>>>(c->act[kLayers], c->wq + kHeadOffset, c->wq + kHeadOffset + kC, B, HW, nullptr,
                                  labels, (float)pos_weight, c->dzh, c->loss_part);
  SADMM_LAUNCH_CHECK();
  head_bwd_w_kernel<<<kC + 1, 256, 0, st>>>(c->act[kLayers], c->dzh, B, HW, grad + kHeadOffset, grad + kHeadOffset + kC);
  SADMM_LAUNCH_CHECK();
  const size_t nact = (size_t)B * kC * HW;
  const int tx = div_up(c->W, kTileXY);
  const dim3 grid(tiles(*c), B);
  for (int l = kLayers - 1; l >= 0; --l) {
    // dZ_l = dA_l * gelu'(pre_l); dA of the last layer comes from the head
    gelu_bwd_kernel<<<div_up((long long)nact, 256), 256, 0, st>>>(c->pre[l], c->da,
                                                                    l == kLayers - 1 ? c->dzh : nullptr,
                                                                    c->wq + kHeadOffset, B, HW, c->dz);
    SADMM_LAUNCH_CHECK();
    const int cin = l == 0 ? kCin0 : kC;
    const float* inl = l == 0 ? in : c->act[l];
    float* dw = grad + layer_offset(l);
    float* db = dw + conv_w_size(cin);
    conv3x3_bwd_w_kernel<<<kC * cin, 256, 0, st>>>(inl, c->dz, cin, B, c->H, c->W, dw, db);
    SADMM_LAUNCH_CHECK();
    if (l > 0) {
      prep_transpose_kernel<<<div_up(conv_w_size(kC), 256), 256, 0, st>>>(c->wq + layer_offset(l), kC, c->wt);
      SADMM_LAUNCH_CHECK();
      conv3x3_kernel<kC, kC, kOutGroup><<<dim3(grid.x, grid.y, kC / kOutGroup), kTileXY * kTileXY, 0, st>>>(
          c->dz, c->wt, nullptr, nullptr, c->da, c->H, c->W, tx);
      SADMM_LAUNCH_CHECK();
    }
  }
  if (loss) {
    std::vector<double> lp(nb);
    SADMM_CUDA_TRY(cudaMemcpyAsync(lp.data(), c->loss_part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : lp) s += v;
    *loss = s;
  }
  return SADMM_OK;
}

int sadmm_cnn_adam_step(sadmm_cnn_t c, const float* grad, double lr, void* stream) {
  using namespace sadmm;
  if (!c || !grad || !(lr > 0.0)) return SADMM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  c->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)c->adam_t), c2 = 1.f - powf(b2, (float)c->adam_t);
  adam_kernel<<<div_up(kParams, 256), 256, 0, st>>>(c->master, c->adam_m, c->adam_v, grad, kParams, (float)lr, b1, b2,
                                                    1e-8f, c1, c2);
  SADMM_LAUNCH_CHECK();
  round_bf16_kernel<<<div_up(kParams, 256), 256, 0, st>>>(c->master, c->wq, kParams);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

void sadmm_cnn_destroy(sadmm_cnn_t c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (void* p : c->owned) cudaFree(p);
  delete c;
}

}  // extern "C"
