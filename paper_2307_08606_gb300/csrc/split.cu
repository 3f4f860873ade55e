// Split-precision operator: A = A_hi + A_lo with both planes in BF16 or FP16
// (pixel-major, (re, im) pairs of 16-bit values, 4 bytes per complex entry per
// plane).  The forward and adjoint products read one or both planes and
// accumulate in FP32; hi + lo is exact in FP32, so with both planes the
// product sees the rounded operator hi + lo (relative error 2^-17 for BF16,
// 2^-22 for FP16 pairs).  Reading the hi plane alone halves the operator
// bytes of the FP32 path; the solver then adds a lo-plane correction that is
// refreshed every few iterations.
#include "common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace sadmm {

namespace {

constexpr int kSpThreads = 128;             // one uint4 (4 complex) per thread and plane
constexpr int kSpRows = 4 * kSpThreads;     // complex rows per CTA slice
constexpr int kSpStage = 512;
constexpr int kSpUnroll = 8;

__device__ __forceinline__ uint4 ld_stream_u4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// 16-bit pair (re, im) packed in one 32-bit word -> two floats.
template <int KIND>
__device__ __forceinline__ float2 unpack(uint32_t w) {
  if constexpr (KIND == kSplitBF16) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
  } else {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
  }
}

template <int KIND>
__device__ __forceinline__ void unpack4(const uint4& u, float (&f)[8]) {
  const float2 a = unpack<KIND>(u.x), b = unpack<KIND>(u.y), c = unpack<KIND>(u.z), d = unpack<KIND>(u.w);
  f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y; f[4] = c.x; f[5] = c.y; f[6] = d.x; f[7] = d.y;
}

__device__ __forceinline__ float v_split(VMode mode, const SolverView& sv, int q, int pix, const float* vexp) {
  if (mode == kVExplicit) return vexp[pix];
  const float xq = sv.x[(size_t)q * sv.N + pix];
  if (mode == kVX) return xq;
  if (mode == kVNegX) return -xq;
  return xq - sv.xbar[pix] + sv.zbar[pix] - sv.s[pix];
}

// Partial sums of sum_p (A_hi + A_lo)[:, idx[p]] v[idx[p]] (planes as selected),
// written in the float4 layout of the FP32 forward partials.
template <int KIND, bool HI, bool LO, bool CONS>
__global__ void __launch_bounds__(kSpThreads)
split_forward_partial_kernel(const __grid_constant__ SetBlock<SplitSet> sets, int KM, int chunks,
                             int cols_per_chunk, VMode mode, const __grid_constant__ SolverView sv,
                             float4* __restrict__ partial) {
  const SplitSet& cs = sets.v[blockIdx.z];
  const int c = blockIdx.y;
  const int p0 = c * cols_per_chunk;
  const int p1 = min(cs.n, p0 + cols_per_chunk);
  const int row4 = blockIdx.x * kSpThreads + threadIdx.x;    // uint4 index within a column
  const bool active_row = row4 * 4 < KM;
  __shared__ float s_v[kSpStage];
  __shared__ int s_off[kSpStage];
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
  const uint4* H = reinterpret_cast<const uint4*>(cs.hi);
  const uint4* L = reinterpret_cast<const uint4*>(cs.lo);
  const size_t col4 = (size_t)KM / 4;
  for (int b0 = p0; b0 < p1; b0 += kSpStage) {
    const int nb = min(kSpStage, p1 - b0);
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += kSpThreads) {
      const int pix = cs.idx[b0 + t];
      s_v[t] = CONS ? sv.zbar[pix] - sv.u[(size_t)cs.q * sv.N + pix] : v_split(mode, sv, cs.q, pix, cs.vexp);
      s_off[t] = pix;
    }
    __syncthreads();
    if (!active_row) continue;
    int j = 0;
    for (; j + kSpUnroll <= nb; j += kSpUnroll) {
      uint4 h[kSpUnroll], l[kSpUnroll];
#pragma unroll
      for (int u = 0; u < kSpUnroll; ++u) {
        const size_t off = (size_t)s_off[j + u] * col4 + row4;
        if (HI) h[u] = ld_stream_u4(H + off);
        if (LO) l[u] = ld_stream_u4(L + off);
      }
#pragma unroll
      for (int u = 0; u < kSpUnroll; ++u) {
        float a[8], b[8];
        if (HI) unpack4<KIND>(h[u], a);
        if (LO) unpack4<KIND>(l[u], b);
        const float v = s_v[j + u];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float e = HI ? (LO ? a[k] + b[k] : a[k]) : b[k];     // hi + lo is exact in FP32
          acc[k] = fmaf(e, v, acc[k]);
        }
      }
    }
    for (; j < nb; ++j) {
      const size_t off = (size_t)s_off[j] * col4 + row4;
      float a[8], b[8];
      if (HI) unpack4<KIND>(ld_stream_u4(H + off), a);
      if (LO) unpack4<KIND>(ld_stream_u4(L + off), b);
      const float v = s_v[j];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float e = HI ? (LO ? a[k] + b[k] : a[k]) : b[k];
        acc[k] = fmaf(e, v, acc[k]);
      }
    }
  }
  if (active_row) {
    float4* out = partial + ((size_t)blockIdx.z * chunks + c) * (KM / 2) + 2 * row4;
    out[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    out[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  }
}

// out[r] = base[r] - sum_c partial[c][r] (+ optional second subtrahend).
__global__ void split_reduce_kernel(const __grid_constant__ SetBlock<SplitSet> sets, int KM, int chunks,
                                    const float4* __restrict__ partial) {
  const SplitSet& cs = sets.v[blockIdx.y];
  const int row2 = blockIdx.x * blockDim.x + threadIdx.x;
  if (row2 * 2 >= KM) return;
  const size_t col2 = (size_t)KM / 2;
  const float4* p = partial + (size_t)blockIdx.y * chunks * col2 + row2;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int c = 0; c < chunks; ++c) {
    const float4 t = p[(size_t)c * col2];
    acc.x += t.x; acc.y += t.y; acc.z += t.z; acc.w += t.w;
  }
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
  if (cs.base) b = reinterpret_cast<const float4*>(cs.base)[row2];
  float4 r = make_float4(b.x - acc.x, b.y - acc.y, b.z - acc.z, b.w - acc.w);
  if (cs.out2) reinterpret_cast<float4*>(cs.out2)[row2] = acc;      // the product itself
  if (cs.out) reinterpret_cast<float4*>(cs.out)[row2] = r;
}

int split_chunks(int nsets, int KM, int max_cols) {
  const int tiles = div_up(KM, kSpRows);
  int want = div_up(152 * 16, (long long)tiles * nsets);
  int cap = div_up(max_cols, 64);
  return max(1, min(want, cap));
}

// ------------------------------------------------------------------ adjoint
constexpr int kSaWarps = 8;
// columns per warp: a template parameter of split_adjoint_kernel (8, or 2
// in the chunked form when that fills the last wave of CTAs better)
constexpr int kSaUnroll = 4;
constexpr int kSaChunk = 1024;        // uint4 of a column per staged chunk of w (4096 complex, 32 KB)

// g = Re((A_hi + A_lo)[:, idx[p]]^H w) (planes as selected).  Epilogue:
// update -> x = v + mu (g + gcorr[pix]) with the ring entry; else g[p] = g and,
// if gcorr_out is set, gcorr_out[pix] = g (the lo-plane correction store).
// One column's products over the rows [c0, c0 + cn) of w staged in s_w (from
// row c0): plain mode adds them to cs (FP32 partials per lane); exact mode
// (two-product per term, double-float sum) to (h_, l_).
template <int KIND, bool HI, bool LO, bool EXACT>
__device__ __forceinline__ void split_adj_accumulate(const uint4* __restrict__ H, const uint4* __restrict__ L,
                                                     size_t base, int cn, int lane, const float4* s_w, float& cs,
                                                     float& h_, float& l_) {
  float acc[kSaUnroll];
#pragma unroll
  for (int u = 0; u < kSaUnroll; ++u) acc[u] = 0.f;
  for (int i0 = 0; i0 < cn; i0 += 32 * kSaUnroll) {
    uint4 h[kSaUnroll], l[kSaUnroll];
#pragma unroll
    for (int u = 0; u < kSaUnroll; ++u) {
      const int i = i0 + lane + 32 * u;
      if (i < cn) {
        if (HI) h[u] = ld_stream_u4(H + base + i);
        if (LO) l[u] = ld_stream_u4(L + base + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kSaUnroll; ++u) {
      const int i = i0 + lane + 32 * u;
      if (i < cn) {
        float a[8], b[8];
        if (HI) unpack4<KIND>(h[u], a);
        if (LO) unpack4<KIND>(l[u], b);
        const float4 wa = s_w[2 * i], wb = s_w[2 * i + 1];
        const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        if constexpr (EXACT) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float e = HI ? (LO ? a[k] + b[k] : a[k]) : b[k];
            const float p = e * wv[k];
            const float pe = fmaf(e, wv[k], -p);     // e w = p + pe exactly
            const float t = h_ + p;                   // two-sum h_ + p = t + err
            const float bp = t - h_;
            l_ += ((h_ - (t - bp)) + (p - bp)) + pe;
            h_ = t;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float e = HI ? (LO ? a[k] + b[k] : a[k]) : b[k];
            acc[u] = fmaf(e, wv[k], acc[u]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kSaUnroll; ++u) cs += acc[u];
}

// Warp reduction of a column's sums and the epilogue: exact mode writes the
// pair (g, g_lo) (+ the correction); else the x-update (update) or g.
template <bool EXACT>
__device__ __forceinline__ void split_adj_finish(const SplitSet& as, const SolverView& sv, bool update, int p,
                                                 int pix, int lane, float g, float h_, float l_) {
  if constexpr (EXACT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h_, o);
      const float ol = __shfl_xor_sync(0xffffffffu, l_, o);
      const float t = h_ + oh;
      const float bp = t - h_;
      l_ += ((h_ - (t - bp)) + (oh - bp)) + ol;
      h_ = t;
    }
    if (lane == 0) {
      if (as.gcorr_in) {
        const float c = as.gcorr_in[pix];
        const float t = h_ + c;
        const float bp = t - h_;
        l_ += (h_ - (t - bp)) + (c - bp);
        h_ = t;
      }
      const float hh = h_ + l_;
      as.g[p] = hh;
      as.g_lo[p] = l_ - (hh - h_);
      if (as.gcorr_out) as.gcorr_out[pix] = hh;
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if (lane == 0) {
    if (update) {
      const float gc = as.gcorr_in ? as.gcorr_in[pix] : 0.f;
      const size_t xi = (size_t)as.q * sv.N + pix;
      const float xo = sv.x[xi];
      const float v = v_admm(sv, as.q, pix, xo);
      const float xn = fmaf(sv.mu, g + gc, v);
      sv.ring[((size_t)sv.slot * sv.Q + as.q) * sv.N + pix] = xn - xo;
      sv.x[xi] = xn;
    } else {
      if (as.g) as.g[p] = g + (as.gcorr_in ? as.gcorr_in[pix] : 0.f);
      if (as.gcorr_out) as.gcorr_out[pix] = g;
    }
  }
}

// g = Re((A_hi + A_lo)[:, idx[p]]^H w) (planes as selected).  EXACT: the
// launch's sets ask for g as an exact pair (g_lo set, no update): each
// uint4's eight products are formed exactly and summed in double-float, so
// that g carries no rounding of the long 2KM-term sum (the primal x-update
// amplifies it by up to cond(rho I + mu B^T B)).  WHOLE: w fits one staged
// chunk and each column is summed in one pass; otherwise w is staged in
// chunks and each warp keeps its columns' sums across them, so that large KM
// keeps several CTAs per SM resident.
template <int KIND, bool HI, bool LO, bool EXACT, bool WHOLE, int COLS>
__global__ void __launch_bounds__(kSaWarps * 32)
split_adjoint_kernel(const __grid_constant__ SetBlock<SplitSet> sets, int KM, bool update,
                     const __grid_constant__ SolverView sv) {
  extern __shared__ float4 s_w[];                    // one chunk of w: up to 2 kSaChunk float4
  const SplitSet& as = sets.v[blockIdx.y];
  const int pbeg = blockIdx.x * kSaWarps * COLS;
  if (pbeg >= as.n) return;
  const float4* w4 = reinterpret_cast<const float4*>(as.w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n4 = KM / 4;                              // uint4 (4 complex) per column and plane
  const uint4* H = reinterpret_cast<const uint4*>(as.hi);
  const uint4* L = reinterpret_cast<const uint4*>(as.lo);
  if constexpr (WHOLE) {
    for (int t = threadIdx.x; t < 2 * n4; t += blockDim.x) s_w[t] = w4[t];
    __syncthreads();
    for (int cw = 0; cw < COLS; ++cw) {
      const int p = pbeg + warp * COLS + cw;
      if (p >= as.n) break;
      const int pix = as.idx[p];
      float g = 0.f, h_ = 0.f, l_ = 0.f;
      split_adj_accumulate<KIND, HI, LO, EXACT>(H, L, (size_t)pix * n4, n4, lane, s_w, g, h_, l_);
      split_adj_finish<EXACT>(as, sv, update, p, pix, lane, g, h_, l_);
    }
    return;
  }
  float cs[COLS], dh[COLS], dl[COLS];
  int pixs[COLS];
#pragma unroll
  for (int cw = 0; cw < COLS; ++cw) {
    cs[cw] = 0.f; dh[cw] = 0.f; dl[cw] = 0.f;
    const int p = pbeg + warp * COLS + cw;
    pixs[cw] = p < as.n ? as.idx[p] : -1;
  }
  for (int c0 = 0; c0 < n4; c0 += kSaChunk) {
    const int cn = min(kSaChunk, n4 - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * cn; t += blockDim.x) s_w[t] = w4[2 * c0 + t];
    __syncthreads();
#pragma unroll 1
    for (int cw = 0; cw < COLS; ++cw) {
      const int pix = pixs[cw];
      if (pix < 0) break;
      float g = cs[cw], h_ = dh[cw], l_ = dl[cw];
      split_adj_accumulate<KIND, HI, LO, EXACT>(H, L, (size_t)pix * n4 + c0, cn, lane, s_w, g, h_, l_);
      cs[cw] = g; dh[cw] = h_; dl[cw] = l_;
    }
  }
#pragma unroll 1
  for (int cw = 0; cw < COLS; ++cw) {
    const int pix = pixs[cw];
    if (pix < 0) break;
    split_adj_finish<EXACT>(as, sv, update, pbeg + warp * COLS + cw, pix, lane, cs[cw], dh[cw], dl[cw]);
  }
}

// -------------------------------------------------------------- conversion
template <int KIND>
__global__ void split_convert_kernel(const float* __restrict__ a, uint16_t* __restrict__ hi,
                                     uint16_t* __restrict__ lo, float* __restrict__ P, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float x = a[i];
    float pair;
    if constexpr (KIND == kSplitBF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      hi[i] = *reinterpret_cast<const uint16_t*>(&h);
      lo[i] = *reinterpret_cast<const uint16_t*>(&l);
      pair = __bfloat162float(h) + __bfloat162float(l);
    } else {
      const __half h = __float2half_rn(x);
      const __half l = __float2half_rn(x - __half2float(h));
      hi[i] = *reinterpret_cast<const uint16_t*>(&h);
      lo[i] = *reinterpret_cast<const uint16_t*>(&l);
      pair = __half2float(h) + __half2float(l);
    }
    if (P) P[i] = pair;
  }
}

template <int KIND, bool HI, bool LO>
int launch_split_forward_t(const SetBlock<SplitSet>& blk, int nsets, int KM, int chunks, int per, VMode mode,
                           const SolverView& sv, float2* partial, cudaStream_t st) {
  dim3 grid(div_up(KM, kSpRows), chunks, nsets);
  if (mode == kVCons)
    split_forward_partial_kernel<KIND, HI, LO, true><<<grid, kSpThreads, 0, st>>>(
        blk, KM, chunks, per, mode, sv, reinterpret_cast<float4*>(partial));
  else
    split_forward_partial_kernel<KIND, HI, LO, false><<<grid, kSpThreads, 0, st>>>(
        blk, KM, chunks, per, mode, sv, reinterpret_cast<float4*>(partial));
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// Fraction of the last wave that a grid of `blocks` CTAs fills, given the
// resident CTAs per SM of its kernel (0 if the query fails).
double last_wave_fill(const void* f, size_t smem, long long blocks) {
  static int sms = 0;
  if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  int r = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, f, kSaWarps * 32, smem) != cudaSuccess || r <= 0) {
    cudaGetLastError();
    return 0.0;
  }
  const long long wave = (long long)r * sms;
  return (double)blocks / (double)(div_up(blocks, wave) * wave);
}

// The chunked form takes eight or two columns per warp, whichever fills the
// last wave of resident CTAs better (by more than 2 %); the whole-w form eight.
template <int KIND, bool HI, bool LO, bool EXACT>
int launch_split_adjoint_e(const SetBlock<SplitSet>& blk, int nsets, int KM, int max_cols, bool update,
                           const SolverView& sv, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(split_adjoint_kernel<KIND, HI, LO, EXACT, false, 8>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    SADMM_CUDA_TRY(cudaFuncSetAttribute(split_adjoint_kernel<KIND, HI, LO, EXACT, false, 2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  const size_t smem = (size_t)std::min(KM / 4, kSaChunk) * 2 * sizeof(float4);
  if (KM / 4 <= kSaChunk) {
    dim3 grid(div_up(max_cols, kSaWarps * 8), nsets);
    split_adjoint_kernel<KIND, HI, LO, EXACT, true, 8><<<grid, kSaWarps * 32, smem, st>>>(blk, KM, update, sv);
  } else {
    const long long b8 = (long long)div_up(max_cols, kSaWarps * 8) * nsets;
    const long long b2 = (long long)div_up(max_cols, kSaWarps * 2) * nsets;
    const double f8 = last_wave_fill((const void*)split_adjoint_kernel<KIND, HI, LO, EXACT, false, 8>, smem, b8);
    const double f2 = last_wave_fill((const void*)split_adjoint_kernel<KIND, HI, LO, EXACT, false, 2>, smem, b2);
    if (f2 > f8 + 0.02) {
      dim3 grid(div_up(max_cols, kSaWarps * 2), nsets);
      split_adjoint_kernel<KIND, HI, LO, EXACT, false, 2><<<grid, kSaWarps * 32, smem, st>>>(blk, KM, update, sv);
    } else {
      dim3 grid(div_up(max_cols, kSaWarps * 8), nsets);
      split_adjoint_kernel<KIND, HI, LO, EXACT, false, 8><<<grid, kSaWarps * 32, smem, st>>>(blk, KM, update, sv);
    }
  }
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// exact double-float g when the sets ask for (g, g_lo) and no update
template <int KIND, bool HI, bool LO>
int launch_split_adjoint_t(const SetBlock<SplitSet>& blk, int nsets, int KM, int max_cols, bool update,
                           const SolverView& sv, cudaStream_t st) {
  if (blk.v[0].g_lo != nullptr && !update)
    return launch_split_adjoint_e<KIND, HI, LO, true>(blk, nsets, KM, max_cols, update, sv, st);
  return launch_split_adjoint_e<KIND, HI, LO, false>(blk, nsets, KM, max_cols, update, sv, st);
}

}  // namespace

size_t split_partial_bytes(int nsets, int KM, int max_cols) {
  return (size_t)nsets * split_chunks(nsets, KM, max_cols) * KM * sizeof(float2);
}

int launch_split_forward(const SplitSet* sets, int nsets, int KM, int kind, int planes, VMode mode,
                         const SolverView& sv, float2* partial, size_t partial_cap, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets || KM % 4 != 0 || planes < 1 || planes > 3 ||
      (kind != kSplitBF16 && kind != kSplitFP16)) {
    set_error("launch_split_forward: bad arguments");
    return SADMM_EINVAL;
  }
  SetBlock<SplitSet> blk;
  int max_cols = 0;
  for (int i = 0; i < nsets; ++i) { blk.v[i] = sets[i]; max_cols = max(max_cols, sets[i].n); }
  const int chunks = split_chunks(nsets, KM, max(max_cols, 1));
  const int per = max(1, div_up(max_cols, chunks));
  if ((size_t)nsets * chunks * KM * sizeof(float2) > partial_cap) {
    set_error("launch_split_forward: partial buffer too small");
    return SADMM_EINVAL;
  }
  // planes: 1 = hi only, 2 = lo only, 3 = hi + lo
  int rc;
  if (kind == kSplitBF16) {
    rc = planes == 3 ? launch_split_forward_t<kSplitBF16, true, true>(blk, nsets, KM, chunks, per, mode, sv, partial, st)
       : planes == 1 ? launch_split_forward_t<kSplitBF16, true, false>(blk, nsets, KM, chunks, per, mode, sv, partial, st)
                     : launch_split_forward_t<kSplitBF16, false, true>(blk, nsets, KM, chunks, per, mode, sv, partial, st);
  } else {
    rc = planes == 3 ? launch_split_forward_t<kSplitFP16, true, true>(blk, nsets, KM, chunks, per, mode, sv, partial, st)
       : planes == 1 ? launch_split_forward_t<kSplitFP16, true, false>(blk, nsets, KM, chunks, per, mode, sv, partial, st)
                     : launch_split_forward_t<kSplitFP16, false, true>(blk, nsets, KM, chunks, per, mode, sv, partial, st);
  }
  SADMM_TRY(rc);
  dim3 g2(div_up(KM / 2, 256), nsets);
  split_reduce_kernel<<<g2, 256, 0, st>>>(blk, KM, chunks, reinterpret_cast<const float4*>(partial));
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_split_adjoint(const SplitSet* sets, int nsets, int KM, int kind, int planes, bool update,
                         const SolverView& sv, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets || KM % 4 != 0 || KM > 16384 || planes < 1 || planes > 3 ||
      (kind != kSplitBF16 && kind != kSplitFP16)) {
    set_error("launch_split_adjoint: bad arguments");
    return SADMM_EINVAL;
  }
  SetBlock<SplitSet> blk;
  int max_cols = 0;
  for (int i = 0; i < nsets; ++i) { blk.v[i] = sets[i]; max_cols = max(max_cols, sets[i].n); }
  if (max_cols == 0) return SADMM_OK;
  if (kind == kSplitBF16) {
    return planes == 3 ? launch_split_adjoint_t<kSplitBF16, true, true>(blk, nsets, KM, max_cols, update, sv, st)
         : planes == 1 ? launch_split_adjoint_t<kSplitBF16, true, false>(blk, nsets, KM, max_cols, update, sv, st)
                       : launch_split_adjoint_t<kSplitBF16, false, true>(blk, nsets, KM, max_cols, update, sv, st);
  }
  return planes == 3 ? launch_split_adjoint_t<kSplitFP16, true, true>(blk, nsets, KM, max_cols, update, sv, st)
       : planes == 1 ? launch_split_adjoint_t<kSplitFP16, true, false>(blk, nsets, KM, max_cols, update, sv, st)
                     : launch_split_adjoint_t<kSplitFP16, false, true>(blk, nsets, KM, max_cols, update, sv, st);
}

int launch_split_convert(const float* A, size_t nfloats, int kind, uint16_t* hi, uint16_t* lo, cudaStream_t st,
                         float* P) {
  if (nfloats == 0) return SADMM_OK;
  const int grid = (int)std::min<size_t>(div_up((long long)nfloats, 256), 152 * 64);
  if (kind == kSplitBF16) split_convert_kernel<kSplitBF16><<<grid, 256, 0, st>>>(A, hi, lo, P, nfloats);
  else if (kind == kSplitFP16) split_convert_kernel<kSplitFP16><<<grid, 256, 0, st>>>(A, hi, lo, P, nfloats);
  else { set_error("launch_split_convert: bad kind"); return SADMM_EINVAL; }
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
