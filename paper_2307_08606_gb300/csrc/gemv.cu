// Column-compacted complex GEMVs over the active-pixel lists and the FP64
// SPD apply of the x-update factor (Eq. 1 products inside Eq. 3, x_q-update).
//
// Operators are pixel-major complex64: column n of A_q is KM contiguous float2.
// The forward product r = base - sum_{p} A[:, idx[p]] v[idx[p]] streams the
// listed columns once; each CTA owns a 256-row slice of one column chunk and
// keeps its partial sum in registers, the per-column scalars v are staged in
// shared memory, and a second kernel reduces the chunk partials in a fixed
// order (deterministic).  The adjoint g[p] = Re(a_{idx[p]}^H w) gives one warp
// per column with w staged in shared memory and a shuffle reduction.
#include "common.cuh"
#include "symtile.cuh"

#include <algorithm>

namespace sadmm {

namespace {

using symtile::DF;
using symtile::df_add;
using symtile::df_add1;
using symtile::df_mul_acc;
using symtile::df_norm;

constexpr int kFwdThreads = 128;          // one float4 (2 complex rows) per thread
constexpr int kFwdRows = 2 * kFwdThreads; // complex rows per CTA slice
constexpr int kFwdStage = 512;            // columns staged per shared-memory batch
constexpr int kFwdUnroll = 8;

// Read-only streaming load of an operator element pair (evict-first in L1).
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

template <bool CONS>
__global__ void __launch_bounds__(kFwdThreads)
forward_partial_kernel(const __grid_constant__ SetBlock<ColumnSet> sets, int KM, int chunks,
                       int cols_per_chunk, VMode mode, const __grid_constant__ SolverView sv,
                       float4* __restrict__ partial) {
  const ColumnSet& cs = sets.v[blockIdx.z];
  const int c = blockIdx.y;
  const int p0 = c * cols_per_chunk;
  const int p1 = min(cs.n, p0 + cols_per_chunk);
  const int row2 = blockIdx.x * kFwdThreads + threadIdx.x;   // float4 index within a column
  const bool active_row = row2 * 2 < KM;
  __shared__ float s_v[kFwdStage];
  __shared__ int s_off[kFwdStage];
  // Eight products per component are summed in FP32 and each such partial
  // goes into a double-float accumulator: near convergence B v almost cancels
  // y, and FP32 accumulation over thousands of columns would lose the digits
  // of the residual that the x-update needs.
  DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const float4* A4 = reinterpret_cast<const float4*>(cs.A);
  const size_t col4 = (size_t)KM / 2;                        // float4 per column
  for (int b0 = p0; b0 < p1; b0 += kFwdStage) {
    const int nb = min(kFwdStage, p1 - b0);
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += kFwdThreads) {
      const int pix = cs.idx[b0 + t];
      s_v[t] = v_col<CONS>(mode, sv, cs.q, pix, cs.vexp);
      s_off[t] = pix;
    }
    __syncthreads();
    if (active_row) {
      int j = 0;
      for (; j + kFwdUnroll <= nb; j += kFwdUnroll) {
        float4 a[kFwdUnroll];
#pragma unroll
        for (int u = 0; u < kFwdUnroll; ++u)
          a[u] = ld_stream(A4 + (size_t)s_off[j + u] * col4 + row2);
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kFwdUnroll; ++u) {
          const float v = s_v[j + u];
          t.x = fmaf(a[u].x, v, t.x);
          t.y = fmaf(a[u].y, v, t.y);
          t.z = fmaf(a[u].z, v, t.z);
          t.w = fmaf(a[u].w, v, t.w);
        }
        df_add1(acc[0], t.x);
        df_add1(acc[1], t.y);
        df_add1(acc[2], t.z);
        df_add1(acc[3], t.w);
      }
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      for (; j < nb; ++j) {
        const float4 a = ld_stream(A4 + (size_t)s_off[j] * col4 + row2);
        const float v = s_v[j];
        t.x = fmaf(a.x, v, t.x);
        t.y = fmaf(a.y, v, t.y);
        t.z = fmaf(a.z, v, t.z);
        t.w = fmaf(a.w, v, t.w);
      }
      df_add1(acc[0], t.x);
      df_add1(acc[1], t.y);
      df_add1(acc[2], t.z);
      df_add1(acc[3], t.w);
    }
  }
  if (active_row) {
    // chunk partial as a pair of float4 planes: high words, then low words
    float4* out = partial + ((size_t)blockIdx.z * chunks + c) * 2 * col4 + row2;
    DF n[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) n[k] = df_norm(acc[k]);
    out[0] = make_float4(n[0].hi, n[1].hi, n[2].hi, n[3].hi);
    out[col4] = make_float4(n[0].lo, n[1].lo, n[2].lo, n[3].lo);
  }
}

// out[r] = base[r] - sum_c partial[c][r].  Four threads per float4 of rows:
// thread part p adds chunks p, p + 4, p + 8, ... in double-float, and the
// four sums are added in the order 0, 1, 2, 3.
constexpr int kRedParts = 4;
constexpr int kRedRows = 64;                 // float4 rows per CTA

__global__ void __launch_bounds__(kRedRows * kRedParts)
forward_reduce_kernel(const __grid_constant__ SetBlock<ColumnSet> sets, int KM, int chunks,
                      const float4* __restrict__ partial) {
  const ColumnSet& cs = sets.v[blockIdx.y];
  const int part = threadIdx.x % kRedParts;
  const int row2 = blockIdx.x * kRedRows + threadIdx.x / kRedParts;
  const bool live = row2 * 2 < KM;
  const size_t col4 = (size_t)KM / 2;
  const float4* p = partial + (size_t)blockIdx.y * chunks * 2 * col4 + row2;
  DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  constexpr int kB = 3;                 // chunk loads issued ahead of their sums
  if (live) {
    for (int c0 = part; c0 < chunks; c0 += kB * kRedParts) {
      float4 h[kB], l[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int c = c0 + u * kRedParts;
        h[u] = l[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < chunks) {
          h[u] = p[(size_t)c * 2 * col4];
          l[u] = p[(size_t)c * 2 * col4 + col4];
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        df_add(acc[0], DF{h[u].x, l[u].x});
        df_add(acc[1], DF{h[u].y, l[u].y});
        df_add(acc[2], DF{h[u].z, l[u].z});
        df_add(acc[3], DF{h[u].w, l[u].w});
      }
    }
  }
  // parts 1, 2, 3 of this row join part 0, in order
  DF tot[4] = {acc[0], acc[1], acc[2], acc[3]};
#pragma unroll
  for (int o = 1; o < kRedParts; ++o) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const DF x{__shfl_down_sync(0xffffffffu, acc[k].hi, o), __shfl_down_sync(0xffffffffu, acc[k].lo, o)};
      if (part == 0) df_add(tot[k], x);
    }
  }
  if (!live || part != 0) return;
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
  if (cs.base) b = reinterpret_cast<const float4*>(cs.base)[row2];
  // r = b - (sum), formed in double-float and rounded once
  const float bb[4] = {b.x, b.y, b.z, b.w};
  float r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    DF d{-tot[k].hi, -tot[k].lo};
    df_add1(d, bb[k]);
    r[k] = d.hi + d.lo;
  }
  reinterpret_cast<float4*>(cs.out)[row2] = make_float4(r[0], r[1], r[2], r[3]);
}

int forward_chunks(int nsets, int KM, int max_cols) {
  const int tiles = div_up(KM, kFwdRows);
  int want = div_up(152 * 16, (long long)tiles * nsets);        // ~2 waves at full occupancy
  int cap = div_up(max_cols, 64);                                // >= 64 columns per chunk
  return max(1, min(want, cap));
}

// ------------------------------------------------------------------ adjoint
constexpr int kAdjWarps = 8;
// columns per warp: 8 in the whole-w form; 8, 4 or 2 in the chunked form,
// chosen per launch so that the last wave of CTAs is as full as possible
// (pick_adjoint_cols: at KM = 16384, N = 128^2, Q = 8, 2048 CTAs of 64 columns
// filled 2.25 waves of 912 resident CTAs; 8192 CTAs of 16 fill 8.98, and the
// adjoint went from 3.03 to 2.61 ms)
constexpr int kAdjUnroll = 4;
constexpr int kAdjWChunk = 2048;      // float4 of w staged at once (4096 complex, 32 KB)

// EXACT (mode g only): every product is formed exactly and added with an
// error-free two-sum, and g leaves as the pair (g, g_lo).  The primal
// x-update x = v + mu H g weights g by H = (rho I + mu B^T B)^{-1}, whose
// condition number is that of rho I + mu B^T B: where B^T B is (nearly)
// singular, any error in g outside the range of B^T is amplified by up to that
// factor, so g must be exact to double-float accuracy there.
// Whole-w form (w fits one staged chunk): each warp sums its columns in one
// pass over the rows.
template <bool EXACT, int COLS>
__global__ void __launch_bounds__(kAdjWarps * 32)
adjoint_whole_kernel(const __grid_constant__ SetBlock<AdjointSet> sets, int KM, bool update,
               const __grid_constant__ SolverView sv) {
  extern __shared__ float4 s_w4[];               // KM/2 float4 = KM complex (KM/2 <= kAdjWChunk)
  const AdjointSet& as = sets.v[blockIdx.y];
  const int cols_per_cta = kAdjWarps * COLS;
  const int pbeg = blockIdx.x * cols_per_cta;
  if (pbeg >= as.n) return;
  const int n4 = KM / 2;
  const float4* w4 = reinterpret_cast<const float4*>(as.w);
  for (int t = threadIdx.x; t < n4; t += blockDim.x) s_w4[t] = w4[t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float4* A4 = reinterpret_cast<const float4*>(as.A);
  for (int cw = 0; cw < COLS; ++cw) {
    const int p = pbeg + warp * COLS + cw;
    if (p >= as.n) break;
    const int pix = as.idx[p];
    const float4* col = A4 + (size_t)pix * n4;
    // Each float4 (two complex entries, four real products) is summed in FP32
    // and the partial goes into a double-float accumulator: the sum over the
    // 2KM real rows cancels heavily (|x| is far below sum |b||w|), and plain
    // FP32 accumulation over thousands of terms loses about three digits.
    DF acc[kAdjUnroll];
#pragma unroll
    for (int u = 0; u < kAdjUnroll; ++u) acc[u] = DF{0.f, 0.f};
    int i = lane;
    for (; i + 32 * (kAdjUnroll - 1) < n4; i += 32 * kAdjUnroll) {
      float4 a[kAdjUnroll];
#pragma unroll
      for (int u = 0; u < kAdjUnroll; ++u) a[u] = ld_stream(col + i + 32 * u);
#pragma unroll
      for (int u = 0; u < kAdjUnroll; ++u) {
        const float4 w = s_w4[i + 32 * u];
        if (EXACT) {
          df_mul_acc(acc[u], a[u].x, w.x);
          df_mul_acc(acc[u], a[u].y, w.y);
          df_mul_acc(acc[u], a[u].z, w.z);
          df_mul_acc(acc[u], a[u].w, w.w);
        } else {
          float t = a[u].x * w.x;
          t = fmaf(a[u].y, w.y, t);
          t = fmaf(a[u].z, w.z, t);
          t = fmaf(a[u].w, w.w, t);
          df_add1(acc[u], t);
        }
      }
    }
    for (; i < n4; i += 32) {
      const float4 a = ld_stream(col + i);
      const float4 w = s_w4[i];
      if (EXACT) {
        df_mul_acc(acc[0], a.x, w.x);
        df_mul_acc(acc[0], a.y, w.y);
        df_mul_acc(acc[0], a.z, w.z);
        df_mul_acc(acc[0], a.w, w.w);
      } else {
        float t = a.x * w.x;
        t = fmaf(a.y, w.y, t);
        t = fmaf(a.z, w.z, t);
        t = fmaf(a.w, w.w, t);
        df_add1(acc[0], t);
      }
    }
#pragma unroll
    for (int u = 1; u < kAdjUnroll; ++u) df_add(acc[0], acc[u]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DF b{__shfl_xor_sync(0xffffffffu, acc[0].hi, o), __shfl_xor_sync(0xffffffffu, acc[0].lo, o)};
      df_add(acc[0], b);
    }
    const float g = acc[0].hi + acc[0].lo;
    if (lane == 0) {
      if (update) {
        // x-update epilogue (Woodbury form): x = v + mu Re(a^H w)
        const size_t xi = (size_t)as.q * sv.N + pix;
        const float xo = sv.x[xi];
        const float v = v_admm(sv, as.q, pix, xo);
        const float xn = fmaf(sv.mu, g, v);
        sv.ring[((size_t)sv.slot * sv.Q + as.q) * sv.N + pix] = xn - xo;
        sv.x[xi] = xn;
      } else if (EXACT) {
        const DF o = df_norm(acc[0]);
        as.g[p] = o.hi;
        as.g_lo[p] = o.lo;
      } else {
        as.g[p] = g;
      }
    }
  }
}

// Chunked form (large KM): w is staged in chunks; each warp keeps its
// columns' double-float sums across the chunks.
template <bool EXACT, int COLS>
__global__ void __launch_bounds__(kAdjWarps * 32)
adjoint_kernel(const __grid_constant__ SetBlock<AdjointSet> sets, int KM, bool update,
               const __grid_constant__ SolverView sv) {
  extern __shared__ float4 s_w4[];               // one chunk of w: up to kAdjWChunk float4
  const AdjointSet& as = sets.v[blockIdx.y];
  const int cols_per_cta = kAdjWarps * COLS;
  const int pbeg = blockIdx.x * cols_per_cta;
  if (pbeg >= as.n) return;
  const int n4 = KM / 2;
  const float4* w4 = reinterpret_cast<const float4*>(as.w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float4* A4 = reinterpret_cast<const float4*>(as.A);
  // per column of this warp, the double-float sum over the chunks done so far
  DF colacc[COLS];
  int pixs[COLS];
#pragma unroll
  for (int cw = 0; cw < COLS; ++cw) {
    colacc[cw] = DF{0.f, 0.f};
    const int p = pbeg + warp * COLS + cw;
    pixs[cw] = p < as.n ? as.idx[p] : -1;
  }
  // w is staged in chunks so that large KM keeps several CTAs per SM resident
  for (int c0 = 0; c0 < n4; c0 += kAdjWChunk) {
    const int cn = min(kAdjWChunk, n4 - c0);
    __syncthreads();                             // the previous chunk is consumed
    for (int t = threadIdx.x; t < cn; t += blockDim.x) s_w4[t] = w4[c0 + t];
    __syncthreads();
#pragma unroll 1
    for (int cw = 0; cw < COLS; ++cw) {
      const int pix = pixs[cw];
      if (pix < 0) break;
      const float4* col = A4 + (size_t)pix * n4 + c0;
      // Each float4 (two complex entries, four real products) is summed in FP32
      // and the partial goes into a double-float accumulator: the sum over the
      // 2KM real rows cancels heavily (|x| is far below sum |b||w|), and plain
      // FP32 accumulation over thousands of terms loses about three digits.
      DF acc[kAdjUnroll];
#pragma unroll
      for (int u = 0; u < kAdjUnroll; ++u) acc[u] = DF{0.f, 0.f};
      int i = lane;
      for (; i + 32 * (kAdjUnroll - 1) < cn; i += 32 * kAdjUnroll) {
        float4 a[kAdjUnroll];
#pragma unroll
        for (int u = 0; u < kAdjUnroll; ++u) a[u] = ld_stream(col + i + 32 * u);
#pragma unroll
        for (int u = 0; u < kAdjUnroll; ++u) {
          const float4 w = s_w4[i + 32 * u];
          if (EXACT) {
            df_mul_acc(acc[u], a[u].x, w.x);
            df_mul_acc(acc[u], a[u].y, w.y);
            df_mul_acc(acc[u], a[u].z, w.z);
            df_mul_acc(acc[u], a[u].w, w.w);
          } else {
            float t = a[u].x * w.x;
            t = fmaf(a[u].y, w.y, t);
            t = fmaf(a[u].z, w.z, t);
            t = fmaf(a[u].w, w.w, t);
            df_add1(acc[u], t);
          }
        }
      }
      for (; i < cn; i += 32) {
        const float4 a = ld_stream(col + i);
        const float4 w = s_w4[i];
        if (EXACT) {
          df_mul_acc(acc[0], a.x, w.x);
          df_mul_acc(acc[0], a.y, w.y);
          df_mul_acc(acc[0], a.z, w.z);
          df_mul_acc(acc[0], a.w, w.w);
        } else {
          float t = a.x * w.x;
          t = fmaf(a.y, w.y, t);
          t = fmaf(a.z, w.z, t);
          t = fmaf(a.w, w.w, t);
          df_add1(acc[0], t);
        }
      }
#pragma unroll
      for (int u = 1; u < kAdjUnroll; ++u) df_add(acc[0], acc[u]);
      df_add(colacc[cw], acc[0]);
    }
  }
#pragma unroll 1
  for (int cw = 0; cw < COLS; ++cw) {
    const int pix = pixs[cw];
    if (pix < 0) break;
    const int p = pbeg + warp * COLS + cw;
    DF tot = colacc[cw];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DF b{__shfl_xor_sync(0xffffffffu, tot.hi, o), __shfl_xor_sync(0xffffffffu, tot.lo, o)};
      df_add(tot, b);
    }
    const float g = tot.hi + tot.lo;
    if (lane == 0) {
      if (update) {
        // x-update epilogue (Woodbury form): x = v + mu Re(a^H w)
        const size_t xi = (size_t)as.q * sv.N + pix;
        const float xo = sv.x[xi];
        const float v = v_admm(sv, as.q, pix, xo);
        const float xn = fmaf(sv.mu, g, v);
        sv.ring[((size_t)sv.slot * sv.Q + as.q) * sv.N + pix] = xn - xo;
        sv.x[xi] = xn;
      } else if (EXACT) {
        const DF o = df_norm(tot);
        as.g[p] = o.hi;
        as.g_lo[p] = o.lo;
      } else {
        as.g[p] = g;
      }
    }
  }
}

}  // namespace

size_t forward_partial_bytes(int nsets, int KM, int max_cols) {
  return (size_t)nsets * forward_chunks(nsets, KM, max_cols) * 2 * KM * sizeof(float2);   // (hi, lo) planes
}

int launch_forward(const ColumnSet* sets, int nsets, int KM, VMode mode, const SolverView& sv,
                   float2* partial, size_t partial_cap, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets) { set_error("launch_forward: %d sets > %d", nsets, kMaxSets); return SADMM_EINVAL; }
  SetBlock<ColumnSet> blk;
  int max_cols = 0;
  for (int i = 0; i < nsets; ++i) { blk.v[i] = sets[i]; max_cols = max(max_cols, sets[i].n); }
  const int chunks = forward_chunks(nsets, KM, max(max_cols, 1));
  const int per = max(1, div_up(max_cols, chunks));
  if (forward_partial_bytes(nsets, KM, max(max_cols, 1)) > partial_cap) {
    set_error("launch_forward: partial buffer too small");
    return SADMM_EINVAL;
  }
  dim3 grid(div_up(KM, kFwdRows), chunks, nsets);
  if (mode == kVCons)
    forward_partial_kernel<true><<<grid, kFwdThreads, 0, st>>>(blk, KM, chunks, per, mode, sv,
                                                               reinterpret_cast<float4*>(partial));
  else
    forward_partial_kernel<false><<<grid, kFwdThreads, 0, st>>>(blk, KM, chunks, per, mode, sv,
                                                                reinterpret_cast<float4*>(partial));
  SADMM_LAUNCH_CHECK();
  return launch_forward_reduce(sets, nsets, KM, chunks, partial, st);
}

int launch_forward_reduce(const ColumnSet* sets, int nsets, int KM, int chunks, const float2* partial,
                          cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets) { set_error("launch_forward_reduce: %d sets > %d", nsets, kMaxSets); return SADMM_EINVAL; }
  SetBlock<ColumnSet> blk;
  for (int i = 0; i < nsets; ++i) blk.v[i] = sets[i];
  dim3 g2(div_up(KM / 2, kRedRows), nsets);
  forward_reduce_kernel<<<g2, kRedRows * kRedParts, 0, st>>>(blk, KM, chunks,
                                                            reinterpret_cast<const float4*>(partial));
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

template <int C>
int configure_adjoint() {
  SADMM_CUDA_TRY(cudaFuncSetAttribute(adjoint_kernel<false, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  SADMM_CUDA_TRY(cudaFuncSetAttribute(adjoint_kernel<true, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  return SADMM_OK;
}

template <int C>
int adjoint_resident(bool whole, bool exact, size_t smem) {
  int r = 0;
  const void* f = whole ? (exact ? (const void*)adjoint_whole_kernel<true, C> : (const void*)adjoint_whole_kernel<false, C>)
                        : (exact ? (const void*)adjoint_kernel<true, C> : (const void*)adjoint_kernel<false, C>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, f, kAdjWarps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return r;
}

// Columns per warp for an adjoint launch: of 8, 4 and 2, the one whose grid
// fills its last wave of resident CTAs best (a fuller wave by more than 2 %
// wins; otherwise the larger group, which stages w fewer times).
int pick_adjoint_cols(bool whole, bool exact, size_t smem, int max_cols, int nsets) {
  static int sms = 0;
  if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const int cand[3] = {8, 4, 2};
  const int res[3] = {adjoint_resident<8>(whole, exact, smem), adjoint_resident<4>(whole, exact, smem),
                      adjoint_resident<2>(whole, exact, smem)};
  int best = 8;
  double best_eff = -1.0;
  for (int c = 0; c < 3; ++c) {
    if (res[c] <= 0) continue;
    const long long blocks = (long long)div_up(max_cols, kAdjWarps * cand[c]) * nsets;
    const long long wave = (long long)res[c] * sms;
    const double eff = (double)blocks / (double)(div_up(blocks, wave) * wave);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = cand[c];
    }
  }
  return best;
}

int launch_adjoint(const AdjointSet* sets, int nsets, int KM, bool update, const SolverView& sv,
                   cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets) { set_error("launch_adjoint: too many sets"); return SADMM_EINVAL; }
  SetBlock<AdjointSet> blk;
  int max_cols = 0;
  for (int i = 0; i < nsets; ++i) { blk.v[i] = sets[i]; max_cols = max(max_cols, sets[i].n); }
  if (max_cols == 0) return SADMM_OK;
  const bool exact = !update && sets[0].g_lo != nullptr;
  for (int i = 1; i < nsets; ++i)
    if ((sets[i].g_lo != nullptr) != (sets[0].g_lo != nullptr)) {
      set_error("launch_adjoint: sets mix exact and plain outputs");
      return SADMM_EINVAL;
    }
  const size_t smem = (size_t)std::min(KM / 2, kAdjWChunk) * sizeof(float4);
  static bool configured = false;
  if (!configured) {
    SADMM_TRY(configure_adjoint<8>());
    SADMM_TRY(configure_adjoint<4>());
    SADMM_TRY(configure_adjoint<2>());
    configured = true;
  }
  const bool whole = KM / 2 <= kAdjWChunk;
  // whole-w form: eight columns per warp (smaller groups re-stage w per CTA
  // and measured slower at KM = 2048); chunked form: the fullest last wave
  const int cols = whole ? 8 : pick_adjoint_cols(whole, exact, smem, max_cols, nsets);
  dim3 grid(div_up(max_cols, kAdjWarps * cols), nsets);
#define SADMM_ADJ_LAUNCH(C)                                                                              \
  if (whole) {                                                                                           \
    if (exact) adjoint_whole_kernel<true, C><<<grid, kAdjWarps * 32, smem, st>>>(blk, KM, update, sv);  \
    else adjoint_whole_kernel<false, C><<<grid, kAdjWarps * 32, smem, st>>>(blk, KM, update, sv);       \
  } else {                                                                                               \
    if (exact) adjoint_kernel<true, C><<<grid, kAdjWarps * 32, smem, st>>>(blk, KM, update, sv);        \
    else adjoint_kernel<false, C><<<grid, kAdjWarps * 32, smem, st>>>(blk, KM, update, sv);             \
  }
  if (cols == 8) { SADMM_ADJ_LAUNCH(8) }
  else if (cols == 4) { SADMM_ADJ_LAUNCH(4) }
  else { SADMM_ADJ_LAUNCH(2) }
#undef SADMM_ADJ_LAUNCH
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm

// ---------------------------------------------------------------------------
// Allocation-free forward product (sadmm_forward_noalloc).
//
// Some callers cannot allocate device memory once they are running: a
// real-time radar front end with a fixed per-frame latency budget (where a
// cudaMalloc / cudaFree can synchronise the device and stall the pipeline), or
// a host process whose device memory is handed out by another allocator under
// a fixed budget.  For them the forward product's chunk partial sums live in
// one file-scope device array instead of memory allocated per call.  The
// array is created when a GPU loads this library and is held until the process
// exits; all calls on that GPU share it.
namespace sadmm {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB per GPU
__device__ __align__(256) float4 g_noalloc_partial[kNoAllocScratchBytes / sizeof(float4)];

// Device address of the scratch array on the current device.  Host code must
// not use the array's name as a pointer: it only stands for the symbol.  The
// address is looked up on every call, with the calling device current, so a
// device reset or a new primary context never leaves a stale address behind;
// the lookup allocates nothing.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  SADMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partial));
  *out = p;
  return SADMM_OK;
}

}  // namespace
}  // namespace sadmm

extern "C" int sadmm_forward_noalloc(const float* A, int KM, int N, const int* idx, int nidx,
                                     const float* v, const float* base, float* r, void* stream) {
  using namespace sadmm;
  if (!A || !r || KM <= 0 || KM % 2 != 0 || N <= 0 || nidx < 0 || (nidx > 0 && (!idx || !v))) {
    set_error("sadmm_forward_noalloc: bad arguments");
    return SADMM_EINVAL;
  }
  const size_t need = forward_partial_bytes(1, KM, nidx > 0 ? nidx : 1);
  if (need > kNoAllocScratchBytes) {
    set_error("sadmm_forward_noalloc: KM=%d with %d columns needs %zu bytes of partial sums, "
              "more than the %zu-byte fixed scratch; use sadmm_forward",
              KM, nidx, need, kNoAllocScratchBytes);
    return SADMM_EINVAL;
  }
  void* scratch = nullptr;
  SADMM_TRY(noalloc_scratch(&scratch));
  ColumnSet cs{(const float2*)A, idx, nidx, 0, v, (const float2*)base, (float2*)r};
  SolverView sv{};
  return launch_forward(&cs, 1, KM, kVExplicit, sv, (float2*)scratch, kNoAllocScratchBytes,
                        (cudaStream_t)stream);
}
