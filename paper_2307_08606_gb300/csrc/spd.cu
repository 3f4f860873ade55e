// Symmetric factor apply out = F u (Eq. 3, x_q-update: the Woodbury matrix W
// or the primal inverse H), for F symmetric positive definite held as
// double-float pairs (hi, lo) with hi = fl32(F), lo = fl32(F - hi).
//
// Precision.  The residual u lies mostly where F is small, so |F u| is far
// below sum |F||u| and plain FP32 loses several digits, while GB300's FP64
// pipe is too slow for a per-iteration pass.  Every product is formed exactly
// in FP32 (p + e = hi u via FMA, plus the small lo u term) and accumulated as
// an unevaluated FP32 pair with the error-free two-sum (Knuth), about 48
// significant bits.
//
// Layout and traffic.  Only the upper triangle is stored, in 64 x 64 tiles
// (I <= J, row-block-major; each tile row-major and contiguous, zero-padded
// past n), so one iteration streams n^2/2 pairs instead of n^2.  A tile (I, J)
// contributes F_IJ u_J to block row I and, off the diagonal, F_IJ^T u_I to
// block row J.  Persistent CTAs (six per SM, so that one CTA's copy overlaps
// the others' arithmetic) pull tiles with one bulk asynchronous copy each
// (cp.async.bulk into shared memory, completion on an mbarrier), then 64
// threads form the row sums and 64 the column sums of the tile: the row
// threads read column pairs as one 16-byte load along skewed diagonals, the
// column threads walk the rows in order (their loads hit distinct banks by
// column and their u values are broadcasts), so that shared-memory accesses
// do not conflict.  Per-tile partial sums (pairs) go to a scratch buffer; a second
// kernel adds them in a fixed order and applies the epilogue.
#include "common.cuh"
#include "symtile.cuh"

namespace sadmm {
namespace {

using namespace symtile;
constexpr int kTileBytes = kT * kT * (int)sizeof(float2);

// Polls of the tile-copy wait before the apply gives up (sadmm_set_wait_limit
// lowers it so that tests can make the wait run out; the drain wait that
// follows a timeout always uses the full limit).
__device__ long long g_spd_wait_limit = kWaitLimit;
constexpr int kSpdThreads = 2 * kT;           // 64 row threads + 64 column threads

// item -> (set, tile): items are numbered set after set
__device__ __forceinline__ int item_set(const SetBlock<SpdSet>& sets, int nsets, int item, int& t) {
  int s = 0;
  while (s + 1 < nsets && item >= sets.v[s + 1].tile0) ++s;
  t = item - sets.v[s].tile0;
  return s;
}

// ULO: the input is the pair u + u_lo (every set of the launch has u_lo).
template <bool ULO>
__global__ void __launch_bounds__(kSpdThreads)
spd_tile_kernel(const __grid_constant__ SetBlock<SpdSet> sets, int nsets, int items, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);           // 64 x 64 pairs
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(16) float s_u[2][kT];                    // u_I, u_J
  __shared__ __align__(16) float s_ul[ULO ? 2 : 1][ULO ? kT : 4];  // their low words (ULO)
  const int tid = threadIdx.x;
  const int lt = tid;                                            // < 64: row lt, else column lt - 64
  if ((int)blockIdx.x >= items) return;
  if (tid == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned phase = 0u;
  const int r = lt & (kT - 1);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    int t, s = item_set(sets, nsets, item, t);
    const SpdSet& ss = sets.v[s];
    const int nt = ntiles_side(ss.n);
    int I, J;
    tile_ij(t, nt, I, J);
    // the previous tile is consumed (closing barrier): reuse the buffer
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_load(tile, ss.P + (size_t)t * kT * kT, kTileBytes, &bar);
    }
    {
      const int blk = lt < kT ? I : J;
      const int i = blk * kT + r;
      s_u[lt >> 6][r] = i < ss.n ? ss.u[i] : 0.f;
      if (ULO) s_ul[lt >> 6][r] = i < ss.n ? ss.u_lo[i] : 0.f;
    }
    __syncthreads();                                   // s_u written
    const bool ok = mbar_wait(&bar, phase, g_spd_wait_limit);
    if (!__syncthreads_and(ok)) {
      // give up on this apply, but only after the one copy in flight (the one
      // that timed out) has landed: it writes this CTA's shared memory, which
      // must stay allocated until then (bounded by the full limit)
      if (tid == 0) {
        mbar_wait(&bar, phase);
        atomicExch(err, 1);
      }
      return;
    }
    phase ^= 1u;
    DF acc0{0.f, 0.f}, acc1{0.f, 0.f};
    if (lt < kT) {
      // row r of F_IJ times u_J, two columns per 16-byte load: pairs
      // (b, b + 1) with b = (2r + c) mod 64, so that the eight threads of a
      // quarter-warp hit eight different bank groups
      const float* uJ = s_u[1];
      const float4* row = reinterpret_cast<const float4*>(tile + r * kT);
#pragma unroll 8
      for (int c = 0; c < kT; c += 4) {
        const int b0 = (2 * r + c) & (kT - 2), b1 = (2 * r + c + 2) & (kT - 2);
        const float4 f0 = row[b0 >> 1], f1 = row[b1 >> 1];
        const float2 u0 = *reinterpret_cast<const float2*>(uJ + b0);
        const float2 u1 = *reinterpret_cast<const float2*>(uJ + b1);
        if (ULO) {
          const float2 l0 = *reinterpret_cast<const float2*>(&s_ul[1][b0]);
          const float2 l1 = *reinterpret_cast<const float2*>(&s_ul[1][b1]);
          df_acc2(acc0, f0.x, f0.y, u0.x, l0.x);
          df_acc2(acc0, f0.z, f0.w, u0.y, l0.y);
          df_acc2(acc1, f1.x, f1.y, u1.x, l1.x);
          df_acc2(acc1, f1.z, f1.w, u1.y, l1.y);
        } else {
          df_acc(acc0, f0.x, f0.y, u0.x);
          df_acc(acc0, f0.z, f0.w, u0.y);
          df_acc(acc1, f1.x, f1.y, u1.x);
          df_acc(acc1, f1.z, f1.w, u1.y);
        }
      }
    } else if (I != J) {
      // column r of F_IJ times u_I (the transposed contribution to block row
      // J): every thread reads row i of the tile at its own column, so the
      // loads are conflict-free and u_I[i] is a broadcast
      const float* uI = s_u[0];
#pragma unroll 4
      for (int i = 0; i < kT; i += 4) {
        const float4 u4 = *reinterpret_cast<const float4*>(uI + i);
        const float2 f0 = tile[i * kT + r], f1 = tile[(i + 1) * kT + r];
        const float2 f2 = tile[(i + 2) * kT + r], f3 = tile[(i + 3) * kT + r];
        if (ULO) {
          const float4 l4 = *reinterpret_cast<const float4*>(&s_ul[0][i]);
          df_acc2(acc0, f0.x, f0.y, u4.x, l4.x);
          df_acc2(acc1, f1.x, f1.y, u4.y, l4.y);
          df_acc2(acc0, f2.x, f2.y, u4.z, l4.z);
          df_acc2(acc1, f3.x, f3.y, u4.w, l4.w);
        } else {
          df_acc(acc0, f0.x, f0.y, u4.x);
          df_acc(acc1, f1.x, f1.y, u4.y);
          df_acc(acc0, f2.x, f2.y, u4.z);
          df_acc(acc1, f3.x, f3.y, u4.w);
        }
      }
    }
    df_add(acc0, acc1);
    const DF o = df_norm(acc0);
    ss.part[(size_t)t * 2 * kT + lt] = make_float2(o.hi, o.lo);
    __syncthreads();                                   // tile and s_u consumed
  }
}

// out_I[i] = sum_{J >= I} row part of tile (I, J) + sum_{J < I} column part of
// tile (J, I), in a fixed order; then the epilogue.
__global__ void __launch_bounds__(kT)
spd_reduce_kernel(const __grid_constant__ SetBlock<SpdSet> sets, bool update, const __grid_constant__ SolverView sv) {
  const SpdSet& ss = sets.v[blockIdx.y];
  const int nt = ntiles_side(ss.n);
  const int I = blockIdx.x;
  if (I >= nt) return;
  const int i = I * kT + threadIdx.x;
  DF acc{0.f, 0.f};
  constexpr int kB = 8;                 // loads issued ahead of their sums
  for (int J0 = 0; J0 < nt; J0 += kB) {
    float2 p[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int J = J0 + u;
      p[u] = make_float2(0.f, 0.f);
      if (J < nt) {
        const int a = min(I, J), b = max(I, J);
        const int t = tile_index(a, b, nt);
        p[u] = ss.part[(size_t)t * 2 * kT + (J >= I ? 0 : kT) + threadIdx.x];
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) df_add(acc, DF{p[u].x, p[u].y});
  }
  if (i >= ss.n) return;
  const float g = acc.hi + acc.lo;
  if (update) {
    // x-update epilogue (primal form): x_J = v_J + mu H g
    const int pix = ss.idx[i];
    const size_t xi = (size_t)ss.q * sv.N + pix;
    const float xo = sv.x[xi];
    const float v = v_admm(sv, ss.q, pix, xo);
    const float xn = fmaf(sv.mu, g, v);
    sv.ring[((size_t)sv.slot * sv.Q + ss.q) * sv.N + pix] = xn - xo;
    sv.x[xi] = xn;
  } else if (ss.outd) {
    ss.outd[(size_t)i * ss.ldd] = (double)acc.hi + (double)acc.lo;
  } else {
    ss.out[i] = g;
  }
}

__global__ void pack_sym_kernel(const double* __restrict__ F, int ld, int n, float2* __restrict__ P) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  const int nt = ntiles_side(n);
  const size_t t = tile_index(I, J, nt);
  float2* out = P + t * kT * kT;
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
    const int r = I * kT + e / kT, c = J * kT + e % kT;
    const double x = (r < n && c < n) ? F[(size_t)r * ld + c] : 0.0;
    const float h = (float)x;
    out[e] = make_float2(h, (float)(x - (double)h));
  }
}

}  // namespace

int set_spd_wait_limit(long long polls) {
  const long long v = polls < 0 ? kWaitLimit : polls;
  SADMM_CUDA_TRY(cudaMemcpyToSymbol(g_spd_wait_limit, &v, sizeof(v)));
  return SADMM_OK;
}

size_t sym_packed_pairs(int n) {
  const size_t nt = ntiles_side(n);
  return nt * (nt + 1) / 2 * kT * kT;
}

size_t sym_part_pairs(int n) {
  const size_t nt = ntiles_side(n);
  return nt * (nt + 1) / 2 * 2 * kT;
}

int launch_pack_sym(const double* F, int ld, int n, float2* P, cudaStream_t st) {
  if (n <= 0) return SADMM_OK;
  const int nt = ntiles_side(n);
  pack_sym_kernel<<<dim3(nt, nt), 256, 0, st>>>(F, ld, n, P);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_spd_apply(const SpdSet* sets, int nsets, bool update, const SolverView& sv, int* err, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets) { set_error("launch_spd_apply: too many sets"); return SADMM_EINVAL; }
  SetBlock<SpdSet> blk;
  int items = 0, nt_max = 0;
  for (int i = 0; i < nsets; ++i) {
    blk.v[i] = sets[i];
    blk.v[i].tile0 = items;
    const int nt = ntiles_side(sets[i].n);
    items += nt * (nt + 1) / 2;
    nt_max = max(nt_max, nt);
  }
  if (items == 0) return SADMM_OK;
  const bool ulo = sets[0].u_lo != nullptr;
  for (int i = 1; i < nsets; ++i)
    if ((sets[i].u_lo != nullptr) != ulo) { set_error("launch_spd_apply: sets mix pair and plain inputs"); return SADMM_EINVAL; }
  const int smem = kTileBytes;
  static bool configured = false;
  if (!configured) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(spd_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    SADMM_CUDA_TRY(cudaFuncSetAttribute(spd_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured = true;
  }
  const int grid = min(items, 152 * 6);           // six 32 KB tiles in flight per SM
  if (ulo) spd_tile_kernel<true><<<grid, kSpdThreads, smem, st>>>(blk, nsets, items, err);
  else spd_tile_kernel<false><<<grid, kSpdThreads, smem, st>>>(blk, nsets, items, err);
  SADMM_LAUNCH_CHECK();
  spd_reduce_kernel<<<dim3(nt_max, nsets), kT, 0, st>>>(blk, update, sv);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
