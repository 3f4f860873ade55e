// Batched sharing ADMM: S scenes that share one geometry (the operators A_q
// and therefore the factors) iterate together, so every operator byte read
// from HBM serves S scenes.  The per-iteration products become GEMMs with S
// right-hand sides (Eq. 3, x_q-update, for all scenes at once):
//   R_q (KM x S) = Y'_q - A_q V_q          V_q[j][s] = x - x_bar + z_bar - s  (scene s)
//   U_q (n x S)  = F_q R_q                 (factor; exact BF16 digit GEMMs on the
//                                           tensor cores, bapply_tc.cu)
//   X_q[j][s]    = V_q[j][s] + mu Re(a_j^H U_q[:, s])
// followed by the per-scene prox / dual / residual step (Eq. 3, x_G- and dual
// updates).  Pixel elimination is not used in this form (every scene keeps
// the full active set, so the shared factor stays valid).
//
// Layout: scene index fastest everywhere: X_q [pixel][scene], x_bar / z_bar /
// s [pixel][scene], Y'_q, R_q, U_q [row][scene] (complex as float2).
#include "common.cuh"
#include "symtile.cuh"
#include "digits.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace sadmm {

namespace {

constexpr int kBS = 16;              // scenes per batch (fixed tile width)

struct BatchDev {
  int Q, N, KM, S;
  float mu, rho;
  const float* lam_over_rho;     // S
  float* X;                      // Q x N x S
  float* dX;                     // Q x N x S  (x^{k+1} - x^k)
  float* xbar;                   // N x S
  float* zbar;                   // N x S
  float* sd;                     // N x S
};

// ------------------------------------------------------------------ forward
// The products B_q V_q for the 16 scenes run on the tensor cores (tc.cu,
// 3xTF32 tcgen05 GEMM into partial[q][split][row][scene]); the splits are added
// here in order and subtracted from y'.
__global__ void bfwd_reduce_kernel(const float2* __restrict__ partial, const float2* const* __restrict__ Yq,
                                   float2* const* __restrict__ Rq, int KM, int chunks) {
  const int q = blockIdx.y;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)KM * kBS) return;
  const float2* p = partial + (size_t)q * chunks * KM * kBS + e;
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < chunks; ++c) {
    const float2 t = p[(size_t)c * KM * kBS];
    acc.x += t.x;
    acc.y += t.y;
  }
  const float2 y = Yq[q][e];
  Rq[q][e] = make_float2(y.x - acc.x, y.y - acc.y);
}

// ------------------------------------------------- packed symmetric apply
// U[i][s] = sum_j F[i][j] u_s[j] for 16 right-hand sides with F symmetric, packed
// as upper-triangular 64 x 64 tiles of double-float pairs (as the
// single-scene apply): exact products, two-sum accumulation, about 48 bits.
// A tile (I, J) is a pair of small GEMMs, OUT_I += F_IJ U_J and (off the
// diagonal) OUT_J += F_IJ^T U_I, with 64 x 16 right-hand sides.  Persistent
// CTAs (five per SM, so that copies overlap other CTAs' arithmetic) pull tiles
// by bulk asynchronous copy (mbarrier, bounded waits); 64 threads hold 4 rows x 4 scenes of F_IJ U_J and 64 threads 4
// columns x 4 scenes of F_IJ^T U_I, stepping along skewed diagonals so that
// shared-memory reads do not conflict.  Per-tile partials go to a scratch
// buffer that bspd_reduce_cols_kernel adds in a fixed order.  This serves the
// multi-column applies of the single-scene factor updates
// (launch_multi_apply_cols); the batched iteration uses the tensor-core digit
// apply (bapply_tc.cu).
using namespace symtile;

constexpr int kBtThreads = 128;
constexpr int kBtTileBytes = kT * kT * (int)sizeof(float2);
constexpr int kBtPart = 2 * kT * kBS;          // float2 partials per tile (row part, column part)

__device__ __forceinline__ size_t cidx(int j, int s) { return ((size_t)(j >> 1) * kBS + s) * 2 + (j & 1); }

// The 16 values of u this thread stages for tile (I, J): thread t covers
// slice t / 64 (u_I, then u_J), row t % 64 of it.
__device__ __forceinline__ void bt_load_u(const float* __restrict__ u, int n, int I, int J, int t, float (&v)[16]) {
  const int blk = (t >> 6) ? J : I;
  const int j = blk * kT + (t & 63);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float4 x = j < n ? reinterpret_cast<const float4*>(u + (size_t)j * kBS)[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    v[4 * e] = x.x; v[4 * e + 1] = x.y; v[4 * e + 2] = x.z; v[4 * e + 3] = x.w;
  }
}

// ... and writes them to the staged slices su[2][64][16].
__device__ __forceinline__ void bt_store_u(float* su, int t, const float (&v)[16]) {
  float* base = su + (size_t)(t >> 6) * kT * kBS + (t & 63) * kBS;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    reinterpret_cast<float4*>(base)[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
}

__global__ void __launch_bounds__(kBtThreads)
bspd_tile_kernel(const float2* const* __restrict__ Pq, const float* const* __restrict__ uq, float2* __restrict__ part,
                 size_t part_stride, int n, int items, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);                        // 64 x 64 pairs
  float* su = reinterpret_cast<float*>(smem_raw + kBtTileBytes);            // (u_I, u_J) x 64 x 16
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int nt = ntiles_side(n);
  const int tiles = nt * (nt + 1) / 2;
  if ((int)blockIdx.x >= items) return;
  if (tid == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned phase = 0u;
  const bool rowpart = tid < 64;
  const int grp = (tid & 63) >> 2;        // row group (rows 4 grp..) or column group
  const int g = tid & 3;                  // scenes 4g .. 4g + 3
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = item / tiles, t = item % tiles;
    int I, J;
    tile_ij(t, nt, I, J);
    // the previous tile and u slices are consumed (closing barrier)
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_load(tile, Pq[q] + (size_t)t * kT * kT, kBtTileBytes, &bar);
    }
    {
      float v[16];
      bt_load_u(uq[q], n, I, J, tid, v);
      bt_store_u(su, tid, v);
    }
    __syncthreads();                                        // su written
    const bool ok = mbar_wait(&bar, phase);
    if (!__syncthreads_and(ok)) {
      // the timed-out copy writes this CTA's shared memory: let it land
      // (bounded) before the CTA exits
      if (tid == 0) {
        mbar_wait(&bar, phase);
        atomicExch(err, 1);
      }
      return;
    }
    phase ^= 1u;
    const float* uI = su;
    const float* uJ = uI + kT * kBS;
    DF acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.f, 0.f};
    if (rowpart) {
      // OUT_I[4 grp + a][4 g + b] += F[4 grp + a][k'] u_J[k'][4 g + b]
#pragma unroll 4
      for (int k0 = 0; k0 < kT; ++k0) {
        const int kk = (k0 + grp) & (kT - 1);
        const float4 u4 = reinterpret_cast<const float4*>(uJ + kk * kBS)[g];
        const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 f = tile[(4 * grp + a) * kT + kk];
#pragma unroll
          for (int b = 0; b < 4; ++b) df_acc(acc[a][b], f.x, f.y, uv[b]);
        }
      }
    } else if (I != J) {
      // OUT_J[4 grp + a][4 g + b] += F[i'][4 grp + a] u_I[i'][4 g + b]
#pragma unroll 4
      for (int k0 = 0; k0 < kT; ++k0) {
        const int ii = (k0 + grp) & (kT - 1);
        const float4 u4 = reinterpret_cast<const float4*>(uI + ii * kBS)[g];
        const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
        const float4 f01 = reinterpret_cast<const float4*>(tile + ii * kT + 4 * grp)[0];
        const float4 f23 = reinterpret_cast<const float4*>(tile + ii * kT + 4 * grp)[1];
        const float fh[4] = {f01.x, f01.z, f23.x, f23.z}, fl[4] = {f01.y, f01.w, f23.y, f23.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) df_acc(acc[a][b], fh[a], fl[a], uv[b]);
      }
    }
    float2* pt = part + (size_t)q * part_stride + (size_t)t * kBtPart + (rowpart ? 0 : kT * kBS);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const DF o0 = df_norm(acc[a][0]), o1 = df_norm(acc[a][1]), o2 = df_norm(acc[a][2]), o3 = df_norm(acc[a][3]);
      float4* dst = reinterpret_cast<float4*>(pt + (4 * grp + a) * kBS + 4 * g);
      dst[0] = make_float4(o0.hi, o0.lo, o1.hi, o1.lo);
      dst[1] = make_float4(o2.hi, o2.lo, o3.hi, o3.lo);
    }
    __syncthreads();                                        // tile and su consumed
  }
}

// OUT[i][s] = sum over the k ranges of the digit apply's partial results
// (double-float, in a fixed order), then the epilogue:
// mode 0 (Woodbury): U written as complex [row][scene]
// mode 1 (primal):   x-update X = V + mu U (row i is pixel i: the full active set)
__global__ void __launch_bounds__(256)
bapply_reduce_kernel(const float2* __restrict__ part, int ksplit, int rows_pad, float* const* __restrict__ outq,
                     int n, int mode, BatchDev b) {
  const int q = blockIdx.y;
  const int e = blockIdx.x * 256 + threadIdx.x;
  const int i = e / kBS, s = e % kBS;
  if (i >= n) return;
  DF acc{0.f, 0.f};
  for (int k = 0; k < ksplit; ++k) {
    const float2 v = part[(((size_t)q * ksplit + k) * rows_pad + i) * kBS + s];
    df_add(acc, DF{v.x, v.y});
  }
  const float g = acc.hi + acc.lo;
  if (mode == 0) {
    outq[q][cidx(i, s)] = g;
  } else {
    const size_t o = ((size_t)q * b.N + i) * kBS + s;
    const size_t pp = (size_t)i * kBS + s;
    const float xo = b.X[o];
    const float v = xo - b.xbar[pp] + b.zbar[pp] - b.sd[pp];
    const float xn = fmaf(b.mu, g, v);
    b.dX[o] = xn - xo;
    b.X[o] = xn;
  }
}

// ------------------------------------------------------------------ adjoint
// G_q = Re(A_q^H W_q) for the 16 scenes runs on the tensor cores (tc.cu,
// 3xTF32 tcgen05 GEMM into gpart[q][split][pixel][scene]); the splits of the
// row range are added here in order, followed by the x-update epilogue.
__global__ void badj_reduce_kernel(const float* __restrict__ gpart, int splits, float* const* __restrict__ gq,
                                   int mode, BatchDev b) {
  const int q = blockIdx.y;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t NS = (size_t)b.N * kBS;
  if (e >= NS) return;
  const float* p = gpart + (size_t)q * splits * NS + e;
  float g = 0.f;
  for (int k = 0; k < splits; ++k) g += p[(size_t)k * NS];
  if (mode == 1) {
    gq[q][e] = g;
  } else {
    const size_t o = (size_t)q * NS + e;
    const float xo = b.X[o];
    const float v = xo - b.xbar[e] + b.zbar[e] - b.sd[e];
    const float xn = fmaf(b.mu, g, v);
    b.dX[o] = xn - xo;
    b.X[o] = xn;
  }
}

// ------------------------------------------------------- prox / residuals
// Per (pixel, scene): x_bar, z_bar = soft(x_bar + s, lambda_s / rho), s update,
// and per-scene FP64 partial sums (same eight sums as the single-scene path).
constexpr int kBrThreads = 256;   // 16 pixels x 16 scenes
constexpr int kBrSums = 8;

__global__ void __launch_bounds__(kBrThreads)
bresid_kernel(BatchDev b, double* __restrict__ partials) {
  const int s = threadIdx.x % kBS, pl = threadIdx.x / kBS;
  const int j = blockIdx.x * (kBrThreads / kBS) + pl;
  double acc[kBrSums];
#pragma unroll
  for (int k = 0; k < kBrSums; ++k) acc[k] = 0.0;
  if (j < b.N) {
    const size_t p = (size_t)j * kBS + s;
    float sx = 0.f;
    for (int q = 0; q < b.Q; ++q) sx += b.X[((size_t)q * b.N + j) * kBS + s];
    const float xb = sx / (float)b.Q;
    const float xo = b.xbar[p], zo = b.zbar[p], so = b.sd[p];
    const float t = xb + so;
    const float zb = copysignf(fmaxf(fabsf(t) - b.lam_over_rho[s], 0.f), t);
    const float sn = (so + xb) - zb;
    const double dxb = (double)xb - xo, dzb = (double)zb - zo, e = (double)xb - zb;
    acc[0] = e * e;
    for (int q = 0; q < b.Q; ++q) {
      const size_t o = ((size_t)q * b.N + j) * kBS + s;
      const double xq = b.X[o], dx = b.dX[o];
      const double zq = xq - (double)xb + (double)zb, dz = dx - dxb + dzb;
      acc[1] += xq * xq;
      acc[2] += zq * zq;
      acc[3] += dz * dz;
      acc[5] += dx * dx;
    }
    acc[4] = (double)sn * sn;
    acc[6] = (double)zb * zb;
    acc[7] = dzb * dzb;
    b.xbar[p] = xb;
    b.zbar[p] = zb;
    b.sd[p] = sn;
  }
  // reduce over the 16 pixels of this block for each scene (fixed order)
  __shared__ double red[kBrThreads / kBS][kBS][kBrSums];
#pragma unroll
  for (int k = 0; k < kBrSums; ++k) red[pl][s][k] = acc[k];
  __syncthreads();
  if (pl == 0) {
    for (int k = 0; k < kBrSums; ++k) {
      double t = 0.0;
      for (int r = 0; r < kBrThreads / kBS; ++r) t += red[r][s][k];
      partials[((size_t)blockIdx.x * kBS + s) * kBrSums + k] = t;
    }
  }
}

__global__ void __launch_bounds__(kBrSums * 32)
bresid_final_kernel(const double* __restrict__ partials, int nblk, BatchDev b, double eps_abs,
                    double eps_rel, int k_after, IterScalars* __restrict__ out) {
  const int s = blockIdx.x;                        // scene
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;   // warp k reduces sum k
  __shared__ double tot[kBrSums];
  double t = 0.0;
  for (int blk = lane; blk < nblk; blk += 32) t += partials[((size_t)blk * kBS + s) * kBrSums + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) tot[k] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double Q = b.Q, QN = (double)b.Q * b.N;
  IterScalars r;
  r.r_pri = sqrt(Q) * sqrt(tot[0]);
  const double xn = sqrt(tot[1]), zn = sqrt(tot[2]);
  r.eps_pri = sqrt(QN) * eps_abs + eps_rel * fmax(xn, zn);
  r.d = (double)b.rho * sqrt(tot[3]);
  r.eps_dual = sqrt(QN) * eps_abs + eps_rel * (double)b.rho * sqrt(Q) * sqrt(tot[4]);
  r.relchange = xn > 0.0 ? sqrt(tot[5]) / xn : INFINITY;
  r.xg_norm = Q * sqrt(tot[6]);
  r.dxg_norm = Q * sqrt(tot[7]);
  r.xnorm = xn;
  r.k = k_after;
  r.gate = 0;
  r.changed = 0;
  double chk = 0.0;
  for (int j = 0; j < kBrSums; ++j) chk += tot[j];
  r.nonfinite = isfinite(chk) ? 0 : 1;
  out[s] = r;
}

__global__ void bscale_kernel(const float* __restrict__ zbar, float Q, float* __restrict__ out, int N) {
  // out[s][j] = Q z_bar[j][s] (scene-major output)
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)N * kBS) return;
  const int j = (int)(e / kBS), s = (int)(e % kBS);
  out[(size_t)s * N + j] = Q * zbar[e];
}

// interleave per-scene measurement vectors y[s][q] (KM complex) -> Y'_q [row][scene]
__global__ void bload_y_kernel(const float2* __restrict__ y, float2* const* __restrict__ Yq, int Q, int KM) {
  const int q = blockIdx.y;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)KM * kBS) return;
  const int r = (int)(e / kBS), s = (int)(e % kBS);
  Yq[q][e] = y[((size_t)s * Q + q) * KM + r];
}

// X_q [pixel][scene] -> out [pixel] for one scene
__global__ void bget_x_kernel(const float* __restrict__ X, int N, int scene, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) out[j] = X[(size_t)j * kBS + scene];
}


// ------------------------------------------- multi-column apply (factor updates)
// P[:, c] = F B[:, E_c] for up to 16 columns at a time (the W U product of a
// rank update of the factor, Eq. 3, x_q-update with changed active sets):
// the columns are gathered into a [row][16] block and pushed through the same
// packed-tile 16-RHS kernel as the batched apply; the reduction writes FP64.
struct ColJob {
  const float2* A;      // operator of the sensor (pixel-major)
  const int* E;         // columns (pixels), device
  int e;                // columns in this call's window [c0, c0 + 16)
  float* U;             // n x 16 staging
  double* P;            // n x 32 output (row-major), columns c0 .. c0 + 15 written
};

__global__ void gather_cols_kernel(const __grid_constant__ SetBlock<ColJob> jobs, int n, int c0) {
  const ColJob& jb = jobs.v[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * kBS) return;
  const int j = idx / kBS, c = idx % kBS;
  float v = 0.f;
  if (c < jb.e) v = reinterpret_cast<const float*>(jb.A)[(size_t)jb.E[c0 + c] * n + j];
  jb.U[idx] = v;
}

__global__ void __launch_bounds__(256)
bspd_reduce_cols_kernel(const float2* __restrict__ part, size_t part_stride, const __grid_constant__ SetBlock<ColJob> jobs,
                        int n, int c0) {
  const int q = blockIdx.y, I = blockIdx.x;
  const ColJob& jb = jobs.v[q];
  const int nt = ntiles_side(n);
  const int i = I * kT + (threadIdx.x >> 2), s0 = 4 * (threadIdx.x & 3);
  DF acc[4] = {DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}};
  const float2* pq = part + (size_t)q * part_stride;
  for (int J = 0; J < nt; ++J) {
    const int a = min(I, J), c = max(I, J);
    const float2* p = pq + (size_t)tile_index(a, c, nt) * kBtPart + (J >= I ? 0 : kT * kBS) +
                      (threadIdx.x >> 2) * kBS + s0;
    const float4 x = reinterpret_cast<const float4*>(p)[0], y = reinterpret_cast<const float4*>(p)[1];
    df_add(acc[0], DF{x.x, x.y});
    df_add(acc[1], DF{x.z, x.w});
    df_add(acc[2], DF{y.x, y.y});
    df_add(acc[3], DF{y.z, y.w});
  }
  if (i >= n) return;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int c = s0 + e;
    if (c < jb.e) jb.P[(size_t)i * kDowndateMax + c0 + c] = (double)acc[e].hi + (double)acc[e].lo;
  }
}

}  // namespace

struct BatchCtx {
  int Q = 0, M = 0, K = 0, N = 0, KM = 0, S = kBS;
  double rho = 1.0, mu = 1.0;
  sadmm_criterion crit{};
  cudaStream_t st = nullptr;
  sadmm_t single = nullptr;        // owns the operators and the FP64 factors
  std::vector<void*> owned;
  float *X = nullptr, *dX = nullptr, *xbar = nullptr, *zbar = nullptr, *sd = nullptr, *lor = nullptr;
  float2 **dY = nullptr, **dR = nullptr;
  DigitApply dapp;                 // factor digits and the apply's scratch (bapply_tc.cu)
  bool dapp_bound = false;
  std::vector<const float2*> hA, hR, hU;   // host copies of the per-sensor device pointers
  std::vector<void*> hY, hG;
  int* berr = nullptr;             // set if a factor tile copy timed out
  float **dU = nullptr, **dG = nullptr;
  float2* partial = nullptr;
  double* rpart = nullptr;
  IterScalars* scal = nullptr;
  float2* ybuf = nullptr;
  float* xout = nullptr;
  int chunks = 1, n = 0, ld = 0, woodbury = 1;
  int asplits = 1;                 // row splits of the adjoint GEMM
  int chunks0 = 1, asplits0 = 1;   // the default splits (the tuner's starting points)
  int chunks_cap = 1, asplits_cap = 1;     // the largest splits the scratch holds
  float* gpart = nullptr;          // Q x asplits x N x 16 partial adjoint sums
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  bool ready = false;              // factors exported and packed for the current operators
  unsigned epoch = 0;              // changes whenever the work one iteration launches changes
  int kernels_per_iter = 0;
  int k = 0;
  IterScalars h_scal[kBS];         // last iteration's per-scene scalars (host copy)
  int h_err = 0;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  }
  BatchDev view() const {
    return BatchDev{Q, N, KM, S, (float)mu, (float)rho, lor, X, dX, xbar, zbar, sd};
  }
  void invalidate() {
    ready = false;
    graph_valid = false;
    ++epoch;
  }
};

// Accessors implemented in api.cu (the batch form reuses a single-scene
// context for operator storage and the FP64 factor pipeline).
int single_export(sadmm_t h, int q, const float2** A, const double** F, int* n, int* ld, int* woodbury);

namespace {

int launch_bapply(BatchCtx& c, const float* const* u, float* const* out, int mode, const BatchDev& bv) {
  SADMM_TRY(launch_digit_apply(c.dapp, u, mode == 0 ? 0 : 1, c.berr, c.st));
  bapply_reduce_kernel<<<dim3(div_up((long long)c.n * kBS, 256), c.Q), 256, 0, c.st>>>(
      c.dapp.part, c.dapp.ksplit, c.dapp.rows_pad, out, c.n, mode, bv);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_forward_products(BatchCtx& c, int chunks, const BatchDev& bv) {
  SADMM_TRY(launch_tc_forward(c.hA.data(), bv.X, bv.xbar, bv.zbar, bv.sd, c.partial, c.Q, c.N, c.KM, chunks, c.berr,
                              c.st));
  bfwd_reduce_kernel<<<dim3(div_up((long long)c.KM * kBS, 256), c.Q), 256, 0, c.st>>>(c.partial, c.dY, c.dR, c.KM,
                                                                                     chunks);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// mode 0: x-update epilogue from W R (Woodbury form); mode 1: G = Re(A^H R) only
int launch_adjoint_products(BatchCtx& c, int splits, const float2* const* in, int mode, const BatchDev& bv) {
  SADMM_TRY(launch_tc_adjoint(c.hA.data(), in, c.gpart, c.Q, c.N, c.KM, splits, c.berr, c.st));
  badj_reduce_kernel<<<dim3(div_up((long long)c.N * kBS, 256), c.Q), 256, 0, c.st>>>(c.gpart, splits, c.dG, mode,
                                                                                    bv);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int batch_launch_iteration(BatchCtx& c) {
  const BatchDev bv = c.view();
  SADMM_TRY(launch_forward_products(c, c.chunks, bv));
  if (c.woodbury) {
    SADMM_TRY(launch_bapply(c, (const float* const*)c.dR, c.dU, 0, bv));
    SADMM_TRY(launch_adjoint_products(c, c.asplits, c.hU.data(), 0, bv));
  } else {
    SADMM_TRY(launch_adjoint_products(c, c.asplits, c.hR.data(), 1, bv));
    SADMM_TRY(launch_bapply(c, (const float* const*)c.dG, nullptr, 1, bv));
  }
  const int nblk = div_up(c.N, kBrThreads / kBS);
  bresid_kernel<<<nblk, kBrThreads, 0, c.st>>>(bv, c.rpart);
  SADMM_LAUNCH_CHECK();
  bresid_final_kernel<<<kBS, kBrSums * 32, 0, c.st>>>(c.rpart, nblk, bv, c.crit.eps_abs, c.crit.eps_rel, 0, c.scal);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// Factors for the current operators (FP64, from the single-scene context),
// cut into the tensor-core apply's digit planes; the apply's scratch.
// Synchronises b.st.
int batch_setup(BatchCtx& b) {
  SADMM_TRY(sadmm_prepare(b.single));
  if (b.ready) return SADMM_OK;
  b.hA.assign(b.Q, nullptr);
  for (int q = 0; q < b.Q; ++q) {
    const float2* A = nullptr;
    const double* F = nullptr;
    SADMM_TRY(single_export(b.single, q, &A, &F, &b.n, &b.ld, &b.woodbury));
    if (!b.dapp_bound) {
      digit_apply_dims(b.dapp, b.Q, b.n);
      void* mem = b.dalloc(digit_apply_bytes(b.dapp));
      if (!mem) { set_error("batched form: factor digit allocation failed"); return SADMM_ENOMEM; }
      SADMM_TRY(digit_apply_bind(b.dapp, mem));
      b.dapp_bound = true;
    }
    SADMM_TRY(launch_factor_digits(b.dapp, q, F, b.ld, b.st));
    b.hA[q] = A;
  }
  SADMM_CUDA_TRY(cudaStreamSynchronize(b.st));
  b.ready = true;
  return SADMM_OK;
}

// One iteration captured as a graph, replayed once per iteration.
int batch_capture(BatchCtx& b) {
  if (b.graph) { cudaGraphExecDestroy(b.graph); b.graph = nullptr; }
  b.graph_valid = false;
  cudaStream_t cap;
  SADMM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t saved = b.st;
  b.st = cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  const long long n0 = sadmm_launch_count();
  int rc = e == cudaSuccess ? batch_launch_iteration(b) : SADMM_ECUDA;
  b.kernels_per_iter = (int)(sadmm_launch_count() - n0);
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &g) : cudaSuccess;
  b.st = saved;
  cudaStreamDestroy(cap);
  if (rc != SADMM_OK) { if (g) cudaGraphDestroy(g); return rc; }
  SADMM_CUDA_TRY(e);
  SADMM_CUDA_TRY(e2);
  e = cudaGraphInstantiate(&b.graph, g, 0);
  cudaGraphDestroy(g);
  SADMM_CUDA_TRY(e);
  b.graph_valid = true;
  return SADMM_OK;
}

// Zero state, measurements y (S x Q x KM complex, host or device) into Y'.
int batch_reset(BatchCtx& b, const float* y, cudaStream_t st) {
  const size_t QNS = (size_t)b.Q * b.N * kBS, NS = (size_t)b.N * kBS;
  SADMM_CUDA_TRY(cudaMemsetAsync(b.X, 0, QNS * 4, st));
  SADMM_CUDA_TRY(cudaMemsetAsync(b.dX, 0, QNS * 4, st));
  SADMM_CUDA_TRY(cudaMemsetAsync(b.xbar, 0, NS * 4, st));
  SADMM_CUDA_TRY(cudaMemsetAsync(b.zbar, 0, NS * 4, st));
  SADMM_CUDA_TRY(cudaMemsetAsync(b.sd, 0, NS * 4, st));
  SADMM_CUDA_TRY(cudaMemcpyAsync(b.ybuf, y, (size_t)kBS * b.Q * b.KM * sizeof(float2), cudaMemcpyDefault, st));
  bload_y_kernel<<<dim3(div_up((long long)b.KM * kBS, 256), b.Q), 256, 0, st>>>(b.ybuf, b.dY, b.Q, b.KM);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// x_G of every scene to x_out (may be NULL); the last iteration's scalars and
// the error flag to the host copies (read after the stream is synchronised).
int batch_collect(BatchCtx& b, float* x_out, cudaStream_t st) {
  const size_t NS = (size_t)b.N * kBS;
  if (x_out) {
    bscale_kernel<<<div_up(NS, 256), 256, 0, st>>>(b.zbar, (float)b.Q, b.xout, b.N);
    SADMM_LAUNCH_CHECK();
    SADMM_CUDA_TRY(cudaMemcpyAsync(x_out, b.xout, NS * 4, cudaMemcpyDefault, st));
  }
  SADMM_CUDA_TRY(cudaMemcpyAsync(b.h_scal, b.scal, sizeof b.h_scal, cudaMemcpyDeviceToHost, st));
  SADMM_CUDA_TRY(cudaMemcpyAsync(&b.h_err, b.berr, sizeof(int), cudaMemcpyDeviceToHost, st));
  return SADMM_OK;
}

int batch_finish(BatchCtx& b, int iters, sadmm_stats* st, double ms) {
  b.k = iters;
  if (b.h_err) {
    SADMM_CUDA_TRY(cudaMemset(b.berr, 0, sizeof(int)));
    b.h_err = 0;
    set_error("batched form: a tile copy or tensor-core pipeline wait did not complete within its limit");
    return SADMM_ETIMEOUT;
  }
  for (int s = 0; s < kBS; ++s)
    if (iters > 0 && b.h_scal[s].nonfinite) { set_error("non-finite value in scene %d", s); return SADMM_ENONFINITE; }
  if (st) {
    const IterScalars& h = b.h_scal[0];
    memset(st, 0, sizeof *st);
    st->iters = iters;
    st->active_total = b.Q * b.N * kBS;
    st->r_pri = h.r_pri; st->eps_pri = h.eps_pri; st->d = h.d; st->eps_dual = h.eps_dual;
    st->relchange = h.relchange;
    st->ms_total = ms;
    st->bytes_iter = (double)iters * ((double)b.Q * b.KM * b.N * 16.0 + (double)b.Q * b.dapp.rows_pad * b.dapp.kpad * 8.0);
  }
  return SADMM_OK;
}

// Up to eight split counts from a quarter to four times the default, in [1, cap].
std::vector<int> split_candidates(int base, int cap) {
  std::vector<int> v;
  const int f[8] = {base / 4, base / 2, (3 * base) / 4, base, (3 * base) / 2, 2 * base, 3 * base, 4 * base};
  for (int x : f) {
    x = std::max(1, std::min(x, cap));
    if (std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
  }
  std::sort(v.begin(), v.end());
  return v;
}

}  // namespace

size_t multi_apply_part_pairs(int n) {
  const size_t nt = ntiles_side(n);
  return nt * (nt + 1) / 2 * kBtPart;
}

int launch_multi_apply_cols(const float2* const* F, const float2* const* A, const int* const* E, const int* e, double* const* P,
                            int njobs, int n, int c0, float* U, void** dptrs, float2* part, int* err, cudaStream_t st) {
  if (njobs <= 0) return SADMM_OK;
  if (njobs > kMaxSets || n % kT != 0) { set_error("launch_multi_apply_cols: bad sizes"); return SADMM_EINVAL; }
  SetBlock<ColJob> blk;
  std::vector<const void*> hp(2 * njobs);
  for (int j = 0; j < njobs; ++j) {
    blk.v[j] = ColJob{A[j], E[j], std::max(0, std::min(kBS, e[j] - c0)), U + (size_t)j * n * kBS, P[j]};
    hp[j] = F[j];
    hp[njobs + j] = blk.v[j].U;
  }
  SADMM_CUDA_TRY(cudaMemcpyAsync(dptrs, hp.data(), hp.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
  gather_cols_kernel<<<dim3(div_up(n * kBS, 256), njobs), 256, 0, st>>>(blk, n, c0);
  SADMM_LAUNCH_CHECK();
  const int nt = div_up(n, kT), items = njobs * nt * (nt + 1) / 2;
  const int smem = kBtTileBytes + 2 * kT * kBS * (int)sizeof(float);
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(bspd_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    conf = true;
  }
  const size_t stride = multi_apply_part_pairs(n);
  bspd_tile_kernel<<<std::min(items, 152 * 5), kBtThreads, smem, st>>>(
      reinterpret_cast<const float2* const*>(dptrs), reinterpret_cast<const float* const*>(dptrs + njobs), part, stride,
      n, items, err);
  SADMM_LAUNCH_CHECK();
  bspd_reduce_cols_kernel<<<dim3(nt, njobs), 256, 0, st>>>(part, stride, blk, n, c0);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm

struct sadmm_batch_ctx : sadmm::BatchCtx {};

struct sadmm_batch_group_ctx {
  std::vector<sadmm::BatchCtx*> b;
  std::vector<unsigned> epochs;
  std::vector<cudaStream_t> side;  // one capture branch per batch
  std::vector<cudaEvent_t> ev;     // fork, then one join per batch
  cudaStream_t st = nullptr;
  cudaGraphExec_t graph = nullptr;
  int kernels_per_iter = 0;
};

extern "C" {

int sadmm_batch_create(int Q, int M, int K, int N, int S, double rho, const double* lambda,
                       const sadmm_criterion* crit, sadmm_batch_t* out) {
  using namespace sadmm;
  if (!out || !lambda || S != kBS) {
    set_error("sadmm_batch_create: S must be %d and lambda / out non-NULL", kBS);
    return SADMM_EINVAL;
  }
  *out = nullptr;
  sadmm_criterion c;
  if (crit) c = *crit; else sadmm_default_criterion(&c);
  if (c.consensus) {
    set_error("sadmm_batch_create: the batched form runs the sharing formulation (consensus = 0)");
    return SADMM_EINVAL;
  }
  c.elim = 0;
  c.precision = 0;
  for (int s = 0; s < S; ++s)
    if (!(lambda[s] >= 0.0) || !std::isfinite(lambda[s])) { set_error("sadmm_batch_create: bad lambda"); return SADMM_EINVAL; }
  sadmm_t single = nullptr;
  SADMM_TRY(sadmm_create(Q, M, K, N, rho, lambda[0], &c, &single));
  sadmm_batch_ctx* b = new (std::nothrow) sadmm_batch_ctx();
  if (!b) { sadmm_destroy(single); return SADMM_ENOMEM; }
  b->Q = Q; b->M = M; b->K = K; b->N = N; b->KM = K * M; b->S = S;
  b->rho = rho; b->mu = c.mu; b->crit = c; b->single = single;
  bool ok = true;
  auto A = [&](size_t bytes) { void* p = b->dalloc(bytes); if (!p) ok = false; return p; };
  const size_t QNS = (size_t)Q * N * kBS, NS = (size_t)N * kBS, KS = (size_t)b->KM * kBS;
  b->X = (float*)A(QNS * 4); b->dX = (float*)A(QNS * 4);
  b->xbar = (float*)A(NS * 4); b->zbar = (float*)A(NS * 4); b->sd = (float*)A(NS * 4);
  b->lor = (float*)A(kBS * 4);
  b->dY = (float2**)A(Q * sizeof(void*));
  b->dR = (float2**)A(Q * sizeof(void*));
  b->dU = (float**)A(Q * sizeof(void*)); b->dG = (float**)A(Q * sizeof(void*));
  b->chunks = b->chunks0 = tc_forward_splits(Q, N, b->KM);
  b->asplits = b->asplits0 = tc_adjoint_splits(Q, N, b->KM);
  b->chunks_cap = std::min(4 * b->chunks0, tc_forward_max_splits(N));
  b->asplits_cap = std::min(4 * b->asplits0, tc_adjoint_max_splits(b->KM));
  b->gpart = (float*)A((size_t)Q * b->asplits_cap * NS * sizeof(float));
  b->partial = (float2*)A((size_t)Q * b->chunks_cap * KS * sizeof(float2));
  b->rpart = (double*)A((size_t)div_up(N, kBrThreads / kBS) * kBS * kBrSums * sizeof(double));
  b->scal = (IterScalars*)A(kBS * sizeof(IterScalars));
  b->berr = (int*)A(sizeof(int));
  b->ybuf = (float2*)A((size_t)S * Q * b->KM * sizeof(float2));
  b->xout = (float*)A((size_t)S * N * 4);
  std::vector<void*> R(Q), U(Q);
  b->hY.assign(Q, nullptr);
  b->hG.assign(Q, nullptr);
  for (int q = 0; q < Q && ok; ++q) {
    b->hY[q] = A(KS * sizeof(float2));
    R[q] = A(KS * sizeof(float2));
    U[q] = A(2 * KS * sizeof(float));
    b->hG[q] = A(NS * sizeof(float));
  }
  for (int q = 0; q < Q; ++q) {
    b->hR.push_back((const float2*)R[q]);
    b->hU.push_back((const float2*)U[q]);
  }
  if (!ok) {
    for (void* p : b->owned) cudaFree(p);
    sadmm_destroy(single);
    delete b;
    set_error("sadmm_batch_create: device allocation failed");
    return SADMM_ENOMEM;
  }
  std::vector<float> lor(kBS);
  for (int s = 0; s < kBS; ++s) lor[s] = (float)(lambda[s] / rho);
  if (cudaMemcpy(b->lor, lor.data(), kBS * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dY, b->hY.data(), Q * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dR, R.data(), Q * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dU, U.data(), Q * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dG, b->hG.data(), Q * sizeof(void*), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->berr, 0, sizeof(int)) != cudaSuccess) {
    for (void* p : b->owned) cudaFree(p);
    sadmm_destroy(single);
    delete b;
    set_error("sadmm_batch_create: initialisation failed");
    return SADMM_ECUDA;
  }
  *out = b;
  return SADMM_OK;
}

int sadmm_batch_set_stream(sadmm_batch_t b, void* stream) {
  using namespace sadmm;
  if (!b) return SADMM_EINVAL;
  SADMM_CUDA_TRY(cudaStreamSynchronize(b->st));
  b->st = (cudaStream_t)stream;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  b->graph_valid = false;
  return sadmm_set_stream(b->single, stream);
}

int sadmm_batch_set_operator(sadmm_batch_t b, int q, const float* A_q) {
  using namespace sadmm;
  if (!b) return SADMM_EINVAL;
  b->invalidate();
  return sadmm_set_operator(b->single, q, A_q);
}

int sadmm_batch_solve(sadmm_batch_t b, const float* y, float* x_out, int iters, sadmm_stats* st) {
  using namespace sadmm;
  if (!b || !y || iters < 0) { set_error("sadmm_batch_solve: bad arguments"); return SADMM_EINVAL; }
  const auto t0 = std::chrono::steady_clock::now();
  SADMM_TRY(batch_setup(*b));
  if (!b->graph_valid) SADMM_TRY(batch_capture(*b));
  SADMM_TRY(batch_reset(*b, y, b->st));
  for (int it = 0; it < iters; ++it) {
    SADMM_CUDA_TRY(cudaGraphLaunch(b->graph, b->st));
    for (int kk = 0; kk < b->kernels_per_iter; ++kk) count_launch();
  }
  SADMM_TRY(batch_collect(*b, x_out, b->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(b->st));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return batch_finish(*b, iters, st, ms);
}

int sadmm_batch_tune(sadmm_batch_t b, int reps, sadmm_batch_tuning* out) {
  using namespace sadmm;
  if (!b || reps < 1) { set_error("sadmm_batch_tune: bad arguments"); return SADMM_EINVAL; }
  SADMM_TRY(batch_setup(*b));
  // defined inputs for the timed launches (the next solve resets the state)
  const size_t QNS = (size_t)b->Q * b->N * kBS, NS = (size_t)b->N * kBS, KS = (size_t)b->KM * kBS;
  for (float* p : {b->X, b->dX}) SADMM_CUDA_TRY(cudaMemsetAsync(p, 0, QNS * 4, b->st));
  for (float* p : {b->xbar, b->zbar, b->sd}) SADMM_CUDA_TRY(cudaMemsetAsync(p, 0, NS * 4, b->st));
  for (int q = 0; q < b->Q; ++q) {
    SADMM_CUDA_TRY(cudaMemsetAsync(b->hY[q], 0, KS * sizeof(float2), b->st));
    SADMM_CUDA_TRY(cudaMemsetAsync((void*)b->hR[q], 0, KS * sizeof(float2), b->st));
    SADMM_CUDA_TRY(cudaMemsetAsync((void*)b->hU[q], 0, 2 * KS * sizeof(float), b->st));
  }
  const BatchDev bv = b->view();
  cudaEvent_t e0, e1;
  SADMM_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); set_error("sadmm_batch_tune: event"); return SADMM_ECUDA; }
  sadmm_batch_tuning t;
  memset(&t, 0, sizeof t);
  int rc = SADMM_OK;
  auto time_it = [&](auto&& launch, double* ms) -> int {
    int r = launch();                                  // untimed first launch
    if (r != SADMM_OK) return r;
    if (cudaEventRecord(e0, b->st) != cudaSuccess) return SADMM_ECUDA;
    for (int i = 0; i < reps && r == SADMM_OK; ++i) r = launch();
    if (r != SADMM_OK) return r;
    if (cudaEventRecord(e1, b->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SADMM_ECUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return SADMM_ECUDA;
    *ms = (double)f / reps;
    return SADMM_OK;
  };
  const std::vector<int> fc = split_candidates(b->chunks0, b->chunks_cap);
  const std::vector<int> ac = split_candidates(b->asplits0, b->asplits_cap);
  const float2* const* adj_in = b->woodbury ? b->hU.data() : b->hR.data();
  int best_f = b->chunks0, best_a = b->asplits0;
  double tf = 1e300, ta = 1e300;
  for (size_t i = 0; i < fc.size() && rc == SADMM_OK; ++i) {
    const int c = fc[i];
    rc = time_it([&] { return launch_forward_products(*b, c, bv); }, &t.fwd_ms[i]);
    t.fwd_splits[i] = c;
    t.n_fwd = (int)i + 1;
    if (rc == SADMM_OK && t.fwd_ms[i] < tf) { tf = t.fwd_ms[i]; best_f = c; }
  }
  for (size_t i = 0; i < ac.size() && rc == SADMM_OK; ++i) {
    const int a = ac[i];
    rc = time_it([&] { return launch_adjoint_products(*b, a, adj_in, 1, bv); }, &t.adj_ms[i]);
    t.adj_splits[i] = a;
    t.n_adj = (int)i + 1;
    if (rc == SADMM_OK && t.adj_ms[i] < ta) { ta = t.adj_ms[i]; best_a = a; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SADMM_OK) return rc;
  int herr = 0;
  SADMM_CUDA_TRY(cudaMemcpy(&herr, b->berr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    SADMM_CUDA_TRY(cudaMemset(b->berr, 0, sizeof(int)));
    set_error("sadmm_batch_tune: a tensor-core pipeline wait did not complete within its limit");
    return SADMM_ETIMEOUT;
  }
  b->chunks = best_f;
  b->asplits = best_a;
  t.fwd_choice = best_f;
  t.adj_choice = best_a;
  t.fwd_default = b->chunks0;
  t.adj_default = b->asplits0;
  b->graph_valid = false;
  ++b->epoch;
  if (out) *out = t;
  return SADMM_OK;
}

int sadmm_batch_get_xq(sadmm_batch_t b, int scene, int q, float* out) {
  using namespace sadmm;
  if (!b || scene < 0 || scene >= b->S || q < 0 || q >= b->Q || !out) return SADMM_EINVAL;
  bget_x_kernel<<<div_up(b->N, 256), 256, 0, b->st>>>(b->X + (size_t)q * b->N * kBS, b->N, scene, b->xout);
  SADMM_LAUNCH_CHECK();
  SADMM_CUDA_TRY(cudaMemcpyAsync(out, b->xout, b->N * 4, cudaMemcpyDefault, b->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(b->st));
  return SADMM_OK;
}

void sadmm_batch_destroy(sadmm_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->owned) cudaFree(p);
  sadmm_destroy(b->single);
  delete b;
}

// ------------------------------------------------------------ batch groups

static void group_release(sadmm_batch_group_t g) {
  if (g->graph) cudaGraphExecDestroy(g->graph);
  for (cudaStream_t s : g->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
}

int sadmm_batch_group_create(const sadmm_batch_t* batches, int n, sadmm_batch_group_t* out) {
  using namespace sadmm;
  if (!out || !batches || n < 1 || n > 64) { set_error("sadmm_batch_group_create: 1..64 batches required"); return SADMM_EINVAL; }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!batches[i]) { set_error("sadmm_batch_group_create: batch %d is NULL", i); return SADMM_EINVAL; }
    for (int j = 0; j < i; ++j)
      if (batches[j] == batches[i]) { set_error("sadmm_batch_group_create: batch %d repeated", i); return SADMM_EINVAL; }
  }
  sadmm_batch_group_t g = new (std::nothrow) sadmm_batch_group_ctx();
  if (!g) return SADMM_ENOMEM;
  for (int i = 0; i < n; ++i) g->b.push_back(batches[i]);
  g->epochs.assign(n, ~0u);
  for (int i = 0; i < n; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      group_release(g);
      set_error("sadmm_batch_group_create: stream creation failed");
      return SADMM_ECUDA;
    }
    g->side.push_back(s);
  }
  for (int i = 0; i <= n; ++i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      group_release(g);
      set_error("sadmm_batch_group_create: event creation failed");
      return SADMM_ECUDA;
    }
    g->ev.push_back(e);
  }
  *out = g;
  return SADMM_OK;
}

int sadmm_batch_group_set_stream(sadmm_batch_group_t g, void* stream) {
  using namespace sadmm;
  if (!g) return SADMM_EINVAL;
  SADMM_CUDA_TRY(cudaStreamSynchronize(g->st));
  g->st = (cudaStream_t)stream;
  return SADMM_OK;
}

// One iteration of every batch, each on its own branch of one graph.
static int group_capture(sadmm_batch_group_t g) {
  using namespace sadmm;
  if (g->graph) { cudaGraphExecDestroy(g->graph); g->graph = nullptr; }
  cudaStream_t cap;
  SADMM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? SADMM_OK : SADMM_ECUDA;
  const long long n0 = sadmm_launch_count();
  if (rc == SADMM_OK && cudaEventRecord(g->ev[0], cap) != cudaSuccess) rc = SADMM_ECUDA;
  for (size_t i = 0; i < g->b.size() && rc == SADMM_OK; ++i) {
    BatchCtx& b = *g->b[i];
    if (cudaStreamWaitEvent(g->side[i], g->ev[0], 0) != cudaSuccess) { rc = SADMM_ECUDA; break; }
    cudaStream_t saved = b.st;
    b.st = g->side[i];
    rc = batch_launch_iteration(b);
    b.st = saved;
    if (rc == SADMM_OK && (cudaEventRecord(g->ev[i + 1], g->side[i]) != cudaSuccess ||
                           cudaStreamWaitEvent(cap, g->ev[i + 1], 0) != cudaSuccess))
      rc = SADMM_ECUDA;
  }
  g->kernels_per_iter = (int)(sadmm_launch_count() - n0);
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &graph) : cudaSuccess;
  cudaStreamDestroy(cap);
  if (rc != SADMM_OK || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rc == SADMM_OK) set_error("batch group: graph capture failed (%s)", cudaGetErrorString(e2));
    return rc != SADMM_OK ? rc : SADMM_ECUDA;
  }
  e = cudaGraphInstantiate(&g->graph, graph, 0);
  cudaGraphDestroy(graph);
  SADMM_CUDA_TRY(e);
  for (size_t i = 0; i < g->b.size(); ++i) g->epochs[i] = g->b[i]->epoch;
  return SADMM_OK;
}

int sadmm_batch_group_solve(sadmm_batch_group_t g, const float* const* y, float* const* x_out, int iters,
                            sadmm_stats* st) {
  using namespace sadmm;
  if (!g || !y || iters < 0) { set_error("sadmm_batch_group_solve: bad arguments"); return SADMM_EINVAL; }
  const int n = (int)g->b.size();
  for (int i = 0; i < n; ++i)
    if (!y[i]) { set_error("sadmm_batch_group_solve: y[%d] is NULL", i); return SADMM_EINVAL; }
  const auto t0 = std::chrono::steady_clock::now();
  bool stale = !g->graph;
  for (int i = 0; i < n; ++i) {
    BatchCtx& b = *g->b[i];
    SADMM_CUDA_TRY(cudaStreamSynchronize(b.st));
    SADMM_TRY(batch_setup(b));
    if (g->epochs[i] != b.epoch) stale = true;
  }
  if (stale) SADMM_TRY(group_capture(g));
  for (int i = 0; i < n; ++i) SADMM_TRY(batch_reset(*g->b[i], y[i], g->st));
  for (int it = 0; it < iters; ++it) {
    SADMM_CUDA_TRY(cudaGraphLaunch(g->graph, g->st));
    for (int kk = 0; kk < g->kernels_per_iter; ++kk) count_launch();
  }
  for (int i = 0; i < n; ++i) SADMM_TRY(batch_collect(*g->b[i], x_out ? x_out[i] : nullptr, g->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(g->st));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int rc = SADMM_OK;
  for (int i = 0; i < n; ++i) {
    const int r = batch_finish(*g->b[i], iters, st ? &st[i] : nullptr, ms);
    if (rc == SADMM_OK) rc = r;
  }
  return rc;
}

void sadmm_batch_group_destroy(sadmm_batch_group_t g) {
  if (!g) return;
  cudaStreamSynchronize(g->st);
  group_release(g);
}

}  // extern "C"
