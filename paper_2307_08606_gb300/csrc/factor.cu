// FP64 factor of the x-update system (Eq. 3, x_q-update):
//   F = (rho I + mu G)^{-1},  G = B_J B_J^T (Woodbury form, 2KM x 2KM) or
//                             G = B_J^T B_J (primal form, |J| x |J|),
// with B_J the real form of the active columns, rows interleaved (re, im) per
// sample so that column p of B_J is the pixel-major column idx[p] of A read as
// 2KM floats.  Steps: Gram (SIMT FP64, 64x64 tiles), right-looking blocked
// Cholesky (diagonal block factor + its inverse, panel solve as a GEMM with
// the inverse, trailing update), blocked inverse of the Cholesky factor by
// block rows, and F = L^{-T} L^{-1}.  Matrices are padded to a multiple of 64
// with an identity block so that every tile is full.
#include "common.cuh"
#include <math.h>

#include <algorithm>
#include <vector>

namespace sadmm {

namespace {

constexpr int T = kTile;      // 64
constexpr int KB = 16;        // k-slab staged in shared memory
constexpr int kThreads = 256; // 16 x 16 threads, 4 x 4 outputs each

using JobBlock = SetBlock<FactorJob>;

// acc[a][b] += sum_k As[k][ty + 16a] * Bs[k][tx + 16b]
__device__ __forceinline__ void mma_slab(double (&acc)[4][4], const double (*As)[T],
                                         const double (*Bs)[T], int ty, int tx) {
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = As[k][ty + 16 * u]; b[u] = Bs[k][tx + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
}

__device__ __forceinline__ void zero_acc(double (&acc)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
}

// Linear index of a lower-triangular tile -> (row, col), row >= col.
__device__ __forceinline__ void tri_decode(int t, int& r, int& c) {
  r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  c = t - r * (r + 1) / 2;
}

// ---------------------------------------------------------------- Gram
__global__ void __launch_bounds__(kThreads)
gram_kernel(const __grid_constant__ JobBlock jobs, int KM, double mu, double rho) {
  const FactorJob& jb = jobs.v[blockIdx.z];
  const int Tn = jb.npad / T;
  int bi, bj;
  tri_decode(blockIdx.x, bi, bj);
  if (bi >= Tn) return;
  __shared__ double As[KB][T], Bs[KB][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  double acc[4][4];
  zero_acc(acc);
  const float* Af = reinterpret_cast<const float*>(jb.A);
  const size_t twoKM = 2 * (size_t)KM;
  if (jb.woodbury) {
    // G[r1][r2] = sum_p B[r1][p] B[r2][p], B[r][p] = Af[idx[p] * 2KM + r]
    const int K = jb.ncols;
    for (int k0 = 0; k0 < K; k0 += KB) {
      for (int e = tid; e < KB * T; e += kThreads) {
        const int kk = e / T, ii = e % T, p = k0 + kk;
        double a = 0.0, b = 0.0;
        if (p < K) {
          const size_t base = (size_t)jb.idx[p] * twoKM;
          a = Af[base + bi * T + ii];
          b = Af[base + bj * T + ii];
        }
        As[kk][ii] = a;
        Bs[kk][ii] = b;
      }
      __syncthreads();
      mma_slab(acc, As, Bs, ty, tx);
      __syncthreads();
    }
  } else {
    // G[a][b] = sum_r B[r][a] B[r][b] over the 2KM rows
    const int K = 2 * KM, n = jb.n;
    for (int k0 = 0; k0 < K; k0 += KB) {
      for (int e = tid; e < KB * T; e += kThreads) {
        const int ii = e / KB, kk = e % KB;
        const int ra = bi * T + ii, rb = bj * T + ii;
        As[kk][ii] = ra < n ? (double)Af[(size_t)jb.idx[ra] * twoKM + k0 + kk] : 0.0;
        Bs[kk][ii] = rb < n ? (double)Af[(size_t)jb.idx[rb] * twoKM + k0 + kk] : 0.0;
      }
      __syncthreads();
      mma_slab(acc, As, Bs, ty, tx);
      __syncthreads();
    }
  }
  const int n = jb.n, ld = jb.npad;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = bi * T + ty + 16 * u, j = bj * T + tx + 16 * v;
      double val;
      if (i < n && j < n) val = mu * acc[u][v] + (i == j ? rho : 0.0);
      else val = (i == j) ? 1.0 : 0.0;
      jb.out[(size_t)i * ld + j] = val;
      if (bi != bj) jb.out[(size_t)j * ld + i] = val;
    }
}

// ---------------------------------------------------------------- Cholesky
// Factor the diagonal block kb in shared memory (unblocked right-looking),
// write L_kk (upper part zero) and its inverse Dinv_kk.
__global__ void __launch_bounds__(kThreads)
potrf_diag_kernel(const __grid_constant__ JobBlock jobs, int kb, int* status) {
  const FactorJob& jb = jobs.v[blockIdx.x];
  if (kb >= jb.npad / T) return;
  extern __shared__ double sm[];
  double (*a)[T + 1] = reinterpret_cast<double (*)[T + 1]>(sm);
  double (*inv)[T + 1] = reinterpret_cast<double (*)[T + 1]>(sm + T * (T + 1));
  const int tid = threadIdx.x, ld = jb.npad;
  double* blk = jb.out + (size_t)kb * T * ld + (size_t)kb * T;
  for (int e = tid; e < T * T; e += kThreads) a[e / T][e % T] = blk[(size_t)(e / T) * ld + e % T];
  __syncthreads();
  for (int j = 0; j < T; ++j) {
    double d = a[j][j];
    __syncthreads();
    if (!(d > 0.0) || !isfinite(d)) {
      if (tid == 0) status[blockIdx.x] = 1;
      d = 1.0;
    }
    d = sqrt(d);
    for (int i = j + tid; i < T; i += kThreads) a[i][j] = (i == j) ? d : a[i][j] / d;
    __syncthreads();
    for (int e = tid; e < T * T; e += kThreads) {
      const int i = e / T, c = e % T;
      if (c > j && i >= c) a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, row by row (threads over columns)
  for (int i = 0; i < T; ++i) {
    if (tid < T) {
      const int c = tid;
      double v = 0.0;
      if (c <= i) {
        double s = (c == i) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s = fma(-a[i][k], inv[k][c], s);
        v = s / a[i][i];
      }
      inv[i][c] = v;
    }
    __syncthreads();
  }
  double* dv = jb.dinv + (size_t)kb * T * T;
  for (int e = tid; e < T * T; e += kThreads) {
    const int i = e / T, c = e % T;
    blk[(size_t)i * ld + c] = c <= i ? a[i][c] : 0.0;
    dv[e] = inv[i][c];
  }
}

// L_ib,kb = A_ib,kb * Dinv_kb^T for the blocks below the diagonal.
__global__ void __launch_bounds__(kThreads)
trsm_kernel(const __grid_constant__ JobBlock jobs, int kb) {
  const FactorJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.npad / T, ib = kb + 1 + blockIdx.x;
  if (ib >= Tn) return;
  __shared__ double As[KB][T], Bs[KB][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16, ld = jb.npad;
  double* blk = jb.out + (size_t)ib * T * ld + (size_t)kb * T;
  const double* dv = jb.dinv + (size_t)kb * T * T;
  double acc[4][4];
  zero_acc(acc);
  for (int k0 = 0; k0 < T; k0 += KB) {
    for (int e = tid; e < KB * T; e += kThreads) {
      const int ii = e / KB, kk = e % KB;
      As[kk][ii] = blk[(size_t)ii * ld + k0 + kk];   // A[i][k]
      Bs[kk][ii] = dv[ii * T + k0 + kk];             // Dinv[j][k]
    }
    __syncthreads();
    mma_slab(acc, As, Bs, ty, tx);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) blk[(size_t)(ty + 16 * u) * ld + tx + 16 * v] = acc[u][v];
}

// A_ij -= L_ik L_jk^T on the trailing lower tiles (i >= j > kb).
__global__ void __launch_bounds__(kThreads)
syrk_update_kernel(const __grid_constant__ JobBlock jobs, int kb) {
  const FactorJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.npad / T, m = Tn - kb - 1;
  if ((int)blockIdx.x >= m * (m + 1) / 2) return;
  int r, c;
  tri_decode(blockIdx.x, r, c);
  const int ib = kb + 1 + r, jbk = kb + 1 + c;
  __shared__ double As[KB][T], Bs[KB][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16, ld = jb.npad;
  const double* Li = jb.out + (size_t)ib * T * ld + (size_t)kb * T;
  const double* Lj = jb.out + (size_t)jbk * T * ld + (size_t)kb * T;
  double acc[4][4];
  zero_acc(acc);
  for (int k0 = 0; k0 < T; k0 += KB) {
    for (int e = tid; e < KB * T; e += kThreads) {
      const int ii = e / KB, kk = e % KB;
      As[kk][ii] = Li[(size_t)ii * ld + k0 + kk];
      Bs[kk][ii] = Lj[(size_t)ii * ld + k0 + kk];
    }
    __syncthreads();
    mma_slab(acc, As, Bs, ty, tx);
    __syncthreads();
  }
  double* Cb = jb.out + (size_t)ib * T * ld + (size_t)jbk * T;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Cb[(size_t)(ty + 16 * u) * ld + tx + 16 * v] -= acc[u][v];
}

// ------------------------------------------------------------- L^{-1}
// tmp diagonal blocks <- Dinv (upper parts zero from the diagonal factor)
__global__ void linv_diag_kernel(const __grid_constant__ JobBlock jobs) {
  const FactorJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.npad / T, b = blockIdx.x;
  if (b >= Tn) return;
  const double* dv = jb.dinv + (size_t)b * T * T;
  double* dst = jb.tmp + (size_t)b * T * jb.npad + (size_t)b * T;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) dst[(size_t)(e / T) * jb.npad + e % T] = dv[e];
}

// Block row i of L^{-1}: X_ij = -Dinv_i * sum_{k=j}^{i-1} L_ik X_kj, j < i.
__global__ void __launch_bounds__(kThreads)
linv_row_kernel(const __grid_constant__ JobBlock jobs, int i) {
  const FactorJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.npad / T, j = blockIdx.x;
  if (i >= Tn || j >= i) return;
  __shared__ double As[KB][T], Bs[KB][T];
  __shared__ double Ts[T][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16, ld = jb.npad;
  double acc[4][4];
  zero_acc(acc);
  for (int k = j; k < i; ++k) {
    const double* Lik = jb.out + (size_t)i * T * ld + (size_t)k * T;
    const double* Xkj = jb.tmp + (size_t)k * T * ld + (size_t)j * T;
    for (int k0 = 0; k0 < T; k0 += KB) {
      for (int e = tid; e < KB * T; e += kThreads) {
        const int ii = e / KB, kk = e % KB;
        As[kk][ii] = Lik[(size_t)ii * ld + k0 + kk];       // L[i][k]
        const int kk2 = e / T, jj = e % T;
        Bs[kk2][jj] = Xkj[(size_t)(k0 + kk2) * ld + jj];   // X[k][j]
      }
      __syncthreads();
      mma_slab(acc, As, Bs, ty, tx);
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Ts[ty + 16 * u][tx + 16 * v] = acc[u][v];
  __syncthreads();
  const double* dv = jb.dinv + (size_t)i * T * T;
  zero_acc(acc);
  for (int k0 = 0; k0 < T; k0 += KB) {
    for (int e = tid; e < KB * T; e += kThreads) {
      const int ii = e / KB, kk = e % KB;
      As[kk][ii] = dv[ii * T + k0 + kk];                   // Dinv[i][m]
      const int kk2 = e / T, jj = e % T;
      Bs[kk2][jj] = Ts[k0 + kk2][jj];                      // T1[m][j]
    }
    __syncthreads();
    mma_slab(acc, As, Bs, ty, tx);
    __syncthreads();
  }
  double* dst = jb.tmp + (size_t)i * T * ld + (size_t)j * T;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[(size_t)(ty + 16 * u) * ld + tx + 16 * v] = -acc[u][v];
}

// F_ab = sum_{k >= a} X_ka^T X_kb for a >= b, mirrored to the upper triangle.
__global__ void __launch_bounds__(kThreads)
inverse_kernel(const __grid_constant__ JobBlock jobs) {
  const FactorJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.npad / T;
  if ((int)blockIdx.x >= Tn * (Tn + 1) / 2) return;
  int a, b;
  tri_decode(blockIdx.x, a, b);
  __shared__ double As[KB][T], Bs[KB][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16, ld = jb.npad;
  double acc[4][4];
  zero_acc(acc);
  for (int k = a; k < Tn; ++k) {
    const double* Xa = jb.tmp + (size_t)k * T * ld + (size_t)a * T;
    const double* Xb = jb.tmp + (size_t)k * T * ld + (size_t)b * T;
    for (int k0 = 0; k0 < T; k0 += KB) {
      for (int e = tid; e < KB * T; e += kThreads) {
        const int kk = e / T, ii = e % T;
        As[kk][ii] = Xa[(size_t)(k0 + kk) * ld + ii];
        Bs[kk][ii] = Xb[(size_t)(k0 + kk) * ld + ii];
      }
      __syncthreads();
      mma_slab(acc, As, Bs, ty, tx);
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = a * T + ty + 16 * u, j = b * T + tx + 16 * v;
      jb.out[(size_t)i * ld + j] = acc[u][v];
      if (a != b) jb.out[(size_t)j * ld + i] = acc[u][v];
    }
}

// ---------------------------------------------------------------- downdate
constexpr int DM = kDowndateMax;          // 32
constexpr int kFewColumns = 6;            // single-column applies up to this many columns per job
constexpr int kDdWarps = 8;
constexpr int kDdChunk = 512;             // rows of U staged per shared-memory pass
using DdBlock = SetBlock<DowndateJob>;

// P = W U: one warp per row of W, lanes stride the row; U (the removed
// columns of B as doubles) is staged in shared memory column by column in
// chunks of rows (consecutive lanes read consecutive rows: no bank conflicts).
template <int EB>
struct DdShape {
  static constexpr int rows = EB <= 8 ? 4 : (EB <= 16 ? 2 : 1);   // rows per warp
};

template <int EB>
__global__ void __launch_bounds__(kDdWarps * 32)
dd_p_kernel(const __grid_constant__ DdBlock jobs, int KM) {
  constexpr int RPW = DdShape<EB>::rows;
  extern __shared__ double s_u[];                 // [EB][kDdChunk]
  const DowndateJob& jb = jobs.v[blockIdx.y];
  const int n = jb.n, e = jb.e;
  const int rbeg = blockIdx.x * kDdWarps * RPW;
  if (rbeg >= n) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* Af = reinterpret_cast<const float*>(jb.A);
  const size_t twoKM = 2 * (size_t)KM;
  double acc[RPW][EB];
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int c = 0; c < EB; ++c) acc[r][c] = 0.0;
  for (int j0 = 0; j0 < n; j0 += kDdChunk) {
    const int nj = min(kDdChunk, n - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < kDdChunk * EB; t += blockDim.x) {
      const int c = t / kDdChunk, jj = t % kDdChunk;
      double v = 0.0;
      if (c < e && jj < nj) v = (double)Af[(size_t)jb.E[c] * twoKM + j0 + jj];
      s_u[c * kDdChunk + jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int i = rbeg + warp * RPW + r;
      if (i >= n) break;
      const double* row = jb.Wsrc + (size_t)i * n + j0;
      for (int jj = lane; jj < nj; jj += 32) {
        const double w = __ldcs(row + jj);
#pragma unroll
        for (int c = 0; c < EB; ++c) acc[r][c] = fma(w, s_u[c * kDdChunk + jj], acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int i = rbeg + warp * RPW + r;
#pragma unroll
    for (int c = 0; c < EB; ++c) {
      double v = acc[r][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (i < n && lane == c) jb.P[(size_t)i * DM + c] = (c < e) ? v : 0.0;
    }
  }
  // columns EB..DM-1 of P are never written by this kernel: zero them
  if constexpr (EB < DM) {
    for (int t = threadIdx.x; t < kDdWarps * RPW * (DM - EB); t += blockDim.x) {
      const int i = rbeg + t / (DM - EB), c = EB + t % (DM - EB);
      if (i < n) jb.P[(size_t)i * DM + c] = 0.0;
    }
  }
}

// Spart[blk][a][b] = sum over 256 rows of U[i][a] P[i][b] (fixed order per thread).
__global__ void dd_s_kernel(const __grid_constant__ DdBlock jobs, int KM) {
  const DowndateJob& jb = jobs.v[blockIdx.y];
  const int a = threadIdx.x / DM, b = threadIdx.x % DM;
  const int i0 = blockIdx.x * 256;
  if (i0 >= jb.n) return;
  double acc = 0.0;
  if (a < jb.e && b < jb.e) {
    const float* col = reinterpret_cast<const float*>(jb.A) + (size_t)jb.E[a] * 2 * KM;
    const int i1 = min(jb.n, i0 + 256);
    for (int i = i0; i < i1; ++i) acc = fma((double)col[i], jb.P[(size_t)i * DM + b], acc);
  }
  jb.Spart[((size_t)blockIdx.x * DM + a) * DM + b] = acc;
}

// S = I - mu sum_blk Spart[blk]; Cholesky S = L L^T and L^{-1} in shared memory
// (identity beyond e); writes L^{-1} to jb.S.
__global__ void __launch_bounds__(DM * DM)
dd_chol_kernel(const __grid_constant__ DdBlock jobs, double mu, int* status) {
  const DowndateJob& jb = jobs.v[blockIdx.x];
  __shared__ double L[DM][DM + 1], Li[DM][DM + 1];
  const int a = threadIdx.x / DM, b = threadIdx.x % DM;
  const int nblk = (jb.n + 255) / 256;
  double sum = 0.0;
  for (int k = 0; k < nblk; ++k) sum += jb.Spart[((size_t)k * DM + a) * DM + b];
  L[a][b] = (a < jb.e && b < jb.e) ? ((a == b ? 1.0 : 0.0) - jb.sign * mu * sum) : (a == b ? 1.0 : 0.0);
  __syncthreads();
  for (int j = 0; j < DM; ++j) {
    double d = L[j][j];
    __syncthreads();
    if (!(d > 0.0) || !isfinite(d)) {
      if (threadIdx.x == 0) status[jb.slot] = 1;
      d = 1.0;
    }
    d = sqrt(d);
    if (b == j && a >= j) L[a][j] = (a == j) ? d : L[a][j] / d;
    __syncthreads();
    if (b > j && a >= b) L[a][b] = fma(-L[a][j], L[b][j], L[a][b]);
    __syncthreads();
  }
  for (int i = 0; i < DM; ++i) {
    if (threadIdx.x < DM) {
      const int c = threadIdx.x;
      double v = 0.0;
      if (c <= i) {
        double s = (c == i) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s = fma(-L[i][k], Li[k][c], s);
        v = s / L[i][i];
      }
      Li[i][c] = v;
    }
    __syncthreads();
  }
  jb.S[a * DM + b] = Li[a][b];
}

// T = P L^{-T} row by row, in place in P.
__global__ void dd_t_kernel(const __grid_constant__ DdBlock jobs) {
  const DowndateJob& jb = jobs.v[blockIdx.y];
  __shared__ double Li[DM][DM];
  for (int t = threadIdx.x; t < DM * DM; t += blockDim.x) Li[t / DM][t % DM] = jb.S[t];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= jb.n) return;
  double p[DM];
#pragma unroll
  for (int c = 0; c < DM; ++c) p[c] = jb.P[(size_t)i * DM + c];
#pragma unroll
  for (int c = 0; c < DM; ++c) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k <= c; ++k) t = fma(p[k], Li[c][k], t);
    jb.P[(size_t)i * DM + c] = t;
  }
}

// Wdst = Wsrc + mu T T^T on the lower 64x64 tiles, written to both triangles.
__global__ void __launch_bounds__(kThreads)
dd_w_kernel(const __grid_constant__ DdBlock jobs, double mu) {
  const DowndateJob& jb = jobs.v[blockIdx.y];
  const int Tn = jb.n / T;
  if ((int)blockIdx.x >= Tn * (Tn + 1) / 2) return;
  int bi, bj;
  tri_decode(blockIdx.x, bi, bj);
  __shared__ double Ti[DM][T], Tj[DM][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  for (int t = tid; t < DM * T; t += kThreads) {
    const int r = t / DM, c = t % DM;
    Ti[c][r] = jb.P[(size_t)(bi * T + r) * DM + c];
    Tj[c][r] = jb.P[(size_t)(bj * T + r) * DM + c];
  }
  __syncthreads();
  double acc[4][4];
  zero_acc(acc);
  for (int c = 0; c < jb.e; ++c) {
    double x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { x[u] = Ti[c][ty + 16 * u]; y[u] = Tj[c][tx + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
  }
  const size_t n = jb.n;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const size_t i = bi * T + ty + 16 * u, j = bj * T + tx + 16 * v;
      const double val = jb.Wsrc[i * n + j] + jb.sign * mu * acc[u][v];
      jb.Wdst[i * n + j] = val;
      if (bi != bj) jb.Wdst[j * n + i] = val;
    }
}

// Fdst = Fsrc + sign mu T T^T on the packed upper-triangular 64x64 tiles of
// (hi, lo) pairs.  T (n x 32 FP64, columns >= e zero) is split into pairs in
// shared memory; each element accumulates its e products T_ik T_jk in
// double-float arithmetic (hi*hi exactly by FMA, plus the two cross terms),
// is scaled by sign mu (a pair) and added to the stored pair with a two-sum.
__device__ __forceinline__ void dfp_add(float& sh, float& sl, float p, float e) {
  const float t = sh + p;
  const float bp = t - sh;
  sl += ((sh - (t - bp)) + (p - bp)) + e;
  sh = t;
}

__global__ void __launch_bounds__(kThreads)
ddw_pairs_kernel(const __grid_constant__ DdBlock jobs, double mu) {
  const DowndateJob& jb = jobs.v[blockIdx.y];
  const int nt = jb.n / T;
  const int ntile = nt * (nt + 1) / 2;
  if ((int)blockIdx.x >= ntile) return;
  // tile number -> (I, J), I <= J, row-block-major (the packed order)
  int I = 0, t = blockIdx.x;
  while (t >= nt - I) { t -= nt - I; ++I; }
  const int J = I + t;
  __shared__ float Ih[DM][T], Il[DM][T], Jh[DM][T], Jl[DM][T];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  for (int q = tid; q < DM * T; q += kThreads) {
    const int r = q / DM, c = q % DM;
    const double a = jb.P[(size_t)(I * T + r) * DM + c], b = jb.P[(size_t)(J * T + r) * DM + c];
    const float ah = (float)a, bh = (float)b;
    Ih[c][r] = ah; Il[c][r] = (float)(a - (double)ah);
    Jh[c][r] = bh; Jl[c][r] = (float)(b - (double)bh);
  }
  __syncthreads();
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { sh[u][v] = 0.f; sl[u][v] = 0.f; }
  for (int c = 0; c < jb.e; ++c) {
    float xh[4], xl[4], yh[4], yl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xh[u] = Ih[c][ty + 16 * u]; xl[u] = Il[c][ty + 16 * u];
      yh[u] = Jh[c][tx + 16 * u]; yl[u] = Jl[c][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float p = xh[u] * yh[v];
        float e = fmaf(xh[u], yh[v], -p);
        e = fmaf(xh[u], yl[v], fmaf(xl[u], yh[v], e));
        dfp_add(sh[u][v], sl[u][v], p, e);
      }
  }
  const double smu = jb.sign * mu;
  const float mh = (float)smu, ml = (float)(smu - (double)mh);
  const size_t tile = (size_t)I * nt - (size_t)I * (I - 1) / 2 + (J - I);
  const float2* src = jb.Fsrc + tile * T * T;
  float2* dst = jb.Fdst + tile * T * T;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int e = (ty + 16 * u) * T + tx + 16 * v;
      // (mh + ml) (sh + sl), then added to the stored pair
      const float p = mh * sh[u][v];
      float err = fmaf(mh, sh[u][v], -p);
      err = fmaf(mh, sl[u][v], fmaf(ml, sh[u][v], err));
      const float2 w = src[e];
      float h = w.x, l = w.y;
      dfp_add(h, l, p, err);
      const float hn = h + l;
      dst[e] = make_float2(hn, l - (hn - h));
    }
}

template <int EB>
int launch_dd_p(const DdBlock& blk, int njobs, int n_max, int KM, cudaStream_t st) {
  const size_t smem = (size_t)kDdChunk * EB * sizeof(double);
  static bool configured = false;
  if (!configured) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(dd_p_kernel<EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    configured = true;
  }
  dd_p_kernel<EB><<<dim3(div_up(n_max, kDdWarps * DdShape<EB>::rows), njobs), kDdWarps * 32, smem, st>>>(blk, KM);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace

size_t downdate_scratch_doubles(int n) {
  return (size_t)(div_up(n, 256) + 1) * DM * DM;
}

int run_downdate(const DowndateJob* jobs, int njobs, int KM, double mu, int* d_status, cudaStream_t st) {
  if (njobs <= 0) return SADMM_OK;
  if (njobs > kMaxSets) { set_error("run_downdate: too many jobs"); return SADMM_EINVAL; }
  DdBlock blk;
  int n_max = 0, e_max = 0;
  for (int i = 0; i < njobs; ++i) {
    blk.v[i] = jobs[i];
    if (jobs[i].e < 1 || jobs[i].e > DM || jobs[i].n % T != 0) {
      set_error("run_downdate: bad job (e=%d n=%d)", jobs[i].e, jobs[i].n);
      return SADMM_EINVAL;
    }
    n_max = max(n_max, jobs[i].n);
    e_max = max(e_max, jobs[i].e);
  }
  if (e_max <= 4) SADMM_TRY(launch_dd_p<4>(blk, njobs, n_max, KM, st));
  else if (e_max <= 8) SADMM_TRY(launch_dd_p<8>(blk, njobs, n_max, KM, st));
  else if (e_max <= 16) SADMM_TRY(launch_dd_p<16>(blk, njobs, n_max, KM, st));
  else SADMM_TRY(launch_dd_p<32>(blk, njobs, n_max, KM, st));
  dd_s_kernel<<<dim3(div_up(n_max, 256), njobs), DM * DM, 0, st>>>(blk, KM);
  SADMM_LAUNCH_CHECK();
  dd_chol_kernel<<<njobs, DM * DM, 0, st>>>(blk, mu, d_status);
  SADMM_LAUNCH_CHECK();
  dd_t_kernel<<<dim3(div_up(n_max, 128), njobs), 128, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  const int Tn = n_max / T;
  dd_w_kernel<<<dim3(Tn * (Tn + 1) / 2, njobs), kThreads, 0, st>>>(blk, mu);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int run_downdate_pairs(const DowndateJob* jobs, int njobs, int KM, double mu, const DdScratch& scr, int* d_status,
                       int* err, cudaStream_t st) {
  if (njobs <= 0) return SADMM_OK;
  if (njobs > kMaxSets) { set_error("run_downdate_pairs: too many jobs"); return SADMM_EINVAL; }
  DdBlock blk;
  int n_max = 0, e_max = 0;
  std::vector<const float2*> F(njobs), A(njobs);
  std::vector<const int*> E(njobs);
  std::vector<int> e(njobs);
  std::vector<double*> P(njobs);
  for (int i = 0; i < njobs; ++i) {
    blk.v[i] = jobs[i];
    if (jobs[i].e < 1 || jobs[i].e > DM || jobs[i].n % T != 0 || !jobs[i].Fsrc || !jobs[i].Fdst ||
        (i > 0 && jobs[i].n != jobs[0].n)) {
      set_error("run_downdate_pairs: bad job (e=%d n=%d)", jobs[i].e, jobs[i].n);
      return SADMM_EINVAL;
    }
    n_max = max(n_max, jobs[i].n);
    e_max = max(e_max, jobs[i].e);
    F[i] = jobs[i].Fsrc; A[i] = jobs[i].A; E[i] = jobs[i].E; e[i] = jobs[i].e; P[i] = jobs[i].P;
    // columns e..31 of P must be zero for the kernels below
    SADMM_CUDA_TRY(cudaMemsetAsync(jobs[i].P, 0, (size_t)jobs[i].n * DM * sizeof(double), st));
  }
  // P = W U.  A few columns: one single-column symmetric apply each (its
  // arithmetic is one product per element); more: sixteen columns per
  // packed-tile pass (one read of W for all of them).
  if (e_max <= kFewColumns) {
    std::vector<int> Eh((size_t)njobs * DM);
    for (int i = 0; i < njobs; ++i)
      SADMM_CUDA_TRY(cudaMemcpyAsync(Eh.data() + (size_t)i * DM, jobs[i].E, jobs[i].e * sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<SpdSet> sets;
    const size_t stride = sym_part_pairs(n_max);
    for (int i = 0; i < njobs; ++i)
      for (int c = 0; c < jobs[i].e; ++c) {
        SpdSet s{};
        s.P = jobs[i].Fsrc;
        s.n = jobs[i].n;
        s.u = reinterpret_cast<const float*>(jobs[i].A) + (size_t)Eh[(size_t)i * DM + c] * 2 * KM;
        s.part = scr.part + (size_t)(sets.size() % kMaxSets) * stride;
        s.outd = jobs[i].P + c;
        s.ldd = DM;
        sets.push_back(s);
      }
    SolverView sv{};
    for (size_t b = 0; b < sets.size(); b += kMaxSets)
      SADMM_TRY(launch_spd_apply(sets.data() + b, (int)std::min<size_t>(kMaxSets, sets.size() - b), false, sv, err, st));
  } else {
    for (int c0 = 0; c0 < e_max; c0 += 16)
      SADMM_TRY(launch_multi_apply_cols(F.data(), A.data(), E.data(), e.data(), P.data(), njobs, n_max, c0, scr.U,
                                        scr.dptrs, scr.part, err, st));
  }
  dd_s_kernel<<<dim3(div_up(n_max, 256), njobs), DM * DM, 0, st>>>(blk, KM);
  SADMM_LAUNCH_CHECK();
  dd_chol_kernel<<<njobs, DM * DM, 0, st>>>(blk, mu, d_status);
  SADMM_LAUNCH_CHECK();
  dd_t_kernel<<<dim3(div_up(n_max, 128), njobs), 128, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  const int Tn = n_max / T;
  ddw_pairs_kernel<<<dim3(Tn * (Tn + 1) / 2, njobs), kThreads, 0, st>>>(blk, mu);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// ------------------------------------------------------- primal downdate
// Removing the pixels E from the ordered list J_old leaves the principal
// submatrix M_RR of M = rho I + mu B_J^T B_J, and (M_RR)^{-1} is the Schur
// complement of H_EE in H = M^{-1}:  H_RR - H_RE H_EE^{-1} H_ER.  With
// H_EE = L L^T and V = H_RE L^{-T} that is H_RR - V V^T, O(n^2 e) in FP64
// instead of the Gram, Cholesky and inverse of a refactorisation.
namespace {

using PddBlock = SetBlock<PrimalDdJob>;

// old positions: kept row p sits at p + #{E < J[p]}, removed row k at
// k + #{J < E[k]} (both lists ascending and disjoint)
__global__ void pdd_pos_kernel(const __grid_constant__ PddBlock jobs) {
  const PrimalDdJob& jb = jobs.v[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= jb.n_new + jb.e) return;
  const bool kept = t < jb.n_new;
  const int x = kept ? jb.J[t] : jb.E[t - jb.n_new];
  const int* other = kept ? jb.E : jb.J;
  int lo = 0, hi = kept ? jb.e : jb.n_new;            // count of other[] < x
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (other[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  jb.pos[t] = (kept ? t : t - jb.n_new) + lo;
}

// V[i][k] = H[pos_i][pos_{n+k}] (zero past e)
__global__ void pdd_gather_kernel(const __grid_constant__ PddBlock jobs) {
  const PrimalDdJob& jb = jobs.v[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= jb.n_new) return;
  const double* row = jb.H + (size_t)jb.pos[i] * jb.ldh;
#pragma unroll 4
  for (int k = 0; k < DM; ++k) jb.V[(size_t)i * DM + k] = k < jb.e ? row[jb.pos[jb.n_new + k]] : 0.0;
}

// L^{-1} of H_EE = L L^T (identity past e), into V + n_new * DM
__global__ void __launch_bounds__(DM * DM)
pdd_chol_kernel(const __grid_constant__ PddBlock jobs, int* status) {
  const PrimalDdJob& jb = jobs.v[blockIdx.x];
  __shared__ double L[DM][DM + 1], Li[DM][DM + 1];
  const int a = threadIdx.x / DM, b = threadIdx.x % DM;
  L[a][b] = (a < jb.e && b < jb.e) ? jb.H[(size_t)jb.pos[jb.n_new + a] * jb.ldh + jb.pos[jb.n_new + b]]
                                   : (a == b ? 1.0 : 0.0);
  __syncthreads();
  for (int j = 0; j < DM; ++j) {
    double d = L[j][j];
    __syncthreads();
    if (!(d > 0.0) || !isfinite(d)) {
      if (threadIdx.x == 0) status[jb.slot] = 1;
      d = 1.0;
    }
    d = sqrt(d);
    if (b == j && a >= j) L[a][j] = (a == j) ? d : L[a][j] / d;
    __syncthreads();
    if (b > j && a >= b) L[a][b] = fma(-L[a][j], L[b][j], L[a][b]);
    __syncthreads();
  }
  for (int i = 0; i < DM; ++i) {
    if (threadIdx.x < DM) {
      const int c = threadIdx.x;
      double v = 0.0;
      if (c <= i) {
        double s = (c == i) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s = fma(-L[i][k], Li[k][c], s);
        v = s / L[i][i];
      }
      Li[i][c] = v;
    }
    __syncthreads();
  }
  jb.V[(size_t)jb.n_new * DM + a * DM + b] = Li[a][b];
}

// V = H_RE L^{-T}, row by row in place
__global__ void pdd_t_kernel(const __grid_constant__ PddBlock jobs) {
  const PrimalDdJob& jb = jobs.v[blockIdx.y];
  __shared__ double Li[DM][DM];
  for (int t = threadIdx.x; t < DM * DM; t += blockDim.x) Li[t / DM][t % DM] = jb.V[(size_t)jb.n_new * DM + t];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= jb.n_new) return;
  double p[DM];
#pragma unroll
  for (int c = 0; c < DM; ++c) p[c] = jb.V[(size_t)i * DM + c];
#pragma unroll
  for (int c = 0; c < DM; ++c) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k <= c; ++k) t = fma(p[k], Li[c][k], t);
    jb.V[(size_t)i * DM + c] = t;
  }
}

// Hn[i][j] = H[pos_i][pos_j] - sum_k V[i][k] V[j][k] for i, j < n_new; the
// identity on the padding up to ldn.  16 x 16 threads per 16 x 16 block,
// the two blocks of V rows staged in shared memory.
__global__ void __launch_bounds__(256)
pdd_update_kernel(const __grid_constant__ PddBlock jobs) {
  const PrimalDdJob& jb = jobs.v[blockIdx.z];
  __shared__ double Vi[16][DM + 1], Vj[16][DM + 1];
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  if (i0 >= jb.ldn || j0 >= jb.ldn) return;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  for (int t = threadIdx.x; t < 16 * DM; t += 256) {
    const int r = t / DM, k = t % DM;
    Vi[r][k] = (i0 + r < jb.n_new) ? jb.V[(size_t)(i0 + r) * DM + k] : 0.0;
    Vj[r][k] = (j0 + r < jb.n_new) ? jb.V[(size_t)(j0 + r) * DM + k] : 0.0;
  }
  __syncthreads();
  const int i = i0 + ty, j = j0 + tx;
  double h;
  if (i < jb.n_new && j < jb.n_new) {
    h = jb.H[(size_t)jb.pos[i] * jb.ldh + jb.pos[j]];
    for (int k = 0; k < jb.e; ++k) h = fma(-Vi[ty][k], Vj[tx][k], h);
  } else {
    h = (i == j) ? 1.0 : 0.0;
  }
  jb.Hn[(size_t)i * jb.ldn + j] = h;
}

}  // namespace

namespace {
// out = the ascending merge of two ascending, disjoint lists: element t of a
// goes to t + #{b < a[t]}, element t of b to t + #{a < b[t]}
__global__ void merge_lists_kernel(const int* __restrict__ a, int na, const int* __restrict__ b, int nb,
                                   int* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= na + nb) return;
  const bool in_a = t < na;
  const int x = in_a ? a[t] : b[t - na];
  const int* other = in_a ? b : a;
  int lo = 0, hi = in_a ? nb : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (other[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  out[(in_a ? t : t - na) + lo] = x;
}
}  // namespace

int launch_merge_lists(const int* a, int na, const int* b, int nb, int* out, cudaStream_t st) {
  if (na + nb <= 0) return SADMM_OK;
  merge_lists_kernel<<<div_up(na + nb, 256), 256, 0, st>>>(a, na, b, nb, out);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int run_primal_downdate(const PrimalDdJob* jobs, int njobs, int* d_status, cudaStream_t st) {
  if (njobs <= 0) return SADMM_OK;
  if (njobs > kMaxSets) { set_error("run_primal_downdate: too many jobs"); return SADMM_EINVAL; }
  PddBlock blk;
  int nmax = 1, ldmax = 1;
  for (int i = 0; i < njobs; ++i) {
    const PrimalDdJob& j = jobs[i];
    if (j.e < 1 || j.e > DM || j.n_new < 1 || j.ldn < j.n_new || j.ldn % T != 0) {
      set_error("run_primal_downdate: bad sizes");
      return SADMM_EINVAL;
    }
    blk.v[i] = j;
    nmax = max(nmax, j.n_new + j.e);
    ldmax = max(ldmax, j.ldn);
  }
  pdd_pos_kernel<<<dim3(div_up(nmax, 256), njobs), 256, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  pdd_gather_kernel<<<dim3(div_up(nmax, 128), njobs), 128, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  pdd_chol_kernel<<<njobs, DM * DM, 0, st>>>(blk, d_status);
  SADMM_LAUNCH_CHECK();
  pdd_t_kernel<<<dim3(div_up(nmax, 128), njobs), 128, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  pdd_update_kernel<<<dim3(ldmax / 16, ldmax / 16, njobs), 256, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int run_gram(const FactorJob& job, int KM, double mu, double rho, int* d_status, cudaStream_t st, int gram) {
  if (job.npad % T != 0 || job.n > job.npad) {
    set_error("run_gram: bad padding");
    return SADMM_EINVAL;
  }
  if (gram == 0) {
    const size_t bytes = gram_tc_scratch_bytes(job, KM);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      set_error("run_gram: %zu bytes of Gram scratch unavailable", bytes);
      return SADMM_ENOMEM;
    }
    const int rc = launch_gram_tc(job, KM, mu, rho, scratch, bytes, d_status, st);
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (rc != SADMM_OK) return rc;
    SADMM_CUDA_TRY(fe);
    return SADMM_OK;
  }
  JobBlock blk;
  blk.v[0] = job;
  const int Tn = job.npad / T;
  gram_kernel<<<dim3(Tn * (Tn + 1) / 2, 1, 1), kThreads, 0, st>>>(blk, KM, mu, rho);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int run_factor(const FactorJob* jobs, int njobs, int KM, double mu, double rho, int* d_status,
               cudaStream_t st, int gram) {
  if (njobs <= 0) return SADMM_OK;
  if (njobs > kMaxSets) { set_error("run_factor: too many jobs"); return SADMM_EINVAL; }
  JobBlock blk;
  int Tmax = 0;
  for (int i = 0; i < njobs; ++i) {
    blk.v[i] = jobs[i];
    if (jobs[i].npad % T != 0 || jobs[i].n > jobs[i].npad) {
      set_error("run_factor: bad padding");
      return SADMM_EINVAL;
    }
    Tmax = max(Tmax, jobs[i].npad / T);
  }
  if (Tmax == 0) return SADMM_OK;
  static bool configured = false;
  const size_t potrf_smem = 2 * T * (T + 1) * sizeof(double);
  if (!configured) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(potrf_diag_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_smem));
    configured = true;
  }
  const int ntri = Tmax * (Tmax + 1) / 2;
  if (gram == 0) {
    // tensor-core Gram, one job after another (each fills the GPU), in one
    // transient digit buffer sized for the largest job
    size_t bytes = 0;
    for (int i = 0; i < njobs; ++i) bytes = std::max(bytes, gram_tc_scratch_bytes(jobs[i], KM));
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      set_error("run_factor: %zu bytes of Gram scratch unavailable", bytes);
      return SADMM_ENOMEM;
    }
    int rc = SADMM_OK;
    for (int i = 0; i < njobs && rc == SADMM_OK; ++i)
      rc = launch_gram_tc(jobs[i], KM, mu, rho, scratch, bytes, d_status + i, st);
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (rc != SADMM_OK) return rc;
    SADMM_CUDA_TRY(fe);
  } else {
    gram_kernel<<<dim3(ntri, 1, njobs), kThreads, 0, st>>>(blk, KM, mu, rho);
    SADMM_LAUNCH_CHECK();
  }
  for (int kb = 0; kb < Tmax; ++kb) {
    potrf_diag_kernel<<<njobs, kThreads, potrf_smem, st>>>(blk, kb, d_status);
    SADMM_LAUNCH_CHECK();
    const int m = Tmax - kb - 1;
    if (m > 0) {
      trsm_kernel<<<dim3(m, njobs), kThreads, 0, st>>>(blk, kb);
      SADMM_LAUNCH_CHECK();
      syrk_update_kernel<<<dim3(m * (m + 1) / 2, njobs), kThreads, 0, st>>>(blk, kb);
      SADMM_LAUNCH_CHECK();
    }
  }
  linv_diag_kernel<<<dim3(Tmax, njobs), 256, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  for (int i = 1; i < Tmax; ++i) {
    linv_row_kernel<<<dim3(i, njobs), kThreads, 0, st>>>(blk, i);
    SADMM_LAUNCH_CHECK();
  }
  inverse_kernel<<<dim3(ntri, njobs), kThreads, 0, st>>>(blk);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
