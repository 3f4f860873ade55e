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

}  // namespace

int run_factor(const FactorJob* jobs, int njobs, int KM, double mu, double rho, int* d_status,
               cudaStream_t st) {
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
  gram_kernel<<<dim3(ntri, 1, njobs), kThreads, 0, st>>>(blk, KM, mu, rho);
  SADMM_LAUNCH_CHECK();
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
