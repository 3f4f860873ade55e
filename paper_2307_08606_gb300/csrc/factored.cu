// Factored (matrix-free) operator products for the signal model of Eq. 1.
//
// After dechirping, sample k of receiver m for pixel n with round-trip delay
// tau[m][n] is A[(m, k), n] = exp(j 2 pi tau (f0 + k df)): a geometric
// progression in k.  Writing k = 16 a + b splits every entry into
//   A[(m, 16 a + b), n] = C[m][a][n] * D[m][b][n],
//   C = exp(j 2 pi tau (f0 + 16 a df)),  D = exp(j 2 pi tau b df),
// so the K x N block of antenna m is stored as (K/16 + 16) x N factors instead
// of K x N entries (8x fewer bytes at K = 256).  Each factor is computed in
// FP64 and rounded to complex64, so a factored entry is within about three
// FP32 roundings of the exact one (the stored operator: one).
//
// Products (Eq. 3, x_q-update, per sensor over the active columns J):
//   forward  r[m][16a+b] = base - sum_{n in J} v_n C[m][a][n] D[m][b][n]:
//            per pixel a (K/16) x 16 outer product, accumulated per CTA over
//            a chunk of pixels staged through shared memory (two buffers:
//            the next stage's tables and the stage after's pixel indices and
//            v are loaded while the current stage is summed); the FP32 sums
//            over the 16 even and the 16 odd pixels of each 32-pixel stage go
//            into double-float accumulators, and the chunk partials are added
//            by the forward product's reduction.
//   adjoint  g_n = sum_m sum_a Re(conj(C[m][a][n]) t_a),
//            t_a = sum_b conj(D[m][b][n]) w[m][16a+b]:
//            one lane per pixel, antennas in order; 64 registers a thread,
//            so that every pixel of a paper-scale launch is resident at once
//            and other warps cover each warp's table loads; the 16-term sums
//            t_a are FP32 and the (m, a) terms go into a double-float
//            accumulator.
// The tables are pixel-fastest ([m][a][n], [m][b][n]), so a warp's loads
// for consecutive pixels are contiguous.
#include "common.cuh"
#include "symtile.cuh"

#include <algorithm>
#include <cmath>

namespace sadmm {
namespace {

using symtile::DF;
using symtile::df_add;
using symtile::df_add1;
using symtile::df_norm;

constexpr int kMaxK1 = 32;           // K <= 512

// ---------------------------------------------------------------- tables
// A[n][m K + k] (pixel-major, as sadmm_set_operator takes it).
__global__ void op_entries_kernel(const double* __restrict__ tau, int M, int K, int N, double f0, double df,
                                  float2* __restrict__ A) {
  const size_t KM = (size_t)M * K, total = KM * (size_t)N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / KM);
    const int r = (int)(e % KM);
    const int m = r / K, k = r % K;
    double cyc = tau[(size_t)m * N + n] * (f0 + k * df);
    cyc -= floor(cyc);
    double s, c;
    sincospi(2.0 * cyc, &s, &c);
    A[e] = make_float2((float)c, (float)s);
  }
}

// C[m][a][n] and D[m][b][n] from the same FP64 phases.
__global__ void op_factors_kernel(const double* __restrict__ tau, int M, int K, int N, double f0, double df,
                                  float2* __restrict__ C, float2* __restrict__ D) {
  const int K1 = K / kFacB;
  const size_t nc = (size_t)M * N * K1, total = nc + (size_t)M * N * kFacB;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double cyc;
    if (e < nc) {                                   // C[m][a][n]
      const size_t ma = e / N;
      const int n = (int)(e % N), a = (int)(ma % K1), m = (int)(ma / K1);
      cyc = tau[(size_t)m * N + n] * (f0 + (double)(kFacB * a) * df);
    } else {                                        // D[m][b][n]
      const size_t e2 = e - nc, mb = e2 / N;
      const int n = (int)(e2 % N), b = (int)(mb % kFacB), m = (int)(mb / kFacB);
      cyc = tau[(size_t)m * N + n] * ((double)b * df);
    }
    cyc -= floor(cyc);
    double s, c;
    sincospi(2.0 * cyc, &s, &c);
    if (e < nc) C[e] = make_float2((float)c, (float)s);
    else D[e - nc] = make_float2((float)c, (float)s);
  }
}

// ---------------------------------------------------------------- forward
// grid (chunks, M, sets); K1 = K/16 is a template parameter so that index
// arithmetic is shifts and the loops unroll.  Thread (h, bp) = (t / 8, t % 8)
// forms rows 16 a + 2 bp and 16 a + 2 bp + 1 of antenna m for AB values of
// a (a = h and, when AB = 2, a = h + K1/2): each 16-byte shared-memory load
// of a table pair then feeds 8 AB multiply-adds.
template <int K1>
struct FwdCfg {
  static constexpr int AB = K1 >= 2 ? 2 : 1;                     // values of a per thread
  static constexpr int NT = K1 * 8 / AB > 32 ? K1 * 8 / AB : 32;
  static constexpr int P = 32;                                    // pixels per stage
  static constexpr int CE = (K1 * P + NT - 1) / NT;              // C elements a thread stages
  static constexpr int DE = (kFacB * P + NT - 1) / NT;           // D elements a thread stages
};

template <int K1>
__global__ void __launch_bounds__(FwdCfg<K1>::NT, 640 / FwdCfg<K1>::NT)
factored_forward_kernel(const __grid_constant__ SetBlock<FactoredSet> sets, int M, int N, int chunks, int per,
                        VMode mode, const __grid_constant__ SolverView sv, float2* __restrict__ partial) {
  using Cf = FwdCfg<K1>;
  constexpr int NT = Cf::NT, P = Cf::P, CE = Cf::CE, DE = Cf::DE, AB = Cf::AB, K = K1 * kFacB;
  const FactoredSet& fs = sets.v[blockIdx.z];
  const int m = blockIdx.y, c = blockIdx.x;
  const int t = threadIdx.x, h = t >> 3, bp = t & 7;
  const bool owner = t < K1 * 8 / AB;
  const int p0 = c * per, p1 = min(fs.n, p0 + per);
  const int nst = p1 > p0 ? (p1 - p0 + P - 1) / P : 0;
  // v_n C[m][a][n] by rows of a (pixel pairs read as one 16-byte load), and
  // D[m][b][n] by rows of pixels (pairs of b read as one 16-byte load);
  // both padded so that stores and loads spread over the banks
  __shared__ __align__(16) float2 s_u[2][K1][P + 2];
  __shared__ __align__(16) float2 s_d[2][P][kFacB + 2];
  __shared__ int s_pix[2][P];
  __shared__ float s_v[2][P];
  const float2* Cm = fs.C + (size_t)m * K1 * N;
  const float2* Dm = fs.D + (size_t)m * kFacB * N;
  auto stage_np = [&](int s) { return min(P, p1 - (p0 + s * P)); };
  float2 rc[CE], rd[DE];
  // loads stage s's tables into registers (pixel indices from s_pix[buf])
  auto fetch = [&](int s, int buf) {
    const int np = stage_np(s);
#pragma unroll
    for (int j = 0; j < CE; ++j) {
      const int e = t + j * NT, aa = e / P, p = e % P;
      rc[j] = (e < K1 * P && p < np) ? Cm[(size_t)aa * N + s_pix[buf][p]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < DE; ++j) {
      const int e = t + j * NT, bb = e / P, p = e % P;
      rd[j] = (e < kFacB * P && p < np) ? Dm[(size_t)bb * N + s_pix[buf][p]] : make_float2(0.f, 0.f);
    }
  };
  // stores them into buffer buf, C scaled by the stage's v
  auto store = [&](int buf) {
#pragma unroll
    for (int j = 0; j < CE; ++j) {
      const int e = t + j * NT, aa = e / P, p = e % P;
      if (e < K1 * P) {
        const float v = s_v[buf][p];
        s_u[buf][aa][p] = make_float2(rc[j].x * v, rc[j].y * v);
      }
    }
#pragma unroll
    for (int j = 0; j < DE; ++j) {
      const int e = t + j * NT, bb = e / P, p = e % P;
      if (e < kFacB * P) s_d[buf][p][bb] = rd[j];
    }
  };
  DF acc[AB][4];                                                  // (re, im) of rows 2bp, 2bp + 1, per a
#pragma unroll
  for (int j = 0; j < AB; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = DF{0.f, 0.f};
  if (nst > 0) {
    // prologue: stage 0 into buffer 0, stage 1's pixels into s_pix[1]
    for (int i = t; i < P; i += NT) {
      const bool ok = i < stage_np(0);
      const int pix = ok ? fs.idx[p0 + i] : 0;
      s_pix[0][i] = pix;
      s_v[0][i] = ok ? v_of(mode, sv, fs.q, pix, fs.vexp) : 0.f;
    }
    __syncthreads();
    fetch(0, 0);
    for (int i = t; i < P; i += NT) {
      const bool ok = nst > 1 && i < stage_np(1);
      const int pix = ok ? fs.idx[p0 + P + i] : 0;
      s_pix[1][i] = pix;
      s_v[1][i] = ok ? v_of(mode, sv, fs.q, pix, fs.vexp) : 0.f;
    }
    store(0);
    __syncthreads();
  }
  for (int s = 0; s < nst; ++s) {
    const int b = s & 1, np = stage_np(s);
    if (s + 1 < nst) fetch(s + 1, b ^ 1);                         // next stage's tables
    int npix = 0;
    float nv = 0.f;
    const bool have2 = t < P && s + 2 < nst && t < stage_np(s + 2);
    if (have2) {                                                  // the stage after's pixels
      npix = fs.idx[p0 + (s + 2) * P + t];
      nv = v_of(mode, sv, fs.q, npix, fs.vexp);
    }
    if (owner) {
      // per value of a: rows (2bp, 2bp + 1) x pixels (even, odd) -> 8 sums
      float tt[AB][8];
#pragma unroll
      for (int j = 0; j < AB; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) tt[j][i] = 0.f;
      int p = 0;
#pragma unroll 2
      for (; p + 1 < np; p += 2) {
        const float4 dx = *reinterpret_cast<const float4*>(&s_d[b][p][2 * bp]);     // D_{2bp}, D_{2bp+1} at p
        const float4 dy = *reinterpret_cast<const float4*>(&s_d[b][p + 1][2 * bp]); // ... at p + 1
#pragma unroll
        for (int j = 0; j < AB; ++j) {
          const float4 uw = *reinterpret_cast<const float4*>(&s_u[b][h + j * (K1 / 2)][p]);  // pixels p, p + 1
          float* q = tt[j];
          q[0] = fmaf(uw.x, dx.x, q[0]); q[0] = fmaf(-uw.y, dx.y, q[0]);
          q[1] = fmaf(uw.x, dx.y, q[1]); q[1] = fmaf(uw.y, dx.x, q[1]);
          q[2] = fmaf(uw.x, dx.z, q[2]); q[2] = fmaf(-uw.y, dx.w, q[2]);
          q[3] = fmaf(uw.x, dx.w, q[3]); q[3] = fmaf(uw.y, dx.z, q[3]);
          q[4] = fmaf(uw.z, dy.x, q[4]); q[4] = fmaf(-uw.w, dy.y, q[4]);
          q[5] = fmaf(uw.z, dy.y, q[5]); q[5] = fmaf(uw.w, dy.x, q[5]);
          q[6] = fmaf(uw.z, dy.z, q[6]); q[6] = fmaf(-uw.w, dy.w, q[6]);
          q[7] = fmaf(uw.z, dy.w, q[7]); q[7] = fmaf(uw.w, dy.z, q[7]);
        }
      }
      if (p < np) {
        const float4 dx = *reinterpret_cast<const float4*>(&s_d[b][p][2 * bp]);
#pragma unroll
        for (int j = 0; j < AB; ++j) {
          const float2 u = s_u[b][h + j * (K1 / 2)][p];
          float* q = tt[j];
          q[0] = fmaf(u.x, dx.x, q[0]); q[0] = fmaf(-u.y, dx.y, q[0]);
          q[1] = fmaf(u.x, dx.y, q[1]); q[1] = fmaf(u.y, dx.x, q[1]);
          q[2] = fmaf(u.x, dx.z, q[2]); q[2] = fmaf(-u.y, dx.w, q[2]);
          q[3] = fmaf(u.x, dx.w, q[3]); q[3] = fmaf(u.y, dx.z, q[3]);
        }
      }
#pragma unroll
      for (int j = 0; j < AB; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          df_add1(acc[j][i], tt[j][i]);
          df_add1(acc[j][i], tt[j][i + 4]);
        }
    }
    // buffer b ^ 1 was last read in stage s - 1 (before the previous
    // barrier); s_pix[b] / s_v[b] (stage s) are no longer needed
    if (s + 1 < nst) store(b ^ 1);
    if (t < P) {
      s_pix[b][t] = npix;
      s_v[b][t] = nv;
    }
    __syncthreads();
  }
  if (!owner) return;
  const int KM = M * K;
  float2* pp = partial + ((size_t)blockIdx.z * chunks + c) * 2 * KM;
#pragma unroll
  for (int j = 0; j < AB; ++j) {
    const int r = m * K + (h + j * (K1 / 2)) * kFacB + 2 * bp;   // even: two complex rows = one float4
    DF o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = df_norm(acc[j][i]);
    reinterpret_cast<float4*>(pp + r)[0] = make_float4(o[0].hi, o[1].hi, o[2].hi, o[3].hi);
    reinterpret_cast<float4*>(pp + KM + r)[0] = make_float4(o[0].lo, o[1].lo, o[2].lo, o[3].lo);
  }
}

// ---------------------------------------------------------------- adjoint
// grid (pixel groups of 128, sets); 4 warps, one lane per pixel; every lane
// runs all M antennas in order (eight CTAs per SM: 64 registers a thread).
constexpr int kMaxKM = 16384;                // w (M K complex) staged in shared memory
constexpr int kAdjPix = 128;

template <int K1>
__global__ void __launch_bounds__(kAdjPix, 8)
factored_adjoint_kernel(const __grid_constant__ SetBlock<FactoredSet> sets, int M, int N, bool update,
                        const __grid_constant__ SolverView sv) {
  constexpr int K = K1 * kFacB;
  extern __shared__ __align__(16) float4 s_w4[];                 // w: M K complex
  const FactoredSet& fs = sets.v[blockIdx.y];
  const int pbeg = blockIdx.x * kAdjPix;
  if (pbeg >= fs.n) return;
  {
    const float4* w4 = reinterpret_cast<const float4*>(fs.w);
    for (int i = threadIdx.x; i < M * K / 2; i += kAdjPix) s_w4[i] = w4[i];
  }
  __syncthreads();
  const int p = pbeg + threadIdx.x;
  if (p >= fs.n) return;
  const int pix = fs.idx[p];
  DF g{0.f, 0.f};
  for (int m = 0; m < M; ++m) {
    float2 d[kFacB];
#pragma unroll
    for (int b = 0; b < kFacB; ++b) d[b] = fs.D[((size_t)m * kFacB + b) * N + pix];
    const float2* Cp = fs.C + (size_t)m * K1 * N + pix;
    const float4* wm = s_w4 + (size_t)m * K / 2;
#pragma unroll 4
    for (int a = 0; a < K1; ++a) {
      const float2 cv = Cp[(size_t)a * N];
      // t_a = sum_b conj(D_b) w_{16a+b}, in two chains (even and odd b)
      float tr0 = 0.f, ti0 = 0.f, tr1 = 0.f, ti1 = 0.f;
#pragma unroll
      for (int i = 0; i < kFacB / 2; ++i) {
        const float4 w = wm[a * (kFacB / 2) + i];                 // w_{16a+2i}, w_{16a+2i+1}
        const float2 e0 = d[2 * i], e1 = d[2 * i + 1];
        tr0 = fmaf(e0.x, w.x, tr0); tr0 = fmaf(e0.y, w.y, tr0);
        ti0 = fmaf(e0.x, w.y, ti0); ti0 = fmaf(-e0.y, w.x, ti0);
        tr1 = fmaf(e1.x, w.z, tr1); tr1 = fmaf(e1.y, w.w, tr1);
        ti1 = fmaf(e1.x, w.w, ti1); ti1 = fmaf(-e1.y, w.z, ti1);
      }
      df_add1(g, fmaf(cv.x, tr0 + tr1, cv.y * (ti0 + ti1)));     // Re(conj(C_a) t_a)
    }
  }
  const float gv = g.hi + g.lo;
  if (update) {
    // x-update epilogue (Woodbury form): x = v + mu Re(a^H w)
    const size_t xi = (size_t)fs.q * sv.N + pix;
    const float xo = sv.x[xi];
    const float v = v_admm(sv, fs.q, pix, xo);
    const float xn = fmaf(sv.mu, gv, v);
    sv.ring[((size_t)sv.slot * sv.Q + fs.q) * sv.N + pix] = xn - xo;
    sv.x[xi] = xn;
  } else {
    fs.g[p] = gv;
  }
}

template <int K1>
int launch_forward_k1(const SetBlock<FactoredSet>& blk, int nsets, int M, int N, int chunks, int per, VMode mode,
                      const SolverView& sv, float2* partial, cudaStream_t st) {
  factored_forward_kernel<K1><<<dim3(chunks, M, nsets), FwdCfg<K1>::NT, 0, st>>>(blk, M, N, chunks, per, mode, sv,
                                                                                  partial);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

template <int K1>
int launch_adjoint_k1(const SetBlock<FactoredSet>& blk, int nsets, int M, int N, int max_cols, bool update,
                      const SolverView& sv, cudaStream_t st) {
  const size_t smem = (size_t)M * K1 * kFacB * sizeof(float2);
  static bool configured = false;
  if (!configured) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(factored_adjoint_kernel<K1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kMaxKM * (int)sizeof(float2)));
    configured = true;
  }
  factored_adjoint_kernel<K1><<<dim3(div_up(max_cols, kAdjPix), nsets), kAdjPix, smem, st>>>(blk, M, N, update, sv);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// Resident forward CTAs per SM (queried once per K1), so that the grid can be
// sized to whole waves.
int forward_residency(int K) {
  static int cached[kMaxK1 + 1] = {};
  const int K1 = K / kFacB;
  if (K1 < 1 || K1 > kMaxK1) return 1;
  if (!cached[K1]) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (K1) {
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<1>, FwdCfg<1>::NT, 0); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<2>, FwdCfg<2>::NT, 0); break;
      case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<4>, FwdCfg<4>::NT, 0); break;
      case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<8>, FwdCfg<8>::NT, 0); break;
      case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<16>, FwdCfg<16>::NT, 0); break;
      case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, factored_forward_kernel<32>, FwdCfg<32>::NT, 0); break;
    }
    cached[K1] = (e == cudaSuccess && nb > 0) ? nb : 4;
  }
  return cached[K1];
}

}  // namespace

bool factored_supported(int K) {
  const int K1 = K / kFacB;
  return K % kFacB == 0 && K1 >= 1 && K1 <= kMaxK1 && (K1 & (K1 - 1)) == 0;
}

int operator_tables(const double* tau, int M, int K, int N, double f0, double df, float2* A, float2* C, float2* D,
                    cudaStream_t st) {
  if (M <= 0 || K <= 0 || N <= 0 || !tau) { set_error("operator_tables: bad sizes"); return SADMM_EINVAL; }
  if (A) {
    op_entries_kernel<<<152 * 8, 256, 0, st>>>(tau, M, K, N, f0, df, A);
    SADMM_LAUNCH_CHECK();
  }
  if (C && D) {
    if (!factored_supported(K)) { set_error("operator_tables: K must be 16, 32, 64, 128, 256 or 512"); return SADMM_EINVAL; }
    op_factors_kernel<<<152 * 8, 256, 0, st>>>(tau, M, K, N, f0, df, C, D);
    SADMM_LAUNCH_CHECK();
  }
  return SADMM_OK;
}

int factored_chunks(int nsets, int M, int K, int max_cols) {
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)sms * forward_residency(K);
  const int want = std::max(1LL, slots / ((long long)M * nsets));   // one full wave of CTAs
  const int cap = div_up(max_cols, 256);                             // at least 256 pixels per chunk
  return std::max(1, std::min(want, cap));
}

size_t factored_partial_bytes(int nsets, int M, int K, int max_cols) {
  return (size_t)nsets * factored_chunks(nsets, M, K, max_cols) * 2 * (size_t)M * K * sizeof(float2);
}

int launch_factored_forward(const FactoredSet* sets, int nsets, int M, int K, int N, VMode mode, const SolverView& sv,
                            float2* partial, size_t partial_cap, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets || !factored_supported(K) || M < 1) {
    set_error("launch_factored_forward: bad sizes (K = 16, 32, ..., 512; at most %d sets)", kMaxSets);
    return SADMM_EINVAL;
  }
  SetBlock<FactoredSet> blk;
  SetBlock<ColumnSet> red;
  int max_cols = 1;
  for (int i = 0; i < nsets; ++i) {
    blk.v[i] = sets[i];
    max_cols = std::max(max_cols, sets[i].n);
    red.v[i] = ColumnSet{nullptr, nullptr, 0, sets[i].q, nullptr, sets[i].base, sets[i].out};
  }
  const int chunks = factored_chunks(nsets, M, K, max_cols);
  if (factored_partial_bytes(nsets, M, K, max_cols) > partial_cap) {
    set_error("launch_factored_forward: partial buffer too small");
    return SADMM_EINVAL;
  }
  const int per = div_up(max_cols, chunks);
  int rc = SADMM_EINVAL;
  switch (K / kFacB) {
    case 1: rc = launch_forward_k1<1>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
    case 2: rc = launch_forward_k1<2>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
    case 4: rc = launch_forward_k1<4>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
    case 8: rc = launch_forward_k1<8>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
    case 16: rc = launch_forward_k1<16>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
    case 32: rc = launch_forward_k1<32>(blk, nsets, M, N, chunks, per, mode, sv, partial, st); break;
  }
  SADMM_TRY(rc);
  return launch_forward_reduce(red.v, nsets, M * K, chunks, partial, st);
}

int launch_factored_adjoint(const FactoredSet* sets, int nsets, int M, int K, int N, bool update, const SolverView& sv,
                            cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  if (nsets > kMaxSets || !factored_supported(K) || M < 1 || M * K > kMaxKM) {
    set_error("launch_factored_adjoint: bad sizes (M K up to %d, K = 16, 32, ..., 512)", kMaxKM);
    return SADMM_EINVAL;
  }
  SetBlock<FactoredSet> blk;
  int max_cols = 1;
  for (int i = 0; i < nsets; ++i) {
    blk.v[i] = sets[i];
    max_cols = std::max(max_cols, sets[i].n);
  }
  switch (K / kFacB) {
    case 1: return launch_adjoint_k1<1>(blk, nsets, M, N, max_cols, update, sv, st);
    case 2: return launch_adjoint_k1<2>(blk, nsets, M, N, max_cols, update, sv, st);
    case 4: return launch_adjoint_k1<4>(blk, nsets, M, N, max_cols, update, sv, st);
    case 8: return launch_adjoint_k1<8>(blk, nsets, M, N, max_cols, update, sv, st);
    case 16: return launch_adjoint_k1<16>(blk, nsets, M, N, max_cols, update, sv, st);
    case 32: return launch_adjoint_k1<32>(blk, nsets, M, N, max_cols, update, sv, st);
  }
  return SADMM_EINVAL;
}

}  // namespace sadmm

extern "C" {

int sadmm_operator_tables(const double* tau, int M, int K, int N, double f0, double df, float* A, float* C,
                          float* D, void* stream) {
  using namespace sadmm;
  if (!tau || M <= 0 || K <= 0 || N <= 0 || (!C) != (!D) || !std::isfinite(f0) || !std::isfinite(df)) {
    set_error("sadmm_operator_tables: bad arguments");
    return SADMM_EINVAL;
  }
  return operator_tables(tau, M, K, N, f0, df, reinterpret_cast<float2*>(A), reinterpret_cast<float2*>(C),
                         reinterpret_cast<float2*>(D), (cudaStream_t)stream);
}

int sadmm_forward_factored(const float* C, const float* D, int M, int K, int N, const int* idx, int nidx,
                           const float* v, const float* base, float* r, void* stream) {
  using namespace sadmm;
  if (!C || !D || !r || M <= 0 || !factored_supported(K) || N <= 0 || nidx < 0 ||
      (nidx > 0 && (!idx || !v))) {
    set_error("sadmm_forward_factored: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  FactoredSet fs{reinterpret_cast<const float2*>(C), reinterpret_cast<const float2*>(D), idx, nidx, 0, v,
                 reinterpret_cast<const float2*>(base), reinterpret_cast<float2*>(r), nullptr, nullptr};
  SolverView sv{};
  const size_t cap = factored_partial_bytes(1, M, K, std::max(nidx, 1));
  void* part = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&part, cap, st));
  int rc = launch_factored_forward(&fs, 1, M, K, N, kVExplicit, sv, (float2*)part, cap, st);
  cudaError_t e = cudaFreeAsync(part, st);
  if (rc != SADMM_OK) return rc;
  SADMM_CUDA_TRY(e);
  return SADMM_OK;
}

int sadmm_adjoint_factored(const float* C, const float* D, int M, int K, int N, const int* idx, int nidx,
                           const float* w, float* g, void* stream) {
  using namespace sadmm;
  if (!C || !D || !w || M <= 0 || !factored_supported(K) || M * K > 16384 || N <= 0 || nidx < 0 ||
      (nidx > 0 && (!idx || !g))) {
    set_error("sadmm_adjoint_factored: bad arguments");
    return SADMM_EINVAL;
  }
  FactoredSet fs{reinterpret_cast<const float2*>(C), reinterpret_cast<const float2*>(D), idx, nidx, 0, nullptr,
                 nullptr, nullptr, reinterpret_cast<const float2*>(w), g};
  SolverView sv{};
  return launch_factored_adjoint(&fs, 1, M, K, N, false, sv, (cudaStream_t)stream);
}

}  // extern "C"
