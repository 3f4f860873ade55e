// Factor apply with 16 right-hand sides on the tensor cores, for the batched
// form (Eq. 3, x_q-update: U = W R in the Woodbury form, H G in the primal
// form, for 16 scenes at once).
//
// Exact integer slices.  Row i of the factor is scaled by 2^-e_i (e_i the
// least exponent with max_j |F_ij| <= 2^e_i) and column s of the right-hand
// sides by 2^-f_s; a scaled value v in [-1, 1] is written as
//   v = 2^-7 (d_0 + 2^-8 d_1 + 2^-16 d_2 + 2^-24 d_3) + t,
// integers |d_a| <= 128 (exact in BF16), |t| <= 2^-32.  Then
//   (F u)_is = 2^(e_i + f_s - 14) sum_{o = 0..3} 2^(-8 o) T_o(i, s),
//   T_o(i, s) = sum_{a + b = o} sum_j d_a(F_ij) d_b(u_js),
// ten digit GEMMs (M 128, N 16, K 16 per tcgen05.mma kind::f16).  Every digit
// product is an integer of magnitude <= 2^14, and an order sum over a chunk of
// 256 values of j (at most four products per j) stays within 2^24, so each
// chunk's order sums are exact in the FP32 accumulator; after each chunk the
// four sums go into double-float running totals (orders 0..2 by error-free
// two-sums, order 3 into the low word: about 2^-46 of the total per chunk).
// The dropped orders (>= 4) and the two slicing remainders contribute at most
// about 5 2^-32 per term (of 2^(e_i + f_s)).  The factor digits take 8 bytes
// per entry, as the double-float pair copy of the single-scene apply.
//
// bapply_tc_kernel is a persistent, warp-specialised pipeline over work items
// (sensor q, block of 128 rows, range of k):
//   warp 0      TMA producer: per 64-k stage the four digit tiles of the row
//               block (128 x 64, one box each) and the four digit tiles of the
//               right-hand sides (16 x 64, one box of 64 rows), 128-byte
//               swizzle (the SW128 K-major operand layout of the MMA), three
//               stages of 72 KB;
//   warp 1      MMA issuer: per 16-k step ten MMAs into the four order
//               accumulators (16 columns each) of one of two TMEM sets
//               (alternating per 256-k chunk);
//   warps 2-5   epilogue: per chunk, tcgen05.ld of the four accumulators (one
//               32-lane quarter per warp: one thread per row, 16 columns),
//               double-float update; per item, the scaled partial result.
// Every wait is bounded; on a timeout the CTA flags *err, waits (bounded) for
// its copies in flight, frees its tensor memory and exits.
#include "digits.cuh"
#include "sadmm.h"

#include <cuda_bf16.h>
#include <cstring>

namespace sadmm {
namespace {

constexpr int kAM = 128;                               // rows per item (TMEM lanes)
constexpr int kAN = 16;                                // right-hand sides
constexpr int kAK = 64;                                // k per stage: one 128-byte BF16 row
constexpr int kAChunk = 256;                           // k per exact chunk
constexpr int kASPC = kAChunk / kAK;                   // stages per chunk
constexpr int kADig = 4;
constexpr int kAATile = kAM * kAK * 2;                 // 16 KB per factor digit
constexpr int kABTile = kAN * kAK * 2;                 // 2 KB per right-hand-side digit
constexpr int kAStage = kADig * (kAATile + kABTile);   // 72 KB
constexpr int kAS = 3;                                 // stages
constexpr int kASmem = kAS * kAStage + 1024;           // + alignment slack
constexpr int kAThreads = 192;                         // producer, MMA issuer, 4 epilogue warps
constexpr int kAEpi = 128;
constexpr int kASetCols = kADig * kAN;                 // four order accumulators
constexpr int kATmemCols = 128;                        // two sets (power of two >= 32)
constexpr long long kAWait = 1ll << 26;
constexpr int kTargetItems = 4 * 152;

// kind::f16, D = F32, A = B = BF16, both K-major, N = 16, M = 128
constexpr uint32_t kAIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kAN >> 3) << 17) |
                             ((uint32_t)(kAM >> 4) << 24);

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// SW128 K-major descriptor: 8-row atoms of 128-byte rows, atoms 1024 bytes apart
__device__ __forceinline__ uint64_t sw128(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma16(unsigned tmem, uint64_t a, uint64_t b, unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kAIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ bool wait(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kAWait; ++it) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void tma2d(unsigned dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// s += x, error-free up to the low word's own rounding (x an FP32 value)
__device__ __forceinline__ void two_add(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

// Digits of t = v 2^7 (|v| <= 1): rint, then the remainder times 2^8; every
// step is exact in the input's own precision.
__device__ __forceinline__ void digits_d(double t, __nv_bfloat16 (&d)[kADig]) {
#pragma unroll
  for (int a = 0; a < kADig; ++a) {
    const double r = rint(t);
    d[a] = __float2bfloat16_rn((float)r);
    t = (t - r) * 256.0;
  }
}
__device__ __forceinline__ void digits_f(float t, __nv_bfloat16 (&d)[kADig]) {
#pragma unroll
  for (int a = 0; a < kADig; ++a) {
    const float r = rintf(t);
    d[a] = __float2bfloat16_rn(r);
    t = (t - r) * 256.f;
  }
}

// least e with m <= 2^e (0 for m = 0)
__device__ __forceinline__ int exponent_of(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);
  return e;
}

// value (j, s) of the right-hand sides in either layout
__device__ __forceinline__ float u_at(const float* __restrict__ u, int umode, int j, int s) {
  return umode == 1 ? u[(size_t)j * kAN + s] : u[((size_t)(j >> 1) * kAN + s) * 2 + (j & 1)];
}

// ----------------------------------------------------------- factor digits
// One CTA per padded row: the row maximum (FP64), then eight columns per
// thread and step; rows >= n and columns >= n are zero.
__global__ void __launch_bounds__(256)
factor_digits_kernel(const double* __restrict__ F, int ld, int n, int rows_pad, int kpad,
                     __nv_bfloat16* __restrict__ D, int* __restrict__ expo) {
  const int i = blockIdx.x, tid = threadIdx.x;
  const double* row = i < n ? F + (size_t)i * ld : nullptr;
  __shared__ double s_max[8];
  double m = 0.0;
  if (row)
    for (int j = tid; j < n; j += 256) m = fmax(m, fabs(row[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) s_max[tid >> 5] = m;
  __syncthreads();
  m = s_max[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmax(m, s_max[w]);
  const int e = exponent_of(m);
  if (tid == 0) expo[i] = e;
  const double sc = ldexp(1.0, 7 - e);
  const size_t plane = (size_t)rows_pad * kpad;
  for (int j0 = 8 * tid; j0 < kpad; j0 += 8 * 256) {
    unsigned w[kADig][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      __nv_bfloat16 d0[kADig], d1[kADig];
      const double v0 = (row && j0 + u < n) ? row[j0 + u] : 0.0;
      const double v1 = (row && j0 + u + 1 < n) ? row[j0 + u + 1] : 0.0;
      digits_d(v0 * sc, d0);
      digits_d(v1 * sc, d1);
#pragma unroll
      for (int a = 0; a < kADig; ++a) w[a][u / 2] = pack2(d0[a], d1[a]);
    }
#pragma unroll
    for (int a = 0; a < kADig; ++a)
      *reinterpret_cast<uint4*>(D + a * plane + (size_t)i * kpad + j0) = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
  }
}

// ------------------------------------------------ right-hand-side digits
// Column maxima of the 16 right-hand sides (float bits; non-negative floats
// order as integers).  One thread per row j.
__global__ void __launch_bounds__(256)
rhs_max_kernel(const float* const* __restrict__ uq, int umode, int n, int* __restrict__ maxbits) {
  const int q = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  const float* u = uq[q];
#pragma unroll
  for (int s = 0; s < kAN; ++s) {
    float m = j < n ? fabsf(u_at(u, umode, j, s)) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(maxbits + q * kAN + s, __float_as_int(m));
  }
}

// Digits of the right-hand sides, [q][digit][s][k]: one CTA per 128 rows j,
// staged in shared memory so that the writes run along k.
constexpr int kURow = 136;                 // padded shared row (BF16 elements)

__global__ void __launch_bounds__(256)
rhs_digits_kernel(const float* const* __restrict__ uq, int umode, int n, int kpad, const int* __restrict__ maxbits,
                  __nv_bfloat16* __restrict__ D, int* __restrict__ expo) {
  __shared__ __align__(16) __nv_bfloat16 sD[kADig][kAN][kURow];
  const int q = blockIdx.y, j0 = blockIdx.x * 128, tid = threadIdx.x;
  const float* u = uq[q];
  const int s = tid & 15, jj = tid >> 4;
  const float m = __int_as_float(maxbits[q * kAN + s]);
  const int e = exponent_of((double)m);
  if (blockIdx.x == 0 && tid < kAN) expo[q * kAN + s] = e;
  const float sc = ldexpf(1.f, 7 - e);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int jl = jj + 16 * r, j = j0 + jl;
    const float v = j < n ? u_at(u, umode, j, s) : 0.f;
    __nv_bfloat16 d[kADig];
    digits_f(v * sc, d);
#pragma unroll
    for (int a = 0; a < kADig; ++a) sD[a][s][jl] = d[a];
  }
  __syncthreads();
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int idx = tid + 256 * w;       // 1024 16-byte pieces: 64 rows x 16
    const int rw = idx >> 4, c8 = idx & 15;
    const int a = rw >> 4, ss = rw & 15;
    const uint4 val = *reinterpret_cast<const uint4*>(&sD[a][ss][c8 * 8]);
    *reinterpret_cast<uint4*>(D + ((size_t)(q * kADig + a) * kAN + ss) * kpad + j0 + c8 * 8) = val;
  }
}

// ------------------------------------------------------------- the GEMM
struct ApplyArgs {
  int Q, rows_pad, kpad, ksplit;
  const int* expoF;
  const int* expoU;
  float2* part;
};

__device__ __forceinline__ void item_decode(int it, const ApplyArgs& aa, int& q, int& I, int& ks) {
  const int nI = aa.rows_pad / kAM;
  ks = it % aa.ksplit;
  const int r = it / aa.ksplit;
  I = r % nI;
  q = r / nI;
}

__global__ void __launch_bounds__(kAThreads, 1)
bapply_tc_kernel(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmU,
                 const __grid_constant__ ApplyArgs aa, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kAS], empty[kAS], accfull[2], accempty[2];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int items = aa.Q * (aa.rows_pad / kAM) * aa.ksplit;
  const int kper = aa.kpad / aa.ksplit;
  const int nchunks = kper / kAChunk;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kATmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < kAS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&accfull[b], 1);
      bar_init(&accempty[b], kAEpi);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s_tmem;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int t = 0;
      const int nst = kper / kAK;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int q, I, ks;
        item_decode(it, aa, q, I, ks);
        for (int sl = 0; sl < nst && ok; ++sl, ++t) {
          const int s = t % kAS;
          if (t >= kAS) ok = wait(&empty[s], ((t / kAS) - 1) & 1);
          if (!ok) break;
          const unsigned st = su32(smem + s * kAStage);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])), "r"(kAStage)
                       : "memory");
          const int x = ks * kper + sl * kAK;
#pragma unroll
          for (int d = 0; d < kADig; ++d)
            tma2d(st + d * kAATile, &tmF, x, (q * kADig + d) * aa.rows_pad + I * kAM, &full[s]);
          tma2d(st + kADig * kAATile, &tmU, x, q * kADig * kAN, &full[s]);
        }
      }
      // copies still in flight when stopping early: wait for them (bounded)
      if (!ok)
        for (int u = max(0, t - kAS); u < t; ++u) wait(&full[u % kAS], (u / kAS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------- MMA issuer
      int t = 0, gc = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        for (int c = 0; c < nchunks && ok; ++c, ++gc) {
          const int b = gc & 1;
          if (gc >= 2) ok = wait(&accempty[b], ((gc / 2) - 1) & 1);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned d0 = tmem + b * kASetCols;
          for (int sc = 0; sc < kASPC && ok; ++sc, ++t) {
            const int s = t % kAS;
            ok = wait(&full[s], (t / kAS) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sa = su32(smem + s * kAStage), sb = sa + kADig * kAATile;
#pragma unroll
            for (int ks = 0; ks < kAK / 16; ++ks) {
              const unsigned f = (sc > 0 || ks > 0) ? 1u : 0u;
              uint64_t A[kADig], B[kADig];
#pragma unroll
              for (int d = 0; d < kADig; ++d) {
                A[d] = sw128(sa + d * kAATile + ks * 32);
                B[d] = sw128(sb + d * kABTile + ks * 32);
              }
              mma16(d0, A[0], B[0], f);                       // order 0
              mma16(d0 + kAN, A[0], B[1], f);                 // order 1
              mma16(d0 + kAN, A[1], B[0], 1u);
              mma16(d0 + 2 * kAN, A[0], B[2], f);             // order 2
              mma16(d0 + 2 * kAN, A[1], B[1], 1u);
              mma16(d0 + 2 * kAN, A[2], B[0], 1u);
              mma16(d0 + 3 * kAN, A[0], B[3], f);             // order 3
              mma16(d0 + 3 * kAN, A[1], B[2], 1u);
              mma16(d0 + 3 * kAN, A[2], B[1], 1u);
              mma16(d0 + 3 * kAN, A[3], B[0], 1u);
            }
            commit(&empty[s]);
          }
          if (ok) commit(&accfull[b]);
        }
      }
    }
  } else {
    // -------------------------------------------------------------- epilogue
    const int quarter = warp & 3;            // TMEM lanes 32 quarter .. + 31
    const int row = quarter * 32 + lane;     // row of the block
    int gc = 0;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int q, I, ks;
      item_decode(it, aa, q, I, ks);
      float th[kAN], tl[kAN];
#pragma unroll
      for (int j = 0; j < kAN; ++j) { th[j] = 0.f; tl[j] = 0.f; }
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = gc & 1;
        ok = wait(&accfull[b], (gc / 2) & 1);
        ok = __all_sync(0xffffffffu, ok);       // tcgen05.ld below is warp-collective
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + b * kASetCols;
        float s0[16], s1[16], s2[16], s3[16];
        tld16(ta, s0);
        tld16(ta + kAN, s1);
        tld16(ta + 2 * kAN, s2);
        tld16(ta + 3 * kAN, s3);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        bar_arrive(&accempty[b]);
#pragma unroll
        for (int j = 0; j < kAN; ++j) {
          two_add(th[j], tl[j], s0[j]);
          two_add(th[j], tl[j], s1[j] * 0x1p-8f);
          two_add(th[j], tl[j], s2[j] * 0x1p-16f);
          tl[j] += s3[j] * 0x1p-24f;
          const float h = th[j] + tl[j];        // renormalise
          tl[j] -= h - th[j];
          th[j] = h;
        }
      }
      if (!ok) break;
      const int i = I * kAM + row;
      const int ei = aa.expoF[(size_t)q * aa.rows_pad + i];
      float4* dst = reinterpret_cast<float4*>(aa.part + (((size_t)q * aa.ksplit + ks) * aa.rows_pad + i) * kAN);
#pragma unroll
      for (int j = 0; j < kAN; j += 2) {
        const int s0e = ei + aa.expoU[q * kAN + j] - 14, s1e = ei + aa.expoU[q * kAN + j + 1] - 14;
        dst[j / 2] = make_float4(ldexpf(th[j], s0e), ldexpf(tl[j], s0e), ldexpf(th[j + 1], s1e),
                                 ldexpf(tl[j + 1], s1e));
      }
    }
  }
  if (!ok) atomicExch(err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kATmemCols) : "memory");
}

// out[i][s] = the sum of the k ranges' partial results (FP64), i < n.
__global__ void digit_out_kernel(const float2* __restrict__ part, int ksplit, int rows_pad, int n,
                                 double* __restrict__ out) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  const int i = e / kAN, s = e % kAN;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = 0; k < ksplit; ++k) {
    const float2 v = part[((size_t)k * rows_pad + i) * kAN + s];
    acc += (double)v.x + (double)v.y;
  }
  out[e] = acc;
}

}  // namespace

void digit_apply_dims(DigitApply& d, int Q, int n) {
  d.Q = Q;
  d.n = n;
  d.rows_pad = round_up(n, kAM);
  const int nI = d.rows_pad / kAM;
  // k ranges of whole chunks: split while the items do not fill the GPU a few
  // times over and the padding stays within an eighth of the chunked length
  const int kc = round_up(n, kAChunk);
  int ks = 1;
  while ((long long)Q * nI * ks < kTargetItems) {
    const int k2 = 2 * ks;
    if ((long long)round_up(div_up(kc, k2), kAChunk) * k2 > kc + kc / 8) break;
    ks = k2;
  }
  d.ksplit = ks;
  d.kpad = round_up(div_up(kc, ks), kAChunk) * ks;
}

static size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }

size_t digit_apply_bytes(const DigitApply& d) {
  return al((size_t)d.Q * kADig * d.rows_pad * d.kpad * 2) + al((size_t)d.Q * d.rows_pad * 4) +
         al((size_t)d.Q * kADig * kAN * d.kpad * 2) + 2 * al((size_t)d.Q * kAN * 4) +
         al((size_t)d.Q * d.ksplit * d.rows_pad * kAN * sizeof(float2));
}

int digit_apply_bind(DigitApply& d, void* mem) {
  char* p = static_cast<char*>(mem);
  d.DF = p;
  p += al((size_t)d.Q * kADig * d.rows_pad * d.kpad * 2);
  d.expoF = reinterpret_cast<int*>(p);
  p += al((size_t)d.Q * d.rows_pad * 4);
  d.DU = p;
  p += al((size_t)d.Q * kADig * kAN * d.kpad * 2);
  d.expoU = reinterpret_cast<int*>(p);
  p += al((size_t)d.Q * kAN * 4);
  d.maxbits = reinterpret_cast<int*>(p);
  p += al((size_t)d.Q * kAN * 4);
  d.part = reinterpret_cast<float2*>(p);
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) { set_error("digit apply: cuTensorMapEncodeTiled unavailable"); return SADMM_ECUDA; }
  memset(&d.tmF, 0, sizeof d.tmF);
  memset(&d.tmU, 0, sizeof d.tmU);
  const cuuint64_t strides[1] = {(cuuint64_t)d.kpad * 2};
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)d.kpad, (cuuint64_t)d.Q * kADig * d.rows_pad};
    const cuuint32_t box[2] = {(cuuint32_t)kAK, (cuuint32_t)kAM};
    const CUresult r = enc(&d.tmF, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, d.DF, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("digit apply: factor tensor map rejected (%d)", (int)r); return SADMM_ECUDA; }
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)d.kpad, (cuuint64_t)d.Q * kADig * kAN};
    const cuuint32_t box[2] = {(cuuint32_t)kAK, (cuuint32_t)(kADig * kAN)};
    const CUresult r = enc(&d.tmU, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, d.DU, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("digit apply: right-hand-side tensor map rejected (%d)", (int)r); return SADMM_ECUDA; }
  }
  return SADMM_OK;
}

int launch_factor_digits(const DigitApply& d, int q, const double* F, int ld, cudaStream_t st) {
  if (q < 0 || q >= d.Q || ld < d.n) { set_error("launch_factor_digits: bad arguments"); return SADMM_EINVAL; }
  const size_t plane = (size_t)d.rows_pad * d.kpad;
  factor_digits_kernel<<<d.rows_pad, 256, 0, st>>>(F, ld, d.n, d.rows_pad, d.kpad,
                                                   static_cast<__nv_bfloat16*>(d.DF) + (size_t)q * kADig * plane,
                                                   d.expoF + (size_t)q * d.rows_pad);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_digit_apply(const DigitApply& d, const float* const* u, int umode, int* err, cudaStream_t st) {
  SADMM_CUDA_TRY(cudaMemsetAsync(d.maxbits, 0, (size_t)d.Q * kAN * sizeof(int), st));
  rhs_max_kernel<<<dim3(div_up(d.n, 256), d.Q), 256, 0, st>>>(u, umode, d.n, d.maxbits);
  SADMM_LAUNCH_CHECK();
  rhs_digits_kernel<<<dim3(d.kpad / 128, d.Q), 256, 0, st>>>(u, umode, d.n, d.kpad, d.maxbits,
                                                             static_cast<__nv_bfloat16*>(d.DU), d.expoU);
  SADMM_LAUNCH_CHECK();
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(bapply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kASmem));
    conf = true;
  }
  const ApplyArgs aa{d.Q, d.rows_pad, d.kpad, d.ksplit, d.expoF, d.expoU, d.part};
  const int items = d.Q * (d.rows_pad / kAM) * d.ksplit;
  bapply_tc_kernel<<<std::min(items, 152), kAThreads, kASmem, st>>>(d.tmF, d.tmU, aa, err);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm

extern "C" int sadmm_digit_apply16(const double* F, int ld, int n, const float* U, double* out, void* stream) {
  using namespace sadmm;
  if (!F || !U || !out || n <= 0 || ld < n) {
    set_error("sadmm_digit_apply16: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DigitApply d;
  digit_apply_dims(d, 1, n);
  const size_t bytes = digit_apply_bytes(d);
  char* mem = nullptr;
  SADMM_CUDA_TRY(cudaMalloc((void**)&mem, bytes + 1024 + 64));
  int* derr = reinterpret_cast<int*>(mem + bytes + 1024);
  const float** uptr = reinterpret_cast<const float**>(mem + bytes + 1024 + 16);
  int rc = digit_apply_bind(d, mem);
  if (rc == SADMM_OK && (cudaMemsetAsync(derr, 0, sizeof(int), st) != cudaSuccess ||
                         cudaMemcpyAsync(uptr, &U, sizeof(void*), cudaMemcpyHostToDevice, st) != cudaSuccess)) {
    set_error("sadmm_digit_apply16: %s", cudaGetErrorString(cudaGetLastError()));
    rc = SADMM_ECUDA;
  }
  if (rc == SADMM_OK) rc = launch_factor_digits(d, 0, F, ld, st);
  if (rc == SADMM_OK) rc = launch_digit_apply(d, uptr, 1, derr, st);
  if (rc == SADMM_OK) {
    digit_out_kernel<<<div_up((long long)n * kAN, 256), 256, 0, st>>>(d.part, d.ksplit, d.rows_pad, n, out);
    if (cudaGetLastError() != cudaSuccess) { set_error("sadmm_digit_apply16: launch failed"); rc = SADMM_ECUDA; }
  }
  int herr = 0;
  if (rc == SADMM_OK && (cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess)) {
    set_error("sadmm_digit_apply16: %s", cudaGetErrorString(cudaGetLastError()));
    rc = SADMM_ECUDA;
  }
  cudaStreamSynchronize(st);
  cudaFree(mem);
  if (rc != SADMM_OK) return rc;
  if (herr) { set_error("sadmm_digit_apply16: a bounded wait of the tensor-core pipeline timed out"); return SADMM_ETIMEOUT; }
  return SADMM_OK;
}
