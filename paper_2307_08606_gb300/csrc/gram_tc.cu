// Gram matrix of the x-update system on the tensor cores (Eq. 3, x_q-update):
//   out = mu G + rho I,  G = B_J^T B_J (primal form: rows are the active
//   pixels, sums over the 2KM real rows) or G = B_J B_J^T (Woodbury form: rows
//   are the 2KM real rows, sums over the active pixels),
// for the FP64 factor, to about 2^-36 of each row's scale (the FP64 Gram of the
// FP32 operator is exact to 2^-53; GB300's FP64 pipe is too narrow for the
// (2KM)^2 |J| or |J|^2 2KM multiply-adds of a large factor).
//
// Exact integer slices.  Each Gram row i (a pixel's column of B, or a real row
// of B) is scaled by 2^-e_i, e_i the least exponent with max |row| <= 2^e_i,
// and each scaled entry v in [-1, 1] is written as
//   v = 2^-7 (d1 + 2^-8 d2 + 2^-16 d3 + 2^-24 d4) + t,  integers |d_a| <= 128,
// |t| <= 2^-32 (t = 0 for FP32 entries with |v| >= 2^-8).  The digits are held
// exactly in BF16, and
//   G_ij = 2^(e_i + e_j - 14) sum_{o >= 2} 2^(-8 (o - 2)) S_o(i, j),
//   S_o(i, j) = sum_{a + b = o} sum_k d_a(i, k) d_b(j, k).
// The orders o = 2..5 are formed (ten digit GEMMs per tile); the dropped
// orders and t contribute at most about 2^-30 per term.  Every digit product
// is an integer of magnitude <= 2^14, exact in the FP32 accumulator, and an
// order sum over a chunk of 256 values of k (at most four products per k)
// stays within 2^24, so each chunk's order sums are exact integers in FP32.
// After every chunk the four sums are read out of tensor memory and added to
// double-float running totals (about 48 bits), which the epilogue scales,
// converts to FP64 and writes with the mirror image.
//
// Kernels: the digit conversions (one per form; the Woodbury form transposes
// through shared memory so that k = pixel is contiguous) write four BF16 digit
// planes [digit][row][k] (rows padded to 128, k to 256, zero-filled) and the
// row exponents; gram_tc_kernel is a persistent, warp-specialised pipeline over
// the upper-triangular tiles (128 rows x 64 columns):
//   warp 0      TMA producer: per 64-k stage, the four digit tiles of the row
//               block (2 boxes of 64 rows each) and of the column block, 128-
//               byte swizzle (the SW128 K-major operand layout of the MMA);
//   warp 1      MMA issuer: per 16-k step ten tcgen05.mma kind::f16 (BF16 in,
//               FP32 accumulate, M 128 N 64 K 16) into the four order
//               accumulators of one of two TMEM sets (alternating per chunk);
//   warps 2-9   epilogue: per chunk, tcgen05.ld of the four accumulators (one
//               32-lane quarter and 32 of the 64 columns per warp),
//               double-float update; per tile, the scaled FP64 output.
// Every wait is bounded; on a timeout the CTA flags *err, waits (bounded) for
// its copies in flight, frees its tensor memory and exits.
#include "common.cuh"
#include "tmap.cuh"

#include <cuda_bf16.h>
#include <cstring>

namespace sadmm {
namespace {

constexpr int kGM = 128;                            // tile rows (TMEM lanes)
constexpr int kGN = 64;                             // tile columns
constexpr int kGK = 64;                             // k per stage: one 128-byte BF16 row
constexpr int kChunk = 256;                         // k per exact chunk
constexpr int kStagesPerChunk = kChunk / kGK;       // 4
constexpr int kDigits = 4;
constexpr int kBox = 64;                            // rows per TMA box
constexpr int kATile = kGM * kGK * 2;               // 16 KB per digit
constexpr int kBTile = kGN * kGK * 2;               // 8 KB per digit
constexpr int kStage = kDigits * (kATile + kBTile); // 96 KB
constexpr int kGS = 2;                              // stages
constexpr int kGSmem = kGS * kStage + 1024;         // + alignment slack
constexpr int kGThreads = 320;                     // producer, MMA issuer, 8 epilogue warps
constexpr int kEpi = 256;                           // epilogue threads
constexpr int kSetCols = 4 * kGN;                   // four order accumulators
constexpr int kGTmemCols = 2 * kSetCols;            // two sets: 512 columns
constexpr long long kGWait = 1ll << 26;

// kind::f16, D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t kGIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) |
                             ((uint32_t)(kGM >> 4) << 24);

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

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t a, uint64_t b, unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kGIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ bool wait(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kGWait; ++it) {
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

// Digits of v * 2^7 (|v| <= 1): four integers in [-128, 128], exact in BF16.
__device__ __forceinline__ void digits4(float t, __nv_bfloat16 (&d)[kDigits]) {
#pragma unroll
  for (int a = 0; a < kDigits; ++a) {
    const float r = rintf(t);
    d[a] = __float2bfloat16_rn(r);
    t = (t - r) * 256.f;                  // exact: |t - r| <= 1/2 is a multiple of ulp(t)
  }
}

// two BF16 values as one word, the first in the low half (memory order)
__device__ __forceinline__ unsigned pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

// least e with m <= 2^e (m >= 0; 0 for m = 0)
__device__ __forceinline__ int row_exponent(float m) {
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);                          // m = f 2^e, f in [1/2, 1)
  return e;
}

struct GramArgs {
  int rows_pad;        // digit-plane rows (multiple of 128)
  int kpad;            // digit-plane k (multiple of 256)
  int n;               // valid rows
  int ld;              // output leading dimension (rows >= ld are not written)
  const int* expo;     // rows_pad row exponents
  double* out;
  double mu, rho;
};

// ------------------------------------------------------- digit conversions
// Primal form: row p = pixel idx[p]: its 2KM floats are contiguous.  One CTA
// per row: the row maximum, then four floats per thread and step.
__global__ void __launch_bounds__(256)
primal_digits_kernel(const float* __restrict__ Af, const int* __restrict__ idx, int n, int R, int kpad, int rows_pad,
                     __nv_bfloat16* __restrict__ D, int* __restrict__ expo) {
  const int p = blockIdx.x;
  const int tid = threadIdx.x;
  const float* src = p < n ? Af + (size_t)idx[p] * R : nullptr;
  __shared__ float s_max[8];
  float m = 0.f;
  if (src)
    for (int k = 4 * tid; k < R; k += 4 * 256) {
      const float4 a = *reinterpret_cast<const float4*>(src + k);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) s_max[tid >> 5] = m;
  __syncthreads();
  m = s_max[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, s_max[w]);
  const int e = row_exponent(m);
  if (tid == 0) expo[p] = e;
  const float sc = ldexpf(1.f, 7 - e);
  const size_t plane = (size_t)rows_pad * kpad;
  for (int k = 4 * tid; k < kpad; k += 4 * 256) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (src && k < R) a = *reinterpret_cast<const float4*>(src + k);
    __nv_bfloat16 d0[kDigits], d1[kDigits], d2[kDigits], d3[kDigits];
    digits4(a.x * sc, d0);
    digits4(a.y * sc, d1);
    digits4(a.z * sc, d2);
    digits4(a.w * sc, d3);
#pragma unroll
    for (int dg = 0; dg < kDigits; ++dg)
      *reinterpret_cast<uint2*>(D + dg * plane + (size_t)p * kpad + k) =
          make_uint2(pack2(d0[dg], d1[dg]), pack2(d2[dg], d3[dg]));
  }
}

// Woodbury form, pass 1: the maximum |B[r][p]| over the active pixels of every
// real row r (as float bits: non-negative floats order as integers).
__global__ void __launch_bounds__(256)
woodbury_rowmax_kernel(const float* __restrict__ Af, const int* __restrict__ idx, int ncols, int R,
                       int* __restrict__ maxbits) {
  const int r = blockIdx.x * 256 + threadIdx.x;
  if (r >= R) return;
  const int per = (ncols + gridDim.y - 1) / gridDim.y;
  const int p0 = blockIdx.y * per, p1 = min(ncols, p0 + per);
  float m = 0.f;
  for (int p = p0; p < p1; ++p) m = fmaxf(m, fabsf(Af[(size_t)idx[p] * R + r]));
  if (m > 0.f) atomicMax(maxbits + r, __float_as_int(m));
}

// Woodbury form, pass 2: 64 real rows x 64 pixels per CTA, read along the
// rows (contiguous in the pixel-major operand) and written along the pixels.
__global__ void __launch_bounds__(256)
woodbury_digits_kernel(const float* __restrict__ Af, const int* __restrict__ idx, int ncols, int R, int kpad,
                       int rows_pad, const int* __restrict__ maxbits, __nv_bfloat16* __restrict__ D,
                       int* __restrict__ expo) {
  __shared__ float tile[64][65];          // [pixel][row]
  const int r0 = blockIdx.y * 64, p0 = blockIdx.x * 64;
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int pp = e / 64, rr = e % 64;
    const int p = p0 + pp, r = r0 + rr;
    tile[pp][rr] = (p < ncols && r < R) ? Af[(size_t)idx[p] * R + r] : 0.f;
  }
  __syncthreads();
  const int rr = tid >> 2, seg = (tid & 3) * 16;
  const int r = r0 + rr;
  const int e = r < R ? row_exponent(__int_as_float(maxbits[r])) : 0;
  if (blockIdx.x == 0 && (tid & 3) == 0 && r < rows_pad) expo[r] = e;
  const float sc = ldexpf(1.f, 7 - e);
  const size_t plane = (size_t)rows_pad * kpad;
  unsigned w[kDigits][8];                 // 16 digits per plane, two per word
#pragma unroll
  for (int u = 0; u < 16; u += 2) {
    __nv_bfloat16 d0[kDigits], d1[kDigits];
    digits4(tile[seg + u][rr] * sc, d0);
    digits4(tile[seg + u + 1][rr] * sc, d1);
#pragma unroll
    for (int a = 0; a < kDigits; ++a) w[a][u / 2] = pack2(d0[a], d1[a]);
  }
#pragma unroll
  for (int a = 0; a < kDigits; ++a) {
    uint4* dst = reinterpret_cast<uint4*>(D + a * plane + (size_t)r * kpad + p0 + seg);
    dst[0] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
    dst[1] = make_uint4(w[a][4], w[a][5], w[a][6], w[a][7]);
  }
}

// ------------------------------------------------------------- the GEMM
// item -> (row block I, column block Jc), Jc >= 2 I (the column block reaches
// the diagonal block or lies right of it)
__device__ __forceinline__ void item_ij(int it, int nI, int nJ, int& I, int& Jc) {
  I = 0;
  while (it >= nJ - 2 * I) {
    it -= nJ - 2 * I;
    ++I;
  }
  Jc = 2 * I + it;
}

__global__ void __launch_bounds__(kGThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tm, const __grid_constant__ GramArgs ga, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kGS], empty[kGS], accfull[2], accempty[2];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nI = ga.rows_pad / kGM, nJ = ga.rows_pad / kGN;
  const int items = nI * nI + nI;
  const int nchunks = ga.kpad / kChunk;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < kGS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&accfull[b], 1);
      bar_init(&accempty[b], kEpi);
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
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int I, Jc;
        item_ij(it, nI, nJ, I, Jc);
        const int nst = nchunks * kStagesPerChunk;
        for (int sl = 0; sl < nst && ok; ++sl, ++t) {
          const int s = t % kGS;
          if (t >= kGS) ok = wait(&empty[s], ((t / kGS) - 1) & 1);
          if (!ok) break;
          unsigned char* st = smem + s * kStage;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])), "r"(kStage)
                       : "memory");
          const int x = sl * kGK;
#pragma unroll
          for (int d = 0; d < kDigits; ++d) {
            const int yA = d * ga.rows_pad + I * kGM, yB = d * ga.rows_pad + Jc * kGN;
#pragma unroll
            for (int h = 0; h < kGM / kBox; ++h)
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                      su32(st + d * kATile + h * (kBox * kGK * 2))),
                  "l"(reinterpret_cast<uint64_t>(&tm)), "r"(x), "r"(yA + h * kBox), "r"(su32(&full[s]))
                  : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    su32(st + kDigits * kATile + d * kBTile)),
                "l"(reinterpret_cast<uint64_t>(&tm)), "r"(x), "r"(yB), "r"(su32(&full[s]))
                : "memory");
          }
        }
      }
      // copies still in flight when stopping early: wait for them (bounded)
      if (!ok)
        for (int u = max(0, t - kGS); u < t; ++u) wait(&full[u % kGS], (u / kGS) & 1);
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
          const unsigned d0 = tmem + b * kSetCols;
          for (int sc = 0; sc < kStagesPerChunk && ok; ++sc, ++t) {
            const int s = t % kGS;
            ok = wait(&full[s], (t / kGS) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sa = su32(smem + s * kStage), sb = sa + kDigits * kATile;
#pragma unroll
            for (int ks = 0; ks < kGK / 16; ++ks) {
              const unsigned f = (sc > 0 || ks > 0) ? 1u : 0u;
              uint64_t A[kDigits], B[kDigits];
#pragma unroll
              for (int d = 0; d < kDigits; ++d) {
                A[d] = sw128(sa + d * kATile + ks * 32);
                B[d] = sw128(sb + d * kBTile + ks * 32);
              }
              mma_bf16(d0, A[0], B[0], f);                       // order 2
              mma_bf16(d0 + kGN, A[0], B[1], f);                 // order 3
              mma_bf16(d0 + kGN, A[1], B[0], 1u);
              mma_bf16(d0 + 2 * kGN, A[0], B[2], f);             // order 4
              mma_bf16(d0 + 2 * kGN, A[1], B[1], 1u);
              mma_bf16(d0 + 2 * kGN, A[2], B[0], 1u);
              mma_bf16(d0 + 3 * kGN, A[0], B[3], f);             // order 5
              mma_bf16(d0 + 3 * kGN, A[1], B[2], 1u);
              mma_bf16(d0 + 3 * kGN, A[2], B[1], 1u);
              mma_bf16(d0 + 3 * kGN, A[3], B[0], 1u);
            }
            commit(&empty[s]);
          }
          if (ok) commit(&accfull[b]);
        }
      }
    }
  } else {
    // -------------------------------------------------------------- epilogue
    const int quarter = warp & 3;           // TMEM lanes 32 quarter .. + 31
    const int row = quarter * 32 + lane;    // row of the tile
    const int c0 = ((warp - 2) >> 2) * (kGN / 2);   // this warp's 32 columns
    int gc = 0;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int I, Jc;
      item_ij(it, nI, nJ, I, Jc);
      constexpr int kC = kGN / 2;
      float th[kC], tl[kC];
#pragma unroll
      for (int j = 0; j < kC; ++j) { th[j] = 0.f; tl[j] = 0.f; }
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = gc & 1;
        ok = wait(&accfull[b], (gc / 2) & 1);
        ok = __all_sync(0xffffffffu, ok);      // tcgen05.ld below is warp-collective
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + b * kSetCols + c0;
#pragma unroll
        for (int cb = 0; cb < kC / 16; ++cb) {
          float s2[16], s3[16], s4[16], s5[16];
          tld16(ta + cb * 16, s2);
          tld16(ta + kGN + cb * 16, s3);
          tld16(ta + 2 * kGN + cb * 16, s4);
          tld16(ta + 3 * kGN + cb * 16, s5);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = cb * 16 + u;
            two_add(th[j], tl[j], s2[u]);
            two_add(th[j], tl[j], s3[u] * 0x1p-8f);
            tl[j] += fmaf(s4[u], 0x1p-16f, s5[u] * 0x1p-24f);
            const float h = th[j] + tl[j];       // renormalise
            tl[j] -= h - th[j];
            th[j] = h;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        bar_arrive(&accempty[b]);
      }
      if (!ok) break;
      const int i = I * kGM + row;
      if (i < ga.ld) {
        const int ei = ga.expo[i];
#pragma unroll
        for (int j0 = 0; j0 < kC; ++j0) {
          const int j = Jc * kGN + c0 + j0;
          if (j >= ga.ld) continue;
          double v;
          if (i < ga.n && j < ga.n)
            v = ga.mu * ldexp((double)th[j0] + (double)tl[j0], ei + ga.expo[j] - 14) + (i == j ? ga.rho : 0.0);
          else
            v = (i == j) ? 1.0 : 0.0;
          ga.out[(size_t)i * ga.ld + j] = v;
          ga.out[(size_t)j * ga.ld + i] = v;
        }
      }
    }
  }
  if (!ok) atomicExch(err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols) : "memory");
}

void gram_dims(const FactorJob& j, int KM, int* rows_pad, int* kpad) {
  const int R = 2 * KM;
  *rows_pad = round_up(j.woodbury ? R : j.ncols, kGM);
  *kpad = round_up(j.woodbury ? j.ncols : R, kChunk);
}

}  // namespace

size_t gram_tc_scratch_bytes(const FactorJob& j, int KM) {
  int rows_pad, kpad;
  gram_dims(j, KM, &rows_pad, &kpad);
  return (size_t)kDigits * rows_pad * kpad * sizeof(__nv_bfloat16) + 2 * (size_t)rows_pad * sizeof(int) + 256;
}

int launch_gram_tc(const FactorJob& j, int KM, double mu, double rho, void* scratch, size_t scratch_bytes, int* err,
                   cudaStream_t st) {
  const int R = 2 * KM;
  if (R % 4 != 0 || j.ncols <= 0 || j.n != (j.woodbury ? R : j.ncols) || j.npad < j.n) {
    set_error("launch_gram_tc: bad sizes");
    return SADMM_EINVAL;
  }
  if (scratch_bytes < gram_tc_scratch_bytes(j, KM)) {
    set_error("launch_gram_tc: scratch too small");
    return SADMM_EINVAL;
  }
  int rows_pad, kpad;
  gram_dims(j, KM, &rows_pad, &kpad);
  __nv_bfloat16* D = reinterpret_cast<__nv_bfloat16*>(scratch);
  const size_t dbytes = (size_t)kDigits * rows_pad * kpad * sizeof(__nv_bfloat16);
  int* expo = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + dbytes);
  int* maxbits = expo + rows_pad;
  const float* Af = reinterpret_cast<const float*>(j.A);
  SADMM_CUDA_TRY(cudaMemsetAsync(expo, 0, 2 * (size_t)rows_pad * sizeof(int), st));
  if (j.woodbury) {
    SADMM_CUDA_TRY(cudaMemsetAsync(D, 0, dbytes, st));    // rows past R stay zero
    woodbury_rowmax_kernel<<<dim3(div_up(R, 256), std::min(256, div_up(j.ncols, 64))), 256, 0, st>>>(
        Af, j.idx, j.ncols, R, maxbits);
    SADMM_LAUNCH_CHECK();
    woodbury_digits_kernel<<<dim3(kpad / 64, div_up(R, 64)), 256, 0, st>>>(Af, j.idx, j.ncols, R, kpad, rows_pad,
                                                                        maxbits, D, expo);
    SADMM_LAUNCH_CHECK();
  } else {
    primal_digits_kernel<<<rows_pad, 256, 0, st>>>(Af, j.idx, j.ncols, R, kpad, rows_pad, D, expo);
    SADMM_LAUNCH_CHECK();
  }
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) { set_error("launch_gram_tc: cuTensorMapEncodeTiled unavailable"); return SADMM_ECUDA; }
  CUtensorMap tm;
  memset(&tm, 0, sizeof tm);
  const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)kDigits * rows_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)kpad * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kGK, (cuuint32_t)kBox};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, D, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("launch_gram_tc: tensor map rejected (%d)", (int)r); return SADMM_ECUDA; }
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem));
    conf = true;
  }
  GramArgs ga{rows_pad, kpad, j.n, j.npad, expo, j.out, mu, rho};
  const int nI = rows_pad / kGM;
  const int items = nI * nI + nI;
  gram_tc_kernel<<<std::min(items, 152), kGThreads, kGSmem, st>>>(tm, ga, err);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
