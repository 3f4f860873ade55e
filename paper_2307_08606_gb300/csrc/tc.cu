// Tensor-core (tcgen05) adjoint GEMM of the batched form (Eq. 3, x_q-update
// for 16 scenes at once):
//   G[p][s] = Re(a_p^H w_s) = sum_r B[r][p] W[r][s],   r over the 2KM real rows,
// with B the real form of A_q (pixel-major: the 2KM floats of pixel p are
// contiguous, so B^T is K-major) and W the 16 right-hand sides (complex
// [row][scene], real row r = 2m + c at float (m * 16 + s) * 2 + c).
//
// Precision: three TF32 products per term (3xTF32).  Each operand is split
// x = hi + lo, lo = x - hi exact in FP32 (the MMA keeps its top 11 bits): the
// right-hand sides with hi = tf32(x) rounded to nearest, the operator tile
// with hi = x itself (the MMA reads the top 19 bits of an FP32 value, its
// truncation to TF32) and lo = x - trunc(x).  hi*hi, hi*lo and lo*hi
// accumulate in FP32 in tensor memory, added as hi*hi + (hi*lo + lo*hi) at the
// end: each product is within 2^-21 of the FP32 one, the dropped lo*lo term is
// below 2^-21, and the sums over K round as FP32 accumulations do.
//
// Tile: M = 128 pixels (TMEM lanes), N = 16 scenes (TMEM columns), K slabs of
// 32 real rows.  A slab of A arrives by TMA (tensor map over the pixel-major
// operand, 128-byte swizzle: exactly the SW128 K-major operand layout of the
// MMA); W's slab (2 KB) by a bulk copy.  The landed tile is the hi operand
// and a lo tile of the same layout is formed beside it; W goes to one 32-row
// B tile (hi rows 0-15, lo rows 16-31) in the no-swizzle K-major layout (core
// matrices of 8 rows x 16 bytes, K-adjacent cores LBO bytes apart, N-adjacent
// cores SBO bytes apart).  One thread issues, per k-step of 8, an N = 32 MMA
// (A hi against the whole B tile: hi*hi and hi*lo from one read of A) and an
// N = 16 MMA (A lo against the hi rows), tcgen05.mma kind::tf32 (M128 K8);
// the accumulators are read back with tcgen05.ld (32 lanes x 16 columns per
// warp).  A variant with separate rings for the landed tiles and the
// converted operands (more slabs in flight, one more hand-off per slab) ran
// slower on GB300 (adjoint 4.3 ms against 3.2 ms at Q=8, KM=16384, N=128^2).
// The pipeline structure is described at tc_adjoint_kernel.  Every wait is
// bounded; on a timeout the CTA flags *err, waits (bounded) for its copies in
// flight, frees its tensor memory and exits.
#include "common.cuh"

#include "tmap.cuh"

#include <cstring>

namespace sadmm {
namespace {

constexpr int kTcM = 128;              // pixels per CTA
constexpr int kTcN = 16;               // scenes
constexpr int kTcK = 32;               // real rows per slab
constexpr int kTmemCols = 128;         // 2 accumulator sets, power of two
// one set: hi x [hi; lo] (an N = 32 accumulator: hi*hi in columns 0-15, hi*lo
// in 16-31) and lo x hi (columns 32-47); sets 64 columns apart
constexpr int kAccSet = 64;
constexpr long long kTcWaitLimit = 1ll << 26;

// operand tile bytes per plane and buffer
constexpr int kABytes = kTcM * kTcK * 4;          // 16 KB
constexpr int kBBytes = kTcN * kTcK * 4;          // 2 KB: one 16-row plane
// The B operand tile holds 32 rows: the TF32 hi parts of the 16 right-hand
// sides (rows 0-15), then their lo parts (rows 16-31), so that one N = 32 MMA
// forms hi*hi and hi*lo from a single read of the A tile.
// canonical K-major layout strides (bytes)
constexpr int kCore = 128;                         // 8 rows x 16 bytes
constexpr int kB_SBO = kCore;                      // next 8 rows
constexpr int kB_LBO = (2 * kTcN / 8) * kCore;     // next 4 k-elements (512)

// byte offset of (row n, k) in the B tile
__host__ __device__ constexpr int b_off(int n, int k) {
  return (k >> 2) * kB_LBO + (n >> 3) * kB_SBO + (n & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, int lbo, int sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
  return d;                            // base offset 0, no swizzle
}

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 16 or 32
constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}
constexpr uint32_t kIdesc16 = idesc_tf32(kTcN), kIdesc32 = idesc_tf32(2 * kTcN);

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, uint32_t idesc, unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// hi*[hi; lo] and lo*hi for one k-step of 8: two MMAs into one accumulator set
__device__ __forceinline__ void mma_3xtf32(unsigned d, uint64_t a_hi, uint64_t a_lo, uint64_t b, unsigned acc) {
  mma_tf32(d, a_hi, b, kIdesc32, acc);
  mma_tf32(d + 2 * kTcN, a_lo, b, kIdesc16, acc);     // the first 16 rows of the B tile: hi
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
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

// The 16 columns of this warp's 32-lane quarter at taddr (one row per lane).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// hi*hi + (hi*lo + lo*hi) from the three accumulators of one set
__device__ __forceinline__ void tmem_sum3(unsigned taddr, float (&v)[16]) {
  float b[16], c[16];
  tmem_ld16(taddr, v);
  tmem_ld16(taddr + kTcN, b);
  tmem_ld16(taddr + 2 * kTcN, c);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += b[i] + c[i];
}

__device__ __forceinline__ float tf32_rn(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x with its low 13 mantissa bits cleared (truncation to TF32)
__device__ __forceinline__ float tf32_tz(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct TmapSet {
  CUtensorMap m[kMaxSets];     // A_q as a 2-D FP32 tensor: x = real row (2KM), y = pixel (N)
};
struct PtrSet {
  const float* w[kMaxSets];    // W_q as floats
};

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// Persistent, warp-specialised pipeline over work items (sensor, 128-pixel
// tile, row split), kS shared-memory stages deep:
//   warp 0      producer: per slab one TMA tile load of A (128 pixels x 32
//               real rows, 128-byte swizzle) and one bulk copy of the W slab;
//   warp 1      MMA issuer: 4 k-steps x 2 tcgen05.mma per slab into one of two
//               TMEM accumulators (alternating per item), commits free the
//               stage and, at the end of an item, publish the accumulator;
//   warps 2-5   converters: form the lo tile of the landed A tile (same
//               swizzled layout; the tile itself is the hi operand) and the B
//               tile from W; after an item, read its accumulator (each warp
//               its 32-lane quarter of TMEM) and store the 128 x 16 result.
// Barriers: full (TMA landed), conv (operands ready), empty (stage free),
// accfull / accempty (accumulator handoff).  All waits are bounded.
constexpr int kS = 5;
constexpr int kPipeThreads = 192;
constexpr int kStageBytes = 2 * kABytes + 3 * kBBytes;        // A (raw = hi), A lo, B (hi; lo), W raw
constexpr int kPipeSmem = kS * kStageBytes + 1024;            // + alignment slack

// SW128 K-major descriptor: 8-row atoms of 128-byte rows, atoms 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                                      // leading offset: unused for swizzled K-major
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;                 // stride offset: next 8 rows
  d |= (uint64_t)1 << 46;                                      // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                                      // 128-byte swizzle
  return d;
}

__global__ void __launch_bounds__(kPipeThreads, 1)
tc_adjoint_kernel(const __grid_constant__ TmapSet tmaps, const __grid_constant__ PtrSet wq, float* __restrict__ gpart,
                  int Q, int N, int KM, int splits, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kS], conv[kS], empty[kS], accfull[2], accempty[2];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int R = 2 * KM;
  const int mtiles = (N + kTcM - 1) / kTcM;
  const int items = Q * mtiles * splits;
  const int rows_per = (R / splits + kTcK - 1) / kTcK * kTcK;
  auto item_of = [&](int it, int& q, int& mt, int& sp, int& rb, int& ns) {
    sp = it % splits;
    const int qm = it / splits;
    mt = qm % mtiles;
    q = qm / mtiles;
    rb = sp * rows_per;
    ns = max(0, (min(R, rb + rows_per) - rb) / kTcK);
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < kS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 128);
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
      // ---------------------------------------------------------------- producer
      int t = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int q, mt, sp, rb, ns;
        item_of(it, q, mt, sp, rb, ns);
        for (int sl = 0; sl < ns && ok; ++sl, ++t) {
          const int s = t % kS;
          if (t >= kS) ok = bar_wait(&empty[s], ((t / kS) - 1) & 1);
          if (!ok) break;
          unsigned char* st = smem + s * kStageBytes;
          mbar_expect_tx(&full[s], kABytes + kBBytes);
          const int x = rb + sl * kTcK, y = mt * kTcM;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  su32(st)),
              "l"(reinterpret_cast<uint64_t>(&tmaps.m[q])), "r"(x), "r"(y), "r"(su32(&full[s]))
              : "memory");
          const float* wsrc = wq.w[q] + (size_t)x * kTcN;       // real rows x .. x+31 = complex rows x/2 ..
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           su32(st + 2 * kABytes + 2 * kBBytes)),
                       "l"(wsrc), "r"(kBBytes), "r"(su32(&full[s]))
                       : "memory");
        }
      }
      // copies still in flight when stopping early: wait for them (bounded)
      if (!ok)
        for (int u = max(0, t - kS); u < t; ++u) bar_wait(&full[u % kS], (u / kS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA issuer
      int t = 0, i = 0;                 // i counts the non-empty items (accumulator alternation)
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int q, mt, sp, rb, ns;
        item_of(it, q, mt, sp, rb, ns);
        if (ns == 0) continue;
        const int ab = i & 1;
        if (i >= 2) ok = bar_wait(&accempty[ab], ((i / 2) - 1) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned d = tmem + ab * kAccSet;    // three independent accumulation chains
        for (int sl = 0; sl < ns && ok; ++sl, ++t) {
          const int s = t % kS;
          ok = bar_wait(&conv[s], (t / kS) & 1);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned st = su32(smem + s * kStageBytes);
          const unsigned a_hi = st, a_lo = st + kABytes, b = st + 2 * kABytes;
#pragma unroll
          for (int ks = 0; ks < kTcK / 8; ++ks) {
            const unsigned acc0 = (sl > 0 || ks > 0) ? 1u : 0u;
            mma_3xtf32(d, sw128_desc(a_hi + ks * 32), sw128_desc(a_lo + ks * 32),
                       smem_desc(b + ks * 2 * kB_LBO, kB_LBO, kB_SBO), acc0);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accfull[ab]);
        ++i;
      }
    }
  } else {
    // --------------------------------------------------------- converters
    const int ct = tid - 64;                        // 0..127
    const int quarter = warp & 3;                   // TMEM lanes 32 quarter .. +31
    int t = 0, i = 0;                   // i counts the non-empty items
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int q, mt, sp, rb, ns;
      item_of(it, q, mt, sp, rb, ns);
      if (ns == 0) {
        // an empty row split contributes zeros
        const int p = mt * kTcM + quarter * 32 + lane;
        if (p < N) {
          float4* out = reinterpret_cast<float4*>(gpart + (((size_t)q * splits + sp) * N + p) * kTcN);
#pragma unroll
          for (int e = 0; e < 4; ++e) out[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        continue;
      }
      for (int sl = 0; sl < ns && ok; ++sl, ++t) {
        const int s = t % kS;
        ok = bar_wait(&full[s], (t / kS) & 1);
        if (!ok) break;
        unsigned char* st = smem + s * kStageBytes;
        // the landed tile stays in place as the hi operand (the MMA reads the
        // top 19 bits of each FP32 value: its truncation to TF32); the lo tile
        // is the exact remainder
        const float4* ahi = reinterpret_cast<const float4*>(st);
        float4* alo = reinterpret_cast<float4*>(st + kABytes);
#pragma unroll
        for (int w = 0; w < kABytes / 16 / 128; ++w) {
          const int e = ct + 128 * w;
          const float4 x = ahi[e];
          alo[e] = make_float4(x.x - tf32_tz(x.x), x.y - tf32_tz(x.y), x.z - tf32_tz(x.z), x.w - tf32_tz(x.w));
        }
        float* bt = reinterpret_cast<float*>(st + 2 * kABytes);
        {
          // scene n = ct % 16, real rows 4j .. 4j + 3 (complex rows 2j, 2j + 1)
          // with j = ct / 16: one 16-byte chunk of the hi rows and one of the
          // lo rows per thread (a quarter-warp covers eight scenes: the eight
          // chunk positions of a 128-byte line, no bank conflict)
          const float* wr = reinterpret_cast<const float*>(st + 2 * kABytes + 2 * kBBytes);
          const int n = ct & 15, j = ct >> 4;
          const float2 w0 = *reinterpret_cast<const float2*>(wr + ((2 * j) * kTcN + n) * 2);
          const float2 w1 = *reinterpret_cast<const float2*>(wr + ((2 * j + 1) * kTcN + n) * 2);
          const float4 h = make_float4(tf32_rn(w0.x), tf32_rn(w0.y), tf32_rn(w1.x), tf32_rn(w1.y));
          *reinterpret_cast<float4*>(bt + b_off(n, 4 * j) / 4) = h;
          *reinterpret_cast<float4*>(bt + b_off(kTcN + n, 4 * j) / 4) =
              make_float4(w0.x - h.x, w0.y - h.y, w1.x - h.z, w1.y - h.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (!ok) break;
      // epilogue of this item
      const int ii = i++;
      const int ab = ii & 1;
      ok = bar_wait(&accfull[ab], (ii / 2) & 1);
      ok = __all_sync(0xffffffffu, ok);          // tcgen05.ld below is warp-collective
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[16];
      tmem_sum3(tmem + ((unsigned)(quarter * 32) << 16) + ab * kAccSet, v);
      const int p = mt * kTcM + quarter * 32 + lane;
      if (p < N) {
        float4* out = reinterpret_cast<float4*>(gpart + (((size_t)q * splits + sp) * N + p) * kTcN);
#pragma unroll
        for (int e = 0; e < 4; ++e) out[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&accempty[ab]);
    }
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ------------------------------------------------------------------ forward
// D_q (2KM x 16) = B_q V_q for the batched form's forward product (Eq. 3,
// x_q-update: r = y' - B v for 16 scenes), V[p][s] = x - x_bar + z_bar - s of
// scene s at pixel p.  M = 128 real rows (TMEM lanes), N = 16 scenes, K = 32
// pixels per slab; items (sensor, row tile, pixel split) are spread over
// persistent CTAs.  The operator tile arrives by TMA as [32 pixels][128 rows]
// (rows contiguous, no swizzle) and the four 2 KB slabs of x, x_bar, z_bar, s
// by bulk copies; converter warps transpose the tile into the SW128 K-major
// layout as the hi tile (the values themselves, truncated to TF32 by the MMA)
// and the lo tile of exact remainders (row m, pixel quad kq
// lands in 16-byte chunk kq ^ (m mod 8) of its 128-byte row: conflict-free),
// form V and split it into the 32-row B tile.  The MMA issuer and the
// epilogue are as in tc_adjoint_kernel; the epilogue writes partial sums in
// the layout of the SIMT forward (partial[q][split][complex row][scene] as
// float2), which bfwd_reduce_kernel turns into r = y' - sum.
constexpr int kFwdS = 3;
constexpr int kFwdRaw = kTcM * kTcK * 4;                       // [32 pixels][128 rows] floats, 16 KB
constexpr int kVBytes = kTcK * kTcN * 4;                        // one [32 pixels][16 scenes] slab, 2 KB
constexpr int kFwdStage = kFwdRaw + 2 * kABytes + 2 * kBBytes + 4 * kVBytes;   // 60 KB: raw, A hi, A lo, B, V
constexpr int kFwdSmem = kFwdS * kFwdStage + 1024;

struct VSet {
  const float* X;       // Q x N x 16
  const float* xbar;    // N x 16
  const float* zbar;
  const float* sd;
};

__global__ void __launch_bounds__(kPipeThreads, 1)
tc_forward_kernel(const __grid_constant__ TmapSet tmaps, const __grid_constant__ VSet vs, float* __restrict__ partial,
                  int Q, int N, int KM, int splits, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kFwdS], conv[kFwdS], empty[kFwdS], accfull[2], accempty[2];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int R = 2 * KM;
  const int mtiles = (R + kTcM - 1) / kTcM;
  const int items = Q * mtiles * splits;
  const int pix_per = (N / splits + kTcK - 1) / kTcK * kTcK;
  auto item_of = [&](int it, int& q, int& mt, int& sp, int& pb, int& ns) {
    sp = it % splits;
    const int qm = it / splits;
    mt = qm % mtiles;
    q = qm / mtiles;
    pb = sp * pix_per;
    const int pe = min(N, pb + pix_per);
    ns = pe > pb ? (pe - pb + kTcK - 1) / kTcK : 0;
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < kFwdS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s_tmem;
  bool ok = true;
  // stage layout: raw A | A hi | A lo | B hi | B lo | x | x_bar | z_bar | s
  auto stage = [&](int s) { return smem + s * kFwdStage; };
  constexpr int oAhi = kFwdRaw, oAlo = kFwdRaw + kABytes, oB = kFwdRaw + 2 * kABytes, oV = oB + 2 * kBBytes;

  if (warp == 0) {
    if (lane == 0) {
      int t = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int q, mt, sp, pb, ns;
        item_of(it, q, mt, sp, pb, ns);
        for (int sl = 0; sl < ns && ok; ++sl, ++t) {
          const int s = t % kFwdS;
          if (t >= kFwdS) ok = bar_wait(&empty[s], ((t / kFwdS) - 1) & 1);
          if (!ok) break;
          unsigned char* st = stage(s);
          const int p0 = pb + sl * kTcK;
          const int nv = min(kTcK, N - p0);                      // pixels present in this slab
          const unsigned vbytes = (unsigned)nv * kTcN * 4;
          mbar_expect_tx(&full[s], kFwdRaw + 4 * vbytes);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  su32(st)),
              "l"(reinterpret_cast<uint64_t>(&tmaps.m[q])), "r"(mt * kTcM), "r"(p0), "r"(su32(&full[s]))
              : "memory");
          const float* src[4] = {vs.X + ((size_t)q * N + p0) * kTcN, vs.xbar + (size_t)p0 * kTcN,
                                 vs.zbar + (size_t)p0 * kTcN, vs.sd + (size_t)p0 * kTcN};
#pragma unroll
          for (int a = 0; a < 4; ++a)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             su32(st + oV + a * kVBytes)),
                         "l"(src[a]), "r"(vbytes), "r"(su32(&full[s]))
                         : "memory");
        }
      }
      if (!ok)
        for (int u = max(0, t - kFwdS); u < t; ++u) bar_wait(&full[u % kFwdS], (u / kFwdS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int t = 0, i = 0;
      for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int q, mt, sp, pb, ns;
        item_of(it, q, mt, sp, pb, ns);
        if (ns == 0) continue;
        const int ab = i & 1;
        if (i >= 2) ok = bar_wait(&accempty[ab], ((i / 2) - 1) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned d = tmem + ab * kAccSet;    // three independent accumulation chains
        for (int sl = 0; sl < ns && ok; ++sl, ++t) {
          const int s = t % kFwdS;
          ok = bar_wait(&conv[s], (t / kFwdS) & 1);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned st = su32(stage(s));
          const unsigned a_hi = st + oAhi, a_lo = st + oAlo, b = st + oB;
#pragma unroll
          for (int ks = 0; ks < kTcK / 8; ++ks) {
            const unsigned acc0 = (sl > 0 || ks > 0) ? 1u : 0u;
            mma_3xtf32(d, sw128_desc(a_hi + ks * 32), sw128_desc(a_lo + ks * 32),
                       smem_desc(b + ks * 2 * kB_LBO, kB_LBO, kB_SBO), acc0);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accfull[ab]);
        ++i;
      }
    }
  } else {
    const int ct = tid - 64;                        // 0..127: row m of the tile
    const int quarter = warp & 3;
    int t = 0, i = 0;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int q, mt, sp, pb, ns;
      item_of(it, q, mt, sp, pb, ns);
      if (ns == 0) {
        const int r = mt * kTcM + quarter * 32 + lane;
        if (r < R)
          for (int sc = 0; sc < kTcN; ++sc)
            partial[(((size_t)q * splits + sp) * KM + (r >> 1)) * kTcN * 2 + sc * 2 + (r & 1)] = 0.f;
        continue;
      }
      for (int sl = 0; sl < ns && ok; ++sl, ++t) {
        const int s = t % kFwdS;
        ok = bar_wait(&full[s], (t / kFwdS) & 1);
        if (!ok) break;
        unsigned char* st = stage(s);
        const float* raw = reinterpret_cast<const float*>(st);
        const int nv = min(kTcK, N - (pb + sl * kTcK));
        // A: row m = ct, pixel quads kq: transpose + TF32 split into SW128 K-major
        const int m = ct;
#pragma unroll
        for (int kq = 0; kq < kTcK / 4; ++kq) {
          float x[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = raw[(4 * kq + j) * kTcM + m];   // zero-filled beyond N by TMA
          // hi = x itself (the MMA truncates it to TF32), lo = the exact remainder
          const float4 h = make_float4(x[0], x[1], x[2], x[3]);
          const float4 l = make_float4(x[0] - tf32_tz(x[0]), x[1] - tf32_tz(x[1]), x[2] - tf32_tz(x[2]),
                                       x[3] - tf32_tz(x[3]));
          const int off = (m >> 3) * 1024 + (m & 7) * 128 + ((kq ^ (m & 7)) << 4);
          *reinterpret_cast<float4*>(st + oAhi + off) = h;
          *reinterpret_cast<float4*>(st + oAlo + off) = l;
        }
        // B: V[k][n] for scene n = ct % 16 and pixels k = 4j .. 4j + 3, j = ct / 16:
        // one 16-byte chunk of the hi rows and one of the lo rows per thread
        // (a quarter-warp covers eight scenes: no bank conflict)
        {
          const int n = ct & 15, j = ct >> 4;
          const float* xv = reinterpret_cast<const float*>(st + oV);
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = 4 * j + u;
            const int e = k * kTcN + n;
            v[u] = k < nv ? xv[e] - xv[e + kVBytes / 4] + xv[e + 2 * kVBytes / 4] - xv[e + 3 * kVBytes / 4] : 0.f;
          }
          float* bt = reinterpret_cast<float*>(st + oB);
          const float4 h = make_float4(tf32_rn(v[0]), tf32_rn(v[1]), tf32_rn(v[2]), tf32_rn(v[3]));
          *reinterpret_cast<float4*>(bt + b_off(n, 4 * j) / 4) = h;
          *reinterpret_cast<float4*>(bt + b_off(kTcN + n, 4 * j) / 4) =
              make_float4(v[0] - h.x, v[1] - h.y, v[2] - h.z, v[3] - h.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (!ok) break;
      const int ii = i++;
      const int ab = ii & 1;
      ok = bar_wait(&accfull[ab], (ii / 2) & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[16];
      tmem_sum3(tmem + ((unsigned)(quarter * 32) << 16) + ab * kAccSet, v);
      const int r = mt * kTcM + quarter * 32 + lane;           // real row
      if (r < R) {
        float* out = partial + (((size_t)q * splits + sp) * KM + (r >> 1)) * kTcN * 2 + (r & 1);
#pragma unroll
        for (int sc = 0; sc < kTcN; ++sc) out[sc * 2] = v[sc];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&accempty[ab]);
    }
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

// The tensor-map encoder comes from the driver through the runtime, so the
// library needs no link-time dependency on libcuda.
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int tc_adjoint_max_splits(int KM) { return std::max(1, (2 * KM) / (4 * kTcK)); }

int tc_forward_max_splits(int N) { return std::max(1, div_up(N, 4 * kTcK)); }

int tc_adjoint_splits(int Q, int N, int KM) {
  const int tiles = div_up(N, kTcM) * Q;
  const int want = div_up(152 * 4, tiles);                  // about four items per persistent CTA
  return std::max(1, std::min(want, tc_adjoint_max_splits(KM)));
}

int launch_tc_adjoint(const float2* const* Aq, const float2* const* Wq, float* gpart, int Q, int N, int KM, int splits,
                      int* err, cudaStream_t st) {
  if (Q < 1 || Q > kMaxSets || N < 1 || (2 * KM) % kTcK != 0 || splits < 1) {
    set_error("launch_tc_adjoint: bad sizes");
    return SADMM_EINVAL;
  }
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) { set_error("launch_tc_adjoint: cuTensorMapEncodeTiled unavailable"); return SADMM_ECUDA; }
  TmapSet tm;
  PtrSet ws;
  memset(&tm, 0, sizeof tm);
  memset(&ws, 0, sizeof ws);
  for (int q = 0; q < Q; ++q) {
    const cuuint64_t dims[2] = {(cuuint64_t)2 * KM, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * KM * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&tm.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(Aq[q]), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("launch_tc_adjoint: tensor map of sensor %d rejected (%d)", q, (int)r); return SADMM_ECUDA; }
    ws.w[q] = reinterpret_cast<const float*>(Wq[q]);
  }
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(tc_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem));
    conf = true;
  }
  const int items = Q * div_up(N, kTcM) * splits;
  tc_adjoint_kernel<<<std::min(items, 152), kPipeThreads, kPipeSmem, st>>>(tm, ws, gpart, Q, N, KM, splits, err);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int tc_forward_splits(int Q, int N, int KM) {
  const int tiles = div_up(2 * KM, kTcM) * Q;
  const int want = div_up(152 * 4, tiles);
  return std::max(1, std::min(want, tc_forward_max_splits(N)));
}

int launch_tc_forward(const float2* const* Aq, const float* X, const float* xbar, const float* zbar, const float* sd,
                      float2* partial, int Q, int N, int KM, int splits, int* err, cudaStream_t st) {
  if (Q < 1 || Q > kMaxSets || N < 1 || (2 * KM) % 16 != 0 || splits < 1) {
    set_error("launch_tc_forward: bad sizes");
    return SADMM_EINVAL;
  }
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) { set_error("launch_tc_forward: cuTensorMapEncodeTiled unavailable"); return SADMM_ECUDA; }
  TmapSet tm;
  memset(&tm, 0, sizeof tm);
  for (int q = 0; q < Q; ++q) {
    const cuuint64_t dims[2] = {(cuuint64_t)2 * KM, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * KM * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcM, (cuuint32_t)kTcK};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&tm.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(Aq[q]), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("launch_tc_forward: tensor map of sensor %d rejected (%d)", q, (int)r); return SADMM_ECUDA; }
  }
  const VSet vs{X, xbar, zbar, sd};
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(tc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem));
    conf = true;
  }
  const int items = Q * div_up(2 * KM, kTcM) * splits;
  tc_forward_kernel<<<std::min(items, 152), kPipeThreads, kFwdSmem, st>>>(tm, vs, reinterpret_cast<float*>(partial), Q,
                                                                          N, KM, splits, err);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm

extern "C" int sadmm_adjoint16_tc(const float* A, int KM, int N, const float* W, float* G, void* stream) {
  using namespace sadmm;
  if (!A || !W || !G || KM <= 0 || (2 * KM) % kTcK != 0 || N <= 0) {
    set_error("sadmm_adjoint16_tc: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* err = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&err, sizeof(int), st));
  int rc = cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess ? SADMM_OK : SADMM_ECUDA;
  const float2* a = reinterpret_cast<const float2*>(A);
  const float2* w = reinterpret_cast<const float2*>(W);
  if (rc == SADMM_OK) rc = launch_tc_adjoint(&a, &w, G, 1, N, KM, 1, (int*)err, st);
  int herr = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(err, st);
  if (rc != SADMM_OK) return rc;
  if (herr) { set_error("sadmm_adjoint16_tc: a tensor-core pipeline wait timed out"); return SADMM_ETIMEOUT; }
  return SADMM_OK;
}

extern "C" int sadmm_forward16_tc(const float* A, int KM, int N, const float* V, float* R, void* stream) {
  using namespace sadmm;
  if (!A || !V || !R || KM <= 0 || (2 * KM) % 16 != 0 || N <= 0) {
    set_error("sadmm_forward16_tc: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // V = x - x_bar + z_bar - s with x = V and the other three zero
  const size_t vbytes = (size_t)N * kTcN * sizeof(float);
  char* buf = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync((void**)&buf, vbytes + 16, st));
  int* err = reinterpret_cast<int*>(buf + vbytes);
  const float* zero = reinterpret_cast<const float*>(buf);
  int rc = (cudaMemsetAsync(buf, 0, vbytes + 16, st) == cudaSuccess) ? SADMM_OK : SADMM_ECUDA;
  const float2* a = reinterpret_cast<const float2*>(A);
  if (rc == SADMM_OK)
    rc = launch_tc_forward(&a, V, zero, zero, zero, reinterpret_cast<float2*>(R), 1, N, KM, 1, err, st);
  int herr = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(buf, st);
  if (rc != SADMM_OK) return rc;
  if (herr) { set_error("sadmm_forward16_tc: a tensor-core pipeline wait timed out"); return SADMM_ETIMEOUT; }
  return SADMM_OK;
}
