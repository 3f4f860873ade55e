// Device helpers shared by the symmetric factor applies (spd.cu, batch.cu) and
// the adjoint (gemv.cu): double-float accumulation with exact products, bulk
// asynchronous copies
// completing on an mbarrier (with bounded waits), and the packed
// upper-triangular tile numbering.
#pragma once
#include "common.cuh"

namespace sadmm {
namespace symtile {

constexpr int kT = kSymTile;
constexpr long long kWaitLimit = 1ll << 26;   // mbarrier polls before giving up

struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_acc(DF& s, float w_hi, float w_lo, float u) {
  const float p = w_hi * u;
  float e = fmaf(w_hi, u, -p);          // w_hi u = p + e exactly
  e = fmaf(w_lo, u, e);
  const float t = s.hi + p;             // two-sum s.hi + p = t + err
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

// s += (w_hi + w_lo)(u + u_lo) to double-float accuracy (the products of the
// two low words are below the error)
__device__ __forceinline__ void df_acc2(DF& s, float w_hi, float w_lo, float u, float u_lo) {
  const float p = w_hi * u;
  float e = fmaf(w_hi, u, -p);
  e = fmaf(w_lo, u, e);
  e = fmaf(w_hi, u_lo, e);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

// s += a b with the product formed exactly (p + e = a b)
__device__ __forceinline__ void df_mul_acc(DF& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

__device__ __forceinline__ void df_add(DF& s, DF b) {
  const float t = s.hi + b.hi;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (b.hi - bp);
  s.hi = t;
  s.lo += err + b.lo;
}

// s += x (a single FP32 term), error-free up to the low word's own rounding
__device__ __forceinline__ void df_add1(DF& s, float x) {
  const float t = s.hi + x;
  const float bp = t - s.hi;
  s.lo += (s.hi - (t - bp)) + (x - bp);
  s.hi = t;
}

__device__ __forceinline__ DF df_norm(DF s) {
  const float t = s.hi + s.lo;
  return DF{t, s.lo - (t - s.hi)};
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Waits for phase `parity` of the barrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__host__ __device__ __forceinline__ int ntiles_side(int n) { return (n + kT - 1) / kT; }

__host__ __device__ __forceinline__ int tile_index(int I, int J, int nt) { return I * nt - I * (I - 1) / 2 + (J - I); }

// tile number t of an nt x nt upper triangle -> (I, J).  Row block I starts
// at tile I nt - I (I - 1) / 2; I is the largest with that start <= t, the
// smaller root of I^2 - (2 nt + 1) I + 2 t = 0 rounded down (an FP32 estimate,
// then corrected exactly in integers).
__device__ __forceinline__ int tile_row_start(int I, int nt) { return I * nt - I * (I - 1) / 2; }

__device__ __forceinline__ void tile_ij(int t, int nt, int& I, int& J) {
  const float b = 2.f * (float)nt + 1.f;
  int i = (int)((b - sqrtf(fmaxf(b * b - 8.f * (float)t, 0.f))) * 0.5f);
  i = max(0, min(i, nt - 1));
  while (i > 0 && tile_row_start(i, nt) > t) --i;
  while (i + 1 < nt && tile_row_start(i + 1, nt) <= t) ++i;
  I = i;
  J = i + (t - tile_row_start(i, nt));
}


}  // namespace symtile
}  // namespace sadmm
