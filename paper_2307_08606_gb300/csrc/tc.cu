// Tensor-core (tcgen05) adjoint GEMM of the batched form (Eq. 3, x_q-update
// for 16 scenes at once):
//   G[p][s] = Re(a_p^H w_s) = sum_r B[r][p] W[r][s],   r over the 2KM real rows,
// with B the real form of A_q (pixel-major: the 2KM floats of pixel p are
// contiguous, so B^T is K-major) and W the 16 right-hand sides (complex
// [row][scene], real row r = 2m + c at float (m * 16 + s) * 2 + c).
//
// Precision: three TF32 products per term (3xTF32).  Each operand is split
// x = hi + lo with hi = tf32(x) (round to nearest) and lo = x - hi (exact in
// FP32; the MMA keeps its top 11 bits), and hi*hi + hi*lo + lo*hi is
// accumulated in FP32 in tensor memory: each product is within 2^-21 of the
// FP32 one, the dropped lo*lo term is below 2^-22, and the sum over K rounds
// as an FP32 accumulation does.
//
// Tile: M = 128 pixels per CTA (TMEM lanes), N = 16 scenes (TMEM columns), K
// slabs of 32 real rows.  Per slab every thread converts one pixel's 32 floats
// (and 4 values of W) into hi and lo operand tiles in shared memory, in the
// canonical K-major no-swizzle layout (core matrices of 8 rows x 16 bytes;
// K-adjacent cores LBO bytes apart, M/N-adjacent cores SBO bytes apart); one
// thread then issues 4 k-steps x 3 products of tcgen05.mma kind::tf32
// (M128 N16 K8) and commits them to an mbarrier.  Two operand buffers let the
// conversion of slab i+1 overlap the MMAs of slab i.  The accumulator is read
// back with tcgen05.ld (32 lanes x 16 columns per warp).  Every wait is
// bounded; on a timeout the CTA flags *err, waits (bounded) for its
// outstanding MMAs, frees its tensor memory and exits.
#include "common.cuh"

namespace sadmm {
namespace {

constexpr int kTcM = 128;              // pixels per CTA
constexpr int kTcN = 16;               // scenes
constexpr int kTcK = 32;               // real rows per slab
constexpr int kTcThreads = 128;
constexpr int kTmemCols = 32;          // power of two >= 32, >= kTcN
constexpr long long kTcWaitLimit = 1ll << 26;

// operand tile bytes per plane and buffer
constexpr int kABytes = kTcM * kTcK * 4;          // 16 KB
constexpr int kBBytes = kTcN * kTcK * 4;          // 2 KB
// canonical K-major layout strides (bytes)
constexpr int kCore = 128;                         // 8 rows x 16 bytes
constexpr int kA_SBO = kCore;                      // next 8 pixels
constexpr int kA_LBO = (kTcM / 8) * kCore;         // next 4 k-elements (2048)
constexpr int kB_SBO = kCore;                      // next 8 scenes
constexpr int kB_LBO = (kTcN / 8) * kCore;         // next 4 k-elements (256)
constexpr int kBufBytes = 2 * kABytes + 2 * kBBytes;   // A hi, A lo, B hi, B lo
constexpr int kTcSmem = 2 * kBufBytes;

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, int lbo, int sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
  return d;                            // base offset 0, no swizzle
}

// kind::tf32, D = F32, A = B = TF32, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
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

__device__ __forceinline__ float tf32_rn(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(kTcThreads)
tc_adjoint_kernel(const float2* const* __restrict__ Aq, const float2* const* __restrict__ Wq, float* __restrict__ gpart,
                  int N, int KM, int splits, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int q = blockIdx.y, split = blockIdx.z;
  const int p0 = blockIdx.x * kTcM;
  const int R = 2 * KM;                                    // real rows
  const int rows_per = (R / splits + kTcK - 1) / kTcK * kTcK;
  const int rb = split * rows_per, re = min(R, rb + rows_per);
  const int nslab = max(0, (re - rb) / kTcK);
  const float* A = reinterpret_cast<const float*>(Aq[q]);
  const float* W = reinterpret_cast<const float*>(Wq[q]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s_tmem;

  // this thread's pixel and its W quad (complex row m_l, scenes 2 (tid % 8), +1)
  const int p = p0 + tid;
  const bool pv = p < N;
  const float4* arow = reinterpret_cast<const float4*>(A + (size_t)(pv ? p : 0) * R);
  const int wm = tid >> 3, ws = 2 * (tid & 7);
  // two register sets: the loads of slab i + 2 are in flight while slabs i
  // and i + 1 are converted and multiplied
  float4 raA[kTcK / 4], raB[kTcK / 4];
  float4 rwA, rwB;
  auto load = [&](int slab, float4 (&ra)[kTcK / 4], float4& rw) {
    const int r0 = rb + slab * kTcK;
#pragma unroll
    for (int e = 0; e < kTcK / 4; ++e) ra[e] = pv ? __ldcs(arow + r0 / 4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    rw = reinterpret_cast<const float4*>(W + ((size_t)(r0 / 2 + wm) * kTcN + ws) * 2)[0];
  };
  unsigned phase = 0u;          // bit b: parity to wait for on buffer b
  unsigned pending = 0u;        // bit b: a commit on buffer b is outstanding
  bool ok = true;
  // convert slab `slab` from registers into operand buffer slab & 1, refill
  // the registers with slab + 2, and issue the slab's MMAs
  auto step = [&](int slab, float4 (&ra)[kTcK / 4], float4& rw) -> bool {
    const int b = slab & 1;
    unsigned char* base = smem + b * kBufBytes;
    float* Ahi = reinterpret_cast<float*>(base);
    float* Alo = reinterpret_cast<float*>(base + kABytes);
    float* Bhi = reinterpret_cast<float*>(base + 2 * kABytes);
    float* Blo = reinterpret_cast<float*>(base + 2 * kABytes + kBBytes);
    // the MMAs that last read this buffer (slab - 2) must be done
    if ((pending >> b) & 1u) {
      ok = bar_wait(&bar[b], (phase >> b) & 1u);
      phase ^= 1u << b;
      pending &= ~(1u << b);
      if (!__syncthreads_and(ok)) return false;
    }
    // A: element (m = tid, k = 4e + j) -> core (tid / 8, e), row tid % 8
#pragma unroll
    for (int e = 0; e < kTcK / 4; ++e) {
      const float4 x = ra[e];
      const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
      const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      const int off = (e * kA_LBO + tid * 16) / 4;
      reinterpret_cast<float4*>(Ahi + off)[0] = h;
      reinterpret_cast<float4*>(Alo + off)[0] = l;
    }
    // B: W real rows 2 wm (re), 2 wm + 1 (im) for scenes ws, ws + 1
    {
      const float v[4] = {rw.x, rw.y, rw.z, rw.w};       // (ws re, ws im, ws+1 re, ws+1 im)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int s = ws + (u >> 1), k = 2 * wm + (u & 1);
        const int off = ((k >> 2) * kB_LBO + (s >> 3) * kB_SBO + (s & 7) * 16 + (k & 3) * 4) / 4;
        const float h = tf32_rn(v[u]);
        Bhi[off] = h;
        Blo[off] = v[u] - h;
      }
    }
    if (slab + 2 < nslab) load(slab + 2, ra, rw);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a_hi = su32(Ahi), a_lo = su32(Alo), b_hi = su32(Bhi), b_lo = su32(Blo);
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const int ao = ks * 2 * kA_LBO, bo = ks * 2 * kB_LBO;
        const unsigned acc0 = (slab > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, smem_desc(a_hi + ao, kA_LBO, kA_SBO), smem_desc(b_hi + bo, kB_LBO, kB_SBO), acc0);
        mma_tf32(tmem, smem_desc(a_hi + ao, kA_LBO, kA_SBO), smem_desc(b_lo + bo, kB_LBO, kB_SBO), 1u);
        mma_tf32(tmem, smem_desc(a_lo + ao, kA_LBO, kA_SBO), smem_desc(b_hi + bo, kB_LBO, kB_SBO), 1u);
      }
      mma_commit(&bar[b]);
    }
    pending |= 1u << b;
    return true;
  };
  if (nslab > 0) load(0, raA, rwA);
  if (nslab > 1) load(1, raB, rwB);
  for (int slab = 0; slab < nslab; slab += 2) {
    if (!step(slab, raA, rwA)) break;
    if (slab + 1 < nslab && !step(slab + 1, raB, rwB)) break;
  }
  // drain: wait for every outstanding commit (bounded)
  for (int b = 0; b < 2; ++b) {
    if ((pending >> b) & 1u) {
      const bool w = bar_wait(&bar[b], (phase >> b) & 1u);
      ok = ok && w;
      phase ^= 1u << b;
    }
  }
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nslab > 0) {
    unsigned r[16];
    const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (pv) {
      float4* out = reinterpret_cast<float4*>(gpart + (((size_t)q * splits + split) * N + p) * kTcN);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        out[e] = make_float4(__uint_as_float(r[4 * e]), __uint_as_float(r[4 * e + 1]), __uint_as_float(r[4 * e + 2]),
                             __uint_as_float(r[4 * e + 3]));
    }
  } else if (!ok && tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

int tc_adjoint_splits(int Q, int N, int KM) {
  const int ctas = div_up(N, kTcM) * Q;
  const int want = div_up(152 * 3 * 4, ctas);          // about four waves of resident CTAs
  return std::max(1, std::min(want, (2 * KM) / (4 * kTcK)));
}

int launch_tc_adjoint(const float2* const* Aq, const float2* const* Wq, float* gpart, int Q, int N, int KM, int splits,
                      int* err, cudaStream_t st) {
  if ((2 * KM) % kTcK != 0 || splits < 1) { set_error("launch_tc_adjoint: bad sizes"); return SADMM_EINVAL; }
  static bool conf = false;
  if (!conf) {
    SADMM_CUDA_TRY(cudaFuncSetAttribute(tc_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    conf = true;
  }
  tc_adjoint_kernel<<<dim3(div_up(N, kTcM), Q, splits), kTcThreads, kTcSmem, st>>>(Aq, Wq, gpart, N, KM, splits, err);
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
  void *ptrs = nullptr, *err = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&ptrs, 2 * sizeof(void*), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&err, sizeof(int), st));
  const void* hp[2] = {A, W};
  int rc = cudaMemcpyAsync(ptrs, hp, sizeof hp, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                   cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess
               ? SADMM_OK
               : SADMM_ECUDA;
  if (rc == SADMM_OK)
    rc = launch_tc_adjoint((const float2* const*)ptrs, (const float2* const*)ptrs + 1, G, 1, N, KM, 1, (int*)err, st);
  int herr = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(ptrs, st);
  cudaFreeAsync(err, st);
  if (rc != SADMM_OK) return rc;
  if (herr) { set_error("sadmm_adjoint16_tc: a tensor-core wait timed out"); return SADMM_ETIMEOUT; }
  return SADMM_OK;
}
