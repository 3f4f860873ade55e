// Learned elimination support for the solver (an extension of Algorithm 1;
// the paper has no counterpart): the per-pixel features the proposal network
// reads, and the re-admission test that returns frozen pixels whose
// optimality residual has grown.
//
// Features of pixel i after k completed iterations (six channels, NCHW with
// one image of the square pixel grid):
//   c0 = log(1 + sum_q |x_q,i|),  c1 = log(1 + max_q |x_q,i|),
//   c2+j = log10(||dx_{.,i}^{(k-j)}||_2 / eps_p + 1e-4) / 4,  j = 0..3,
// where dx^{(t)} is the update of iteration t over the sensors (from the ring
// of the last Kp updates; frozen pixels contribute zero updates).
//
// Re-admission: a frozen pixel i of sensor q re-enters when the correction a
// single-coordinate x-update would make exceeds thr:
//   |c| / (mu ||a_i||^2 + rho) > thr,  c = mu Re(a_i^H (A_q x_q - y_q)) + rho s_i,
// c being the pixel's entry of the optimality condition of Eq. 2.
#include "common.cuh"

namespace sadmm {
namespace {

__global__ void features_kernel(const __grid_constant__ SolverView sv, int k_done, float inv_eps_p,
                                float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sv.N) return;
  const size_t N = sv.N;
  float sum = 0.f, mx = 0.f;
  for (int q = 0; q < sv.Q; ++q) {
    const float a = fabsf(sv.x[q * N + i]);
    sum += a;
    mx = fmaxf(mx, a);
  }
  out[i] = log1pf(sum);
  out[N + i] = log1pf(mx);
  for (int j = 0; j < 4; ++j) {
    float u = 0.f;
    if (j < sv.Kp && k_done - j >= 1) {
      const int slot = ((k_done - 1 - j) % sv.Kp + sv.Kp) % sv.Kp;
      const float* ring = sv.ring + (size_t)slot * sv.Q * N;
      for (int q = 0; q < sv.Q; ++q) {
        const float d = ring[q * N + i];
        u = fmaf(d, d, u);
      }
      u = sqrtf(u);
    }
    out[(2 + j) * N + i] = 0.25f * log10f(u * inv_eps_p + 1e-4f);
  }
}

struct ListSet {
  int* J;
  int* F;
};

// Per sensor CTA: mask[q][i] = 1 for i in J_q, then F_q = sorted complement.
__global__ void __launch_bounds__(1024)
frozen_lists_kernel(const __grid_constant__ SetBlock<ListSet> sets, int N, const int* __restrict__ counts,
                    uint8_t* __restrict__ mask, int* __restrict__ fcounts) {
  const int q = blockIdx.x;
  uint8_t* m = mask + (size_t)q * 2 * N;          // [0, N): active, [N, 2N): re-admit flags
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) m[i] = 0;
  __syncthreads();
  const int n = counts[q];
  for (int p = threadIdx.x; p < n; p += blockDim.x) m[sets.v[q].J[p]] = 1;
  __syncthreads();
  __shared__ int s_w[32];
  __shared__ int s_base, s_tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  for (int b0 = 0; b0 < N; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const bool fr = i < N && !m[i];
    const unsigned bal = __ballot_sync(0xffffffffu, fr);
    __syncthreads();
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
      const int v = lane < nw ? s_w[lane] : 0;
      int inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane < nw) s_w[lane] = inc - v;
      if (lane == 31) s_tot = inc;
    }
    __syncthreads();
    if (fr) sets.v[q].F[s_base + s_w[warp] + __popc(bal & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0) s_base += s_tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) fcounts[q] = s_base;
}

constexpr int kRaWarps = 8;

// One warp per frozen column: g = Re(a^H r), ||a||^2; flag re-admission.
__global__ void __launch_bounds__(kRaWarps * 32)
readmit_check_kernel(const __grid_constant__ SetBlock<ReadmitSet> sets, int KM, const __grid_constant__ SolverView sv,
                     float thr, uint8_t* __restrict__ mask) {
  const ReadmitSet& rs = sets.v[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kRaWarps + warp;
  if (p >= rs.n) return;
  const int pix = rs.F[p];
  const float4* col = reinterpret_cast<const float4*>(rs.A + (size_t)pix * KM);
  const float4* r4 = reinterpret_cast<const float4*>(rs.r);
  float g = 0.f, nrm = 0.f;
  for (int i = lane; i < KM / 2; i += 32) {
    const float4 a = col[i], r = r4[i];
    g = fmaf(a.x, r.x, fmaf(a.y, r.y, fmaf(a.z, r.z, fmaf(a.w, r.w, g))));
    nrm = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, nrm))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g += __shfl_xor_sync(0xffffffffu, g, o);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  }
  if (lane != 0) return;
  // A x - y = -(y' - A_J x_J) = -r, so the optimality entry is -mu g + rho s
  const float c = -sv.mu * g + sv.rho * sv.s[pix];
  const float move = fabsf(c) / (sv.mu * nrm + sv.rho);
  if (move > thr) mask[(size_t)rs.q * 2 * sv.N + sv.N + pix] = 1;
}

struct RebuildSet {
  int* J;
  int* R;
};

// Per sensor CTA, after the SSC pass: the active flags are re-marked from the
// current J_q, then J_q = sorted {i : active or re-admitted} and R_q = sorted
// re-admitted pixels, whose ring entries are set to `fill` so that the window
// of Algorithm 1 does not drop them at once.
__global__ void __launch_bounds__(1024)
rebuild_lists_kernel(const __grid_constant__ SetBlock<RebuildSet> sets, const __grid_constant__ SolverView sv,
                     uint8_t* __restrict__ mask, int* __restrict__ counts, int* __restrict__ rcounts,
                     float fill, uint8_t* __restrict__ tag, int* __restrict__ tally) {
  const int q = blockIdx.x;
  const int N = sv.N;
  uint8_t* act = mask + (size_t)q * 2 * N;
  const uint8_t* re = act + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) act[i] = 0;
  __syncthreads();
  const int n = counts[q];
  for (int p = threadIdx.x; p < n; p += blockDim.x) act[sets.v[q].J[p]] = 1;
  __syncthreads();
  __shared__ int s_a[32], s_r[32];
  __shared__ int s_ba, s_br, s_ta, s_tr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) { s_ba = 0; s_br = 0; }
  for (int b0 = 0; b0 < N; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const bool r = i < N && re[i];
    const bool a = i < N && (act[i] || r);
    const unsigned ba = __ballot_sync(0xffffffffu, a), br = __ballot_sync(0xffffffffu, r);
    __syncthreads();
    if (lane == 0) { s_a[warp] = __popc(ba); s_r[warp] = __popc(br); }
    __syncthreads();
    if (warp == 0) {
      const int va = lane < nw ? s_a[lane] : 0, vr = lane < nw ? s_r[lane] : 0;
      int ia = va, ir = vr;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int ta = __shfl_up_sync(0xffffffffu, ia, o), tr = __shfl_up_sync(0xffffffffu, ir, o);
        if (lane >= o) { ia += ta; ir += tr; }
      }
      if (lane < nw) { s_a[lane] = ia - va; s_r[lane] = ir - vr; }
      if (lane == 31) { s_ta = ia; s_tr = ir; }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    if (a) sets.v[q].J[s_ba + s_a[warp] + __popc(ba & lt)] = i;
    if (r) {
      sets.v[q].R[s_br + s_r[warp] + __popc(br & lt)] = i;
      for (int t = 0; t < sv.Kp; ++t) sv.ring[((size_t)t * sv.Q + q) * N + i] = fill;
      if (tag && tag[(size_t)q * N + i]) {       // a proposal's removal undone: a false elimination
        tag[(size_t)q * N + i] = 0;
        atomicAdd(tally + sv.Q + q, 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_ba += s_ta; s_br += s_tr; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    counts[q] = s_ba;
    rcounts[q] = s_br;
  }
}

}  // namespace

int launch_features(const SolverView& sv, int k_done, double eps_p, float* out, cudaStream_t st) {
  features_kernel<<<div_up(sv.N, 256), 256, 0, st>>>(sv, k_done, (float)(1.0 / eps_p), out);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_frozen_lists(const SolverView& sv, int* const* J, const int* counts, uint8_t* mask, int* const* F,
                        int* fcounts, cudaStream_t st) {
  SetBlock<ListSet> blk;
  for (int q = 0; q < sv.Q; ++q) blk.v[q] = ListSet{J[q], F[q]};
  frozen_lists_kernel<<<sv.Q, 1024, 0, st>>>(blk, sv.N, counts, mask, fcounts);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_readmit_check(const ReadmitSet* sets, int nsets, int KM, const SolverView& sv, double thr,
                         uint8_t* mask, cudaStream_t st) {
  if (nsets <= 0) return SADMM_OK;
  SetBlock<ReadmitSet> blk;
  int mx = 0;
  for (int i = 0; i < nsets; ++i) { blk.v[i] = sets[i]; mx = max(mx, sets[i].n); }
  if (mx == 0) return SADMM_OK;
  readmit_check_kernel<<<dim3(div_up(mx, kRaWarps), nsets), kRaWarps * 32, 0, st>>>(blk, KM, sv, (float)thr, mask);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_rebuild_lists(const SolverView& sv, int* const* J, int* const* R, uint8_t* mask, int* counts,
                         int* rcounts, double ring_fill, cudaStream_t st, uint8_t* tag, int* tally) {
  SetBlock<RebuildSet> blk;
  for (int q = 0; q < sv.Q; ++q) blk.v[q] = RebuildSet{J[q], R[q]};
  rebuild_lists_kernel<<<sv.Q, 1024, 0, st>>>(blk, sv, mask, counts, rcounts, (float)ring_fill,
                                             tally ? tag : nullptr, tally);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
