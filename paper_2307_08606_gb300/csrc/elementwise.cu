// Fused prox + dual + residual reductions (Eq. 3, x_G- and dual updates, and the primal /
// dual residuals that gate Algorithm 1) and the SSC stream compaction
// (Algorithm 1) of the sharing-ADMM iteration.
#include "common.cuh"

#include <algorithm>

namespace sadmm {

namespace {

constexpr int kResThreads = 128;
constexpr int kNumSums = 8;
constexpr int kSscThreads = 1024;

// Deterministic block reduction of kNumSums doubles (fixed shuffle tree, then
// warp totals summed in warp order by warp 0).
__device__ __forceinline__ void block_reduce(double (&v)[kNumSums], double (*s_red)[kNumSums]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) s_red[warp][j] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) {
      double t = lane < nw ? s_red[lane][j] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[j] = t;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float soft_threshold(float t, float thr) {
  return copysignf(fmaxf(fabsf(t) - thr, 0.f), t);
}

// One thread per pixel i:
//   x_bar' = mean_q x_q[i];  z_bar' = soft(x_bar' + s, lambda/rho);  s' = s + x_bar' - z_bar'
// and FP64 partial sums of the residual norms.  The last CTA to finish (ticket)
// reduces the per-CTA partials in CTA order and writes the scalars.
__global__ void __launch_bounds__(kResThreads)
residual_kernel(const __grid_constant__ SolverView sv, double* __restrict__ partials,
                unsigned int* ticket, IterScalars* __restrict__ out, int k_after, double eps_abs,
                double eps_rel, int elim, int Kp, int ssc_every) {
  __shared__ double s_red[kResThreads / 32][kNumSums];
  __shared__ bool s_last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) acc[j] = 0.0;
  if (i < sv.N && sv.u) {
    // consensus form: z' = soft(x_bar + u_bar, lambda / (Q rho)) (lam_over_rho
    // holds lambda / (Q rho)), u_q' = u_q + x_q - z'; sums for
    // r_pri = ||X - z'||, ||X||, sqrt(Q) ||z'||, the dual residual
    // rho sqrt(Q) ||z' - z||, ||U'||, ||dX||, ||z'||, ||z' - z||
    const size_t N = sv.N;
    float sx = 0.f, su = 0.f;
    for (int q = 0; q < sv.Q; ++q) {
      sx += sv.x[q * N + i];
      su += sv.u[q * N + i];
    }
    const float xb = sx / (float)sv.Q, ub = su / (float)sv.Q;
    const float z_old = sv.zbar[i];
    const float z = soft_threshold(xb + ub, sv.lam_over_rho);
    const float dz = z - z_old;
    const float* ring = sv.ring + (size_t)sv.slot * sv.Q * N;
    float a0 = 0.f, a1 = 0.f, a4 = 0.f, a5 = 0.f;
    for (int q = 0; q < sv.Q; ++q) {
      const float xq = sv.x[q * N + i], dx = ring[q * N + i];
      const float e = xq - z;
      const float un = sv.u[q * N + i] + e;
      sv.u[q * N + i] = un;
      a0 = fmaf(e, e, a0);
      a1 = fmaf(xq, xq, a1);
      a4 = fmaf(un, un, a4);
      a5 = fmaf(dx, dx, a5);
    }
    acc[0] = a0;
    acc[1] = a1;
    acc[2] = (double)sv.Q * z * z;
    acc[3] = (double)sv.Q * dz * dz;
    acc[4] = a4;
    acc[5] = a5;
    acc[6] = (double)z * z;
    acc[7] = (double)dz * dz;
    sv.xbar[i] = xb;
    sv.zbar[i] = z;
  } else if (i < sv.N) {
    // per-pixel terms in FP32 (a handful per thread; GB300's FP64 pipe is
    // narrow), cross-thread sums in FP64
    const size_t N = sv.N;
    constexpr int kQB = 8;               // sensors whose loads are issued together
    float sx = 0.f;
    for (int q0 = 0; q0 < sv.Q; q0 += kQB) {
      float v[kQB];
#pragma unroll
      for (int u = 0; u < kQB; ++u) v[u] = q0 + u < sv.Q ? sv.x[(q0 + u) * N + i] : 0.f;
#pragma unroll
      for (int u = 0; u < kQB; ++u)
        if (q0 + u < sv.Q) sx += v[u];
    }
    const float xb = sx / (float)sv.Q;
    const float xb_old = sv.xbar[i], zb_old = sv.zbar[i], s_old = sv.s[i];
    const float zb = soft_threshold(xb + s_old, sv.lam_over_rho);
    const float sn = (s_old + xb) - zb;
    const float dxb = xb - xb_old;
    const float dzb = zb - zb_old;
    const float e = xb - zb;
    float a1 = 0.f, a2 = 0.f, a3 = 0.f, a5 = 0.f;
    const float* ring = sv.ring + (size_t)sv.slot * sv.Q * N;
    for (int q0 = 0; q0 < sv.Q; q0 += kQB) {
      float xv[kQB], dv[kQB];
#pragma unroll
      for (int u = 0; u < kQB; ++u) {
        const bool ok = q0 + u < sv.Q;
        xv[u] = ok ? sv.x[(q0 + u) * N + i] : 0.f;
        dv[u] = ok ? ring[(q0 + u) * N + i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kQB; ++u) {
        if (q0 + u >= sv.Q) break;
        const float xq = xv[u], dx = dv[u];
        const float zq = (xq - xb) + zb;
        const float dz = (dx - dxb) + dzb;
        a1 = fmaf(xq, xq, a1);
        a2 = fmaf(zq, zq, a2);
        a3 = fmaf(dz, dz, a3);
        a5 = fmaf(dx, dx, a5);
      }
    }
    acc[0] = (double)e * e;
    acc[1] = a1;
    acc[2] = a2;
    acc[3] = a3;
    acc[5] = a5;
    acc[4] = (double)sn * sn;
    acc[6] = (double)zb * zb;
    acc[7] = (double)dzb * dzb;
    sv.xbar[i] = xb;
    sv.zbar[i] = zb;
    sv.s[i] = sn;
  }
  block_reduce(acc, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) partials[blockIdx.x * kNumSums + j] = acc[j];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[kNumSums];
#pragma unroll
  for (int j = 0; j < kNumSums; ++j) tot[j] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) tot[j] += __ldcg(partials + b * kNumSums + j);
  }
  block_reduce(tot, s_red);
  if (threadIdx.x == 0) {
    const double Q = sv.Q, QN = (double)sv.Q * sv.N;
    IterScalars r;
    const bool cons = sv.u != nullptr;
    r.r_pri = (cons ? 1.0 : sqrt(Q)) * sqrt(tot[0]);
    const double xn = sqrt(tot[1]), zn = sqrt(tot[2]);
    r.eps_pri = sqrt(QN) * eps_abs + eps_rel * fmax(xn, zn);
    r.d = (double)sv.rho * sqrt(tot[3]);
    r.eps_dual = sqrt(QN) * eps_abs + eps_rel * (double)sv.rho * (cons ? 1.0 : sqrt(Q)) * sqrt(tot[4]);
    r.relchange = xn > 0.0 ? sqrt(tot[5]) / xn : INFINITY;
    r.xg_norm = (cons ? 1.0 : Q) * sqrt(tot[6]);
    r.dxg_norm = (cons ? 1.0 : Q) * sqrt(tot[7]);
    r.xnorm = xn;
    r.k = k_after;
    r.gate = (elim && k_after >= Kp && k_after % ssc_every == 0 && r.r_pri <= r.eps_pri) ? 1 : 0;
    r.changed = 0;
    double chk = 0.0;
#pragma unroll
    for (int j = 0; j < kNumSums; ++j) chk += tot[j];
    r.nonfinite = isfinite(chk) ? 0 : 1;
    *out = r;
    *ticket = 0u;            // ready for the next launch
  }
}

struct SscSet {
  int* J;
  int* E;
};

// Algorithm 1, one CTA per sensor: zeta_i = (1/Kp) sum of the last Kp |updates|;
// keep i iff zeta_i >= eps_p.  Order-preserving in-place compaction by a
// block-wide ballot scan; removed pixels go to E, their ring entries are
// cleared (so frozen pixels report a zero update) and, in zero mode, x is set
// to 0.
__global__ void __launch_bounds__(kSscThreads)
ssc_kernel(const __grid_constant__ SetBlock<SscSet> sets, const __grid_constant__ SolverView sv,
           int* __restrict__ counts, double eps_p, int freeze_mode, const IterScalars* sc,
           const float* __restrict__ prob, float theta, int learned_now, uint8_t* __restrict__ tag,
           int* __restrict__ tally) {
  const int q = blockIdx.x;
  const int gate = sc->gate;
  if (!gate && !learned_now) {
    if (threadIdx.x == 0) counts[sv.Q + q] = 0;
    return;
  }
  __shared__ int s_wk[32], s_wr[32];
  __shared__ int s_base_k, s_base_r, s_tot_k, s_tot_r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = counts[q];
  int* J = sets.v[q].J;
  int* E = sets.v[q].E;
  const size_t N = sv.N;
  if (threadIdx.x == 0) { s_base_k = 0; s_base_r = 0; }
  for (int b0 = 0; b0 < n; b0 += blockDim.x) {
    const int p = b0 + threadIdx.x;
    const bool valid = p < n;
    int pix = 0;
    bool keep = false;
    if (valid) {
      pix = J[p];
      double z = 0.0;
      for (int t = 0; t < sv.Kp; ++t) z += fabs((double)sv.ring[((size_t)t * sv.Q + q) * N + pix]);
      z /= (double)sv.Kp;
      keep = gate ? (z >= eps_p) : true;
      // learned proposal: drop pixels the network marks as converged
      if (learned_now && prob[pix] > theta && keep) {
        keep = false;
        if (tag) {                     // removed by the proposal alone
          tag[(size_t)q * N + pix] = 1;
          atomicAdd(tally + q, 1);
        }
      }
    }
    const bool rem = valid && !keep;
    const unsigned bk = __ballot_sync(0xffffffffu, keep);
    const unsigned br = __ballot_sync(0xffffffffu, rem);
    const unsigned lt = (1u << lane) - 1u;
    __syncthreads();                 // every read of J in this round is done
    if (lane == 0) { s_wk[warp] = __popc(bk); s_wr[warp] = __popc(br); }
    __syncthreads();
    if (warp == 0) {
      int vk = lane < nw ? s_wk[lane] : 0, vr = lane < nw ? s_wr[lane] : 0;
      int ik = vk, ir = vr;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int tk = __shfl_up_sync(0xffffffffu, ik, o);
        const int tr = __shfl_up_sync(0xffffffffu, ir, o);
        if (lane >= o) { ik += tk; ir += tr; }
      }
      if (lane < nw) { s_wk[lane] = ik - vk; s_wr[lane] = ir - vr; }
      if (lane == 31) { s_tot_k = ik; s_tot_r = ir; }
    }
    __syncthreads();
    if (keep) J[s_base_k + s_wk[warp] + __popc(bk & lt)] = pix;
    if (rem) {
      E[s_base_r + s_wr[warp] + __popc(br & lt)] = pix;
      for (int t = 0; t < sv.Kp; ++t) sv.ring[((size_t)t * sv.Q + q) * N + pix] = 0.f;
      if (freeze_mode == 1) sv.x[(size_t)q * N + pix] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) { s_base_k += s_tot_k; s_base_r += s_tot_r; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    counts[q] = s_base_k;
    counts[sv.Q + q] = s_base_r;
  }
}

__global__ void xbar_kernel(const __grid_constant__ SolverView sv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sv.N) return;
  float sx = 0.f;
  for (int q = 0; q < sv.Q; ++q) sx += sv.x[(size_t)q * sv.N + i];
  sv.xbar[i] = sx / (float)sv.Q;
}

__global__ void scale_kernel(const float* __restrict__ in, float a, float* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * in[i];
}

}  // namespace

int launch_scale(const float* in, float a, float* out, int n, cudaStream_t st) {
  if (n <= 0) return SADMM_OK;
  scale_kernel<<<div_up(n, 256), 256, 0, st>>>(in, a, out, n);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int residual_blocks(int N) { return div_up(N, kResThreads); }

int launch_residuals(const SolverView& sv, const sadmm_criterion& c, double* partials,
                     unsigned int* ticket, IterScalars* out, int k_after, cudaStream_t st) {
  residual_kernel<<<residual_blocks(sv.N), kResThreads, 0, st>>>(
      sv, partials, ticket, out, k_after, c.eps_abs, c.eps_rel, c.elim, c.Kp, c.ssc_every);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_ssc(const SolverView& sv, int* const* J, int* const* E, int* counts, double eps_p,
               int freeze_mode, const IterScalars* sc, const float* prob, float theta, int learned_now,
               cudaStream_t st, uint8_t* tag, int* tally) {
  if (sv.Q > kMaxSets) return SADMM_EINVAL;
  SetBlock<SscSet> blk;
  for (int q = 0; q < sv.Q; ++q) blk.v[q] = SscSet{J[q], E[q]};
  ssc_kernel<<<sv.Q, kSscThreads, 0, st>>>(blk, sv, counts, eps_p, freeze_mode, sc, prob, theta,
                                           learned_now && prob ? 1 : 0, tally ? tag : nullptr, tally);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

// ------------------------------------------------------- back-projection
// out = -i y (KM complex per sensor, in place after the copy of y).
__global__ void bp_rotate_kernel(const float2* __restrict__ y, float2* __restrict__ out, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = y[i];
    out[i] = make_float2(v.y, -v.x);
  }
}

// out[n] = sum_q |g_q,re[n] + i g_q,im[n]|, sensors in order.
__global__ void bp_combine_kernel(const float* __restrict__ g, int Q, int N, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int q = 0; q < Q; ++q) {
    const float re = g[(size_t)q * 2 * N + n], im = g[(size_t)q * 2 * N + N + n];
    acc += sqrtf(fmaf(re, re, im * im));
  }
  out[n] = acc;
}

int launch_bp_rotate(const float2* y, float2* out, size_t n, cudaStream_t st) {
  if (n == 0) return SADMM_OK;
  bp_rotate_kernel<<<div_up((long long)n, 256), 256, 0, st>>>(y, out, n);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_bp_combine(const float* g, int Q, int N, float* out, cudaStream_t st) {
  bp_combine_kernel<<<div_up(N, 256), 256, 0, st>>>(g, Q, N, out);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

int launch_recompute_xbar(const SolverView& sv, cudaStream_t st) {
  xbar_kernel<<<div_up(sv.N, 256), 256, 0, st>>>(sv);
  SADMM_LAUNCH_CHECK();
  return SADMM_OK;
}

}  // namespace sadmm
