// Shared device/host helpers of the sharing-ADMM library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "sadmm.h"

namespace sadmm {

// Status plumbing: every internal call returns an int status; the message of
// the last failure is kept per host thread.
void set_error(const char* fmt, ...);

#define SADMM_CUDA_TRY(expr)                                                         \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ::sadmm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                  \
                         cudaGetErrorString(e_));                                    \
      return SADMM_ECUDA;                                                            \
    }                                                                                \
  } while (0)

#define SADMM_TRY(expr)                                                              \
  do {                                                                               \
    int s_ = (expr);                                                                 \
    if (s_ != SADMM_OK) return s_;                                                   \
  } while (0)

// Every kernel launch of the library goes through this check, which also
// counts it (process-wide, see sadmm_launch_count).
void count_launch();
#define SADMM_LAUNCH_CHECK()             \
  do {                                   \
    ::sadmm::count_launch();             \
    SADMM_CUDA_TRY(cudaGetLastError());  \
  } while (0)

constexpr int kTile = 64;          // FP64 factor tile edge (Gram, Cholesky, inverse)
constexpr int kMaxSets = 64;       // sensors per batched launch (= maximum Q)

// Per-sensor launch arguments travel by value in the kernel parameter block
// (no device-side argument copies, so launches can be captured in a graph).
template <typename T>
struct SetBlock {
  T v[kMaxSets];
};

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Which source the forward product reads its per-column scalar from.
enum VMode : int {
  kVAdmm = 0,   // v = x_q - x_bar + z_bar - s   (Eq. 3, x_q-update right-hand side)
  kVX = 1,      // v = x_q                       (fold of frozen pixels into y')
  kVExplicit = 2,// v = caller array indexed by pixel
  kVNegX = 3,    // v = -x_q                      (unfold of re-admitted pixels)
  kVCons = 4     // v = z - u_q                   (consensus form's x-update right-hand side)
};

// Device-resident per-iteration scalars written by the residual kernel
// (layout shared with the host; all doubles first).
struct IterScalars {
  double r_pri, eps_pri, d, eps_dual, relchange, xg_norm, dxg_norm, xnorm;
  int k;          // iterations completed after this one
  int gate;       // Algorithm 1 test runs this iteration
  int changed;    // sensors whose active set shrank (written by the SSC kernel)
  int nonfinite;  // a NaN/Inf was seen in the reductions
};

// Device view of the solver state handed to the kernels.
struct SolverView {
  int Q, N, KM, Kp;
  float mu, rho;
  float lam_over_rho;
  float* x;          // Q x N
  float* xbar;       // N
  float* zbar;       // N
  float* s;          // N
  float* ring;       // Kp x Q x N signed updates x^{t+1} - x^t
  int slot;          // ring slot written this iteration
  float* u;          // consensus form: Q x N scaled duals (zbar holds z); null for the sharing form
};

// The x-update's v on pixel pix of sensor q (Eq. 3, x_q-update, read as
// Boyd's sharing step: v = x_q - x_bar + z_bar - s), or, for the consensus
// form, v = z - u_q.
__device__ __forceinline__ float v_admm(const SolverView& sv, int q, int pix, float xq) {
  if (sv.u) return sv.zbar[pix] - sv.u[(size_t)q * sv.N + pix];
  return xq - sv.xbar[pix] + sv.zbar[pix] - sv.s[pix];
}

// ---- kernel launchers (implemented in the .cu files) ----
struct ColumnSet {          // one sensor's column list for a batched launch
  const float2* A;          // pixel-major operator of the sensor
  const int* idx;           // column (pixel) indices
  int n;                    // number of listed columns
  int q;                    // sensor index (row of x, ring)
  const float* vexp;        // explicit v (kVExplicit)
  const float2* base;       // base vector (KM complex) or null
  float2* out;              // KM complex output
};

int launch_forward(const ColumnSet* sets, int nsets, int KM, VMode mode, const SolverView& sv,
                   float2* partial, size_t partial_cap, cudaStream_t st);
size_t forward_partial_bytes(int nsets, int KM, int max_cols);
// out = base - sum over chunks of the double-float chunk partials
// partial[set][chunk][plane][KM] (plane 0 high words, plane 1 low words).
int launch_forward_reduce(const ColumnSet* sets, int nsets, int KM, int chunks, const float2* partial,
                          cudaStream_t st);

// The per-column scalar v of the forward product, by mode.
__device__ __forceinline__ float v_of(VMode mode, const SolverView& sv, int q, int pix, const float* vexp) {
  if (mode == kVExplicit) return vexp[pix];
  const float xq = sv.x[(size_t)q * sv.N + pix];
  if (mode == kVX) return xq;
  if (mode == kVNegX) return -xq;
  return xq - sv.xbar[pix] + sv.zbar[pix] - sv.s[pix];
}

// The per-column scalar with the consensus mode as a compile-time choice: the
// forward kernels are instantiated apart for it, so that the sharing form's
// instantiation keeps the code it had without the consensus read.
template <bool CONS>
__device__ __forceinline__ float v_col(VMode mode, const SolverView& sv, int q, int pix, const float* vexp) {
  if constexpr (CONS) return sv.zbar[pix] - sv.u[(size_t)q * sv.N + pix];
  return v_of(mode, sv, q, pix, vexp);
}

// Factored operator (factored.cu): A[(m, k), n] = C[m][a][n] D[m][b][n] with
// k = 16 a + b, C = exp(j 2 pi tau (f0 + 16 a df)), D = exp(j 2 pi tau b df).
constexpr int kFacB = 16;
struct FactoredSet {
  const float2* C;          // M x K/16 x N (pixel fastest)
  const float2* D;          // M x 16 x N
  const int* idx;           // column (pixel) indices
  int n;
  int q;
  const float* vexp;        // forward: explicit v (kVExplicit)
  const float2* base;       // forward: base vector (KM complex) or null
  float2* out;              // forward: KM complex output
  const float2* w;          // adjoint: KM complex input
  float* g;                 // adjoint: g[p] output (mode g)
};
bool factored_supported(int K);   // K = 16, 32, 64, 128, 256 or 512
int operator_tables(const double* tau, int M, int K, int N, double f0, double df, float2* A, float2* C, float2* D,
                    cudaStream_t st);
int factored_chunks(int nsets, int M, int K, int max_cols);
size_t factored_partial_bytes(int nsets, int M, int K, int max_cols);
int launch_factored_forward(const FactoredSet* sets, int nsets, int M, int K, int N, VMode mode, const SolverView& sv,
                            float2* partial, size_t partial_cap, cudaStream_t st);
int launch_factored_adjoint(const FactoredSet* sets, int nsets, int M, int K, int N, bool update, const SolverView& sv,
                            cudaStream_t st);

struct AdjointSet {
  const float2* A;
  const int* idx;
  int n;
  int q;
  const float2* w;   // KM complex
  float* g;          // output g[p] (mode g) or unused (mode update)
  float* g_lo;       // mode g, optional: g from exact products summed in double-float, written as
                     // the pair (g, g_lo) (the primal x-update amplifies any error in g, see api.cu)
};
int launch_adjoint(const AdjointSet* sets, int nsets, int KM, bool update, const SolverView& sv,
                   cudaStream_t st);

// Batched adjoint on the tensor cores (tc.cu): gpart[q][split][p][s] =
// sum over the split's real rows of B_q[r][p] W_q[r][s] (16 scenes).  Aq and
// Wq are HOST arrays of Q device pointers (the tensor maps are built on the host).
int tc_adjoint_splits(int Q, int N, int KM);
// Batched forward on the tensor cores (tc.cu): partial[q][split][m][s] (float2:
// real rows 2m, 2m+1) = sum over the split's pixels p of B_q[r][p] V[p][s],
// V = x - x_bar + z_bar - s of scene s (16 scenes); Aq: HOST array of Q device pointers.
int tc_forward_splits(int Q, int N, int KM);
// Largest useful split counts (at least four 32-row / 32-pixel slabs per split).
int tc_adjoint_max_splits(int KM);
int tc_forward_max_splits(int N);
int launch_tc_forward(const float2* const* Aq, const float* X, const float* xbar, const float* zbar, const float* sd,
                      float2* partial, int Q, int N, int KM, int splits, int* err, cudaStream_t st);
int launch_tc_adjoint(const float2* const* Aq, const float2* const* Wq, float* gpart, int Q, int N, int KM, int splits,
                      int* err, cudaStream_t st);

// Symmetric factors are stored as packed upper-triangular 64 x 64 tiles of
// double-float pairs (spd.cu).
constexpr int kSymTile = 64;
size_t sym_packed_pairs(int n);      // float2 elements of the packed factor
size_t sym_part_pairs(int n);        // float2 elements of the apply's partial sums
// P (packed pairs) <- the upper triangle of the n x n FP64 matrix F (leading dimension ld)
int launch_pack_sym(const double* F, int ld, int n, float2* P, cudaStream_t st);

struct SpdSet {
  const float2* P;   // packed factor (launch_pack_sym)
  int n;
  const float* u;    // n floats
  float* out;        // n floats (plain) or unused (update)
  const int* idx;    // primal form: pixel of row p (update mode)
  int q;
  float2* part;      // sym_part_pairs(n) scratch
  int tile0;         // set by launch_spd_apply
  double* outd;      // optional: out written as hi + lo in FP64, element i at outd[i * ldd]
  int ldd;
  const float* u_lo; // optional: low words of u (the input is the pair u + u_lo)
};
// out = F u for every set (or, with update, the primal x-update epilogue).
// *err is set to 1 if a tile copy did not complete within the wait limit.
int launch_spd_apply(const SpdSet* sets, int nsets, bool update, const SolverView& sv, int* err,
                     cudaStream_t st);
// Polls of the factor apply's tile-copy wait before it gives up (< 0: the default).
int set_spd_wait_limit(long long polls);

// Back-projection helpers (elementwise.cu): out = -i y; out = sum_q |g_re + i g_im|
// with g laid out per sensor as [re N][im N].
int launch_bp_rotate(const float2* y, float2* out, size_t n, cudaStream_t st);
int launch_bp_combine(const float* g, int Q, int N, float* out, cudaStream_t st);
int launch_residuals(const SolverView& sv, const sadmm_criterion& c, double* partials,
                     unsigned int* ticket, IterScalars* out, int k_after, cudaStream_t st);
int residual_blocks(int N);

// Algorithm 1 on every sensor: reads the gate from `sc`; compacts J[q] in
// place (order kept), lists removed pixels in E[q], zeroes their ring entries
// (and x in zero mode).  counts[q] = new |J_q|, counts[Q + q] = |E_q|.
// tag (Q x N, may be null) / tally (2Q ints): pixels the learned proposal
// removed that Algorithm 1 alone would have kept are tagged and counted in
// tally[q]; the rebuild counts tagged pixels that are re-admitted in
// tally[Q + q] and clears their tags (false eliminations of the proposal).
int launch_ssc(const SolverView& sv, int* const* J, int* const* E, int* counts, double eps_p,
               int freeze_mode, const IterScalars* sc, const float* prob, float theta, int learned_now,
               cudaStream_t st, uint8_t* tag = nullptr, int* tally = nullptr);
// Learned proposal and re-admission (learned.cu)
int launch_features(const SolverView& sv, int k_done, double eps_p, float* out, cudaStream_t st);
int launch_frozen_lists(const SolverView& sv, int* const* J, const int* counts, uint8_t* mask, int* const* F,
                        int* fcounts, cudaStream_t st);
struct ReadmitSet {
  const float2* A;
  const int* F;        // frozen pixels of the sensor
  int n;
  int q;
  const float2* r;     // y'_q - A_J x_J
};
int launch_readmit_check(const ReadmitSet* sets, int nsets, int KM, const SolverView& sv, double thr,
                         uint8_t* mask, cudaStream_t st);
int launch_rebuild_lists(const SolverView& sv, int* const* J, int* const* R, uint8_t* mask, int* counts,
                         int* rcounts, double ring_fill, cudaStream_t st, uint8_t* tag = nullptr,
                         int* tally = nullptr);
int launch_recompute_xbar(const SolverView& sv, cudaStream_t st);
int launch_scale(const float* in, float a, float* out, int n, cudaStream_t st);

// ---- split-precision operator planes (split.cu) ----
constexpr int kSplitBF16 = 1;
constexpr int kSplitFP16 = 2;
struct SplitSet {
  const void* hi;            // 16-bit (re, im) plane, pixel-major
  const void* lo;            // 16-bit residual plane
  const int* idx;            // column (pixel) list
  int n;                     // listed columns
  int q;                     // sensor (row of x and the ring)
  const float* vexp;         // forward, kVExplicit: v by pixel
  const float2* base;        // forward: out = base - product (null: 0)
  float2* out;               // forward: base - product (may be null)
  float2* out2;              // forward: the product itself (may be null)
  const float2* w;           // adjoint input (KM complex)
  float* g;                  // adjoint output in list order (+ gcorr_in when set)
  float* g_lo;               // with g: the low words of an exact double-float g (split adjoint, no update)
  const float* gcorr_in;     // per-pixel correction added to the adjoint
  float* gcorr_out;          // adjoint: per-pixel store of the product
};
int launch_split_forward(const SplitSet* sets, int nsets, int KM, int kind, int planes, VMode mode,
                         const SolverView& sv, float2* partial, size_t partial_cap, cudaStream_t st);
int launch_split_adjoint(const SplitSet* sets, int nsets, int KM, int kind, int planes, bool update,
                         const SolverView& sv, cudaStream_t st);
// hi = RN(a), lo = RN(a - hi) per float; P (may be null) = hi + lo, exact in
// FP32: the pair operator the split products see.
int launch_split_convert(const float* A, size_t nfloats, int kind, uint16_t* hi, uint16_t* lo,
                         cudaStream_t st, float* P = nullptr);
size_t split_partial_bytes(int nsets, int KM, int max_cols);

// FP64 factor: F <- (rho I + mu G)^{-1} for the Gram of the listed columns.
struct FactorJob {
  const float2* A;
  const int* idx;
  int ncols;         // |J|
  int n;             // factor dimension (2KM or |J|)
  int npad;          // round_up(n, kTile), also the leading dimension
  int woodbury;      // 1: G = B_J B_J^T (2KM x 2KM), 0: G = B_J^T B_J
  double* out;       // npad x npad: Gram, then its Cholesky factor, then the inverse (result)
  double* tmp;       // npad x npad scratch (inverse of the Cholesky factor)
  double* dinv;      // (npad / kTile) x kTile x kTile inverses of the diagonal blocks
};
// gram: 0 = tensor-core Gram from exact BF16 digit slices (gram_tc.cu; takes
// transient scratch from the stream-ordered pool), 1 = SIMT FP64 Gram.
// d_status[i] is set to 1 if job i's matrix is not positive definite, 2 if a
// bounded wait of its Gram timed out.
int run_factor(const FactorJob* jobs, int njobs, int KM, double mu, double rho, int* d_status,
               cudaStream_t st, int gram = 0);
// The Gram step alone: job.out = mu G + rho I (identity padding), same methods.
int run_gram(const FactorJob& job, int KM, double mu, double rho, int* d_status, cudaStream_t st, int gram);
size_t gram_tc_scratch_bytes(const FactorJob& j, int KM);
// job.out (npad x npad, leading dimension npad) = mu G + rho I with identity
// padding, G the Gram of the job's form; *err = 2 on a timed-out wait.
int launch_gram_tc(const FactorJob& j, int KM, double mu, double rho, void* scratch, size_t scratch_bytes, int* err,
                   cudaStream_t st);

// Rank-e downdate of a Woodbury-form factor after removing e <= kDowndateMax
// columns E from the active set (Eq. 3's system without those pixels):
//   (G - mu U U^T)^{-1} = W + mu T T^T,  P = W U,  S = I - mu U^T P = L L^T,
//   T = P L^{-T},  U = B_E (interleaved real form of the removed columns);
// with sign = -1 the rank-e update after adding columns back:
//   (G + mu U U^T)^{-1} = W - mu T T^T,  S = I + mu U^T P.
constexpr int kDowndateMax = 32;
struct DowndateJob {
  const float2* A;
  const int* E;          // removed pixels of this pass
  int e;                 // 1..kDowndateMax
  int n;                 // factor dimension 2KM (leading dimension too)
  const double* Wsrc;    // current factor
  double* Wdst;          // updated factor (may alias Wsrc)
  double* P;             // n x kDowndateMax scratch: W U, then T
  double* Spart;         // ceil(n/256) x kDowndateMax^2 partial sums of U^T P
  double* S;             // kDowndateMax^2: the inverse Cholesky factor of S
  int slot;              // index of this job's failure flag in the status array
  int sign;              // +1 remove the columns, -1 add them
  // double-float path (run_downdate_pairs): the packed pair copies of W
  const float2* Fsrc;
  float2* Fdst;          // may alias Fsrc
};
int run_downdate(const DowndateJob* jobs, int njobs, int KM, double mu, int* d_status, cudaStream_t st);

// P[:, c0 + c] = F B[:, E[c0 + c]] for c < min(16, e - c0), per job (batch.cu):
// the 16-column packed-tile apply used by the factor updates.  F, A, E, P:
// HOST arrays of per-job device pointers; U: njobs x n x 16 floats of scratch;
// dptrs: 2 x njobs device pointers of scratch; part: njobs x
// multi_apply_part_pairs(n) float2 of scratch.
size_t multi_apply_part_pairs(int n);
int launch_multi_apply_cols(const float2* const* F, const float2* const* A, const int* const* E, const int* e, double* const* P,
                            int njobs, int n, int c0, float* U, void** dptrs, float2* part, int* err, cudaStream_t st);

// The same rank update applied to the packed (hi, lo) pair copy of W only
// (Fsrc -> Fdst), with W U formed by the 16-column double-float packed-tile
// apply and the rank-e correction accumulated in double-float arithmetic; the
// FP64 Wsrc/Wdst are not used.  All jobs share n.
struct DdScratch {
  float* U;          // jobs x n x 16
  void** dptrs;      // 2 x jobs device pointers
  float2* part;      // jobs x multi_apply_part_pairs(n); also 64 x sym_part_pairs(n) for single-column applies
};
// Downdate of a primal-form factor H = (rho I + mu B_J^T B_J)^{-1} over the
// ordered list J_old when the pixels E leave it (factor.cu): the new factor
// over J_new = J_old \ E is the Schur complement H_RR - H_RE H_EE^{-1} H_ER.
struct PrimalDdJob {
  const double* H;    // old factor, n_old x n_old, leading dimension ldh
  int ldh;
  double* Hn;         // new factor, n_new x n_new (identity-padded to ldn), leading dimension ldn
  int ldn;
  const int* J;       // new ordered list (n_new pixels, ascending)
  const int* E;       // removed pixels (e <= kDowndateMax, ascending)
  int n_new, e;
  int* pos;           // n_new + e scratch: old positions of the kept rows, then of the removed ones
  double* V;          // n_new x kDowndateMax scratch, then kDowndateMax^2 for L^{-1} of H_EE
  int slot;           // status slot
};
int run_primal_downdate(const PrimalDdJob* jobs, int njobs, int* d_status, cudaStream_t st);
// out (na + nb) = ascending merge of the ascending, disjoint lists a and b
int launch_merge_lists(const int* a, int na, const int* b, int nb, int* out, cudaStream_t st);
int run_downdate_pairs(const DowndateJob* jobs, int njobs, int KM, double mu, const DdScratch& scr, int* d_status,
                       int* err, cudaStream_t st);
size_t downdate_scratch_doubles(int n);

}  // namespace sadmm
