// C ABI and host orchestration of the sharing-ADMM solver (Section III:
// Eq. 3 iterated with Algorithm 1).  One context owns the device state of
// one problem; all work goes to the context's stream.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace sadmm {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

namespace {

struct Allocator {
  sadmm_alloc_fn alloc = nullptr;
  sadmm_free_fn release = nullptr;
  void* user = nullptr;
};
Allocator g_alloc;

struct Sensor {
  float2* A = nullptr;       // N x KM pixel-major
  float2* y = nullptr;       // KM
  float2* yp = nullptr;      // KM, y minus frozen contributions
  float2* r = nullptr;       // KM, residual y' - A_J v_J
  float2* w = nullptr;       // KM, W r (Woodbury form)
  float* g = nullptr;        // N, Re(A_J^H r) in list order (primal form)
  float* g_lo = nullptr;     // N, its low words (plain FP32 path: g exact to double-float)
  int* pos = nullptr;        // N, primal-form downdate scratch (elim > 0)
  int* J = nullptr;          // N, active list
  int* E = nullptr;          // N, pixels removed in the last SSC pass
  int* F = nullptr;          // N, frozen pixels at the last learned step (elim = 2)
  int* R = nullptr;          // N, pixels re-admitted at the last learned step (elim = 2)
  int* Jm = nullptr;         // N, intermediate lists of a multi-pass primal downdate
  double* fb[3] = {nullptr, nullptr, nullptr};   // FP64 factor buffers
  float2* fhl[3] = {nullptr, nullptr, nullptr};  // their packed symmetric (hi, lo) pair copies, used every iteration
  double* dinv = nullptr;      // diagonal-block inverses; also the downdate's n x 32 scratch
  double* dd = nullptr;        // downdate scratch (partial sums and the small factor)
  int cum_dd = 0;              // columns downdated since the last full factorisation
  uint16_t* hi = nullptr;      // split-precision planes (precision > 0)
  uint16_t* lo = nullptr;
  float2* P = nullptr;         // the pair operator hi + lo (exact in FP32): what the split
                               // products see, so the factor, fold and updates use it too
  float2* base_corr = nullptr; // y' - A_lo,J v at the last lo refresh (precision 3/4)
  float* gcorr = nullptr;      // Re(a_lo^H w) per pixel at the last lo refresh
  int full = 0;              // buffer holding the full-set factor
  bool full_valid = false;
  int cur = 0;               // buffer in use
  int n = 0;                 // factor dimension in use
  int woodbury = 0;          // form in use
  int cnt = 0;               // |J_q| (host mirror)
  bool op_set = false;
  // factored representation (sadmm_set_operator_delays)
  double* tau = nullptr;       // M x N round-trip delays
  float2* C = nullptr;         // M x K/16 x N
  float2* D = nullptr;         // M x 16 x N
  bool factored = false;
};

uint64_t constexpr kStateMagic = 0x31766174734d4453ull;   // "SDMstav1"

}  // namespace

struct Ctx {
  int Q = 0, M = 0, K = 0, N = 0, KM = 0;
  double rho = 1.0, lam = 0.0;
  sadmm_criterion crit{};
  cudaStream_t st = nullptr;
  Allocator alloc;
  std::vector<void*> owned;
  std::vector<Sensor> s;
  float *x = nullptr, *xbar = nullptr, *zbar = nullptr, *sd = nullptr, *ring = nullptr;
  float* u = nullptr;          // consensus form: Q x N scaled duals
  float* xg = nullptr;
  int* iota = nullptr;
  float2* partial = nullptr;
  size_t partial_cap = 0;
  float2* spd_part = nullptr;  // per-sensor partial sums of the symmetric factor apply
  DdScratch dd{};              // scratch of the factor updates' 16-column applies
  size_t spd_part_stride = 0;
  int* spd_err = nullptr;      // set by the factor apply if a tile copy timed out
  double* red = nullptr;
  unsigned int* ticket = nullptr;
  IterScalars* scal = nullptr;
  int* counts = nullptr;       // 4Q: |J_q|, |E_q|, |F_q|, |R_q|
  int* dstatus = nullptr;      // Q factor status flags
  IterScalars* h_scal = nullptr;
  int* h_counts = nullptr;
  int* h_status = nullptr;
  int npad_max = 0;
  int k = 0;
  // learned proposal and re-admission (elim = 2)
  sadmm_cnn_t cnn = nullptr;   // owned
  int cnn_H = 0, cnn_W = 0;
  float* feat = nullptr;       // 6 x N features
  float* prob = nullptr;       // N proposal probabilities
  uint8_t* mask = nullptr;     // Q x 2N: active flags, re-admission flags
  uint8_t* ptag = nullptr;     // Q x N: removed by the learned proposal alone (until re-admitted)
  int* ptally = nullptr;       // 2Q: proposal removals, re-admissions of those
  bool learned_now = false;    // the iteration last launched ran the learned step
  bool learned_due() const {
    return crit.elim == 2 && cnn != nullptr && (k + 1) % crit.learn_every == 0 && k + 1 >= std::max(crit.Kp, 4);
  }
  std::vector<sadmm_iter_record> hist;
  bool corr_due = true;        // precision 3/4: refresh the lo-plane products next iteration
  int last_corr_k = 0;
  int split_kind() const { return (crit.precision == 1 || crit.precision == 3) ? kSplitBF16 : kSplitFP16; }
  // the operator the iteration solves with: the stored one, or its pair form
  const float2* op(int q) const { return crit.precision > 0 && s[q].P ? s[q].P : s[q].A; }
  int op_kind() const { return crit.precision > 0 ? split_kind() : 0; }
  int factor_kind = -1;        // op_kind() of the operator the full-set factors were formed from
  int ring_kp = 0;             // update-ring capacity (Kp slots)
  int products = SADMM_PRODUCTS_AUTO;
  float2* bp_y = nullptr;      // back-projection scratch: Q x [y, -i y]
  float* bp_g = nullptr;       // Q x [Re, Im] of A^H y
  float* bp_out = nullptr;     // N
  bool all_factored() const {
    for (const Sensor& S : s)
      if (!S.factored) return false;
    return true;
  }
  // the per-iteration products read the factored tables
  // (automatically only while every sensor is in the Woodbury form: the
  // primal form's H g amplifies the factored entries' rounding by the
  // condition number of rho I + mu B^T B, which the stored path avoids with
  // an exact g)
  // the forward product's right-hand side: the sharing or the consensus x-update
  VMode vmode() const { return crit.consensus ? kVCons : kVAdmm; }
  bool use_factored() const {
    if (products == SADMM_PRODUCTS_STORED || crit.precision != 0 || crit.consensus || !all_factored()) return false;
    if (products == SADMM_PRODUCTS_AUTO)
      for (const Sensor& S : s)
        if (S.cnt > 0 && !S.woodbury) return false;
    return true;
  }
  bool periodic() const { return crit.precision >= 3; }
  // profiling: one event pair per (slot, phase); a slot is an iteration not
  // yet collected (one per iteration when the host synchronises each
  // iteration, one per iteration of the whole run otherwise)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<char> ev_used;
  int prof_slot = 0;
  double prof_ms[SADMM_NUM_PHASES] = {};
  long long prof_n[SADMM_NUM_PHASES] = {};

  int ensure_events(int slots) {
    const size_t need = (size_t)slots * SADMM_NUM_PHASES * 2;
    while (ev.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return SADMM_ECUDA;
      ev.push_back(e);
    }
    ev_used.resize(ev.size() / 2, 0);
    return SADMM_OK;
  }
  void mark(int phase, bool begin) {
    if (!prof) return;
    if (ensure_events(prof_slot + 1) != SADMM_OK) { prof = false; return; }
    const size_t pair = (size_t)prof_slot * SADMM_NUM_PHASES + phase;
    cudaEventRecord(ev[2 * pair + (begin ? 0 : 1)], st);
    if (!begin) ev_used[pair] = 1;
  }
  // After a stream synchronisation: fold the recorded phase times in.
  void collect() {
    if (!prof) { prof_slot = 0; return; }
    for (size_t pair = 0; pair < ev_used.size(); ++pair) {
      if (!ev_used[pair]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * pair], ev[2 * pair + 1]) == cudaSuccess) {
        prof_ms[pair % SADMM_NUM_PHASES] += ms;
        prof_n[pair % SADMM_NUM_PHASES] += 1;
      }
      ev_used[pair] = 0;
    }
    prof_slot = 0;
  }
  // device history of per-iteration scalars for runs without per-iteration sync
  IterScalars* hist_dev = nullptr;
  int hist_cap = 0;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (alloc.alloc) {
      p = alloc.alloc(bytes, (void*)st, alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void release_all() {
    cudaStreamSynchronize(st);
    for (void* p : owned) {
      if (alloc.release) alloc.release(p, (void*)st, alloc.user);
      else cudaFree(p);
    }
    owned.clear();
    if (h_scal) cudaFreeHost(h_scal);
    if (h_counts) cudaFreeHost(h_counts);
    if (h_status) cudaFreeHost(h_status);
    if (cnn) sadmm_cnn_destroy(cnn);
    cnn = nullptr;
    for (auto& e : ev) cudaEventDestroy(e);
    ev.clear();
    ev_used.clear();
    h_scal = nullptr;
    h_counts = nullptr;
    h_status = nullptr;
  }
  SolverView view() const {
    SolverView v;
    v.Q = Q; v.N = N; v.KM = KM; v.Kp = crit.Kp;
    v.mu = (float)crit.mu; v.rho = (float)rho;
    v.lam_over_rho = (float)(crit.consensus ? lam / (Q * rho) : lam / rho);
    v.u = crit.consensus ? u : nullptr;
    v.x = x; v.xbar = xbar; v.zbar = zbar; v.s = sd; v.ring = ring;
    v.slot = k % crit.Kp;
    return v;
  }
};

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

__global__ void iota_kernel(int* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

int factor_dims(const Ctx& c, int cnt, int* n, int* woodbury) {
  *woodbury = cnt > 2 * c.KM ? 1 : 0;
  *n = *woodbury ? 2 * c.KM : cnt;
  return SADMM_OK;
}

// Buffers for factors of shrunken active sets (elimination, re-admission,
// restored states): the third FP64 buffer and two more packed pair copies, so
// that the full-set factor (buffer 0 and its pairs) survives.  Contexts that
// never shrink a set (plain SADMM) do without them.
int ensure_set_buffers(Ctx& c) {
  const size_t fbytes = (size_t)c.npad_max * c.npad_max * sizeof(double);
  const size_t pbytes = sym_packed_pairs(c.npad_max) * sizeof(float2);
  for (Sensor& S : c.s) {
    if (!S.fb[2]) S.fb[2] = (double*)c.dalloc(fbytes);
    for (int b = 1; b < 3; ++b)
      if (!S.fhl[b]) S.fhl[b] = (float2*)c.dalloc(pbytes);
    if (!S.Jm) S.Jm = (int*)c.dalloc((size_t)c.N * sizeof(int));
    if (!S.fb[2] || !S.fhl[1] || !S.fhl[2] || !S.Jm) {
      cudaGetLastError();
      set_error("factor buffers for shrunken active sets: device allocation failed");
      return SADMM_ENOMEM;
    }
  }
  return SADMM_OK;
}

// Factor refresh for the listed sensors at their current active sets.
int refresh(Ctx& c, const std::vector<int>& qs, bool full_set) {
  if (!full_set) SADMM_TRY(ensure_set_buffers(c));
  std::vector<FactorJob> jobs;
  std::vector<int> owner, outbuf;
  for (int q : qs) {
    Sensor& S = c.s[q];
    if (S.cnt == 0) { S.n = 0; continue; }
    int n, wb;
    factor_dims(c, S.cnt, &n, &wb);
    int o, t;
    if (full_set) { o = 0; t = 1; }
    else { o = (S.full + 1) % 3; t = (S.full + 2) % 3; }
    FactorJob j;
    j.A = c.op(q); j.idx = full_set ? c.iota : S.J; j.ncols = S.cnt; j.n = n;
    j.npad = round_up(n, kTile); j.woodbury = wb; j.out = S.fb[o]; j.tmp = S.fb[t];
    j.dinv = S.dinv;
    jobs.push_back(j);
    owner.push_back(q);
    outbuf.push_back(o);
  }
  if (jobs.empty()) return SADMM_OK;
  SADMM_CUDA_TRY(cudaMemsetAsync(c.dstatus, 0, sizeof(int) * c.Q, c.st));
  for (size_t b = 0; b < jobs.size(); b += kMaxSets) {
    const int nj = (int)std::min<size_t>(kMaxSets, jobs.size() - b);
    SADMM_TRY(run_factor(jobs.data() + b, nj, c.KM, c.crit.mu, c.rho, c.dstatus + b, c.st));
  }
  SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_status, c.dstatus, sizeof(int) * c.Q, cudaMemcpyDeviceToHost, c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  for (size_t i = 0; i < jobs.size(); ++i) {
    if (c.h_status[i] == 2) {
      set_error("factor of sensor %d: a bounded wait of the tensor-core Gram timed out", owner[i]);
      return SADMM_ETIMEOUT;
    }
    if (c.h_status[i]) {
      set_error("factor of sensor %d is not positive definite (non-finite operator?)", owner[i]);
      return SADMM_ENONFINITE;
    }
    Sensor& S = c.s[owner[i]];
    S.cur = outbuf[i];
    S.n = jobs[i].n;
    S.woodbury = jobs[i].woodbury;
    if (full_set) { S.full = outbuf[i]; S.full_valid = true; }
    S.cum_dd = 0;
    SADMM_TRY(launch_pack_sym(S.fb[S.cur], jobs[i].npad, jobs[i].n, S.fhl[S.cur], c.st));
  }
  return SADMM_OK;
}

// Rank-|E| downdate of Woodbury-form factors, in passes of at most
// kDowndateMax removed columns; with `add` the rank-|R| update for the
// re-admitted columns instead.  The update is applied to the packed (hi, lo)
// pair copy the iteration reads (run_downdate_pairs: W U by the double-float
// symmetric apply, the small system in FP64, the rank correction in
// double-float), so the FP64 factor is only rebuilt on a full refresh.
// Sensors whose update fails (the small system is not numerically positive
// definite) are returned in `failed`.
int downdate(Ctx& c, const std::vector<int>& qs, std::vector<int>* failed, bool add = false) {
  if (qs.empty()) return SADMM_OK;
  SADMM_TRY(ensure_set_buffers(c));
  std::vector<int> dst(c.Q), etot(c.Q);
  int max_e = 0;
  for (int q : qs) {
    Sensor& S = c.s[q];
    dst[q] = (S.cur == S.full) ? (S.full + 1) % 3 : S.cur;
    etot[q] = c.h_counts[(add ? 3 : 1) * c.Q + q];
    max_e = std::max(max_e, etot[q]);
  }
  SADMM_CUDA_TRY(cudaMemsetAsync(c.dstatus, 0, sizeof(int) * c.Q, c.st));
  const int n = 2 * c.KM;
  const size_t nblk = div_up(n, 256);
  for (int off = 0; off < max_e; off += kDowndateMax) {
    std::vector<DowndateJob> jobs;
    for (int q : qs) {
      Sensor& S = c.s[q];
      if (etot[q] <= off) continue;
      DowndateJob j{};
      j.A = c.op(q); j.E = (add ? S.R : S.E) + off; j.e = std::min(kDowndateMax, etot[q] - off); j.n = n;
      j.Fsrc = (off == 0) ? S.fhl[S.cur] : S.fhl[dst[q]];
      j.Fdst = S.fhl[dst[q]];
      j.P = S.dinv; j.Spart = S.dd; j.S = S.dd + nblk * kDowndateMax * kDowndateMax;
      j.slot = q;
      j.sign = add ? -1 : 1;
      jobs.push_back(j);
    }
    SADMM_TRY(run_downdate_pairs(jobs.data(), (int)jobs.size(), c.KM, c.crit.mu, c.dd, c.dstatus, c.spd_err, c.st));
  }
  SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_status, c.dstatus, sizeof(int) * c.Q, cudaMemcpyDeviceToHost, c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  for (int q : qs) {
    Sensor& S = c.s[q];
    if (c.h_status[q]) { failed->push_back(q); continue; }
    S.cur = dst[q];
    S.cum_dd += etot[q];
  }
  return SADMM_OK;
}

int prepare(Ctx& c) {
  std::vector<int> qs;
  if (c.factor_kind != c.op_kind())        // the factors belong to another operator form
    for (Sensor& S : c.s) S.full_valid = false;
  for (int q = 0; q < c.Q; ++q) {
    if (!c.s[q].op_set) {
      set_error("operator of sensor %d not set", q);
      return SADMM_ENOTREADY;
    }
    if (!c.s[q].full_valid) qs.push_back(q);
  }
  if (c.products == SADMM_PRODUCTS_FACTORED) {
    if (c.crit.precision > 0) {
      set_error("factored products need precision 0 (the split forms read the stored planes)");
      return SADMM_EINVAL;
    }
    if (c.crit.consensus) {
      set_error("factored products run the sharing form (consensus = 0)");
      return SADMM_EINVAL;
    }
    for (int q = 0; q < c.Q; ++q)
      if (!c.s[q].factored) {
        set_error("factored products requested but sensor %d has no delays (sadmm_set_operator_delays)", q);
        return SADMM_ENOTREADY;
      }
  }
  if (qs.empty()) return SADMM_OK;
  std::vector<int> saved(c.Q);
  for (int q : qs) { saved[q] = c.s[q].cnt; c.s[q].cnt = c.N; }
  int rc = refresh(c, qs, true);
  for (int q : qs) c.s[q].cnt = saved[q];
  if (rc == SADMM_OK) c.factor_kind = c.op_kind();
  return rc;
}

// Point every sensor at its full-set factor and reset the iterates to zero.
int reset_state(Ctx& c) {
  const size_t QN = (size_t)c.Q * c.N;
  SADMM_CUDA_TRY(cudaMemsetAsync(c.x, 0, QN * sizeof(float), c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.xbar, 0, c.N * sizeof(float), c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.zbar, 0, c.N * sizeof(float), c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.sd, 0, c.N * sizeof(float), c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.ring, 0, (size_t)c.crit.Kp * QN * sizeof(float), c.st));
  if (c.u) SADMM_CUDA_TRY(cudaMemsetAsync(c.u, 0, QN * sizeof(float), c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.ptag, 0, QN, c.st));
  SADMM_CUDA_TRY(cudaMemsetAsync(c.ptally, 0, 2 * c.Q * sizeof(int), c.st));
  std::vector<int> cnts(2 * c.Q, 0);
  for (int q = 0; q < c.Q; ++q) {
    Sensor& S = c.s[q];
    SADMM_CUDA_TRY(cudaMemcpyAsync(S.J, c.iota, c.N * sizeof(int), cudaMemcpyDeviceToDevice, c.st));
    SADMM_CUDA_TRY(cudaMemcpyAsync(S.yp, S.y, c.KM * sizeof(float2), cudaMemcpyDeviceToDevice, c.st));
    S.cnt = c.N;
    cnts[q] = c.N;
    S.cur = S.full;
    S.cum_dd = 0;
    factor_dims(c, c.N, &S.n, &S.woodbury);
  }
  SADMM_CUDA_TRY(cudaMemcpyAsync(c.counts, cnts.data(), cnts.size() * sizeof(int), cudaMemcpyHostToDevice, c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  c.k = 0;
  c.corr_due = true;
  c.last_corr_k = 0;
  return SADMM_OK;
}

// One iteration of Eq. 3 (x-update, prox, dual) and Algorithm 1 (device side).
int launch_split_products_fwd(Ctx& c, const SolverView& sv, bool corr);
int launch_split_products_adj(Ctx& c, const SolverView& sv, bool corr);

// Algorithm 1 on the device.  At a learned iteration (elim = 2) it is preceded
// by the re-admission test of the pixels frozen before this pass (flags in the
// second half of each sensor's mask row) and by the proposal network, whose
// probabilities the SSC pass uses to drop pixels in addition to Algorithm 1.
int launch_elimination(Ctx& c, const SolverView& sv, IterScalars* out) {
  c.learned_now = c.learned_due();
  std::vector<int*> Jp(c.Q), Ep(c.Q), Fp(c.Q);
  for (int q = 0; q < c.Q; ++q) { Jp[q] = c.s[q].J; Ep[q] = c.s[q].E; Fp[q] = c.s[q].F; }
  c.mark(6, true);
  if (c.learned_now) {
    // residual of the whole model, y' - A_J x_J = y - A x, into r (free until the next iteration)
    std::vector<ColumnSet> fw;
    std::vector<ReadmitSet> rs;
    for (int q = 0; q < c.Q; ++q) {
      Sensor& S = c.s[q];
      if (S.cnt > 0) fw.push_back(ColumnSet{c.op(q), S.J, S.cnt, q, nullptr, S.yp, S.r});
      else SADMM_CUDA_TRY(cudaMemcpyAsync(S.r, S.yp, c.KM * sizeof(float2), cudaMemcpyDeviceToDevice, c.st));
      if (S.cnt < c.N) rs.push_back(ReadmitSet{c.op(q), S.F, c.N - S.cnt, q, S.r});
    }
    if (!fw.empty())
      SADMM_TRY(launch_forward(fw.data(), (int)fw.size(), c.KM, kVX, sv, c.partial, c.partial_cap, c.st));
    SADMM_TRY(launch_frozen_lists(sv, Jp.data(), c.counts, c.mask, Fp.data(), c.counts + 2 * c.Q, c.st));
    SADMM_TRY(launch_readmit_check(rs.data(), (int)rs.size(), c.KM, sv, c.crit.readmit * c.crit.eps_p, c.mask,
                                   c.st));
    SADMM_TRY(launch_features(sv, c.k + 1, c.crit.eps_p, c.feat, c.st));
    SADMM_TRY(sadmm_cnn_forward(c.cnn, c.feat, 1, c.prob, (void*)c.st));
  }
  SADMM_TRY(launch_ssc(sv, Jp.data(), Ep.data(), c.counts, c.crit.eps_p, c.crit.freeze_mode, out, c.prob,
                       (float)c.crit.learn_theta, c.learned_now ? 1 : 0, c.st, c.ptag, c.ptally));
  c.mark(6, false);
  return SADMM_OK;
}

int launch_iteration(Ctx& c, IterScalars* out) {
  const SolverView sv = c.view();
  if (c.crit.precision > 0) {
    const bool corr = c.periodic() && (c.corr_due || c.k - c.last_corr_k >= c.crit.correct_every);
    c.mark(0, true);
    SADMM_TRY(launch_split_products_fwd(c, sv, corr));
    c.mark(0, false);
    std::vector<SpdSet> spd_w, spd_p;
    for (int q = 0; q < c.Q; ++q) {
      Sensor& S = c.s[q];
      if (S.cnt == 0) continue;
      const float2* F = S.fhl[S.cur];
      float2* part = c.spd_part + (size_t)q * c.spd_part_stride;
      if (S.woodbury)
        spd_w.push_back(SpdSet{F, S.n, reinterpret_cast<const float*>(S.r), reinterpret_cast<float*>(S.w), nullptr, q,
                               part, 0});
      else   // g from the split adjoint as an exact pair (g, g_lo)
        spd_p.push_back(SpdSet{F, S.n, S.g, nullptr, S.J, q, part, 0, nullptr, 0, S.g_lo});
    }
    c.mark(1, true);
    SADMM_TRY(launch_spd_apply(spd_w.data(), (int)spd_w.size(), false, sv, c.spd_err, c.st));
    c.mark(1, false);
    c.mark(2, true);
    SADMM_TRY(launch_split_products_adj(c, sv, corr));
    c.mark(2, false);
    c.mark(4, true);
    SADMM_TRY(launch_spd_apply(spd_p.data(), (int)spd_p.size(), true, sv, c.spd_err, c.st));
    c.mark(4, false);
    if (corr) { c.corr_due = false; c.last_corr_k = c.k; }
    c.mark(5, true);
    SADMM_TRY(launch_residuals(sv, c.crit, c.red, c.ticket, out, c.k + 1, c.st));
    c.mark(5, false);
    if (c.crit.elim) SADMM_TRY(launch_elimination(c, sv, out));
    return SADMM_OK;
  }
  std::vector<ColumnSet> fw;
  std::vector<SpdSet> spd_w, spd_p;
  std::vector<AdjointSet> adj_w, adj_p;
  std::vector<FactoredSet> ffw, fadj_w, fadj_p;    // factored representation
  const bool fac = c.use_factored();
  for (int q = 0; q < c.Q; ++q) {
    Sensor& S = c.s[q];
    if (S.cnt == 0) continue;
    fw.push_back(ColumnSet{S.A, S.J, S.cnt, q, nullptr, S.yp, S.r});
    ffw.push_back(FactoredSet{S.C, S.D, S.J, S.cnt, q, nullptr, S.yp, S.r, nullptr, nullptr});
    const float2* F = S.fhl[S.cur];
    float2* part = c.spd_part + (size_t)q * c.spd_part_stride;
    if (S.woodbury) {
      spd_w.push_back(SpdSet{F, S.n, reinterpret_cast<const float*>(S.r), reinterpret_cast<float*>(S.w), nullptr, q,
                             part, 0});
      adj_w.push_back(AdjointSet{S.A, S.J, S.cnt, q, S.w, nullptr});
      fadj_w.push_back(FactoredSet{S.C, S.D, S.J, S.cnt, q, nullptr, nullptr, nullptr, S.w, nullptr});
    } else {
      adj_p.push_back(AdjointSet{S.A, S.J, S.cnt, q, S.r, S.g, S.g_lo});
      fadj_p.push_back(FactoredSet{S.C, S.D, S.J, S.cnt, q, nullptr, nullptr, nullptr, S.r, S.g});
      // primal form: g enters H g as an exact pair (the factored entries
      // carry their own rounding, so that path passes g alone)
      spd_p.push_back(SpdSet{F, S.n, S.g, nullptr, S.J, q, part, 0, nullptr, 0, fac ? nullptr : S.g_lo});
    }
  }
  c.mark(0, true);
  if (fac)
    SADMM_TRY(launch_factored_forward(ffw.data(), (int)ffw.size(), c.M, c.K, c.N, c.vmode(), sv, c.partial,
                                      c.partial_cap, c.st));
  else
    SADMM_TRY(launch_forward(fw.data(), (int)fw.size(), c.KM, c.vmode(), sv, c.partial, c.partial_cap, c.st));
  c.mark(0, false);
  if (!spd_w.empty()) {
    c.mark(1, true);
    SADMM_TRY(launch_spd_apply(spd_w.data(), (int)spd_w.size(), false, sv, c.spd_err, c.st));
    c.mark(1, false);
    c.mark(2, true);
    if (fac)
      SADMM_TRY(launch_factored_adjoint(fadj_w.data(), (int)fadj_w.size(), c.M, c.K, c.N, true, sv, c.st));
    else
      SADMM_TRY(launch_adjoint(adj_w.data(), (int)adj_w.size(), c.KM, true, sv, c.st));
    c.mark(2, false);
  }
  if (!spd_p.empty()) {
    c.mark(3, true);
    if (fac)
      SADMM_TRY(launch_factored_adjoint(fadj_p.data(), (int)fadj_p.size(), c.M, c.K, c.N, false, sv, c.st));
    else
      SADMM_TRY(launch_adjoint(adj_p.data(), (int)adj_p.size(), c.KM, false, sv, c.st));
    c.mark(3, false);
    c.mark(4, true);
    SADMM_TRY(launch_spd_apply(spd_p.data(), (int)spd_p.size(), true, sv, c.spd_err, c.st));
    c.mark(4, false);
  }
  c.mark(5, true);
  SADMM_TRY(launch_residuals(sv, c.crit, c.red, c.ticket, out, c.k + 1, c.st));
  c.mark(5, false);
  if (c.crit.elim) SADMM_TRY(launch_elimination(c, sv, out));
  return SADMM_OK;
}

// Split-precision forward product r = y' - (A_hi + A_lo) v.  Pairs read both
// planes every iteration; the periodic modes read hi every iteration and
// refresh base_corr = y' - A_lo v only on correction iterations.
int launch_split_products_fwd(Ctx& c, const SolverView& sv, bool corr) {
  std::vector<SplitSet> a, b;
  for (int q = 0; q < c.Q; ++q) {
    Sensor& S = c.s[q];
    if (S.cnt == 0) continue;
    SplitSet x{};
    x.hi = S.hi; x.lo = S.lo; x.idx = S.J; x.n = S.cnt; x.q = q;
    if (!c.periodic()) {
      x.base = S.yp; x.out = S.r;
      a.push_back(x);
    } else {
      if (corr) {
        SplitSet l = x;
        l.base = S.yp; l.out = S.base_corr;
        b.push_back(l);
      }
      x.base = S.base_corr; x.out = S.r;
      a.push_back(x);
    }
  }
  const int kind = c.split_kind();
  if (!b.empty())
    SADMM_TRY(launch_split_forward(b.data(), (int)b.size(), c.KM, kind, 2, c.vmode(), sv, c.partial, c.partial_cap,
                                   c.st));
  return launch_split_forward(a.data(), (int)a.size(), c.KM, kind, c.periodic() ? 1 : 3, c.vmode(), sv,
                              c.partial, c.partial_cap, c.st);
}

// Split-precision adjoint g = Re((A_hi + A_lo)^H w): with the x-update epilogue
// for Woodbury-form sensors, into S.g for primal-form sensors.
int launch_split_products_adj(Ctx& c, const SolverView& sv, bool corr) {
  std::vector<SplitSet> lo_pass, upd, gout;
  for (int q = 0; q < c.Q; ++q) {
    Sensor& S = c.s[q];
    if (S.cnt == 0) continue;
    SplitSet x{};
    x.hi = S.hi; x.lo = S.lo; x.idx = S.J; x.n = S.cnt; x.q = q;
    x.w = S.woodbury ? S.w : S.r;
    if (c.periodic()) {
      if (corr) {
        SplitSet l = x;
        l.gcorr_out = S.gcorr;
        lo_pass.push_back(l);
      }
      x.gcorr_in = S.gcorr;
    }
    if (S.woodbury) upd.push_back(x);
    else { x.g = S.g; x.g_lo = S.g_lo; gout.push_back(x); }
  }
  const int kind = c.split_kind();
  const int planes = c.periodic() ? 1 : 3;
  if (!lo_pass.empty())
    SADMM_TRY(launch_split_adjoint(lo_pass.data(), (int)lo_pass.size(), c.KM, kind, 2, false, sv, c.st));
  SADMM_TRY(launch_split_adjoint(upd.data(), (int)upd.size(), c.KM, kind, planes, true, sv, c.st));
  return launch_split_adjoint(gout.data(), (int)gout.size(), c.KM, kind, planes, false, sv, c.st);
}

// Primal-form factors whose sets lost e pixels and stay in the primal form:
// H over J_new is the Schur complement of H_EE in H (the inverse of a
// principal submatrix), taken in passes of at most kDowndateMax removed
// pixels in list order; before each pass but the last, the list the pass
// leaves (J_new merged with the pixels still to be removed) is formed in
// S.Jm.  The pair copy is packed once, after the last pass.  Sensors whose
// small block H_EE is not numerically positive definite are returned in
// `failed` (they are refactored).
int primal_downdate(Ctx& c, const std::vector<int>& qs, std::vector<int>* failed) {
  if (qs.empty()) return SADMM_OK;
  SADMM_TRY(ensure_set_buffers(c));
  std::vector<int> etot(c.Q, 0), bad(c.Q, 0);
  int passes = 0;
  for (int q : qs) {
    etot[q] = c.h_counts[c.Q + q];
    passes = std::max(passes, div_up(etot[q], kDowndateMax));
  }
  for (int pass = 0; pass < passes; ++pass) {
    std::vector<PrimalDdJob> jobs;
    std::vector<int> owner, dst;
    for (int q : qs) {
      Sensor& S = c.s[q];
      const int off = pass * kDowndateMax;
      if (bad[q] || off >= etot[q]) continue;
      const int e = std::min(kDowndateMax, etot[q] - off);
      const int rest = etot[q] - off - e;          // removed by later passes
      const int* Jp = S.J;
      if (rest > 0) {
        SADMM_TRY(launch_merge_lists(S.J, S.cnt, S.E + off + e, rest, S.Jm, c.st));
        Jp = S.Jm;
      }
      const int d = (S.cur == S.full) ? (S.full + 1) % 3 : 3 - S.full - S.cur;
      PrimalDdJob j{};
      j.H = S.fb[S.cur];
      j.ldh = round_up(S.n, kTile);
      j.Hn = S.fb[d];
      j.n_new = S.cnt + rest;
      j.ldn = round_up(j.n_new, kTile);
      j.J = Jp;
      j.E = S.E + off;
      j.e = e;
      j.pos = S.pos;
      j.V = S.dinv;
      j.slot = q;
      jobs.push_back(j);
      owner.push_back(q);
      dst.push_back(d);
    }
    if (jobs.empty()) continue;
    SADMM_CUDA_TRY(cudaMemsetAsync(c.dstatus, 0, sizeof(int) * c.Q, c.st));
    SADMM_TRY(run_primal_downdate(jobs.data(), (int)jobs.size(), c.dstatus, c.st));
    SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_status, c.dstatus, sizeof(int) * c.Q, cudaMemcpyDeviceToHost, c.st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
    for (size_t i = 0; i < jobs.size(); ++i) {
      const int q = owner[i];
      Sensor& S = c.s[q];
      if (c.h_status[q]) { bad[q] = 1; failed->push_back(q); continue; }
      S.cur = dst[i];
      S.n = jobs[i].n_new;
      S.cum_dd += jobs[i].e;
    }
  }
  for (int q : qs) {
    if (bad[q]) continue;
    Sensor& S = c.s[q];
    SADMM_TRY(launch_pack_sym(S.fb[S.cur], round_up(S.n, kTile), S.n, S.fhl[S.cur], c.st));
  }
  return SADMM_OK;
}

// A Schur-complement pass costs about 2 n^2 kDowndateMax FP64 flops (n the
// factor's size before it), a refactorisation of the n_new kept pixels about
// n_new^3 (Cholesky, triangular inverse, product; the Gram runs on the tensor
// cores): the passes are taken while they are cheaper.
bool primal_downdate_cheaper(int n_old, int n_new) {
  const double e = n_old - n_new;
  return 2.0 * (double)n_old * n_old * e < (double)n_new * n_new * n_new;
}

// Columns a Woodbury factor may gain or lose by rank updates before it is
// rebuilt from scratch.  Each pass applies the Woodbury identity exactly in
// FP64, so rounding grows with the number of passes only; 2n columns (n = 2KM)
// keeps it far below the FP32 iteration's own rounding.
int refactor_after(const Ctx& c) { return 4 * c.KM; }

// After an SSC pass that shrank some sets: fold frozen pixels into y' (or
// re-average in zero mode) and refresh the factors of those sensors.
int apply_changes(Ctx& c, const std::vector<int>& changed) {
  const SolverView sv = c.view();
  if (c.crit.freeze_mode == 0) {
    std::vector<ColumnSet> fold;
    for (int q : changed) {
      Sensor& S = c.s[q];
      fold.push_back(ColumnSet{c.op(q), S.E, c.h_counts[c.Q + q], q, nullptr, S.yp, S.yp});
    }
    SADMM_TRY(launch_forward(fold.data(), (int)fold.size(), c.KM, kVX, sv, c.partial, c.partial_cap, c.st));
  } else {
    SADMM_TRY(launch_recompute_xbar(sv, c.st));
  }
  // A factor that keeps its form is downdated by the removed columns (a
  // rank-|E| Woodbury update, or the Schur complement of a primal-form
  // factor); a form change, more columns than one primal pass takes, or too
  // many accumulated downdates (rounding) refactor from scratch.
  std::vector<int> dd, pdd, full;
  for (int q : changed) {
    const Sensor& S = c.s[q];
    const int e = c.h_counts[c.Q + q];
    if (S.woodbury && S.cnt > 2 * c.KM && S.cum_dd + e <= refactor_after(c)) dd.push_back(q);
    else if (!S.woodbury && S.pos && S.cnt > 0 && S.n == S.cnt + e && primal_downdate_cheaper(S.n, S.cnt) &&
             S.cum_dd + e <= refactor_after(c))
      pdd.push_back(q);
    else full.push_back(q);
  }
  SADMM_TRY(downdate(c, dd, &full));
  SADMM_TRY(primal_downdate(c, pdd, &full));
  c.corr_due = true;        // y' and the active sets changed: refresh the lo-plane products
  return refresh(c, full, false);
}

// After a learned SSC pass: rebuild each J_q as the ordered union of the kept
// and the re-admitted pixels (flags set by the re-admission test), unfold the
// re-admitted pixels from y' (freeze mode 0) and add their columns to the
// factors (rank update of a Woodbury form, otherwise a refresh).
int readmit(Ctx& c, int* total) {
  *total = 0;
  const SolverView sv = c.view();
  std::vector<int*> Jp(c.Q), Rp(c.Q);
  for (int q = 0; q < c.Q; ++q) { Jp[q] = c.s[q].J; Rp[q] = c.s[q].R; }
  SADMM_TRY(launch_rebuild_lists(sv, Jp.data(), Rp.data(), c.mask, c.counts, c.counts + 3 * c.Q,
                                 2.0 * c.crit.eps_p, c.st, c.ptag, c.ptally));
  SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_counts, c.counts, 4 * c.Q * sizeof(int), cudaMemcpyDeviceToHost, c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  std::vector<int> added;
  std::vector<ColumnSet> unfold;
  for (int q = 0; q < c.Q; ++q) {
    Sensor& S = c.s[q];
    const int nr = c.h_counts[3 * c.Q + q];
    if (nr == 0) continue;
    added.push_back(q);
    S.cnt = c.h_counts[q];
    *total += nr;
    unfold.push_back(ColumnSet{c.op(q), S.R, nr, q, nullptr, S.yp, S.yp});
  }
  if (added.empty()) return SADMM_OK;
  if (c.crit.freeze_mode == 0)
    SADMM_TRY(launch_forward(unfold.data(), (int)unfold.size(), c.KM, kVNegX, sv, c.partial, c.partial_cap, c.st));
  std::vector<int> up, full;
  for (int q : added) {
    const Sensor& S = c.s[q];
    const int e = c.h_counts[3 * c.Q + q];
    if (S.woodbury && S.cum_dd + e <= refactor_after(c)) up.push_back(q);
    else full.push_back(q);
  }
  SADMM_TRY(downdate(c, up, &full, true));
  c.corr_due = true;
  return refresh(c, full, false);
}

double iter_bytes(const Ctx& c) {
  double b = 0.0;
  for (const Sensor& S : c.s) {
    if (S.cnt == 0) continue;
    const double per_entry = c.crit.precision == 0 ? 8.0 : (c.periodic() ? 4.0 : 8.0);
    b += 2.0 * c.KM * (double)S.cnt * per_entry + (double)sym_packed_pairs(S.n) * sizeof(float2);
  }
  return b;
}

sadmm_iter_record make_record(const Ctx& c, const IterScalars& r, int changed, int learned = 0,
                              int readmitted = 0) {
  sadmm_iter_record rec;
  rec.k = r.k; rec.gate = r.gate; rec.changed = changed;
  rec.learned = learned; rec.readmitted = readmitted;
  rec.active_total = 0;
  for (const Sensor& S : c.s) rec.active_total += S.cnt;
  rec.r_pri = r.r_pri; rec.eps_pri = r.eps_pri; rec.d = r.d; rec.eps_dual = r.eps_dual;
  rec.relchange = r.relchange;
  return rec;
}

// Reads and clears the factor apply's timeout flag; SADMM_ETIMEOUT if it was
// set.  A timed-out apply leaves its outputs unwritten, so this status takes
// precedence over a non-finite iterate that it may have caused.
int take_timeout(Ctx& c) {
  int spd_err = 0;
  SADMM_CUDA_TRY(cudaMemcpyAsync(&spd_err, c.spd_err, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  if (!spd_err) return SADMM_OK;
  SADMM_CUDA_TRY(cudaMemsetAsync(c.spd_err, 0, sizeof(int), c.st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
  set_error("factor apply: a tile copy did not complete within the wait limit");
  return SADMM_ETIMEOUT;
}

int run(Ctx& c, float* x_out, int iters, double tol, sadmm_stats* st) {
  const double t0 = now_ms();
  double t_ref = 0.0, bytes = 0.0;
  int refreshes = 0, stop_reason = 0, done = 0, learned_steps = 0, readmitted = 0;
  c.hist.clear();
  // Without elimination and without a residual-based stop nothing decided on
  // the host depends on an iteration's scalars: run the iterations back to
  // back and read all scalars once at the end.
  const bool nosync = !c.crit.elim && !(c.crit.stop == 0 && tol > 0.0) && c.crit.stop != 1;
  if (nosync && iters > 0) {
    if (c.hist_cap < iters) {
      void* p = c.dalloc((size_t)iters * sizeof(IterScalars));
      if (!p) { set_error("history buffer allocation failed"); return SADMM_ENOMEM; }
      c.hist_dev = (IterScalars*)p;
      c.hist_cap = iters;
    }
    for (int it = 0; it < iters; ++it) {
      bytes += iter_bytes(c);
      c.prof_slot = it;
      SADMM_TRY(launch_iteration(c, c.hist_dev + it));
      c.k += 1;
    }
    std::vector<IterScalars> h(iters);
    SADMM_CUDA_TRY(cudaMemcpyAsync(h.data(), c.hist_dev, iters * sizeof(IterScalars), cudaMemcpyDeviceToHost, c.st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
    c.collect();
    done = iters;
    for (int it = 0; it < iters; ++it) {
      if (h[it].nonfinite) {
        SADMM_TRY(take_timeout(c));
        set_error("non-finite value in iteration %d", h[it].k);
        return SADMM_ENONFINITE;
      }
      c.hist.push_back(make_record(c, h[it], 0));
    }
  } else {
    for (int it = 0; it < iters; ++it) {
      bytes += iter_bytes(c);
      SADMM_TRY(launch_iteration(c, c.scal));
      SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_scal, c.scal, sizeof(IterScalars), cudaMemcpyDeviceToHost, c.st));
      SADMM_CUDA_TRY(cudaMemcpyAsync(c.h_counts, c.counts, 4 * c.Q * sizeof(int), cudaMemcpyDeviceToHost, c.st));
      SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
      c.collect();
      c.k += 1;
      done += 1;
      const IterScalars& r = *c.h_scal;
      if (r.nonfinite) {
        SADMM_TRY(take_timeout(c));
        set_error("non-finite value in iteration %d", c.k);
        return SADMM_ENONFINITE;
      }
      std::vector<int> changed;
      if (c.crit.elim && (r.gate || c.learned_now)) {
        for (int q = 0; q < c.Q; ++q) {
          if (c.h_counts[c.Q + q] > 0) {
            changed.push_back(q);
            c.s[q].cnt = c.h_counts[q];
          }
        }
      }
      if (!changed.empty()) {
        const double ta = now_ms();
        c.mark(7, true);
        SADMM_TRY(apply_changes(c, changed));
        c.mark(7, false);
        SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
        c.collect();
        t_ref += now_ms() - ta;
        refreshes += 1;
      }
      int nre = 0;
      if (c.learned_now) {
        const double ta = now_ms();
        c.mark(7, true);
        SADMM_TRY(readmit(c, &nre));
        c.mark(7, false);
        SADMM_CUDA_TRY(cudaStreamSynchronize(c.st));
        c.collect();
        t_ref += now_ms() - ta;
        learned_steps += 1;
        readmitted += nre;
      }
      c.hist.push_back(make_record(c, r, (int)changed.size(), c.learned_now ? 1 : 0, nre));
      if (c.crit.stop == 0 && tol > 0.0 && r.relchange <= tol) { stop_reason = 1; break; }
      if (c.crit.stop == 1 && r.r_pri <= r.eps_pri && r.d <= r.eps_dual) { stop_reason = 2; break; }
    }
  }
  if (x_out) {
    SADMM_TRY(launch_scale(c.zbar, c.crit.consensus ? 1.f : (float)c.Q, c.xg, c.N, c.st));
    SADMM_CUDA_TRY(cudaMemcpyAsync(x_out, c.xg, c.N * sizeof(float), cudaMemcpyDefault, c.st));
  }
  SADMM_TRY(take_timeout(c));
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters = done;
    st->stop_reason = stop_reason;
    st->refreshes = refreshes;
    st->learned_steps = learned_steps;
    st->readmitted = readmitted;
    for (const Sensor& S : c.s) st->active_total += S.cnt;
    if (!c.hist.empty()) {
      const sadmm_iter_record& h = c.hist.back();
      st->r_pri = h.r_pri; st->eps_pri = h.eps_pri; st->d = h.d; st->eps_dual = h.eps_dual;
      st->relchange = h.relchange;
    }
    st->ms_total = now_ms() - t0;
    st->ms_refresh = t_ref;
    st->bytes_iter = bytes;
    std::vector<int> tally(2 * c.Q, 0);
    SADMM_CUDA_TRY(cudaMemcpy(tally.data(), c.ptally, tally.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int q = 0; q < c.Q; ++q) { st->proposed += tally[q]; st->proposed_readmitted += tally[c.Q + q]; }
  }
  return SADMM_OK;
}

bool valid_criterion(const sadmm_criterion& c) {
  return c.mu > 0.0 && c.Kp >= 1 && c.Kp <= 64 && c.eps_p >= 0.0 && c.elim >= 0 && c.elim <= 2 &&
         c.freeze_mode >= 0 && c.freeze_mode <= 1 &&
         !(c.elim == 2 && (c.learn_every < 1 || !(c.eps_p > 0.0) || !(c.learn_theta >= 0.0 && c.learn_theta <= 1.0) ||
                           !(c.readmit >= 0.0))) &&
         c.stop >= 0 && c.stop <= 1 && c.precision >= 0 && c.precision <= 4 && c.correct_every >= 1 &&
         c.ssc_every >= 1 && (c.consensus == 0 || c.consensus == 1) && !(c.consensus && c.elim == 2);
}

int valid_ctx(sadmm_t c) {
  if (!c) { set_error("null context"); return SADMM_EINVAL; }
  return SADMM_OK;
}

}  // namespace
}  // namespace sadmm

using sadmm::Ctx;
using sadmm::set_error;

struct sadmm_ctx : Ctx {};

namespace sadmm {
// Operator and current factor of sensor q (for the batched form, which keeps
// every pixel active and so uses the full-set factor).
int single_export(sadmm_t h, int q, const float2** A, const double** F, int* n, int* ld, int* woodbury) {
  if (!h || q < 0 || q >= h->Q) return SADMM_EINVAL;
  const sadmm::Sensor& S = h->s[q];
  if (!S.full_valid) { set_error("factor of sensor %d not prepared", q); return SADMM_ENOTREADY; }
  *A = S.A;
  *F = S.fb[S.full];
  int nn, wb;
  factor_dims(*h, h->N, &nn, &wb);
  *n = nn;
  *ld = round_up(nn, kTile);
  *woodbury = wb;
  return SADMM_OK;
}
}  // namespace sadmm


extern "C" {

void sadmm_default_criterion(sadmm_criterion* c) {
  if (!c) return;
  c->mu = 1.0;
  c->Kp = 5;
  c->eps_p = 1e-5;
  c->eps_abs = 1e-4;
  c->eps_rel = 1e-2;
  c->elim = 1;
  c->freeze_mode = 0;
  c->stop = 0;
  c->precision = 0;
  c->correct_every = 4;
  c->learn_every = 10;
  c->learn_theta = 0.5;
  c->readmit = 10.0;
  c->ssc_every = 1;
  c->consensus = 0;
}

int sadmm_set_allocator(sadmm_alloc_fn alloc, sadmm_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr)) {
    set_error("allocator and release must both be set or both be NULL");
    return SADMM_EINVAL;
  }
  sadmm::g_alloc.alloc = alloc;
  sadmm::g_alloc.release = release;
  sadmm::g_alloc.user = user;
  return SADMM_OK;
}

int sadmm_create(int Q, int M, int K, int N, double rho, double lambda, const sadmm_criterion* crit,
                 sadmm_t* out) {
  using namespace sadmm;
  if (!out) { set_error("out is NULL"); return SADMM_EINVAL; }
  *out = nullptr;
  sadmm_criterion c;
  if (crit) c = *crit; else sadmm_default_criterion(&c);
  const long long KM = (long long)K * M;
  if (Q < 1 || Q > kMaxSets || M < 1 || K < 1 || N < 1 || KM % 32 != 0 || KM > 16384 ||
      !(rho > 0.0) || !(lambda >= 0.0) || !valid_criterion(c) || !std::isfinite(rho) || !std::isfinite(lambda)) {
    set_error("sadmm_create: invalid sizes or parameters (Q=%d M=%d K=%d N=%d rho=%g lambda=%g)", Q, M,
              K, N, rho, lambda);
    return SADMM_EINVAL;
  }
  if ((long long)N * KM * 8 > (1ll << 40)) { set_error("operator too large"); return SADMM_EINVAL; }
  sadmm_ctx* ctx = new (std::nothrow) sadmm_ctx();
  if (!ctx) return SADMM_ENOMEM;
  ctx->Q = Q; ctx->M = M; ctx->K = K; ctx->N = N; ctx->KM = (int)KM;
  ctx->rho = rho; ctx->lam = lambda; ctx->crit = c;
  ctx->alloc = g_alloc;
  ctx->npad_max = round_up(std::min<long long>(N, 2 * KM), kTile);
  ctx->s.resize(Q);
  bool ok = true;
  auto A = [&](size_t b) { void* p = ctx->dalloc(b); if (!p) ok = false; return p; };
  const size_t fbytes = (size_t)ctx->npad_max * ctx->npad_max * sizeof(double);
  const size_t pbytes = sym_packed_pairs(ctx->npad_max) * sizeof(float2);
  for (int q = 0; q < Q && ok; ++q) {
    Sensor& S = ctx->s[q];
    S.A = (float2*)A((size_t)N * KM * sizeof(float2));
    S.y = (float2*)A(KM * sizeof(float2));
    S.yp = (float2*)A(KM * sizeof(float2));
    S.r = (float2*)A(KM * sizeof(float2));
    S.w = (float2*)A(KM * sizeof(float2));
    S.g = (float*)A((size_t)N * sizeof(float));
    S.g_lo = (float*)A((size_t)N * sizeof(float));
    if (c.elim > 0) S.pos = (int*)A((size_t)N * sizeof(int));
    S.J = (int*)A((size_t)N * sizeof(int));
    S.E = (int*)A((size_t)N * sizeof(int));
    S.F = (int*)A((size_t)N * sizeof(int));
    S.R = (int*)A((size_t)N * sizeof(int));
    for (int b = 0; b < 2; ++b) S.fb[b] = (double*)A(fbytes);   // full-set factor and its scratch
    S.fhl[0] = (float2*)A(pbytes);
    S.dinv = (double*)A((size_t)ctx->npad_max * kTile * sizeof(double));
    S.dd = (double*)A(downdate_scratch_doubles(2 * (int)KM) * sizeof(double));
    if (c.precision > 0) {
      S.hi = (uint16_t*)A((size_t)N * KM * 2 * sizeof(uint16_t));
      S.lo = (uint16_t*)A((size_t)N * KM * 2 * sizeof(uint16_t));
      S.P = (float2*)A((size_t)N * KM * sizeof(float2));
      S.base_corr = (float2*)A(KM * sizeof(float2));
      S.gcorr = (float*)A((size_t)N * sizeof(float));
    }
  }
  const size_t QN = (size_t)Q * N;
  ctx->x = (float*)A(QN * sizeof(float));
  ctx->xbar = (float*)A(N * sizeof(float));
  ctx->zbar = (float*)A(N * sizeof(float));
  ctx->sd = (float*)A(N * sizeof(float));
  ctx->xg = (float*)A(N * sizeof(float));
  ctx->ring = (float*)A((size_t)c.Kp * QN * sizeof(float));
  ctx->ring_kp = c.Kp;
  if (c.consensus) ctx->u = (float*)A(QN * sizeof(float));
  ctx->iota = (int*)A(N * sizeof(int));
  ctx->partial_cap = 0;
  for (int ns = 1; ns <= Q; ++ns) {  // any subset of sensors may be launched together
    ctx->partial_cap = std::max(ctx->partial_cap, forward_partial_bytes(ns, (int)KM, N));
    if (factored_supported(K)) ctx->partial_cap = std::max(ctx->partial_cap, factored_partial_bytes(ns, M, K, N));
    if (c.precision > 0) ctx->partial_cap = std::max(ctx->partial_cap, split_partial_bytes(ns, (int)KM, N));
  }
  ctx->partial = (float2*)A(ctx->partial_cap);
  ctx->spd_part_stride = sym_part_pairs(ctx->npad_max);
  ctx->spd_part = (float2*)A((size_t)Q * ctx->spd_part_stride * sizeof(float2));
  ctx->spd_err = (int*)A(sizeof(int));
  if (c.elim > 0 && ctx->npad_max == 2 * KM) {   // Woodbury-form factors get rank updates
    const int n = 2 * (int)KM;
    ctx->dd.U = (float*)A((size_t)Q * n * 16 * sizeof(float));
    ctx->dd.dptrs = (void**)A((size_t)2 * Q * sizeof(void*));
    ctx->dd.part = (float2*)A(std::max((size_t)Q * multi_apply_part_pairs(n), (size_t)kMaxSets * sym_part_pairs(n)) *
                              sizeof(float2));
  }
  ctx->red = (double*)A((size_t)residual_blocks(N) * 8 * sizeof(double));
  ctx->ticket = (unsigned int*)A(sizeof(unsigned int));
  ctx->scal = (IterScalars*)A(sizeof(IterScalars));
  ctx->counts = (int*)A(4 * Q * sizeof(int));
  ctx->feat = (float*)A((size_t)6 * N * sizeof(float));
  ctx->prob = (float*)A((size_t)N * sizeof(float));
  ctx->mask = (uint8_t*)A((size_t)Q * 2 * N);
  ctx->ptag = (uint8_t*)A((size_t)Q * N);
  ctx->ptally = (int*)A((size_t)2 * Q * sizeof(int));
  ctx->dstatus = (int*)A(Q * sizeof(int));
  if (ok && c.elim > 0 && ensure_set_buffers(*ctx) != SADMM_OK) ok = false;
  if (ok && (cudaMallocHost(&ctx->h_scal, sizeof(IterScalars)) != cudaSuccess ||
             cudaMallocHost(&ctx->h_counts, 4 * Q * sizeof(int)) != cudaSuccess ||
             cudaMallocHost(&ctx->h_status, Q * sizeof(int)) != cudaSuccess))
    ok = false;
  if (!ok) {
    cudaGetLastError();
    set_error("sadmm_create: device allocation failed");
    ctx->release_all();
    delete ctx;
    return SADMM_ENOMEM;
  }
  iota_kernel<<<div_up(N, 256), 256, 0, ctx->st>>>(ctx->iota, N);
  if (cudaMemsetAsync(ctx->ticket, 0, sizeof(unsigned int), ctx->st) != cudaSuccess ||
      cudaMemsetAsync(ctx->spd_err, 0, sizeof(int), ctx->st) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(ctx->st) != cudaSuccess) {
    set_error("sadmm_create: initialisation failed");
    ctx->release_all();
    delete ctx;
    return SADMM_ECUDA;
  }
  *out = ctx;
  return SADMM_OK;
}

int sadmm_set_stream(sadmm_t ctx, void* stream) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  ctx->st = (cudaStream_t)stream;
  return SADMM_OK;
}

int sadmm_set_criterion(sadmm_t ctx, const sadmm_criterion* crit) {
  using namespace sadmm;
  SADMM_TRY(valid_ctx(ctx));
  if (!crit || !valid_criterion(*crit)) { set_error("sadmm_set_criterion: invalid criterion"); return SADMM_EINVAL; }
  const sadmm_criterion c = *crit;
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  const size_t N = ctx->N, KM = ctx->KM, QN = (size_t)ctx->Q * N;
  bool ok = true;
  auto A = [&](size_t b) { void* p = ctx->dalloc(b); if (!p) ok = false; return p; };
  // buffers the new knobs need that the context was created without
  if (c.Kp > ctx->ring_kp) {
    ctx->ring = (float*)A((size_t)c.Kp * QN * sizeof(float));
    ctx->ring_kp = c.Kp;
  }
  if (c.consensus && !ctx->u) ctx->u = (float*)A(QN * sizeof(float));
  const int old_kind = ctx->crit.precision > 0 ? ctx->split_kind() : -1;
  for (int q = 0; q < ctx->Q && ok; ++q) {
    Sensor& S = ctx->s[q];
    if (c.elim > 0 && !S.pos) S.pos = (int*)A(N * sizeof(int));
    if (c.precision > 0 && !S.hi) {
      S.hi = (uint16_t*)A(N * KM * 2 * sizeof(uint16_t));
      S.lo = (uint16_t*)A(N * KM * 2 * sizeof(uint16_t));
      S.P = (float2*)A(N * KM * sizeof(float2));
      S.base_corr = (float2*)A(KM * sizeof(float2));
      S.gcorr = (float*)A(N * sizeof(float));
    }
  }
  if (ok && c.elim > 0 && ctx->npad_max == 2 * (int)KM && !ctx->dd.U) {
    const int n = 2 * (int)KM;
    ctx->dd.U = (float*)A((size_t)ctx->Q * n * 16 * sizeof(float));
    ctx->dd.dptrs = (void**)A((size_t)2 * ctx->Q * sizeof(void*));
    ctx->dd.part = (float2*)A(std::max((size_t)ctx->Q * multi_apply_part_pairs(n),
                                       (size_t)kMaxSets * sym_part_pairs(n)) * sizeof(float2));
  }
  if (ok && c.precision > 0) {
    size_t need = 0;
    for (int ns = 1; ns <= ctx->Q; ++ns) need = std::max(need, split_partial_bytes(ns, (int)KM, (int)N));
    if (need > ctx->partial_cap) {
      ctx->partial = (float2*)A(need);
      ctx->partial_cap = need;
    }
  }
  if (ok && c.elim > 0 && ensure_set_buffers(*ctx) != SADMM_OK) ok = false;
  if (!ok) {
    cudaGetLastError();
    set_error("sadmm_set_criterion: device allocation failed");
    return SADMM_ENOMEM;
  }
  const bool mu_changed = c.mu != ctx->crit.mu;
  ctx->crit = c;
  if (c.precision > 0 && ctx->split_kind() != old_kind)
    for (int q = 0; q < ctx->Q; ++q)
      if (ctx->s[q].op_set)
        SADMM_TRY(launch_split_convert(reinterpret_cast<const float*>(ctx->s[q].A), N * KM * 2, ctx->split_kind(),
                                       ctx->s[q].hi, ctx->s[q].lo, ctx->st, reinterpret_cast<float*>(ctx->s[q].P)));
  if (mu_changed)
    for (Sensor& S : ctx->s) S.full_valid = false;
  ctx->corr_due = true;
  ctx->last_corr_k = 0;
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_set_lambda(sadmm_t ctx, double lambda) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) { set_error("sadmm_set_lambda: lambda must be finite and >= 0"); return SADMM_EINVAL; }
  ctx->lam = lambda;
  return SADMM_OK;
}

int sadmm_set_operator(sadmm_t ctx, int q, const float* A_q) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (q < 0 || q >= ctx->Q || !A_q) { set_error("sadmm_set_operator: bad sensor or pointer"); return SADMM_EINVAL; }
  sadmm::Sensor& S = ctx->s[q];
  S.factored = false;
  SADMM_CUDA_TRY(cudaMemcpyAsync(S.A, A_q, (size_t)ctx->N * ctx->KM * sizeof(float2), cudaMemcpyDefault, ctx->st));
  if (ctx->crit.precision > 0)
    SADMM_TRY(sadmm::launch_split_convert(reinterpret_cast<const float*>(S.A), (size_t)ctx->N * ctx->KM * 2,
                                          ctx->split_kind(), S.hi, S.lo, ctx->st, reinterpret_cast<float*>(S.P)));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  S.op_set = true;
  S.full_valid = false;
  return SADMM_OK;
}

int sadmm_set_operator_delays(sadmm_t ctx, int q, const double* tau, double f0, double df) {
  using namespace sadmm;
  SADMM_TRY(valid_ctx(ctx));
  if (q < 0 || q >= ctx->Q || !tau || !std::isfinite(f0) || !std::isfinite(df)) {
    set_error("sadmm_set_operator_delays: bad sensor, pointer or frequency");
    return SADMM_EINVAL;
  }
  if (!factored_supported(ctx->K)) {
    set_error("sadmm_set_operator_delays: needs K = 16, 32, 64, 128, 256 or 512 (K=%d)", ctx->K);
    return SADMM_EINVAL;
  }
  Sensor& S = ctx->s[q];
  const size_t MN = (size_t)ctx->M * ctx->N;
  if (!S.tau) {
    S.tau = (double*)ctx->dalloc(MN * sizeof(double));
    S.C = (float2*)ctx->dalloc(MN * (ctx->K / kFacB) * sizeof(float2));
    S.D = (float2*)ctx->dalloc(MN * kFacB * sizeof(float2));
    if (!S.tau || !S.C || !S.D) { set_error("sadmm_set_operator_delays: device allocation failed"); return SADMM_ENOMEM; }
  }
  S.factored = false;
  SADMM_CUDA_TRY(cudaMemcpyAsync(S.tau, tau, MN * sizeof(double), cudaMemcpyDefault, ctx->st));
  SADMM_TRY(operator_tables(S.tau, ctx->M, ctx->K, ctx->N, f0, df, S.A, S.C, S.D, ctx->st));
  if (ctx->crit.precision > 0)
    SADMM_TRY(launch_split_convert(reinterpret_cast<const float*>(S.A), (size_t)ctx->N * ctx->KM * 2,
                                   ctx->split_kind(), S.hi, S.lo, ctx->st, reinterpret_cast<float*>(S.P)));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  S.op_set = true;
  S.full_valid = false;
  S.factored = true;
  return SADMM_OK;
}

int sadmm_backprojection(sadmm_t ctx, const float* const* y, float* out) {
  using namespace sadmm;
  SADMM_TRY(valid_ctx(ctx));
  if (!y || !out) { set_error("sadmm_backprojection: bad arguments"); return SADMM_EINVAL; }
  for (int q = 0; q < ctx->Q; ++q) {
    if (!y[q]) { set_error("sadmm_backprojection: y[%d] is NULL", q); return SADMM_EINVAL; }
    if (!ctx->s[q].op_set) { set_error("operator of sensor %d not set", q); return SADMM_ENOTREADY; }
  }
  const bool fac = ctx->use_factored();
  const size_t KM = ctx->KM, N = ctx->N;
  if (!ctx->bp_y) {
    ctx->bp_y = (float2*)ctx->dalloc((size_t)ctx->Q * 2 * KM * sizeof(float2));
    ctx->bp_g = (float*)ctx->dalloc((size_t)ctx->Q * 2 * N * sizeof(float));
    ctx->bp_out = (float*)ctx->dalloc(N * sizeof(float));
    if (!ctx->bp_y || !ctx->bp_g || !ctx->bp_out) { set_error("sadmm_backprojection: device allocation failed"); return SADMM_ENOMEM; }
  }
  std::vector<AdjointSet> as;
  std::vector<FactoredSet> fs;
  for (int q = 0; q < ctx->Q; ++q) {
    float2* yq = ctx->bp_y + (size_t)q * 2 * KM;
    SADMM_CUDA_TRY(cudaMemcpyAsync(yq, y[q], KM * sizeof(float2), cudaMemcpyDefault, ctx->st));
    SADMM_TRY(launch_bp_rotate(yq, yq + KM, KM, ctx->st));
    const Sensor& S = ctx->s[q];
    for (int part = 0; part < 2; ++part) {
      const float2* w = yq + part * KM;
      float* g = ctx->bp_g + ((size_t)q * 2 + part) * N;
      as.push_back(AdjointSet{S.A, ctx->iota, (int)N, q, w, g});
      fs.push_back(FactoredSet{S.C, S.D, ctx->iota, (int)N, q, nullptr, nullptr, nullptr, w, g});
    }
  }
  SolverView sv{};
  for (size_t i0 = 0; i0 < as.size(); i0 += kMaxSets) {
    const int n = (int)std::min<size_t>(kMaxSets, as.size() - i0);
    if (fac) SADMM_TRY(launch_factored_adjoint(fs.data() + i0, n, ctx->M, ctx->K, ctx->N, false, sv, ctx->st));
    else SADMM_TRY(launch_adjoint(as.data() + i0, n, ctx->KM, false, sv, ctx->st));
  }
  SADMM_TRY(launch_bp_combine(ctx->bp_g, ctx->Q, ctx->N, ctx->bp_out, ctx->st));
  SADMM_CUDA_TRY(cudaMemcpyAsync(out, ctx->bp_out, N * sizeof(float), cudaMemcpyDefault, ctx->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_set_products(sadmm_t ctx, int mode) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (mode < SADMM_PRODUCTS_AUTO || mode > SADMM_PRODUCTS_FACTORED) {
    sadmm::set_error("sadmm_set_products: mode %d is not one of 0, 1, 2", mode);
    return SADMM_EINVAL;
  }
  ctx->products = mode;
  return SADMM_OK;
}

int sadmm_prepare(sadmm_t ctx) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  return sadmm::prepare(*ctx);
}

int sadmm_solve(sadmm_t ctx, const float* const* y, float* x_out, int iters, double tol, sadmm_stats* st) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (!y || iters < 0) { set_error("sadmm_solve: bad arguments"); return SADMM_EINVAL; }
  for (int q = 0; q < ctx->Q; ++q)
    if (!y[q]) { set_error("sadmm_solve: y[%d] is NULL", q); return SADMM_EINVAL; }
  SADMM_TRY(sadmm::prepare(*ctx));
  for (int q = 0; q < ctx->Q; ++q)
    SADMM_CUDA_TRY(cudaMemcpyAsync(ctx->s[q].y, y[q], ctx->KM * sizeof(float2), cudaMemcpyDefault, ctx->st));
  SADMM_TRY(sadmm::reset_state(*ctx));
  return sadmm::run(*ctx, x_out, iters, tol, st);
}

int sadmm_resume(sadmm_t ctx, float* x_out, int iters, double tol, sadmm_stats* st) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (iters < 0) { set_error("sadmm_resume: bad arguments"); return SADMM_EINVAL; }
  SADMM_TRY(sadmm::prepare(*ctx));
  return sadmm::run(*ctx, x_out, iters, tol, st);
}

int sadmm_get_xq(sadmm_t ctx, int q, float* out) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (q < 0 || q >= ctx->Q || !out) { set_error("sadmm_get_xq: bad arguments"); return SADMM_EINVAL; }
  SADMM_CUDA_TRY(cudaMemcpyAsync(out, ctx->x + (size_t)q * ctx->N, ctx->N * sizeof(float), cudaMemcpyDefault, ctx->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_get_active(sadmm_t ctx, int q, int* idx, int* count) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (q < 0 || q >= ctx->Q || !count) { set_error("sadmm_get_active: bad arguments"); return SADMM_EINVAL; }
  *count = ctx->s[q].cnt;
  if (idx && ctx->s[q].cnt > 0)
    SADMM_CUDA_TRY(cudaMemcpyAsync(idx, ctx->s[q].J, ctx->s[q].cnt * sizeof(int), cudaMemcpyDefault, ctx->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_history(sadmm_t ctx, sadmm_iter_record* out, int cap) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  const int n = (int)std::min<size_t>(cap < 0 ? 0 : cap, ctx->hist.size());
  if (n > 0 && out) memcpy(out, ctx->hist.data(), n * sizeof(sadmm_iter_record));
  return out ? n : (int)ctx->hist.size();
}

// State blob: header, x (QN), x_bar, z_bar, s (N each), ring (Kp Q N), counts
// (Q int32), J (Q x N int32, first counts[q] valid), y' (Q x KM complex64).
namespace {
struct StateHeader {
  uint64_t magic;
  int32_t Q, N, KM, Kp, k, pad;
};
size_t state_bytes(const Ctx& c) {
  const size_t QN = (size_t)c.Q * c.N;
  return sizeof(StateHeader) + QN * 4 + 3 * (size_t)c.N * 4 + (size_t)c.crit.Kp * QN * 4 + c.Q * 4 +
         QN * 4 + (size_t)c.Q * c.KM * 8 + (c.crit.consensus ? QN * 4 : 0);
}
}  // namespace

int sadmm_get_state(sadmm_t ctx, void* buf, size_t* bytes) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (!bytes) { set_error("bytes is NULL"); return SADMM_EINVAL; }
  const size_t need = state_bytes(*ctx);
  if (!buf) { *bytes = need; return SADMM_OK; }
  if (*bytes < need) { set_error("state buffer too small (%zu < %zu)", *bytes, need); return SADMM_EINVAL; }
  *bytes = need;
  char* p = (char*)buf;
  StateHeader h{sadmm::kStateMagic, ctx->Q, ctx->N, ctx->KM, ctx->crit.Kp, ctx->k, 0};
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  const size_t QN = (size_t)ctx->Q * ctx->N;
  auto d2h = [&](const void* src, size_t b) -> int {
    SADMM_CUDA_TRY(cudaMemcpyAsync(p, src, b, cudaMemcpyDeviceToHost, ctx->st));
    p += b;
    return SADMM_OK;
  };
  SADMM_TRY(d2h(ctx->x, QN * 4));
  SADMM_TRY(d2h(ctx->xbar, ctx->N * 4));
  SADMM_TRY(d2h(ctx->zbar, ctx->N * 4));
  SADMM_TRY(d2h(ctx->sd, ctx->N * 4));
  SADMM_TRY(d2h(ctx->ring, (size_t)ctx->crit.Kp * QN * 4));
  for (int q = 0; q < ctx->Q; ++q) { memcpy(p, &ctx->s[q].cnt, 4); p += 4; }
  for (int q = 0; q < ctx->Q; ++q) SADMM_TRY(d2h(ctx->s[q].J, (size_t)ctx->N * 4));
  for (int q = 0; q < ctx->Q; ++q) SADMM_TRY(d2h(ctx->s[q].yp, (size_t)ctx->KM * 8));
  if (ctx->crit.consensus) SADMM_TRY(d2h(ctx->u, QN * 4));     // consensus duals last
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_set_state(sadmm_t ctx, const void* buf, size_t bytes) {
  using namespace sadmm;
  SADMM_TRY(valid_ctx(ctx));
  if (!buf || bytes != state_bytes(*ctx)) { set_error("sadmm_set_state: size mismatch"); return SADMM_EINVAL; }
  StateHeader h;
  memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.Q != ctx->Q || h.N != ctx->N || h.KM != ctx->KM || h.Kp != ctx->crit.Kp) {
    set_error("sadmm_set_state: incompatible state");
    return SADMM_EINVAL;
  }
  SADMM_TRY(prepare(*ctx));
  const char* p = (const char*)buf + sizeof h;
  const size_t QN = (size_t)ctx->Q * ctx->N;
  const char* ringp = p + QN * 4 + 3 * (size_t)ctx->N * 4;
  const char* cntp = ringp + (size_t)ctx->crit.Kp * QN * 4;
  const char* Jp = cntp + ctx->Q * 4;
  const char* ypp = Jp + QN * 4;
  std::vector<int> cnt(ctx->Q);
  memcpy(cnt.data(), cntp, ctx->Q * 4);
  // ring entries of inactive pixels must read as zero updates
  std::vector<float> ring((size_t)ctx->crit.Kp * QN);
  memcpy(ring.data(), ringp, ring.size() * 4);
  std::vector<int> J(QN);
  memcpy(J.data(), Jp, QN * 4);
  for (int q = 0; q < ctx->Q; ++q) {
    if (cnt[q] < 0 || cnt[q] > ctx->N) { set_error("sadmm_set_state: bad count"); return SADMM_EINVAL; }
    std::vector<char> act(ctx->N, 0);
    int prev = -1;
    for (int i = 0; i < cnt[q]; ++i) {
      const int v = J[(size_t)q * ctx->N + i];
      if (v <= prev || v >= ctx->N) { set_error("sadmm_set_state: active set not sorted/unique"); return SADMM_EINVAL; }
      act[v] = 1;
      prev = v;
    }
    for (int i = 0; i < ctx->N; ++i)
      if (!act[i])
        for (int t = 0; t < ctx->crit.Kp; ++t) ring[((size_t)t * ctx->Q + q) * ctx->N + i] = 0.f;
  }
  auto h2d = [&](void* dst, const void* src, size_t b) -> int {
    SADMM_CUDA_TRY(cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, ctx->st));
    return SADMM_OK;
  };
  SADMM_TRY(h2d(ctx->x, p, QN * 4));
  SADMM_TRY(h2d(ctx->xbar, p + QN * 4, ctx->N * 4));
  SADMM_TRY(h2d(ctx->zbar, p + QN * 4 + ctx->N * 4, ctx->N * 4));
  SADMM_TRY(h2d(ctx->sd, p + QN * 4 + 2 * (size_t)ctx->N * 4, ctx->N * 4));
  SADMM_TRY(h2d(ctx->ring, ring.data(), ring.size() * 4));
  if (ctx->crit.consensus) SADMM_TRY(h2d(ctx->u, ypp + (size_t)ctx->Q * ctx->KM * 8, QN * 4));
  std::vector<int> counts(2 * ctx->Q, 0);
  std::vector<int> changed;
  for (int q = 0; q < ctx->Q; ++q) {
    Sensor& S = ctx->s[q];
    SADMM_TRY(h2d(S.J, J.data() + (size_t)q * ctx->N, (size_t)ctx->N * 4));
    SADMM_TRY(h2d(S.yp, ypp + (size_t)q * ctx->KM * 8, (size_t)ctx->KM * 8));
    S.cnt = cnt[q];
    counts[q] = cnt[q];
    if (cnt[q] == ctx->N) {
      S.cur = S.full;
      S.cum_dd = 0;
      factor_dims(*ctx, ctx->N, &S.n, &S.woodbury);
    } else {
      changed.push_back(q);
    }
  }
  SADMM_TRY(h2d(ctx->counts, counts.data(), counts.size() * 4));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  ctx->k = h.k;
  ctx->corr_due = true;
  return refresh(*ctx, changed, false);
}

int sadmm_set_eliminator(sadmm_t ctx, const float* params, int H, int W) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  if (!params) {
    if (ctx->cnn) sadmm_cnn_destroy(ctx->cnn);
    ctx->cnn = nullptr;
    return SADMM_OK;
  }
  if (H < 1 || W < 1 || (long long)H * W != ctx->N) {
    set_error("sadmm_set_eliminator: grid %d x %d does not hold N = %d pixels", H, W, ctx->N);
    return SADMM_EINVAL;
  }
  if (ctx->cnn && (ctx->cnn_H != H || ctx->cnn_W != W)) {
    sadmm_cnn_destroy(ctx->cnn);
    ctx->cnn = nullptr;
  }
  if (!ctx->cnn) {
    SADMM_TRY(sadmm_cnn_create(H, W, 1, &ctx->cnn));
    ctx->cnn_H = H;
    ctx->cnn_W = W;
  }
  return sadmm_cnn_set_params(ctx->cnn, params);
}

int sadmm_features(sadmm_t ctx, float* out) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  if (!out) { set_error("sadmm_features: out is NULL"); return SADMM_EINVAL; }
  SADMM_TRY(sadmm::launch_features(ctx->view(), ctx->k, ctx->crit.eps_p, ctx->feat, ctx->st));
  SADMM_CUDA_TRY(cudaMemcpyAsync(out, ctx->feat, (size_t)6 * ctx->N * sizeof(float), cudaMemcpyDefault, ctx->st));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  return SADMM_OK;
}

int sadmm_set_profiling(sadmm_t ctx, int on) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  SADMM_CUDA_TRY(cudaStreamSynchronize(ctx->st));
  ctx->prof = on != 0;
  for (int p = 0; p < SADMM_NUM_PHASES; ++p) {
    ctx->prof_ms[p] = 0.0;
    ctx->prof_n[p] = 0;
  }
  std::fill(ctx->ev_used.begin(), ctx->ev_used.end(), 0);
  ctx->prof_slot = 0;
  return SADMM_OK;
}

int sadmm_profile(sadmm_t ctx, double* ms, long long* launches, int cap) {
  SADMM_TRY(sadmm::valid_ctx(ctx));
  const int n = std::max(0, std::min(cap, SADMM_NUM_PHASES));
  for (int p = 0; p < n; ++p) {
    if (ms) ms[p] = ctx->prof_ms[p];
    if (launches) launches[p] = ctx->prof_n[p];
  }
  return n;
}

long long sadmm_launch_count(void) { return sadmm::g_launches.load(); }

void sadmm_destroy(sadmm_t ctx) {
  if (!ctx) return;
  ctx->release_all();
  delete ctx;
}

const char* sadmm_strerror(int status) {
  switch (status) {
    case SADMM_OK: return "ok";
    case SADMM_EINVAL: return "invalid argument";
    case SADMM_ENOMEM: return "out of memory";
    case SADMM_ECUDA: return "CUDA error";
    case SADMM_ETIMEOUT: return "device wait timed out";
    case SADMM_ENOTREADY: return "operator not set";
    case SADMM_ENONFINITE: return "non-finite value";
    default: return "unknown status";
  }
}

const char* sadmm_last_error(void) { return sadmm::g_err.c_str(); }

// ---------------------------------------------------------------- kernel level
int sadmm_forward(const float* A, int KM, int N, const int* idx, int nidx, const float* v,
                  const float* base, float* r, void* stream) {
  using namespace sadmm;
  if (!A || !r || KM <= 0 || KM % 2 != 0 || N <= 0 || nidx < 0 || (nidx > 0 && (!idx || !v))) {
    set_error("sadmm_forward: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ColumnSet cs{(const float2*)A, idx, nidx, 0, v, (const float2*)base, (float2*)r};
  SolverView sv{};
  const size_t cap = forward_partial_bytes(1, KM, std::max(nidx, 1));
  void* part = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&part, cap, st));
  int rc = launch_forward(&cs, 1, KM, kVExplicit, sv, (float2*)part, cap, st);
  cudaError_t e = cudaFreeAsync(part, st);
  if (rc != SADMM_OK) return rc;
  SADMM_CUDA_TRY(e);
  return SADMM_OK;
}

int sadmm_adjoint(const float* A, int KM, int N, const int* idx, int nidx, const float* w, float* g,
                  void* stream) {
  using namespace sadmm;
  if (!A || !w || KM <= 0 || KM % 2 != 0 || KM > 16384 || N <= 0 || nidx < 0 ||
      (nidx > 0 && (!idx || !g))) {
    set_error("sadmm_adjoint: bad arguments");
    return SADMM_EINVAL;
  }
  AdjointSet as{(const float2*)A, idx, nidx, 0, (const float2*)w, g};
  SolverView sv{};
  return launch_adjoint(&as, 1, KM, false, sv, (cudaStream_t)stream);
}

int sadmm_factor(const float* A, int KM, int N, const int* idx, int nidx, double mu, double rho,
                 double* F, int ldf, int* form, void* stream) {
  using namespace sadmm;
  if (!A || !idx || !F || KM <= 0 || KM % 32 != 0 || nidx <= 0 || !(rho > 0.0) || !(mu > 0.0)) {
    set_error("sadmm_factor: bad arguments");
    return SADMM_EINVAL;
  }
  const int wb = nidx > 2 * KM ? 1 : 0;
  const int n = wb ? 2 * KM : nidx;
  const int npad = round_up(n, kTile);
  if (ldf != npad) { set_error("sadmm_factor: ldf must equal roundup(n, 64) = %d", npad); return SADMM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  void *tmp = nullptr, *dinv = nullptr, *status = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)npad * npad * sizeof(double), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&dinv, (size_t)npad * kTile * sizeof(double), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&status, sizeof(int), st));
  SADMM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  FactorJob j{(const float2*)A, idx, nidx, n, npad, wb, F, (double*)tmp, (double*)dinv};
  int rc = run_factor(&j, 1, KM, mu, rho, (int*)status, st);
  int hs = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(tmp, st);
  cudaFreeAsync(dinv, st);
  cudaFreeAsync(status, st);
  if (rc != SADMM_OK) return rc;
  if (hs == 2) { set_error("sadmm_factor: a bounded wait of the tensor-core Gram timed out"); return SADMM_ETIMEOUT; }
  if (hs) { set_error("sadmm_factor: matrix not positive definite"); return SADMM_ENONFINITE; }
  if (form) *form = wb;
  return SADMM_OK;
}

int sadmm_gram(const float* A, int KM, int N, const int* idx, int nidx, double mu, double rho, int method,
               double* F, int ldf, int* form, void* stream) {
  using namespace sadmm;
  if (!A || !idx || !F || KM <= 0 || KM % 2 != 0 || N <= 0 || nidx <= 0 || nidx > N || !(rho >= 0.0) ||
      !(mu > 0.0) || (method != 0 && method != 1) || (method == 1 && KM % 8 != 0)) {
    set_error("sadmm_gram: bad arguments");
    return SADMM_EINVAL;
  }
  const int wb = nidx > 2 * KM ? 1 : 0;
  const int n = wb ? 2 * KM : nidx;
  const int npad = round_up(n, kTile);
  if (ldf != npad) { set_error("sadmm_gram: ldf must equal roundup(n, 64) = %d", npad); return SADMM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  void* status = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&status, sizeof(int), st));
  int rc = cudaMemsetAsync(status, 0, sizeof(int), st) == cudaSuccess ? SADMM_OK : SADMM_ECUDA;
  FactorJob j{(const float2*)A, idx, nidx, n, npad, wb, F, nullptr, nullptr};
  if (rc == SADMM_OK) rc = run_gram(j, KM, mu, rho, (int*)status, st, method);
  int hs = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaError_t fe = cudaFreeAsync(status, st);
  if (rc != SADMM_OK) return rc;
  SADMM_CUDA_TRY(fe);
  if (hs) { set_error("sadmm_gram: a bounded wait of the tensor-core Gram timed out"); return SADMM_ETIMEOUT; }
  if (form) *form = wb;
  return SADMM_OK;
}

int sadmm_factor_downdate(const float* A, int KM, const int* E, int e, double mu, double* W,
                          void* stream) {
  return sadmm_factor_update(A, KM, E, e, mu, 1, W, stream);
}

int sadmm_factor_update(const float* A, int KM, const int* E, int e, double mu, int sign, double* W,
                        void* stream) {
  using namespace sadmm;
  if (!A || !W || KM <= 0 || KM % 32 != 0 || e < 0 || (e > 0 && !E) || !(mu > 0.0) ||
      (sign != 1 && sign != -1)) {
    set_error("sadmm_factor_update: bad arguments");
    return SADMM_EINVAL;
  }
  if (e == 0) return SADMM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = 2 * KM;
  void *P = nullptr, *dd = nullptr, *status = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&P, (size_t)n * kDowndateMax * sizeof(double), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&dd, downdate_scratch_doubles(n) * sizeof(double), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&status, sizeof(int), st));
  SADMM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  int rc = SADMM_OK;
  for (int off = 0; off < e && rc == SADMM_OK; off += kDowndateMax) {
    DowndateJob j{(const float2*)A, E + off, std::min(kDowndateMax, e - off), n, W, W, (double*)P,
                  (double*)dd, (double*)dd + (size_t)div_up(n, 256) * kDowndateMax * kDowndateMax, 0, sign};
    rc = run_downdate(&j, 1, KM, mu, (int*)status, st);
  }
  int hs = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(P, st);
  cudaFreeAsync(dd, st);
  cudaFreeAsync(status, st);
  if (rc != SADMM_OK) return rc;
  if (hs) { set_error("sadmm_factor_update: updated system not positive definite"); return SADMM_ENONFINITE; }
  return SADMM_OK;
}

int sadmm_split_operator(const float* A, size_t n_complex, int kind, void* hi, void* lo, void* stream) {
  using namespace sadmm;
  if (!A || !hi || !lo || (kind != kSplitBF16 && kind != kSplitFP16)) {
    set_error("sadmm_split_operator: bad arguments");
    return SADMM_EINVAL;
  }
  return launch_split_convert(A, 2 * n_complex, kind, (uint16_t*)hi, (uint16_t*)lo, (cudaStream_t)stream);
}

int sadmm_forward_split(const void* hi, const void* lo, int kind, int planes, int KM, int N, const int* idx,
                        int nidx, const float* v, const float* base, float* r, void* stream) {
  using namespace sadmm;
  if (!r || KM <= 0 || KM % 4 != 0 || N <= 0 || nidx < 0 || (nidx > 0 && (!idx || !v)) ||
      planes < 1 || planes > 3 || ((planes & 1) && !hi) || ((planes & 2) && !lo)) {
    set_error("sadmm_forward_split: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SplitSet cs{};
  cs.hi = hi; cs.lo = lo; cs.idx = idx; cs.n = nidx; cs.vexp = v; cs.base = (const float2*)base;
  cs.out = (float2*)r;
  SolverView sv{};
  const size_t cap = split_partial_bytes(1, KM, std::max(nidx, 1));
  void* part = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&part, cap, st));
  int rc = launch_split_forward(&cs, 1, KM, kind, planes, kVExplicit, sv, (float2*)part, cap, st);
  cudaError_t e = cudaFreeAsync(part, st);
  if (rc != SADMM_OK) return rc;
  SADMM_CUDA_TRY(e);
  return SADMM_OK;
}

int sadmm_adjoint_split(const void* hi, const void* lo, int kind, int planes, int KM, int N, const int* idx,
                        int nidx, const float* w, float* g, void* stream) {
  using namespace sadmm;
  if (!w || KM <= 0 || KM % 4 != 0 || KM > 16384 || N <= 0 || nidx < 0 || (nidx > 0 && (!idx || !g)) ||
      planes < 1 || planes > 3 || ((planes & 1) && !hi) || ((planes & 2) && !lo)) {
    set_error("sadmm_adjoint_split: bad arguments");
    return SADMM_EINVAL;
  }
  SplitSet as{};
  as.hi = hi; as.lo = lo; as.idx = idx; as.n = nidx; as.w = (const float2*)w; as.g = g;
  SolverView sv{};
  return launch_split_adjoint(&as, 1, KM, kind, planes, false, sv, (cudaStream_t)stream);
}

int sadmm_set_wait_limit(long long polls) { return sadmm::set_spd_wait_limit(polls); }

int sadmm_spd_apply(const double* F, int n, int ldf, const float* u, float* out, void* stream) {
  using namespace sadmm;
  if (!F || !u || !out || n <= 0 || n > 49152 || ldf < round_up(n, 2) || ldf % 2 != 0) {
    set_error("sadmm_spd_apply: bad arguments");
    return SADMM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void *P = nullptr, *part = nullptr, *err = nullptr;
  SADMM_CUDA_TRY(cudaMallocAsync(&P, sym_packed_pairs(n) * sizeof(float2), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&part, sym_part_pairs(n) * sizeof(float2), st));
  SADMM_CUDA_TRY(cudaMallocAsync(&err, sizeof(int), st));
  int rc = cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess ? SADMM_OK : SADMM_ECUDA;
  if (rc == SADMM_OK) rc = launch_pack_sym(F, ldf, n, (float2*)P, st);
  if (rc == SADMM_OK) {
    SpdSet s{(const float2*)P, n, u, out, nullptr, 0, (float2*)part, 0};
    SolverView sv{};
    rc = launch_spd_apply(&s, 1, false, sv, (int*)err, st);
  }
  int herr = 0;
  if (rc == SADMM_OK) {
    SADMM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SADMM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(P, st);
  cudaFreeAsync(part, st);
  cudaError_t e = cudaFreeAsync(err, st);
  if (rc != SADMM_OK) return rc;
  SADMM_CUDA_TRY(e);
  if (herr) { set_error("sadmm_spd_apply: a tile copy did not complete within the wait limit"); return SADMM_ETIMEOUT; }
  return SADMM_OK;
}

}  // extern "C"
