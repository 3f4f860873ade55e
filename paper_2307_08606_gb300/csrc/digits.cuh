// Factor apply with 16 right-hand sides on the tensor cores (Eq. 3,
// x_q-update: U = F R for the Woodbury factor W, G -> H G for the primal
// inverse H), for the batched form.  The dense factor F (n x n, FP64) and the
// right-hand sides are cut into exact BF16 integer digits (bapply_tc.cu), so
// that every tensor-core product is exact and the order sums are exact
// integers in FP32; the result carries about 2^-30 of (row scale x column
// scale) per term.
#pragma once
#include "common.cuh"
#include "tmap.cuh"

namespace sadmm {

struct DigitApply {
  int Q = 0, n = 0;
  int rows_pad = 0;        // factor rows, padded to 128 (TMEM lanes)
  int kpad = 0;            // k (factor columns / right-hand-side rows), padded to 256 x ksplit
  int ksplit = 1;          // k ranges per row block (work items Q x rows_pad / 128 x ksplit)
  void* DF = nullptr;      // BF16 digits of the factors [q][digit][row][k]
  int* expoF = nullptr;    // [q][row] row exponents
  void* DU = nullptr;      // BF16 digits of the right-hand sides [q][digit][s][k]
  int* expoU = nullptr;    // [q][s] column exponents
  int* maxbits = nullptr;  // [q][s] column maxima (float bits)
  float2* part = nullptr;  // [q][split][row][s] double-float partial results
  CUtensorMap tmF, tmU;
};

// Sizes for Q factors of order n (no allocation).
void digit_apply_dims(DigitApply& d, int Q, int n);
// Bytes of one allocation that holds every buffer.
size_t digit_apply_bytes(const DigitApply& d);
// Carve the buffers out of mem (digit_apply_bytes(d) bytes, 1024-aligned) and
// build the tensor maps.
int digit_apply_bind(DigitApply& d, void* mem);
// Digits of factor q from F (n x n FP64, row-major, leading dimension ld).
int launch_factor_digits(const DigitApply& d, int q, const double* F, int ld, cudaStream_t st);
// d.part = F_q u_q for every q: u[q] is a device pointer (device array of Q
// pointers) to the 16 right-hand sides, umode 1: float [j][s]; umode 0: the
// interleaved real rows of complex [m][s] (real row j = 2m + c at float
// ((m * 16 + s) * 2 + c)).  *err = 2 if a pipeline wait ran out.
int launch_digit_apply(const DigitApply& d, const float* const* u, int umode, int* err, cudaStream_t st);

}  // namespace sadmm
