// FP64-accurate matrix products on the BF16 tensor cores (error-free splitting).
//
// GB300's FP64 rate (~1.1 TFLOP/s) is ~2000x below its BF16 tensor rate, and the FP64 products of
// the residual and Rayleigh-Ritz steps dominate the solve once the filter runs on tensor cores.
// This path computes those products to FP64-level accuracy from BF16 pieces:
//   * each row r of an operand X (logical R x K) is scaled by 2^-e_r so that |x| < 1, then split
//     exactly into S = 7 slices of integers |t| <= 256 (bf16-exact): x = 2^e_r sum_s t_s 2^-8(s+1)
//     + O(2^(e_r - 56));
//   * C(i,j) = sum_k A(i,k) B(j,k) is assembled from the slice products A_s B_t^T with s + t <= S-1
//     (28 products), grouped by level L = s + t.  |t_0| <= 256 and |t_s| <= 128 for s > 0, so over a
//     group of 128 K terms the sum of level L is an integer below 2^24 for L <= 5 and the FP32
//     tensor-core accumulation of those levels is exact; the last level (weight 2^-48) could in the
//     worst case lose one unit, an error below 2^-72 of the product, far under FP64 rounding;
//   * each group's levels are combined as sum_L D_L 2^-8L into a float-float (hi, lo) accumulator
//     (TwoSum), and C(i,j) = 2^(e_i + f_j - 16) (hi + lo) is formed in FP64 at the end.
// The result carries ~2^-48 relative rounding per chunk combination, comparable to an FP64 GEMM's
// own rounding for the shapes used here.
#pragma once
#include "common.cuh"

namespace rchfsi {

constexpr int kOzSlices = 7;

struct OzOperand {
  int64_t R = 0, K = 0, Kp = 0;      // logical rows, reduction length, K padded to a multiple of 64
  int64_t Rp = 0;                    // rows per slice in storage (>= R and >= 32, extra rows zero)
  DevBuf<__nv_bfloat16> sl;          // [S][Rp][Kp] slices, K-major
  DevBuf<int> ex;                    // [R] row exponents
  size_t bytes() const { return sl.bytes() + ex.bytes(); }
};

// Split the logical R x K FP64 matrix X, element (r, k) at X[r * rs + k * ks], into `op`.
void oz_slice(cudaStream_t s, int64_t R, int64_t K, const double* X, int64_t rs, int64_t ks, OzOperand& op);

// C(i, j) = sum_k A(i, k) B(j, k), i < A.R, j < B.R, stored column-major: C[j * ldc + i].
// ws: split-K workspace (grown as needed); err: device flag raised by a bounded-wait timeout.
// symmetric: the caller knows C is symmetric (a Gram matrix Y^T (A Y) with A symmetric, A.R == B.R):
// only the output tiles that reach the upper triangle are computed and the rest is mirrored.
void oz_gemm(cudaStream_t s, int num_sms, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc,
             DevBuf<double>& ws, int* err, bool symmetric = false);

// Operand and workspace buffers lent to a caller's FP64-accurate products (the eigensolver).
struct OzScratch {
  OzOperand* a;
  OzOperand* b;
  DevBuf<double>* ws;
  int* err;
  int num_sms;
};

}  // namespace rchfsi
