// Tensor-core (tcgen05) GEMM with the Chebyshev recurrence fused into its epilogue:
//   out = a * (A R_Y) + b * R_Y + c * R_X + a * W diag(lam)
// A: M x K row-major (K-contiguous), R_Y: K x N column-major (K-contiguous), out/R_X/W: M x N
// column-major.  TF32 takes FP32 storage, BF16 takes bfloat16 storage; accumulation is FP32.
#pragma once
#include "common.cuh"

namespace rchfsi {

struct TcRecur {
  float a, b, c;
  const float* Ry;
  const float* Rx;  // may be null (c term dropped)
  const float* W;   // may be null
  const double* lam;
  float* out;
};

struct TcRecur16 {
  float a, b, c;
  const __nv_bfloat16* Ry;
  const __nv_bfloat16* Rx;
  const __nv_bfloat16* W;
  const double* lam;
  __nv_bfloat16* out;
};

// lda / ldb: row pitch (elements) of A (row-major) and of B (column-major); ldo: leading dimension
// of out / R_Y / R_X / W.  Pitches times the element size must be multiples of 16 bytes (TMA).
// err: device flag set to nonzero when a bounded wait inside the kernel ran out.
void tc_gemm_tf32_recur(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, DevBuf<float>& split, const TcRecur& r, int64_t ldo, int* err);
void tc_gemm_bf16_recur(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A,
                        int64_t lda, const __nv_bfloat16* B, int64_t ldb, DevBuf<float>& split, const TcRecur16& r,
                        int64_t ldo, int* err);

// Floats of split-K partial sums the TF32 GEMM plan needs for this shape (0 when it does not split).
size_t tc_gemm_tf32_split_floats(int num_sms, int64_t M, int64_t N, int64_t K);

// tc_gemm_tf32_recur with caller-provided split-K storage (ws, ws_floats) instead of a DevBuf:
// allocates nothing.  Throws INVALID_ARG when the plan needs more than ws_floats.
void tc_gemm_tf32_recur_ws(cudaStream_t s, int num_sms, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                           const float* B, int64_t ldb, float* ws, size_t ws_floats, const TcRecur& r, int64_t ldo,
                           int* err);

}  // namespace rchfsi
