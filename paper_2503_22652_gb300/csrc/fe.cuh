// Finite-element (cell-matrix) operator: A = sum_c P_c^T A_c P_c over n_cells cells of n_c dofs.
// The paper evaluates this product cell by cell with batched dense GEMMs (Remark in Section 4.2);
// here each kernel gathers a cell's rows of the block, multiplies by the cell matrix and
// scatter-adds the result.
#pragma once
#include <memory>

#include "common.cuh"

namespace rchfsi {

struct FeOp {
  int64_t m = 0, n_cells = 0;
  int nc = 0;
  bool B_shared = false;
  DevBuf<int> dofs;          // n_cells * nc
  DevBuf<double> A64, B64;   // cell matrices, row-major (B64 holds one matrix when shared)
  DevBuf<double> Dinv;       // m
  DevBuf<float> A32;         // FP32 cell matrices for the filter products
  DevBuf<float> Atf;         // TF32-rounded copy
  DevBuf<__nv_bfloat16> A16; // BF16 copy
  DevBuf<float> Dinv32;
  DevBuf<uint8_t> imgtf, img16;  // cell matrices packed as swizzled tensor-core operand images
  DevBuf<uint8_t> imgADtf;       // A_c D_c^-1 (columns scaled by D^-1 at the cell's dofs), TF32 images
  // Owner of each dof (one of the cells that contain it, balanced over the cells): per cell 128
  // entries, own_pos[k] = position of node k among the dofs the cell owns (node order), -1 when it
  // does not own it; own_max = the most dofs one cell owns.
  DevBuf<int8_t> own_pos;
  int own_max = 0;
  int max_mult = 1;              // the most cell listings of one dof (cells sharing it)
  int* err = nullptr;            // device flag raised when a bounded wait in a kernel runs out
  // Complex Hermitian operator A = Ar + i Ai acting on the real embedding [x_r; x_i] of length 2 mc:
  // this object holds Ar (A64) and B, `imag` holds Ai; m = 2 mc, Dinv = [D^-1; D^-1].  Each
  // complex product is four real cell products on the two row halves of the block.
  bool cplx = false;
  int64_t mc = 0;
  std::unique_ptr<FeOp> imag;
  // FP64-accurate tensor-core products (fe_oz.cu): BF16 slice images of the cell matrices and their
  // row exponents, per dof the largest exponent of the cell rows that reach it (the scale of its
  // fixed-point accumulator; made on first use), and per-product scratch (column exponents, slice
  // planes of the input block)
  mutable DevBuf<uint8_t> ozA, ozB;
  mutable DevBuf<int> ozAe, ozBe, ozcexp, ozArow, ozBrow;
  // packed from this operator's matrices (an allocation taken over from a previous operator is not)
  mutable bool oz_packed[2] = {false, false}, rowexp_packed[2] = {false, false};
  bool imgAD_packed = false;
  mutable DevBuf<__nv_bfloat16> ozplanes;
};

// Y (row-major m x n) = Op X, Op = A or B, FP64.  Y is overwritten.
void fe_apply_f64_rows(cudaStream_t s, const FeOp& op, bool useB, const double* X, double* Y, int n);
// AX = A X and/or BX = B X (either output may be null), FP64-accurate, from exact BF16 slices on
// the tensor cores (fe_oz.cu).  X, AX, BX: column-major m x n, leading dimension m; the slices of X
// are made once for both products.  accA, accB: m x n scratch blocks (the fixed-point accumulators)
// for the outputs requested.
void fe_apply_f64_cols_tc(cudaStream_t s, const FeOp& op, const double* X, double* AX, double* BX, int n,
                          int num_sms, double* accA, double* accB);

// Filter product for FE operators on row-major m x n blocks, accumulated into Rx (the
// product-free recurrence terms are applied to Rx beforehand):
//   dmode 0: Rx += a * A Ry,  1: Rx += a * A D^-1 Ry (Algorithm 3),  2: Rx += a * D^-1 A Ry (Algorithm 2)
// precision: RCHFSI_FP32 (FFMA), RCHFSI_TF32 / RCHFSI_BF16 (tensor cores).
void fe_filter_product_f32(cudaStream_t s, FeOp& op, int precision, const float* Ry, float* Rx, int n, float a,
                           int dmode);

// Same for FP64 storage (parity path).
void fe_filter_product_f64(cudaStream_t s, const FeOp& op, const double* Ry, double* Rx, int n, double a,
                           int dmode);

// Elementwise recurrence terms for row-major blocks: Rx = b*Ry + c*Rx + a*W*lam[j]
void recur_terms_rows_f32(cudaStream_t s, int64_t m, int n, const float* Ry, float* Rx, const float* W,
                          const double* lam, double a, double b, double c);
// Same with (a, b, c) = coef[0..2] read on the device (capturable in a CUDA graph).
void recur_terms_rows_f32_dev(cudaStream_t s, int64_t m, int n, const float* Ry, float* Rx, const float* W,
                              const double* lam, const double* coef);
void recur_terms_rows_f64(cudaStream_t s, int64_t m, int n, const double* Ry, double* Rx, const double* W,
                          const double* lam, double a, double b, double c);

}  // namespace rchfsi
