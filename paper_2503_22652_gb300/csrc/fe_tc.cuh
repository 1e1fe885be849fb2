// Tensor-core (tcgen05) cell-matrix product of the FE filter.
#pragma once
#include "fe.cuh"

namespace rchfsi {
// Rx += a * A (D^-1 Ry) (dmode 1) or a * D^-1 A Ry (dmode 2) or a * A Ry (dmode 0) on row-major m x n
// FP32 blocks, products on tcgen05 tensor cores (precision RCHFSI_TF32 or RCHFSI_BF16).
void fe_tc_product(cudaStream_t s, FeOp& op, int precision, const float* Ry, float* Rx, int n, float a, int dmode);

// One real cell-matrix product of a batched launch: Rx += sign * a * A (D^-1 Ry) (dmode as above) with
// a = *coef when coef is set (read on the device), else the value a.  BN = 0 picks the default tile.
struct FeTcPart {
  FeOp* op;
  const float* Ry;
  float* Rx;
  int n;
  float a;
  const double* coef;
  float sign;
  int dmode;
  int BN;
};

// All parts in one persistent launch (at most 64 parts).
void fe_tc_batch(cudaStream_t s, int precision, const FeTcPart* parts, int nparts, int num_sms);

// The parts of one operator product (1 for a real operator, 4 for a complex one); returns the count.
int fe_tc_parts(FeOp& op, const float* Ry, float* Rx, int n, float a, const double* coef, int dmode, int BN,
                FeTcPart* out);

// Pack the tensor-core cell images of the operator (and of its imaginary part) ahead of a capture.
void fe_tc_parts_prepare(cudaStream_t s, FeOp& op, int precision);

// Largest column tile of the precision (TF32 96, BF16 208).
int fe_tc_bn_max(int precision);
}  // namespace rchfsi
