// Tensor-core (tcgen05) cell-matrix product of the FE filter.
#pragma once
#include "fe.cuh"

namespace rchfsi {
// Rx += a * A (D^-1 Ry) (dmode 1) or a * D^-1 A Ry (dmode 2) or a * A Ry (dmode 0) on row-major m x n
// FP32 blocks, products on tcgen05 tensor cores (precision RCHFSI_TF32 or RCHFSI_BF16).
void fe_tc_product(cudaStream_t s, FeOp& op, int precision, const float* Ry, float* Rx, int n, float a, int dmode);
}  // namespace rchfsi
