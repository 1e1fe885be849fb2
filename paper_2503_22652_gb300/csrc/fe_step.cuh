// Fused degree step of the finite-element R-ChFSI filter on the tcgen05 tensor cores (fe_step.cu).
#pragma once
#include "fe.cuh"

namespace rchfsi {

// One real cell-matrix part of a fused step (a complex operator has four: Ar and Ai on the two row
// halves of the embedded block).  With S_j = s_j R_j the scaled iterates of Algorithm 3:
//   U[dofs(c), :] += sign * alpha * (A_c D_c^-1) V[dofs(c), :]            for every cell c
//   U[d, :]       += beta * V[d, :] + omega * W[d, :] diag(lam)          once per dof d (owner terms)
// V, W, U: row-major FP32 blocks of `rows` rows and n columns; lam: n floats (Lambda_{k-1} in FP32).  When coef is set,
// (alpha, beta, omega) = coef[0..2] are read on the device (a captured graph stays valid when the
// coefficients change).  owner = false drops the owner terms (the cross parts of a complex operator).
struct FeStepPart {
  FeOp* op;
  const float* V;
  const float* W;
  float* U;
  const float* lam;
  const double* coef;
  int64_t rows;
  int n;
  float alpha, beta, omega, sign;
  bool owner;
};

// True when the fused step can run: TF32 products, n a multiple of 4 (16-byte rows for TMA),
// n_c <= 128.
bool fe_step_supported(const FeOp& op, int n, int precision);

// The parts of one operator's step (1 real, 4 complex); returns the count.
int fe_step_parts(FeOp& op, const float* V, const float* W, float* U, const float* lam, int n, float alpha,
                  float beta, float omega, const double* coef, FeStepPart* out);

// Pack the operator's scaled cell images (A_c D_c^-1, TF32) and owner masks ahead of a capture.
void fe_step_prepare(cudaStream_t s, FeOp& op);

// All parts (at most 64) in one persistent launch; BN = column tile (32, 64 or 96).
void fe_step_batch(cudaStream_t s, const FeStepPart* parts, int nparts, int BN, int num_sms);

// Column tile for this operator and width, chosen by timing the candidates once per shape on the
// problem's own data (into a scratch output); cached.
int fe_step_tune(cudaStream_t s, int num_sms, FeOp& op, int n, const float* V, const float* W, const float* lam);

}  // namespace rchfsi
