// Symmetrisation of the N x N Gram and projected matrices of the Rayleigh-Ritz step (column-major);
// the Cholesky factor, its inverse and the eigensolver are in small_eig.cu.
#include "common.cuh"

namespace rchfsi {
namespace {

__global__ void symmetrize_kernel(int n, double* A, int lda) {
  const int64_t tot = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    const int col = (int)(t / n), row = (int)(t - (int64_t)col * n);
    if (row > col) {
      const double v = 0.5 * (A[(int64_t)col * lda + row] + A[(int64_t)row * lda + col]);
      A[(int64_t)col * lda + row] = v;
      A[(int64_t)row * lda + col] = v;
    }
  }
}

}  // namespace

void symmetrize_f64(cudaStream_t s, int n, double* A, int lda) {
  symmetrize_kernel<<<64, 256, 0, s>>>(n, A, lda);
  RC_LAUNCH();
}

}  // namespace rchfsi
