// Small dense FP64 kernels of the Rayleigh-Ritz step (N x N, column-major):
// Cholesky factorisation of the B-Gram matrix (the "Cholesky-QR" of the filtered block in the
// B inner product) and the two triangular solves that form L^-1 G_A L^-T and E = L^-T V.
#include "common.cuh"

namespace rchfsi {
namespace {

// Right-looking Cholesky, one CTA, in place on the lower triangle.  info = 0 on success,
// j+1 when the j-th pivot is not positive (or not finite).  The strict upper triangle is zeroed.
__global__ void __launch_bounds__(1024) cholesky_kernel(int n, double* A, int lda, int* info) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * lda + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = j + 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
      A[(int64_t)j * lda + j] = piv;
    }
    __syncthreads();
    if (bad) break;
    const double inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)j * lda + i] *= inv;
    __syncthreads();
    // trailing update of the lower triangle: A(i,k) -= L(i,j) L(k,j) for j < k <= i;
    // one warp per column k, lanes over rows i (contiguous in column-major storage)
    {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int k = j + 1 + warp; k < n; k += nw) {
        const double lkj = A[(int64_t)j * lda + k];
        for (int i = k + lane; i < n; i += 32) A[(int64_t)k * lda + i] -= A[(int64_t)j * lda + i] * lkj;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = bad;
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    const int col = (int)(t / n), row = (int)(t - (int64_t)col * n);
    if (row < col) A[(int64_t)col * lda + row] = 0.0;
  }
}

// Solve L Z = B in place (forward substitution, column-oriented), one CTA per right-hand side.
__global__ void trsm_lower_kernel(int n, int nrhs, const double* __restrict__ L, int ldl, double* B, int ldb) {
  extern __shared__ double z[];
  const int col = blockIdx.x;
  if (col >= nrhs) return;
  double* b = B + (int64_t)col * ldb;
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = b[i];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double zk = z[k] / L[(int64_t)k * ldl + k];
    __syncthreads();
    if (threadIdx.x == 0) z[k] = zk;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) z[i] -= L[(int64_t)k * ldl + i] * zk;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = z[i];
}

// Solve L^T Z = B in place (backward substitution, dot form over column k of L).
__global__ void trsm_lower_trans_kernel(int n, int nrhs, const double* __restrict__ L, int ldl, double* B,
                                        int ldb) {
  extern __shared__ double z[];
  __shared__ double red[32];
  const int col = blockIdx.x;
  if (col >= nrhs) return;
  double* b = B + (int64_t)col * ldb;
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = b[i];
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    double s = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) s = fma(L[(int64_t)k * ldl + i], z[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      z[k] = (z[k] - t) / L[(int64_t)k * ldl + k];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = z[i];
}

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

int cholesky_f64(cudaStream_t s, int n, double* A, int lda, int* d_info) {
  cholesky_kernel<<<1, 1024, 0, s>>>(n, A, lda, d_info);
  RC_LAUNCH();
  return 0;
}

void trsm_lower_left_f64(cudaStream_t s, int n, int nrhs, const double* L, int ldl, double* B, int ldb) {
  RC_CHECK(n <= 6144, RCHFSI_ERR_UNSUPPORTED, "trsm: block larger than 6144");
  trsm_lower_kernel<<<nrhs, 256, n * sizeof(double), s>>>(n, nrhs, L, ldl, B, ldb);
  RC_LAUNCH();
}

void trsm_lower_trans_left_f64(cudaStream_t s, int n, int nrhs, const double* L, int ldl, double* B, int ldb) {
  RC_CHECK(n <= 6144, RCHFSI_ERR_UNSUPPORTED, "trsm: block larger than 6144");
  trsm_lower_trans_kernel<<<nrhs, 256, n * sizeof(double), s>>>(n, nrhs, L, ldl, B, ldb);
  RC_LAUNCH();
}

void symmetrize_f64(cudaStream_t s, int n, double* A, int lda) {
  symmetrize_kernel<<<64, 256, 0, s>>>(n, A, lda);
  RC_LAUNCH();
}

}  // namespace rchfsi
