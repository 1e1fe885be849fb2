// Memory-bound helper kernels: layout changes, casts, column norms, the reconstruction of
// Algorithm 3 (Y_p = D^-1 R_Y + X Lambda_Y), the product-free part of the recurrence update, and
// the small reductions used by the Lanczos estimate.  Grid-stride loops sized to the SM count.
#include "common.cuh"

namespace rchfsi {
namespace {

__device__ __forceinline__ unsigned grid_threads() { return gridDim.x * blockDim.x; }

inline unsigned ew_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

__global__ void transpose_kernel(int64_t rows, int64_t cols, const double* __restrict__ in, int64_t ldin,
                                 double* __restrict__ out, int64_t ldout) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[k][threadIdx.x] = in[r * ldin + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * ldout + r] = t[threadIdx.x][k];
  }
}

// o1(i, j) = (float)(W(i, j) s1), o2(i, j) = (float)(W(i, j) s2): W column-major (leading dimension
// m), o1 and o2 row-major m x n.  32 x 32 shared-memory tiles, rows on blockIdx.x.
__global__ void __launch_bounds__(256) cols_to_rows_f32x2_kernel(int64_t m, int64_t n, const double* __restrict__ W,
                                                                 double s1, double s2, float* __restrict__ o1,
                                                                 float* __restrict__ o2) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int c = ty; c < 32; c += 8) {
    const int64_t i = i0 + tx, j = j0 + c;
    t[c][tx] = (i < m && j < n) ? W[j * m + i] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + tx;
    if (i < m && j < n) {
      const double w = t[tx][r];
      o1[i * n + j] = (float)(w * s1);
      o2[i * n + j] = (float)(w * s2);
    }
  }
}

// Y(i, j) = dinv[i] (rs R(i, j)) + X(i, j) lam[j] (dinv optional): R row-major float (leading
// dimension n); X and Y column-major (leading dimension m).  32 x 32 shared-memory tiles.
__global__ void __launch_bounds__(256) rows_to_cols_recon_kernel(int64_t m, int64_t n, const float* __restrict__ R,
                                                                 double rs, const double* __restrict__ dinv,
                                                                 const double* X, const double* __restrict__ lam,
                                                                 double* Y) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + tx;
    t[r][tx] = (i < m && j < n) ? rs * (double)R[i * n + j] : 0.0;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int64_t i = i0 + tx, j = j0 + c;
    if (i < m && j < n) {
      double v = t[tx][c];
      if (dinv) v *= dinv[i];
      Y[j * m + i] = fma(X[j * m + i], lam[j], v);
    }
  }
}

__global__ void scale_cols_kernel(int64_t m, int64_t n, double* X, int64_t ld, const double* scale) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t j = e / m, i = e - j * m;
    X[j * ld + i] *= scale[j];
  }
}

// One CTA per column: out[j] = ||X(:,j)||_2 (column-major).
__global__ void col_norms_kernel(int64_t m, const double* __restrict__ X, int64_t ld, double* out, int inverse) {
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = X[j * ld + i];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[j] = inverse ? 1.0 / sqrt(s) : sqrt(s);
  }
}

__global__ void scale_rows_kernel(int64_t m, int64_t n, const double* in, double* out, const double* d, int cols) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t i = e / n, j = e - i * n;
    out[e] = in[e] * (cols ? d[j] : d[i]);
  }
}

// Round an FP32 value to TF32 (10 explicit mantissa bits), round-to-nearest, ties away from zero
// (the cvt.rna.tf32.f32 rounding).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void cast_f64_f32_kernel(int64_t n, const double* in, float* out, double scale, int tf32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += grid_threads()) {
    float v = (float)(in[e] * scale);
    out[e] = tf32 ? to_tf32(v) : v;
  }
}

__global__ void cast_f64_bf16_kernel(int64_t n, const double* in, __nv_bfloat16* out, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += grid_threads())
    out[e] = __float2bfloat16_rn((float)(in[e] * scale));
}

__global__ void cast_f32_f64_kernel(int64_t n, const float* in, double* out, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += grid_threads())
    out[e] = scale * (double)in[e];
}

__global__ void scaled_copy_kernel(int64_t n, const double* in, double* out, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += grid_threads())
    out[e] = in[e] * scale;
}

template <typename R>
__device__ __forceinline__ double ld_r(const R* p, int64_t o) { return (double)p[o]; }
template <>
__device__ __forceinline__ double ld_r<__nv_bfloat16>(const __nv_bfloat16* p, int64_t o) {
  return (double)__bfloat162float(p[o]);
}

// Y = D^-1 R + X diag(lam), all column-major m x n with leading dimension m.
template <typename R>
__global__ void reconstruct_kernel(int64_t m, int64_t n, const R* __restrict__ Rr, int64_t ldr,
                                   const double* __restrict__ dinv, const double* __restrict__ X,
                                   const double* __restrict__ lam, double* __restrict__ Y) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t j = e / m, i = e - j * m;
    double r = ld_r(Rr, j * ldr + i);
    if (dinv) r *= dinv[i];
    Y[e] = fma(X[e], lam[j], r);
  }
}

// Rx = b*Ry + c*Rx + a*W*lam[j]  (float storage, column-major)
__global__ void recur_axpby_kernel(int64_t m, int64_t n, const float* __restrict__ Ry, float* __restrict__ Rx,
                                   const float* __restrict__ W, const double* __restrict__ lam, float a, float b,
                                   float c) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t j = e / m;
    float v = b * Ry[e] + c * Rx[e];
    if (W) v += a * W[e] * (float)lam[j];
    Rx[e] = v;
  }
}

__global__ void resid_norms_kernel(int64_t m, const double* __restrict__ W, const double* __restrict__ X,
                                   double* out_abs, double* out_x) {
  __shared__ double red[2][32];
  const int64_t j = blockIdx.x;
  double s = 0.0, t = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double w = W[j * m + i], x = X[j * m + i];
    s = fma(w, w, s);
    t = fma(x, x, t);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = threadIdx.x < (blockDim.x >> 5);
    s = ok ? red[0][threadIdx.x] : 0.0;
    t = ok ? red[1][threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if (threadIdx.x == 0) {
      out_abs[j] = sqrt(s);
      out_x[j] = sqrt(t);
    }
  }
}

// Single-CTA dot product: *out = x . y
__global__ void dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

}  // namespace

void transpose_f64(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin, double* out,
                   int64_t ldout) {
  if (rows <= 0 || cols <= 0) return;
  RC_CHECK(cdiv(rows, 32) <= 65535u, RCHFSI_ERR_INVALID_ARG, "transpose: too many rows for the grid");
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, in, ldin, out, ldout);
  RC_LAUNCH();
}

void scale_cols_f64(cudaStream_t s, int64_t m, int64_t n, double* X, int64_t ld, const double* scale) {
  scale_cols_kernel<<<ew_blocks(m * n), 256, 0, s>>>(m, n, X, ld, scale);
  RC_LAUNCH();
}

void col_norms_f64(cudaStream_t s, int64_t m, int64_t n, const double* X, int64_t ld, double* out) {
  if (n <= 0) return;
  col_norms_kernel<<<(unsigned)n, 256, 0, s>>>(m, X, ld, out, 0);
  RC_LAUNCH();
}

void scale_rows_f64(cudaStream_t s, int64_t m, int64_t n, const double* in, double* out, const double* d,
                    bool cols) {
  scale_rows_kernel<<<ew_blocks(m * n), 256, 0, s>>>(m, n, in, out, d, cols ? 1 : 0);
  RC_LAUNCH();
}

void cols_to_rows_f32x2(cudaStream_t s, int64_t m, int64_t n, const double* W, double s1, double s2, float* o1,
                        float* o2) {
  if (m <= 0 || n <= 0) return;
  RC_CHECK(cdiv(n, 32) <= 65535u, RCHFSI_ERR_INVALID_ARG, "cols_to_rows: too many columns for the grid");
  cols_to_rows_f32x2_kernel<<<dim3(cdiv(m, 32), cdiv(n, 32)), 256, 0, s>>>(m, n, W, s1, s2, o1, o2);
  RC_LAUNCH();
}

void rows_to_cols_recon(cudaStream_t s, int64_t m, int64_t n, const float* R, double rs, const double* dinv,
                        const double* X, const double* lam, double* Y) {
  if (m <= 0 || n <= 0) return;
  RC_CHECK(cdiv(n, 32) <= 65535u, RCHFSI_ERR_INVALID_ARG, "rows_to_cols: too many columns for the grid");
  rows_to_cols_recon_kernel<<<dim3(cdiv(m, 32), cdiv(n, 32)), 256, 0, s>>>(m, n, R, rs, dinv, X, lam, Y);
  RC_LAUNCH();
}

void cast_f64_to_f32(cudaStream_t s, int64_t n, const double* in, float* out, double scale, int round_tf32) {
  cast_f64_f32_kernel<<<ew_blocks(n), 256, 0, s>>>(n, in, out, scale, round_tf32);
  RC_LAUNCH();
}

void cast_f64_to_bf16(cudaStream_t s, int64_t n, const double* in, __nv_bfloat16* out, double scale) {
  cast_f64_bf16_kernel<<<ew_blocks(n), 256, 0, s>>>(n, in, out, scale);
  RC_LAUNCH();
}

void cast_f32_to_f64(cudaStream_t s, int64_t n, const float* in, double* out, double scale) {
  cast_f32_f64_kernel<<<ew_blocks(n), 256, 0, s>>>(n, in, out, scale);
  RC_LAUNCH();
}

namespace {
// A += factor * tr(A) * I (one block: the trace, then the diagonal update)
__global__ void shift_diag_trace_kernel(int n, double* A, int lda, double factor) {
  __shared__ double part[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += A[(int64_t)i * lda + i];
  part[threadIdx.x] = t;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  const double shift = factor * part[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * lda + i] += shift;
}
}  // namespace

void shift_diag_by_trace_f64(cudaStream_t s, int n, double* A, int lda, double factor) {
  shift_diag_trace_kernel<<<1, 256, 0, s>>>(n, A, lda, factor);
  RC_LAUNCH();
}

void fill_zero(cudaStream_t s, void* p, size_t bytes) { RC_CUDA(cudaMemsetAsync(p, 0, bytes, s)); }

void scaled_copy_f64(cudaStream_t s, int64_t n, const double* in, double* out, double scale) {
  scaled_copy_kernel<<<ew_blocks(n), 256, 0, s>>>(n, in, out, scale);
  RC_LAUNCH();
}

void reconstruct_f64(cudaStream_t s, int64_t m, int64_t n, const double* R, int64_t ldr, const double* dinv,
                     const double* X, const double* lam, double* Y) {
  reconstruct_kernel<double><<<ew_blocks(m * n), 256, 0, s>>>(m, n, R, ldr, dinv, X, lam, Y);
  RC_LAUNCH();
}

void reconstruct_f32(cudaStream_t s, int64_t m, int64_t n, const float* R, int64_t ldr, const double* dinv,
                     const double* X, const double* lam, double* Y) {
  reconstruct_kernel<float><<<ew_blocks(m * n), 256, 0, s>>>(m, n, R, ldr, dinv, X, lam, Y);
  RC_LAUNCH();
}

void reconstruct_bf16(cudaStream_t s, int64_t m, int64_t n, const __nv_bfloat16* R, int64_t ldr,
                      const double* dinv, const double* X, const double* lam, double* Y) {
  reconstruct_kernel<__nv_bfloat16><<<ew_blocks(m * n), 256, 0, s>>>(m, n, R, ldr, dinv, X, lam, Y);
  RC_LAUNCH();
}

namespace {
__global__ void cast2d_f32_kernel(int64_t rows, int64_t cols, const double* in, int64_t ldin, float* out,
                                  int64_t ldout, double scale, int tf32) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t r = e / cols, c = e - r * cols;
    const float v = (float)(in[r * ldin + c] * scale);
    out[r * ldout + c] = tf32 ? to_tf32(v) : v;
  }
}
__global__ void cast2d_bf16_kernel(int64_t rows, int64_t cols, const double* in, int64_t ldin, __nv_bfloat16* out,
                                   int64_t ldout, double scale) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += grid_threads()) {
    const int64_t r = e / cols, c = e - r * cols;
    out[r * ldout + c] = __float2bfloat16_rn((float)(in[r * ldin + c] * scale));
  }
}
}  // namespace

void cast2d_f64_to_f32(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin, float* out,
                       int64_t ldout, double scale, int round_tf32) {
  cast2d_f32_kernel<<<ew_blocks(rows * cols), 256, 0, s>>>(rows, cols, in, ldin, out, ldout, scale, round_tf32);
  RC_LAUNCH();
}

void cast2d_f64_to_bf16(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin,
                        __nv_bfloat16* out, int64_t ldout, double scale) {
  cast2d_bf16_kernel<<<ew_blocks(rows * cols), 256, 0, s>>>(rows, cols, in, ldin, out, ldout, scale);
  RC_LAUNCH();
}

void recur_axpby_f32(cudaStream_t s, int64_t m, int64_t n, const float* Ry, float* Rx, const float* W,
                     const double* lam, double a, double b, double c) {
  recur_axpby_kernel<<<ew_blocks(m * n), 256, 0, s>>>(m, n, Ry, Rx, W, lam, (float)a, (float)b, (float)c);
  RC_LAUNCH();
}

void resid_rel_norms(cudaStream_t s, int64_t m, int64_t n, const double* W, const double* X, double* out_abs,
                     double* out_xnorm) {
  if (n <= 0) return;
  resid_norms_kernel<<<(unsigned)n, 256, 0, s>>>(m, W, X, out_abs, out_xnorm);
  RC_LAUNCH();
}

void dot_f64(cudaStream_t s, int64_t n, const double* x, const double* y, double* out) {
  dot_kernel<<<1, 1024, 0, s>>>(n, x, y, out);
  RC_LAUNCH();
}

}  // namespace rchfsi
