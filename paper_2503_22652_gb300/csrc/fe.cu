// SIMT kernels of the finite-element (cell-matrix) operator.
//
// One CTA takes one cell and one tile of block columns: it gathers the cell's n_c rows of the
// input block into shared memory (scaled by D^-1 when the product is A D^-1 R), multiplies by the
// cell matrix (row i of A_c is read as a warp-wide broadcast) and scatter-adds the n_c output rows
// with atomics (a dof shared by several cells receives one add per cell).  This is the FP64 path
// (residuals, Rayleigh-Ritz) and the FP32 "FFMA" filter path; the tensor-core path lives in
// fe_tc.cu.
#include "fe.cuh"
#include "fe_tc.cuh"
#include "prof.cuh"

namespace rchfsi {
namespace {

constexpr int NCMAX = 128;

template <typename T, int TN>
__global__ void __launch_bounds__(256) fe_cell_kernel(int nc, const int* __restrict__ dofs,
                                                      const T* __restrict__ Acells, int64_t a_stride,
                                                      const T* __restrict__ X, T* __restrict__ Y, int n, T alpha,
                                                      const double* __restrict__ dinv, int dmode) {
  __shared__ T xs[NCMAX][TN];
  __shared__ int ids[NCMAX];
  const int64_t cell = blockIdx.x;
  const int j0 = blockIdx.y * TN;
  const int tid = threadIdx.x;
  const T* Ac = Acells + cell * a_stride;
  for (int i = tid; i < nc; i += blockDim.x) ids[i] = dofs[cell * nc + i];
  __syncthreads();
  for (int e = tid; e < nc * TN; e += blockDim.x) {
    const int i = e / TN, j = e % TN;
    const int col = j0 + j;
    T v = T(0);
    if (col < n) {
      const int g = ids[i];
      v = X[(int64_t)g * n + col];
      if (dmode == 1) v *= (T)dinv[g];
    }
    xs[i][j] = v;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int PER = TN / 32;
  for (int i = warp; i < nc; i += 8) {
    T acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = T(0);
    const T* arow = Ac + (int64_t)i * nc;
    for (int k = 0; k < nc; ++k) {
      const T a = arow[k];
#pragma unroll
      for (int q = 0; q < PER; ++q) acc[q] = fma(a, xs[k][lane + 32 * q], acc[q]);
    }
    const int g = ids[i];
    T sc = alpha;
    if (dmode == 2) sc *= (T)dinv[g];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int col = j0 + lane + 32 * q;
      if (col < n) atomicAdd(&Y[(int64_t)g * n + col], sc * acc[q]);
    }
  }
}

// Recurrence update of row-major m x n blocks, Rx = a W lam + b Ry + c Rx (W may be null).  Thread
// (x, y) owns column j = 32 blockIdx.x + x and walks rows y, y + 8 gridDim.y, ...: its lam_j is read
// and converted once (an FP64 conversion per element would occupy the FP64 pipe, and e % n costs a
// 64-bit division), the warp's 32 columns are consecutive (coalesced).
template <typename T>
__global__ void __launch_bounds__(256) recur_rows_kernel(int64_t m, int n, const T* __restrict__ Ry, T* __restrict__ Rx,
                                                         const T* __restrict__ W, const double* __restrict__ lam, T a,
                                                         T b, T c) {
  const int j = blockIdx.x * 32 + threadIdx.x;
  if (j >= n) return;
  const T al = W ? a * (T)lam[j] : T(0);
  for (int64_t i = blockIdx.y * 8 + threadIdx.y; i < m; i += (int64_t)gridDim.y * 8) {
    const int64_t e = i * n + j;
    T v = b * Ry[e];
    if (c != T(0)) v += c * Rx[e];
    if (W) v += al * W[e];
    Rx[e] = v;
  }
}

// Same update with (a, b, c) = coef[0..2] read on the device, so that a captured CUDA graph of the
// filter loop stays valid when the Chebyshev coefficients change between outer iterations.
__global__ void __launch_bounds__(256) recur_rows_dev_kernel(int64_t m, int n, const float* __restrict__ Ry,
                                                             float* __restrict__ Rx, const float* __restrict__ W,
                                                             const double* __restrict__ lam,
                                                             const double* __restrict__ coef) {
  const int j = blockIdx.x * 32 + threadIdx.x;
  if (j >= n) return;
  const float b = (float)coef[1], c = (float)coef[2];
  const float al = W ? (float)(coef[0] * lam[j]) : 0.f;
  for (int64_t i = blockIdx.y * 8 + threadIdx.y; i < m; i += (int64_t)gridDim.y * 8) {
    const int64_t e = i * n + j;
    float v = b * Ry[e];
    if (c != 0.f) v += c * Rx[e];
    if (W) v += al * W[e];
    Rx[e] = v;
  }
}

// Grid of recur_rows kernels: 32-column strips, row blocks for ~16 CTAs per SM.
inline dim3 recur_grid(int64_t m, int n) {
  const unsigned gx = cdiv(n, 32);
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 8), (int64_t)152 * 16 / gx + 1));
  return dim3(gx, (unsigned)std::min<int64_t>(gy, 65535));
}

template <typename T, int TN>
void launch_cells(cudaStream_t s, const FeOp& op, const T* A, int64_t a_stride, const T* X, T* Y, int n, T alpha,
                  int dmode, int cls) {
  RC_CHECK(op.nc <= NCMAX, RCHFSI_ERR_INVALID_ARG, "n_c larger than 128");
  RC_CHECK(op.n_cells <= 0x7fffffff, RCHFSI_ERR_INVALID_ARG, "too many cells");
  dim3 grid((unsigned)op.n_cells, cdiv(n, TN));
  RC_CHECK(grid.y <= 65535u, RCHFSI_ERR_INVALID_ARG, "block too wide");
  const double nc = op.nc, C = (double)op.n_cells, es = sizeof(T);
  // algorithmic bytes: input block read once, output block read+written once, the cell matrices
  prof::Scope ps(s, cls, 2.0 * nc * nc * C * n, es * (3.0 * op.m * n + (a_stride ? C : 1.0) * nc * nc));
  fe_cell_kernel<T, TN><<<grid, 256, 0, s>>>(op.nc, op.dofs.p, A, a_stride, X, Y, n, alpha, op.Dinv.p, dmode);
  RC_LAUNCH();
}

}  // namespace

// A product Y += alpha * Op X on row-major blocks of the (possibly embedded) problem.  For a complex
// operator the block's rows [0, mc) hold real parts and [mc, 2 mc) imaginary parts:
//   Y_r += alpha (Ar X_r - Ai X_i),   Y_i += alpha (Ai X_r + Ar X_i)
// and the real B acts on each half.
template <typename T, class F>
void complex_parts(const FeOp& op, bool useB, const T* X, T* Y, int n, T alpha, F&& one) {
  if (!op.cplx) {
    one(op, X, Y, alpha);
    return;
  }
  const int64_t off = op.mc * (int64_t)n;
  if (useB) {
    one(op, X, Y, alpha);
    one(op, X + off, Y + off, alpha);
    return;
  }
  const FeOp& im = *op.imag;
  one(op, X, Y, alpha);
  one(im, X + off, Y, -alpha);
  one(im, X, Y + off, alpha);
  one(op, X + off, Y + off, alpha);
}

void fe_apply_f64_rows(cudaStream_t s, const FeOp& op, bool useB, const double* X, double* Y, int n) {
  RC_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * op.m * n, s));
  complex_parts<double>(op, useB, X, Y, n, 1.0, [&](const FeOp& o, const double* x, double* y, double al) {
    const double* M = useB ? op.B64.p : o.A64.p;
    const int64_t stride = (useB && op.B_shared) ? 0 : (int64_t)op.nc * op.nc;
    launch_cells<double, 32>(s, o, M, stride, x, y, n, al, 0, RCHFSI_KERNEL_FE_CELL_F64);
  });
}

void fe_filter_product_f64(cudaStream_t s, const FeOp& op, const double* Ry, double* Rx, int n, double a,
                           int dmode) {
  complex_parts<double>(op, false, Ry, Rx, n, a, [&](const FeOp& o, const double* x, double* y, double al) {
    launch_cells<double, 32>(s, o, o.A64.p, (int64_t)o.nc * o.nc, x, y, n, al, dmode, RCHFSI_KERNEL_FE_CELL);
  });
}

// FP32 (FFMA) filter product of one real part.
static void fe_product_f32_one(cudaStream_t s, FeOp& op, const float* Ry, float* Rx, int n, float a, int dmode) {
  const size_t na = (size_t)op.n_cells * op.nc * op.nc;
  if (!op.A32.p) {
    op.A32.ensure(na);
    cast_f64_to_f32(s, na, op.A64.p, op.A32.p, 1.0, 0);
  }
  launch_cells<float, 64>(s, op, op.A32.p, (int64_t)op.nc * op.nc, Ry, Rx, n, a, dmode, RCHFSI_KERNEL_FE_CELL);
}

void fe_filter_product_f32(cudaStream_t s, FeOp& op, int precision, const float* Ry, float* Rx, int n, float a,
                           int dmode) {
  if (precision != RCHFSI_FP32) {
    // tensor cores: the real and imaginary cell products of a complex operator in one launch
    fe_tc_product(s, op, precision, Ry, Rx, n, a, dmode);
    return;
  }
  complex_parts<float>(op, false, Ry, Rx, n, a, [&](const FeOp& o, const float* x, float* y, float al) {
    fe_product_f32_one(s, const_cast<FeOp&>(o), x, y, n, al, dmode);
  });
}

void recur_terms_rows_f32(cudaStream_t s, int64_t m, int n, const float* Ry, float* Rx, const float* W,
                          const double* lam, double a, double b, double c) {
  recur_rows_kernel<float><<<recur_grid(m, n), dim3(32, 8), 0, s>>>(m, n, Ry, Rx, W, lam, (float)a, (float)b,
                                                                     (float)c);
  RC_LAUNCH();
}

void recur_terms_rows_f32_dev(cudaStream_t s, int64_t m, int n, const float* Ry, float* Rx, const float* W,
                              const double* lam, const double* coef) {
  recur_rows_dev_kernel<<<recur_grid(m, n), dim3(32, 8), 0, s>>>(m, n, Ry, Rx, W, lam, coef);
  RC_LAUNCH();
}

void recur_terms_rows_f64(cudaStream_t s, int64_t m, int n, const double* Ry, double* Rx, const double* W,
                          const double* lam, double a, double b, double c) {
  recur_rows_kernel<double><<<recur_grid(m, n), dim3(32, 8), 0, s>>>(m, n, Ry, Rx, W, lam, a, b, c);
  RC_LAUNCH();
}

}  // namespace rchfsi
