// Shared internal definitions of the R-ChFSI CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <stdexcept>
#include <vector>

#include "../../include/rchfsi.h"

namespace rchfsi {

// Error raised inside the library; converted to a status code at the C ABI.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

#define RC_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::rchfsi::Error(RCHFSI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                                 " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)

#define RC_CHECK(cond, code, msg)                    \
  do {                                               \
    if (!(cond)) throw ::rchfsi::Error((code), (msg)); \
  } while (0)

// Count of this library's kernel launches (read through rchfsi_profile_read).
int64_t& launch_counter();

// Raise a kernel's dynamic shared-memory limit on the current device to `bytes`.  The attribute is
// per function and per device and shared by every host thread: this sets it once per (kernel,
// device, size) under a lock, so concurrent callers on any device never launch before it is set.
void set_smem_limit(const void* kernel, int bytes);

// The driver's cuTensorMapEncodeTiled (PFN_cuTensorMapEncodeTiled_v12000), looked up once.
void* tensor_map_encoder();

#define RC_LAUNCH()                                   \
  do {                                                \
    RC_CUDA(cudaGetLastError());                      \
    __atomic_add_fetch(&::rchfsi::launch_counter(), 1, __ATOMIC_RELAXED); \
  } while (0)

// Owning device buffer.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // Ensure capacity for `count` elements (contents are not preserved on growth).
  T* ensure(size_t count) {
    if (count <= n && p) return p;
    release();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error(RCHFSI_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
    return p;
  }
  size_t bytes() const { return n * sizeof(T); }
  // Take over o's allocation (o is left empty); this buffer's own allocation is released.
  void take(DevBuf& o) {
    if (&o == this) return;
    release();
    p = o.p;
    n = o.n;
    o.p = nullptr;
    o.n = 0;
  }
};

inline bool is_device_pointer(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------- kernels (launchers)
// All matrices are dense; "col" = column-major (each column contiguous, leading dim = rows),
// "row" = row-major.  Internal m x N blocks are column-major.

// C = op(A) op(B) consumed by an epilogue.  A(i,k) at A[i*lda+k] if a_kcontig else A[k*lda+i];
// B(k,j) at B[j*ldb+k] if b_kcontig else B[k*ldb+j].
enum EpiKind { EPI_STORE = 0, EPI_RECUR = 1, EPI_AXPY_DIAG = 2, EPI_RESID = 3 };

struct EpiArgs {
  int kind = EPI_STORE;
  // EPI_STORE:     C[j*ldc+i] = alpha*acc + beta*C[j*ldc+i]
  // EPI_RECUR:     Rx = a*acc + b*Ry + c*Rx + a*W*lam[j]   (W may be null; Rx may equal out)
  // EPI_AXPY_DIAG: C = acc + Xadd[j*ldx+i]*lam[j]           (reconstruction with dense D^-1)
  // EPI_RESID:     C = Xadd - acc*lam[j]                    (W = AX - BX Lambda)
  void* C = nullptr;
  int64_t ldc = 0;
  double alpha = 1.0, beta = 0.0;
  double a = 0, b = 0, c = 0;
  const void* Ry = nullptr;
  const void* Rx = nullptr;
  const void* W = nullptr;
  const double* lam = nullptr;
  const void* Xadd = nullptr;
  int64_t ldx = 0;
  int prof_cls = RCHFSI_KERNEL_GEMM_F64;  // kernel class for the opt-in timers
};

void gemm_f64(cudaStream_t s, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool a_kcontig,
              const double* B, int64_t ldb, bool b_kcontig, const EpiArgs& epi);
void gemm_f32(cudaStream_t s, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, bool a_kcontig,
              const float* B, int64_t ldb, bool b_kcontig, const EpiArgs& epi);

// Elementwise / layout kernels.
void transpose_f64(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin, double* out,
                   int64_t ldout);  // out(j,i) = in(i,j), both row-major views
void scale_cols_f64(cudaStream_t s, int64_t m, int64_t n, double* X, int64_t ld, const double* scale);
void col_norms_f64(cudaStream_t s, int64_t m, int64_t n, const double* X, int64_t ld, double* out);
void scale_rows_f64(cudaStream_t s, int64_t m, int64_t n, const double* in, double* out, const double* d,
                    bool cols);  // out = diag(d)*in (cols=false) or in*diag(d) (cols=true); row-major m x n
// o1 = (float)(s1 W), o2 = (float)(s2 W) as row-major m x n blocks, W column-major (leading dim m)
void cols_to_rows_f32x2(cudaStream_t s, int64_t m, int64_t n, const double* W, double s1, double s2, float* o1,
                        float* o2);
// Y = dinv .* (rs R) + X diag(lam), R row-major float m x n, X and Y column-major (leading dim m)
void rows_to_cols_recon(cudaStream_t s, int64_t m, int64_t n, const float* R, double rs, const double* dinv,
                        const double* X, const double* lam, double* Y);
void cast_f64_to_f32(cudaStream_t s, int64_t n, const double* in, float* out, double scale, int round_tf32);
void cast_f64_to_bf16(cudaStream_t s, int64_t n, const double* in, __nv_bfloat16* out, double scale);
void cast_f32_to_f64(cudaStream_t s, int64_t n, const float* in, double* out, double scale = 1.0);
void fill_zero(cudaStream_t s, void* p, size_t bytes);
void scaled_copy_f64(cudaStream_t s, int64_t n, const double* in, double* out, double scale);
// Yp(col) = dinv .* R + X .* lam  (R of type float/double, col-major m x n)
// (R has leading dimension ldr; X and Y have leading dimension m.)
void reconstruct_f64(cudaStream_t s, int64_t m, int64_t n, const double* R, int64_t ldr, const double* dinv,
                     const double* X, const double* lam, double* Y);
void reconstruct_f32(cudaStream_t s, int64_t m, int64_t n, const float* R, int64_t ldr, const double* dinv,
                     const double* X, const double* lam, double* Y);
void reconstruct_bf16(cudaStream_t s, int64_t m, int64_t n, const __nv_bfloat16* R, int64_t ldr,
                      const double* dinv, const double* X, const double* lam, double* Y);
// 2D casts: `rows` rows of `cols` contiguous elements, pitches ldin / ldout (elements).
void cast2d_f64_to_f32(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin, float* out,
                       int64_t ldout, double scale, int round_tf32);
void cast2d_f64_to_bf16(cudaStream_t s, int64_t rows, int64_t cols, const double* in, int64_t ldin,
                        __nv_bfloat16* out, int64_t ldout, double scale);
// Recurrence update without a product (for FE: Rx = b*Ry + c*Rx + a*W*lam), generic storage
void recur_axpby_f32(cudaStream_t s, int64_t m, int64_t n, const float* Ry, float* Rx, const float* W,
                     const double* lam, double a, double b, double c);
// Residual-norm helpers
void resid_rel_norms(cudaStream_t s, int64_t m, int64_t n, const double* W, const double* X, double* out_abs,
                     double* out_xnorm);

// Small dense FP64 kernels (N x N, column-major).
void symmetrize_f64(cudaStream_t s, int n, double* A, int lda);
// A += factor * tr(A) * I (n x n, leading dimension lda)
void shift_diag_by_trace_f64(cudaStream_t s, int n, double* A, int lda, double factor);
// Cholesky G = L L^T and L^-1 (small_eig.cu): A (n x n, col-major) destroyed; L, Linv lower triangular.
int cholesky_inverse_f64(cudaStream_t s, int n, double* A, double* L, double* Linv, int* d_info, int num_sms,
                         DevBuf<double>& scratch);
// Symmetric eigensolver (small_eig.cu: Householder tridiagonalisation, bisection, inverse iteration):
// M destroyed; V (column-major eigenvectors) and evals ascending.  Returns false when it declines the
// problem (order > 3072 or a cluster of close eigenvalues too large for inverse iteration).
// oz: when set, the N x N products of its orthogonalisation step run FP64-accurate on the tensor
// cores (oz_gemm.cuh) instead of as FP64 GEMMs.
struct OzScratch;
bool sym_eig_f64(cudaStream_t s, int n, double* M, double* V, double* evals, DevBuf<double>& ws, int* d_flag,
                 int num_sms, const OzScratch* oz = nullptr);
// Symmetric eigensolver (parallel cyclic Jacobi, jacobi.cu): M destroyed; V, evals ascending.
int jacobi_eig_f64(cudaStream_t s, int n, double* M, double* V, double* evals, DevBuf<double>& ws, double tol,
                   int max_sweeps);

// Real embedding of complex Hermitian problems (cplx.cu).
void cplx_deinterleave(cudaStream_t s, int64_t n, const double* in, double* re, double* im);
void cplx_embed_block(cudaStream_t s, int64_t m, int64_t N, const double* Xc, double* Xe);
void cplx_extract_cols(cudaStream_t s, int64_t m, int64_t ncols, const double* Xe, const int* cols, double* Yc);
void cplx_embed_dense(cudaStream_t s, int64_t m, const double* Ac, double* Ae);
void cplx_embed_blockdiag(cudaStream_t s, int64_t m, const double* B, double* Be);
void cplx_dot(cudaStream_t s, int64_t m, const double* Xe, const double* BXe, int cu, int cv, double* out);
void cplx_axpy(cudaStream_t s, int64_t m, double* Xe, double* AXe, double* BXe, int cu, int cv, double ar,
               double ai, double scale);
void cplx_rebuild(cudaStream_t s, int64_t m, int64_t N, const double* src, const int* cols, double* dst);
void cplx_gram_complete(cudaStream_t s, int64_t N, double* G);  // right half of [[P, Q], [-Q, P]] (2N x 2N)
void gather_cols_f64(cudaStream_t s, int64_t rows, int64_t ncols, const double* src, const int* cols, double* dst);

// Lanczos vector helpers
void dot_f64(cudaStream_t s, int64_t n, const double* x, const double* y, double* out);

}  // namespace rchfsi
