// Real embedding of complex Hermitian problems.
//
// A complex Hermitian pencil (A, B) with real B is solved as the real symmetric pencil of twice
// the size: A_e = [[Ar, -Ai], [Ai, Ar]], B_e = diag(B, B), D_e^-1 = diag(D^-1, D^-1).  A complex
// vector x = xr + i xi maps to [xr; xi]; its multiple i x maps to [-xi; xr].  Every complex
// eigenpair appears twice in the real pencil, with the same eigenvalue.  A block of N complex
// vectors is embedded as the 2m x 2N real block [[Xr, -Xi], [Xi, Xr]] so that its real span is
// closed under multiplication by i.  Complex blocks at the C ABI are row-major interleaved
// (re, im) pairs; embedded blocks are column-major (leading dimension 2m).
#include "common.cuh"

namespace rchfsi {
namespace {

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

__global__ void deinterleave_kernel(int64_t n, const double* __restrict__ in, double* __restrict__ re,
                                    double* __restrict__ im) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    re[e] = in[2 * e];
    im[e] = in[2 * e + 1];
  }
}

// Xc: m x N complex row-major interleaved; Xe: 2m x 2N column-major.
__global__ void embed_block_kernel(int64_t m, int64_t N, const double* __restrict__ Xc, double* __restrict__ Xe) {
  const int64_t total = m * N;
  const int64_t m2 = 2 * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e - i * N;
    const double xr = Xc[2 * e], xi = Xc[2 * e + 1];
    Xe[j * m2 + i] = xr;
    Xe[j * m2 + m + i] = xi;
    Xe[(N + j) * m2 + i] = -xi;
    Xe[(N + j) * m2 + m + i] = xr;
  }
}

// Yc (m x ncols complex row-major) column j = embedded column cols[j] of Xe (2m rows, column-major).
__global__ void extract_cols_kernel(int64_t m, int64_t ncols, const double* __restrict__ Xe,
                                    const int* __restrict__ cols, double* __restrict__ Yc) {
  const int64_t total = m * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, j = e - i * ncols;
    const int64_t c = cols[j];
    Yc[2 * e] = Xe[c * 2 * m + i];
    Yc[2 * e + 1] = Xe[c * 2 * m + m + i];
  }
}

// Ac: m x m complex row-major interleaved -> Ae: 2m x 2m real row-major [[Ar, -Ai], [Ai, Ar]].
__global__ void embed_dense_kernel(int64_t m, const double* __restrict__ Ac, double* __restrict__ Ae) {
  const int64_t total = m * m;
  const int64_t m2 = 2 * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m, k = e - i * m;
    const double ar = Ac[2 * e], ai = Ac[2 * e + 1];
    Ae[i * m2 + k] = ar;
    Ae[i * m2 + m + k] = -ai;
    Ae[(m + i) * m2 + k] = ai;
    Ae[(m + i) * m2 + m + k] = ar;
  }
}

// B (m x m real) -> diag(B, B) (2m x 2m), off-diagonal blocks zero.
__global__ void embed_blockdiag_kernel(int64_t m, const double* __restrict__ B, double* __restrict__ Be) {
  const int64_t total = m * m;
  const int64_t m2 = 2 * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m, k = e - i * m;
    const double b = B[e];
    Be[i * m2 + k] = b;
    Be[i * m2 + m + k] = 0.0;
    Be[(m + i) * m2 + k] = 0.0;
    Be[(m + i) * m2 + m + k] = b;
  }
}

// Complex B-inner products of column pairs of the embedded block: for candidate columns u, v of
// Xe with B-images BXe, out = u^H B v as (re, im) where u_c = u_top + i u_bot:
//   re = u_top . (Bv)_top + u_bot . (Bv)_bot,  im = u_top . (Bv)_bot - u_bot . (Bv)_top
__global__ void cplx_dot_kernel(int64_t m, const double* __restrict__ Xe, const double* __restrict__ BXe, int cu,
                                int cv, double* out) {
  __shared__ double red[2][32];
  const int64_t m2 = 2 * m;
  const double* ut = Xe + (int64_t)cu * m2;
  const double* bv = BXe + (int64_t)cv * m2;
  double re = 0.0, im = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    re += ut[i] * bv[i] + ut[m + i] * bv[m + i];
    im += ut[i] * bv[m + i] - ut[m + i] * bv[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    out[0] = a;
    out[1] = b;
  }
}

// v <- (v - alpha u) * scale in the complex sense, for the column and its A- and B-images:
// column v_c = v_top + i v_bot, alpha = ar + i ai.  Null arrays are skipped.
__global__ void cplx_axpy_kernel(int64_t m, double* Xe, double* AXe, double* BXe, int cu, int cv, double ar,
                                 double ai, double scale) {
  const int64_t m2 = 2 * m;
  double* arrs[3] = {Xe, AXe, BXe};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    for (int which = 0; which < 3; ++which) {
      double* base = arrs[which];
      if (!base) continue;
      const double ur = base[(int64_t)cu * m2 + i], ui = base[(int64_t)cu * m2 + m + i];
      double& vr = base[(int64_t)cv * m2 + i];
      double& vi = base[(int64_t)cv * m2 + m + i];
      const double nr = vr - (ar * ur - ai * ui);
      const double ni = vi - (ar * ui + ai * ur);
      vr = nr * scale;
      vi = ni * scale;
    }
  }
}

// dst (2m x 2N, column-major) = [src(:, cols), J src(:, cols)] with J [x_top; x_bot] = [-x_bot; x_top]
// (multiplication by i).  cols == null means the identity, in which case src may equal dst.
__global__ void rebuild_kernel(int64_t m, int64_t N, const double* src, const int* __restrict__ cols, double* dst) {
  const int64_t total = m * N;
  const int64_t m2 = 2 * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    const int64_t c = cols ? cols[j] : j;
    const double xt = src[c * m2 + i], xb = src[c * m2 + m + i];
    dst[j * m2 + i] = xt;
    dst[j * m2 + m + i] = xb;
    dst[(N + j) * m2 + i] = -xb;
    dst[(N + j) * m2 + m + i] = xt;
  }
}

// Gram matrix of an embedded block Y = [Y1, J Y1] (2N x 2N, column-major) from its left half:
// G = [[P, Q], [-Q, P]], so G(i, N + j) = -G(N + i, j) for i < N and G(i - N, j) for i >= N.
__global__ void gram_complete_kernel(int64_t N, double* G) {
  const int64_t n2 = 2 * N, total = n2 * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n2, i = e - j * n2;
    G[(N + j) * n2 + i] = i < N ? -G[j * n2 + N + i] : G[j * n2 + i - N];
  }
}

// dst(:, j) = src(:, cols[j]) for column-major blocks with `rows` rows.
__global__ void gather_cols_kernel(int64_t rows, int64_t ncols, const double* __restrict__ src,
                                   const int* __restrict__ cols, double* __restrict__ dst) {
  const int64_t total = rows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, i = e - j * rows;
    dst[e] = src[(int64_t)cols[j] * rows + i];
  }
}

}  // namespace

void cplx_gram_complete(cudaStream_t s, int64_t N, double* G) {
  gram_complete_kernel<<<blocks_for(2 * N * N), 256, 0, s>>>(N, G);
  RC_LAUNCH();
}

void gather_cols_f64(cudaStream_t s, int64_t rows, int64_t ncols, const double* src, const int* cols, double* dst) {
  gather_cols_kernel<<<blocks_for(rows * ncols), 256, 0, s>>>(rows, ncols, src, cols, dst);
  RC_LAUNCH();
}

void cplx_deinterleave(cudaStream_t s, int64_t n, const double* in, double* re, double* im) {
  deinterleave_kernel<<<blocks_for(n), 256, 0, s>>>(n, in, re, im);
  RC_LAUNCH();
}

void cplx_embed_block(cudaStream_t s, int64_t m, int64_t N, const double* Xc, double* Xe) {
  embed_block_kernel<<<blocks_for(m * N), 256, 0, s>>>(m, N, Xc, Xe);
  RC_LAUNCH();
}

void cplx_extract_cols(cudaStream_t s, int64_t m, int64_t ncols, const double* Xe, const int* cols, double* Yc) {
  extract_cols_kernel<<<blocks_for(m * ncols), 256, 0, s>>>(m, ncols, Xe, cols, Yc);
  RC_LAUNCH();
}

void cplx_embed_dense(cudaStream_t s, int64_t m, const double* Ac, double* Ae) {
  embed_dense_kernel<<<blocks_for(m * m), 256, 0, s>>>(m, Ac, Ae);
  RC_LAUNCH();
}

void cplx_embed_blockdiag(cudaStream_t s, int64_t m, const double* B, double* Be) {
  embed_blockdiag_kernel<<<blocks_for(m * m), 256, 0, s>>>(m, B, Be);
  RC_LAUNCH();
}

void cplx_dot(cudaStream_t s, int64_t m, const double* Xe, const double* BXe, int cu, int cv, double* out) {
  cplx_dot_kernel<<<1, 1024, 0, s>>>(m, Xe, BXe, cu, cv, out);
  RC_LAUNCH();
}

void cplx_axpy(cudaStream_t s, int64_t m, double* Xe, double* AXe, double* BXe, int cu, int cv, double ar,
               double ai, double scale) {
  cplx_axpy_kernel<<<blocks_for(m), 256, 0, s>>>(m, Xe, AXe, BXe, cu, cv, ar, ai, scale);
  RC_LAUNCH();
}

void cplx_rebuild(cudaStream_t s, int64_t m, int64_t N, const double* src, const int* cols, double* dst) {
  RC_CHECK(cols == nullptr || src != dst, RCHFSI_ERR_INVALID_ARG, "cplx_rebuild: gather must not be in place");
  rebuild_kernel<<<blocks_for(m * N), 256, 0, s>>>(m, N, src, cols, dst);
  RC_LAUNCH();
}

}  // namespace rchfsi
