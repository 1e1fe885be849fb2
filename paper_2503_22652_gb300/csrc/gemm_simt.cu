// SIMT (FFMA / DFMA) tiled GEMM with fused epilogues.
//
// FP64 work on this GPU is bound by the FP64 ALUs (about 1.1 TFLOP/s for the whole chip, 1/64 of
// the FP32 FFMA rate), so a register-tiled SIMT kernel reaches the FP64 roofline; the same code in
// FP32 is the "FP32 arithmetic" filter path of the paper (products in FP32 on the FFMA pipes).
//
// Tile: 64 x 64 outputs per CTA, K step 16, 256 threads, 4 x 4 outputs per thread at stride 16
// (conflict-free shared-memory reads).  The epilogue applies one of:
//   store, the Chebyshev recurrence update (Algorithm 3 / Algorithm 2 loop body),
//   reconstruction with a dense D^-1, or the residual W = AX - BX Lambda.
#include "common.cuh"
#include "prof.cuh"

namespace rchfsi {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
struct EpiDev {
  int kind;
  T* C;
  int64_t ldc;
  T alpha, beta;
  T a, b, c;
  const T* Ry;
  const T* Rx;
  const T* W;
  const double* lam;
  const T* Xadd;
  int64_t ldx;

  __device__ __forceinline__ void operator()(int64_t i, int64_t j, T acc) const {
    const int64_t o = j * ldc + i;
    switch (kind) {
      case EPI_STORE: {
        T v = alpha * acc;
        if (beta != T(0)) v += beta * C[o];
        C[o] = v;
        break;
      }
      case EPI_RECUR: {
        // R_X <- a*P + b*R_Y + c*R_X + a*W*Lambda_Y[j]
        T v = a * acc + b * Ry[o];
        if (Rx) v += c * Rx[o];
        if (W) v += a * W[o] * (T)lam[j];
        C[o] = v;
        break;
      }
      case EPI_AXPY_DIAG:
        C[o] = acc + Xadd[j * ldx + i] * (T)lam[j];
        break;
      case EPI_RESID:
        C[o] = Xadd[j * ldx + i] - acc * (T)lam[j];
        break;
    }
  }
};

template <typename T, bool AK, bool BKC>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A,
                                                       int64_t lda, const T* __restrict__ B, int64_t ldb,
                                                       EpiDev<T> epi) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      const int e = tid + q * NT;
      int ii, kk;
      if (AK) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      T v = T(0);
      if (gi < M && gk < K) v = AK ? A[gi * lda + gk] : A[gk * lda + gi];
      As[kk][ii] = v;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      const int e = tid + q * NT;
      int jj, kk;
      if (BKC) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      const int64_t gj = j0 + jj, gk = k0 + kk;
      T v = T(0);
      if (gj < N && gk < K) v = BKC ? B[gj * ldb + gk] : B[gk * ldb + gj];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t gi = i0 + ty + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gj = j0 + tx + 16 * q;
      if (gj < N) epi(gi, gj, acc[r][q]);
    }
  }
}

template <typename T>
EpiDev<T> to_dev(const EpiArgs& e) {
  EpiDev<T> d;
  d.kind = e.kind;
  d.C = (T*)e.C;
  d.ldc = e.ldc;
  d.alpha = (T)e.alpha;
  d.beta = (T)e.beta;
  d.a = (T)e.a;
  d.b = (T)e.b;
  d.c = (T)e.c;
  d.Ry = (const T*)e.Ry;
  d.Rx = (const T*)e.Rx;
  d.W = (const T*)e.W;
  d.lam = e.lam;
  d.Xadd = (const T*)e.Xadd;
  d.ldx = e.ldx;
  return d;
}

template <typename T>
void gemm_dispatch(cudaStream_t s, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool ak, const T* B,
                   int64_t ldb, bool bk, const EpiArgs& epi) {
  if (M <= 0 || N <= 0) return;
  RC_CHECK(cdiv(M, BM) <= 65535u, RCHFSI_ERR_INVALID_ARG, "gemm: M too large for the grid");
  dim3 grid(cdiv(N, BN), cdiv(M, BM));
  EpiDev<T> d = to_dev<T>(epi);
  const double es = sizeof(T);
  const double extra = (epi.kind == EPI_RECUR) ? (2.0 + (epi.Rx ? 1 : 0) + (epi.W ? 1 : 0)) : 1.0;
  prof::Scope ps(s, epi.prof_cls, 2.0 * M * N * K, es * ((double)M * K + (double)K * N + extra * M * N));
  if (ak && bk) gemm_simt_kernel<T, true, true><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d);
  else if (ak && !bk) gemm_simt_kernel<T, true, false><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d);
  else if (!ak && bk) gemm_simt_kernel<T, false, true><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d);
  else gemm_simt_kernel<T, false, false><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d);
  RC_LAUNCH();
}

}  // namespace

void gemm_f64(cudaStream_t s, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool a_kcontig,
              const double* B, int64_t ldb, bool b_kcontig, const EpiArgs& epi) {
  gemm_dispatch<double>(s, M, N, K, A, lda, a_kcontig, B, ldb, b_kcontig, epi);
}

void gemm_f32(cudaStream_t s, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, bool a_kcontig,
              const float* B, int64_t ldb, bool b_kcontig, const EpiArgs& epi) {
  gemm_dispatch<float>(s, M, N, K, A, lda, a_kcontig, B, ldb, b_kcontig, epi);
}

}  // namespace rchfsi
