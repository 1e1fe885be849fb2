// SIMT (FFMA / DFMA) tiled GEMM with fused epilogues.
//
// FP64 work on this GPU is bound by the FP64 ALUs (about 1.1 TFLOP/s for the whole chip, 1/64 of
// the FP32 FFMA rate), so a register-tiled SIMT kernel is the FP64 path; the same code in FP32 is
// the "FP32 arithmetic" filter path of the paper (products in FP32 on the FFMA pipes).
//
// Tile: 64 x 64 outputs per CTA, K step 16, 256 threads, 4 x 4 outputs per thread at stride 16
// (conflict-free shared-memory reads).  The epilogue applies one of:
//   store, the Chebyshev recurrence update (Algorithm 3 / Algorithm 2 loop body),
//   reconstruction with a dense D^-1, or the residual W = AX - BX Lambda.
// Shapes with few output tiles and a long K (the N x N Gram matrices Y^T A Y, Y^T B Y) are split
// along K across CTAs so that every SM works: each split writes its partial tile to a workspace and
// a second kernel sums the partials in a fixed order (deterministic) and applies the epilogue.
#include <algorithm>

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

// blockIdx.z selects the K slice [z*kslice, min(K, (z+1)*kslice)); with `partial` set the raw
// accumulators go to partial[z][j*M + i] instead of through the epilogue.
template <typename T, bool AK, bool BKC>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A,
                                                       int64_t lda, const T* __restrict__ B, int64_t ldb,
                                                       EpiDev<T> epi, int64_t kslice, T* __restrict__ partial) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int64_t j0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kslice;
  const int64_t kend = min(K, kbeg + kslice);
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      const int e = tid + q * NT;
      int ii, kk;
      if (AK) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      const int64_t gi = i0 + ii, gk = k0 + kk;
      T v = T(0);
      if (gi < M && gk < kend) v = AK ? A[gi * lda + gk] : A[gk * lda + gi];
      As[kk][ii] = v;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      const int e = tid + q * NT;
      int jj, kk;
      if (BKC) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      const int64_t gj = j0 + jj, gk = k0 + kk;
      T v = T(0);
      if (gj < N && gk < kend) v = BKC ? B[gj * ldb + gk] : B[gk * ldb + gj];
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
      if (gj < N) {
        if (partial) partial[((int64_t)blockIdx.z * N + gj) * M + gi] = acc[r][q];
        else epi(gi, gj, acc[r][q]);
      }
    }
  }
}

// Matrix-vector shapes (N <= 4, A K-contiguous): one warp per output row, lanes over K.  The tiled
// kernel would compute a 64-wide tile for each of these columns.
template <typename T, bool BKC>
__global__ void __launch_bounds__(256) gemv_kernel(int64_t M, int N, int64_t K, const T* __restrict__ A, int64_t lda,
                                                   const T* __restrict__ B, int64_t ldb, EpiDev<T> epi) {
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= M) return;
  const T* arow = A + i * lda;
  if (N == 1) {
    // one column: four independent partial sums (no FMA on columns that do not exist; on this GPU
    // a warp-wide FP64 instruction holds the FP64 pipe whether or not its result is used)
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int64_t k = lane;
    for (; k + 96 < K; k += 128) {
      const int64_t s1 = BKC ? 32 : 32 * ldb;
      const T* b = BKC ? B + k : B + k * ldb;
      a0 = fma(arow[k], b[0], a0);
      a1 = fma(arow[k + 32], b[s1], a1);
      a2 = fma(arow[k + 64], b[2 * s1], a2);
      a3 = fma(arow[k + 96], b[3 * s1], a3);
    }
    for (; k < K; k += 32) a0 = fma(arow[k], BKC ? B[k] : B[k * ldb], a0);
    T v = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) epi(i, 0, v);
    return;
  }
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t k = lane; k < K; k += 32) {
    const T a = arow[k];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < N) acc[j] = fma(a, BKC ? B[(int64_t)j * ldb + k] : B[k * ldb + j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane < N) {
    T v = acc[0];
#pragma unroll
    for (int j = 1; j < 4; ++j)
      if (lane == j) v = acc[j];
    epi(i, lane, v);
  }
}

template <typename T>
__global__ void splitk_sum_kernel(int64_t M, int64_t N, int nsplit, const T* __restrict__ partial, EpiDev<T> epi) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / M, i = e - j * M;
    T acc = T(0);
    for (int s = 0; s < nsplit; ++s) acc += partial[(int64_t)s * total + e];
    epi(i, j, acc);
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

// Per-host-thread workspace of split-K partials (calls of one thread run in stream order).
template <typename T>
DevBuf<T>& split_ws() {
  static thread_local DevBuf<T> ws;
  return ws;
}

template <typename T>
void gemm_dispatch(cudaStream_t s, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool ak, const T* B,
                   int64_t ldb, bool bk, const EpiArgs& epi) {
  if (M <= 0 || N <= 0) return;
  if (N <= 4 && ak) {
    EpiDev<T> d = to_dev<T>(epi);
    prof::Scope ps(s, epi.prof_cls, 2.0 * M * N * K, (double)sizeof(T) * ((double)M * K + (double)K * N + M * N));
    if (bk) gemv_kernel<T, true><<<cdiv(M, 8), 256, 0, s>>>(M, (int)N, K, A, lda, B, ldb, d);
    else gemv_kernel<T, false><<<cdiv(M, 8), 256, 0, s>>>(M, (int)N, K, A, lda, B, ldb, d);
    RC_LAUNCH();
    return;
  }
  RC_CHECK(cdiv(M, BM) <= 65535u, RCHFSI_ERR_INVALID_ARG, "gemm: M too large for the grid");
  const int64_t tiles = (int64_t)cdiv(N, BN) * cdiv(M, BM);
  // split K when the output alone cannot fill the GPU (target ~4 CTAs per SM, slices >= 2 BK)
  int nsplit = 1;
  const int64_t want = 152 * 4;
  if (tiles < want && K >= 4 * BK) {
    nsplit = (int)std::min<int64_t>((want + tiles - 1) / tiles, K / (2 * BK));
    nsplit = std::max(nsplit, 1);
    nsplit = std::min(nsplit, 64);
  }
  int64_t kslice = (K + nsplit - 1) / nsplit;
  kslice = (kslice + BK - 1) / BK * BK;
  nsplit = (int)((K + kslice - 1) / kslice);
  if (nsplit < 1) nsplit = 1;
  T* part = nullptr;
  if (nsplit > 1) part = split_ws<T>().ensure((size_t)nsplit * M * N);
  dim3 grid(cdiv(N, BN), cdiv(M, BM), nsplit);
  EpiDev<T> d = to_dev<T>(epi);
  const double es = sizeof(T);
  const double extra = (epi.kind == EPI_RECUR) ? (2.0 + (epi.Rx ? 1 : 0) + (epi.W ? 1 : 0)) : 1.0;
  prof::Scope ps(s, epi.prof_cls, 2.0 * M * N * K, es * ((double)M * K + (double)K * N + extra * M * N));
  if (ak && bk) gemm_simt_kernel<T, true, true><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d, kslice, part);
  else if (ak && !bk) gemm_simt_kernel<T, true, false><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d, kslice, part);
  else if (!ak && bk) gemm_simt_kernel<T, false, true><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d, kslice, part);
  else gemm_simt_kernel<T, false, false><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, d, kslice, part);
  RC_LAUNCH();
  if (nsplit > 1) {
    const int64_t total = M * N;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
    splitk_sum_kernel<T><<<blocks, 256, 0, s>>>(M, N, nsplit, part, d);
    RC_LAUNCH();
  }
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
