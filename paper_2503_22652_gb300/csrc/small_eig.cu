// Small dense FP64 kernels of the Rayleigh-Ritz step (Section 2.1, Algorithm 1): the Cholesky factor
// of the B-Gram matrix with its inverse, and the symmetric eigensolver of the projected matrix.
//
// On this GPU FP64 arithmetic is scarce (about 2 DFMA per clock per SM) and the N x N problems
// (N = 60 ... 2400) are too small to fill the chip, so these steps are bound by the length of
// their sequential dependency chains.  The kernels keep every chain on the device and pay one
// barrier per elimination step:
//   * chol_inv_kernel: right-looking Cholesky G = L L^T (one barrier per column), then L^-1 column
//     by column (each column of L^-1 is an independent forward substitution, owned by one warp);
//   * tridiag_kernel: Householder reduction to tridiagonal form Q^T M Q = T (two barriers per
//     column: after the symmetric matrix-vector product, after the rank-2 update); for one cluster,
//     tridiag_dsmem_kernel exchanges through distributed shared memory and has the owner of the
//     next pivot column compute its Householder scalars during the update;
//   * bisect_kernel: eigenvalues of T by Sturm-sequence multisection, one warp per eigenvalue
//     (32 trial points per step), the Sturm recurrence free of per-step checks (exact zeros are
//     detected off the dependency chain and only then recounted with the substitution);
//   * inviter_kernel: eigenvectors of T by inverse iteration (tridiagonal LU with partial pivoting),
//     Gram-Schmidt inside clusters of numerically equal eigenvalues (gap <= 1e-9 ||T||), then one
//     Newton-Schulz step Z <- Z (3 I - Z^T Z) / 2 (two GEMMs) for the O(eps ||T|| / gap) residue
//     between the others, which leaves each residual at O(eps ||T||);
//   * backtransform_kernel: V = Q Z, one warp per eigenvector.
// The multi-CTA kernels run as one thread-block cluster (barrier.cluster) when the matrix is small,
// or as a cooperative grid (grid-wide barrier) when more SMs pay for the extra barrier cost; the
// "resident" variants keep each CTA's columns in shared memory.  Data written by another CTA is read
// with ld.global.cg (L2), never through a possibly stale L1 line.
#include <cooperative_groups.h>

#include <cfloat>

#include "common.cuh"
#include "oz_gemm.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace rchfsi {
namespace {

constexpr int EIG_THREADS = 512;

template <bool CLUSTER>
__device__ __forceinline__ void all_sync() {
  if constexpr (CLUSTER) {
    cg::this_cluster().sync();
  } else {
    cg::this_grid().sync();
  }
}

// Sum over the CTA; every thread receives the result.  `red` holds 33 doubles.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Two warp sums with their shuffle / add latencies interleaved.
__device__ __forceinline__ void warp_sum2(double& a, double& b) {
  for (int o = 16; o > 0; o >>= 1) {
    const double ta = __shfl_xor_sync(0xffffffffu, a, o), tb = __shfl_xor_sync(0xffffffffu, b, o);
    a += ta;
    b += tb;
  }
}

// The loops below walk rows in warp-uniform chunks of 32, four chunks per iteration with all loads
// issued before the FMAs: an FP64 FMA has ~64 clocks of latency, so a load-FMA-store chain per
// element leaves the FP64 pipe idle, while a chunk that lies past the end is skipped as a whole (on
// this GPU a warp-wide FP64 instruction occupies the SM's FP64 pipe for ~12 clocks whatever its
// active lanes, so the FMA count must stay that of the plain loop).
// Lane partial of sum_{i < rr} mc[i] v[i].
__device__ __forceinline__ double dot_part(const double* mc, const double* v, int rr, int lane) {
  double a0 = 0.0, a1 = 0.0;
  for (int c0 = 0; c0 < rr; c0 += 128) {
    double m[4], x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = c0 + 32 * u + lane;
      m[u] = i < rr ? mc[i] : 0.0;
      x[u] = i < rr ? v[i] : 0.0;
    }
    if (c0 < rr) a0 = fma(m[0], x[0], a0);
    if (c0 + 32 < rr) a1 = fma(m[1], x[1], a1);
    if (c0 + 64 < rr) a0 = fma(m[2], x[2], a0);
    if (c0 + 96 < rr) a1 = fma(m[3], x[3], a1);
  }
  return a0 + a1;
}

// mc[i] -= v[i] wc + w[i] vc for i < rr; with S2, also the lane partial of sum_{i >= 2} mc[i]^2 of
// the new values.
template <bool S2>
__device__ __forceinline__ double rank2_part(double* mc, const double* v, const double* w, double vc, double wc,
                                             int rr, int lane) {
  double s2 = 0.0;
  for (int c0 = 0; c0 < rr; c0 += 128) {
    double m[4], x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = c0 + 32 * u + lane;
      m[u] = i < rr ? mc[i] : 0.0;
      x[u] = i < rr ? v[i] : 0.0;
      y[u] = i < rr ? w[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (c0 + 32 * u < rr) {
        const int i = c0 + 32 * u + lane;
        const double nm = fma(-y[u], vc, fma(-x[u], wc, m[u]));
        if (i < rr) mc[i] = nm;
        if (S2) s2 = fma(i >= 2 && i < rr ? nm : 0.0, nm, s2);
      }
    }
  }
  return s2;
}

// ------------------------------------------------------------------ Cholesky and L^-1
// A (n x n, column-major, symmetric; its lower triangle is destroyed), L and Linv (outputs,
// lower triangular with zero upper part).  info = j + 1 when pivot j is not positive / finite.
// Column k of the trailing matrix is owned by CTA k mod P.
template <bool CLUSTER>
__global__ void __launch_bounds__(EIG_THREADS) chol_inv_kernel(int n, double* A, double* L, double* Linv,
                                                               int* info) {
  extern __shared__ double sm[];
  double* col = sm;      // n: scaled pivot column of the current step
  double* col2 = sm + n; // n: second buffer for the inverse phase
  const int P = gridDim.x, r = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  bool bad = false;
  for (int j = 0; j < n; ++j) {
    const double ajj = __ldcg(A + (int64_t)j * n + j);
    if (!(ajj > 0.0) || !isfinite(ajj)) {
      // every CTA reads the same value, so all leave the loop at the same step
      if (r == 0 && tid == 0) *info = j + 1;
      bad = true;
      break;
    }
    const double piv = sqrt(ajj), inv = 1.0 / piv;
    for (int i = j + 1 + tid; i < n; i += blockDim.x) col[i] = __ldcg(A + (int64_t)j * n + i) * inv;
    __syncthreads();
    if (j % P == r) {
      for (int i = tid; i < n; i += blockDim.x) L[(int64_t)j * n + i] = i < j ? 0.0 : (i == j ? piv : col[i]);
    }
    // trailing update of the owned columns k > j (lower part): A(i,k) -= L(i,j) L(k,j)
    const int k0 = j + 1 + ((r - (j + 1)) % P + P) % P;  // first owned column > j
    for (int k = k0 + warp * P; k < n; k += nw * P) {
      const double lk = col[k];
      double* ak = A + (int64_t)k * n;
      for (int i = k + lane; i < n; i += 32) ak[i] -= col[i] * lk;
    }
    all_sync<CLUSTER>();
  }
  if (bad) return;
  if (r == 0 && tid == 0) *info = 0;
  // L^-1: column c solves L x = e_c; the warp owning c does every step of that column
  for (int c = r + warp * P; c < n; c += nw * P)
    for (int i = lane; i < n; i += 32) Linv[(int64_t)c * n + i] = (i == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double* lc = (k & 1) ? col2 : col;
    for (int i = k + tid; i < n; i += blockDim.x) lc[i] = __ldcg(L + (int64_t)k * n + i);
    __syncthreads();
    const double inv = 1.0 / lc[k];
    for (int c = r + warp * P; c <= k && c < n; c += nw * P) {
      double* x = Linv + (int64_t)c * n;
      const double xk = x[k] * inv;
      __syncwarp();
      if (lane == 0) x[k] = xk;
      for (int i = k + 1 + lane; i < n; i += 32) x[i] -= lc[i] * xk;
      __syncwarp();
    }
    // the other buffer is refilled next step, after every warp has left this one (2 steps apart)
  }
}

// Same factorisation with the owned columns resident in shared memory (nq = ceil(n / P) columns per
// CTA), the pivot column exchanged through a double-buffered L2 slot (xch, 2 n doubles: the owner of
// column j + 1 publishes it during step j while the others may still read column j), one barrier
// per column.  L^-1 then runs as in chol_inv_kernel, with the next column of L prefetched into
// registers (rows tid + 256 t, t < 16, so n <= 4096).
template <bool CLUSTER>
__global__ void __launch_bounds__(256) chol_inv_smem_kernel(int n, const double* __restrict__ A, double* L,
                                                            double* Linv, double* xch, double* dinv, int* info) {
  extern __shared__ double sm[];
  constexpr int MAXT = 16;
  const int P = gridDim.x, r = blockIdx.x;
  const int nq = (n - r + P - 1) / P;
  double* cols = sm;                  // nq x n
  double* col = cols + (size_t)nq * n;  // n (scaled pivot column), later the first L^-1 buffer
  double* col2 = col + n;             // n
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5, bd = blockDim.x;
  for (int q = 0; q < nq; ++q)
    for (int i = tid; i < n; i += bd) cols[(size_t)q * n + i] = A[(size_t)(r + q * P) * n + i];
  __syncthreads();
  if (r == 0)
    for (int i = tid; i < n; i += bd) __stcg(xch + i, cols[i]);
  all_sync<CLUSTER>();
  bool bad = false;
  for (int j = 0; j < n; ++j) {
    const double* xj = xch + (size_t)(j & 1) * n;
    const double ajj = __ldcg(xj + j);
    if (!(ajj > 0.0) || !isfinite(ajj)) {
      if (r == 0 && tid == 0) *info = j + 1;
      bad = true;
      break;
    }
    const double inv = rsqrt(ajj), piv = ajj * inv;
    for (int i = j + 1 + tid; i < n; i += bd) col[i] = __ldcg(xj + i) * inv;
    __syncthreads();
    if (j % P == r) {
      for (int i = tid; i < n; i += bd) L[(size_t)j * n + i] = i < j ? 0.0 : (i == j ? piv : col[i]);
      if (tid == 0) __stcg(dinv + j, inv);
    }
    const int qa = (j + 1 - r + P - 1) / P > 0 ? (j + 1 - r + P - 1) / P : 0;
    for (int q = qa + warp; q < nq; q += nw) {
      const int k = r + q * P;
      const double lk = col[k];
      double* ak = cols + (size_t)q * n;
      for (int i = k + lane; i < n; i += 32) ak[i] -= col[i] * lk;
    }
    __syncthreads();
    if (j + 1 < n && (j + 1) % P == r) {
      const double* ak = cols + (size_t)((j + 1 - r) / P) * n;
      double* xn = xch + (size_t)((j + 1) & 1) * n;
      for (int i = j + 1 + tid; i < n; i += bd) __stcg(xn + i, ak[i]);
    }
    all_sync<CLUSTER>();
  }
  if (bad) return;
  if (r == 0 && tid == 0) *info = 0;
  for (int c = r + warp * P; c < n; c += nw * P)
    for (int i = lane; i < n; i += 32) Linv[(size_t)c * n + i] = (i == c) ? 1.0 : 0.0;
  double cur[MAXT], nxt[MAXT];
  double dcur = __ldcg(dinv), dnxt = 0.0;
#pragma unroll
  for (int t = 0; t < MAXT; ++t) {
    const int i = tid + bd * t;
    cur[t] = i < n ? __ldcg(L + i) : 0.0;
  }
  for (int k = 0; k < n; ++k) {
    double* lc = (k & 1) ? col2 : col;
#pragma unroll
    for (int t = 0; t < MAXT; ++t) {
      const int i = tid + bd * t;
      if (i >= k && i < n) lc[i] = cur[t];
    }
    if (k + 1 < n) {
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        const int i = tid + bd * t;
        nxt[t] = (i >= k + 1 && i < n) ? __ldcg(L + (size_t)(k + 1) * n + i) : 0.0;
      }
      dnxt = __ldcg(dinv + k + 1);
    }
    __syncthreads();
    const double inv = dcur;
    for (int c = r + warp * P; c <= k && c < n; c += nw * P) {
      double* x = Linv + (size_t)c * n;
      const double xk = x[k] * inv;
      __syncwarp();
      if (lane == 0) x[k] = xk;
      for (int i = k + 1 + lane; i < n; i += 32) x[i] -= lc[i] * xk;
      __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < MAXT; ++t) cur[t] = nxt[t];
    dcur = dnxt;
  }
}

// ------------------------------------------------------------------ blocked Cholesky and L^-1
// A = L L^T (A symmetric positive definite, n x n column-major, lower triangle read) and L^-1, on a
// cooperative grid, in 32 x 32 tiles: per block column K, one CTA factors the diagonal tile and
// inverts its factor (DI_K), all CTAs solve the panel L_IK = A_IK DI_K^T and update the trailing
// lower triangle A_IJ -= L_IK L_JK^T; then L^-1 by the right-looking block forward substitution of
// L X = I: X_K,: = DI_K B_K,: and B_I,: -= L_IK X_K,: for I > K.  5 grid barriers per block column
// instead of one per column, and the FP64 work spread over every SM.
// di: scratch of ceil(n / 32) x 32 x 32 doubles; bad: one int of scratch.  info: 0, or j + 1 for the
// first column j whose pivot is not positive (L and L^-1 are then not written in full).
constexpr int CB = 32;

// Rows [r0, r0 + nr) x columns [c0, c0 + nc) of C (+|-)= A B^T or A B, the tiles staged in shared
// memory; 256 threads over the part's outputs.
__device__ __forceinline__ void tile_acc_part(double (*C)[CB + 1], const double (*A)[CB + 1], const double (*B)[CB + 1],
                                              bool btrans, double sign, int r0, int nr, int c0, int nc) {
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int r = r0 + e / nc, c = c0 + e % nc;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
    for (int k = 0; k < CB; k += 2) {
      a0 = fma(A[r][k], btrans ? B[c][k] : B[k][c], a0);
      a1 = fma(A[r][k + 1], btrans ? B[c][k + 1] : B[k + 1][c], a1);
    }
    C[r][c] = fma(sign, a0 + a1, C[r][c]);
  }
}

// Tile (I, J) of a column-major n x n matrix to / from shared memory (zeros outside the matrix).
__device__ __forceinline__ void tile_load(double (*T)[CB + 1], const double* M, int n, int I, int J) {
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    const int c = e / CB, r = e % CB, i = I * CB + r, j = J * CB + c;
    T[r][c] = (i < n && j < n) ? __ldcg(M + (size_t)j * n + i) : 0.0;
  }
}
__device__ __forceinline__ void tile_store(const double (*T)[CB + 1], double* M, int n, int I, int J) {
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    const int c = e / CB, r = e % CB, i = I * CB + r, j = J * CB + c;
    if (i < n && j < n) __stcg(M + (size_t)j * n + i, T[r][c]);
  }
}
__device__ __forceinline__ void tile_store_part(const double (*T)[CB + 1], double* M, int n, int I, int J, int r0,
                                                int nr, int c0, int nc) {
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int c = c0 + e / nr, r = r0 + e % nr, i = I * CB + r, j = J * CB + c;
    if (i < n && j < n) __stcg(M + (size_t)j * n + i, T[r][c]);
  }
}

__global__ void __launch_bounds__(256) chol_inv_blocked_kernel(int n, const double* __restrict__ A, double* L,
                                                               double* Linv, double* di, int* bad, int* info) {
  __shared__ double T0[CB][CB + 1], T1[CB][CB + 1], T2[CB][CB + 1];
  __shared__ double rdiag[CB];  // 1 / L_jj of the diagonal tile
  cg::grid_group grid = cg::this_grid();
  const int P = gridDim.x, r = blockIdx.x, tid = threadIdx.x;
  const int nt = (n + CB - 1) / CB;
  const size_t nn = (size_t)n * n;
  // L = lower(A), Linv = I
  for (size_t e = (size_t)r * blockDim.x + tid; e < nn; e += (size_t)P * blockDim.x) {
    const size_t j = e / n, i = e - j * n;
    __stcg(L + e, i >= j ? A[e] : 0.0);
    __stcg(Linv + e, i == j ? 1.0 : 0.0);
  }
  if (r == 0 && tid == 0) *bad = 0;
  grid.sync();
  for (int K = 0; K < nt; ++K) {
    const int nb = min(CB, n - K * CB);
    // ---- diagonal tile: Cholesky in shared memory, then DI_K = L_KK^-1 (CTA 0)
    if (r == 0) {
      tile_load(T0, L, n, K, K);
      __syncthreads();
      for (int j = 0; j < nb; ++j) {
        const double d = T0[j][j];
        if (!(d > 0.0) || !isfinite(d)) {
          if (tid == 0) {
            *bad = K * CB + j + 1;
            *info = K * CB + j + 1;
          }
          break;
        }
        const double inv = rsqrt(d);
        if (tid == 0) rdiag[j] = inv;
        __syncthreads();
        if (tid > j && tid < nb) T0[tid][j] *= inv;
        __syncthreads();
        // trailing update inside the tile: T0[i][k] -= T0[i][j] T0[k][j], j < k <= i < nb
        for (int e = tid; e < CB * CB; e += blockDim.x) {
          const int i = e / CB, k = e % CB;
          if (k > j && k <= i && i < nb) T0[i][k] = fma(-T0[i][j], T0[k][j], T0[i][k]);
        }
        if (tid == 0) T0[j][j] = d * inv;
        __syncthreads();
      }
      // the update also wrote the tile's upper half: L is lower triangular
      for (int e = tid; e < CB * CB; e += blockDim.x)
        if (e % CB > e / CB) T0[e / CB][e % CB] = 0.0;
      __syncthreads();
      if (*(volatile int*)bad == 0) {
        // DI = L_KK^-1 by forward substitution, 8 threads per column c: x_i = (delta_ic - sum_k
        // L_ik x_k) / L_ii for i >= c, the sum split over the 8 threads
        const int c = tid >> 3, s = tid & 7;
        for (int e = tid; e < CB * CB; e += blockDim.x) T1[e / CB][e % CB] = 0.0;
        __syncthreads();
        for (int i = 0; i < CB; ++i) {
          double part = 0.0;
          if (c < nb && i < nb && i >= c)
            for (int k = c + s; k < i; k += 8) part = fma(T0[i][k], T1[k][c], part);
          part += __shfl_xor_sync(0xffffffffu, part, 1);
          part += __shfl_xor_sync(0xffffffffu, part, 2);
          part += __shfl_xor_sync(0xffffffffu, part, 4);
          if (s == 0 && c < nb && i < nb && i >= c) T1[i][c] = ((i == c ? 1.0 : 0.0) - part) * rdiag[i];
          __syncthreads();
        }
        tile_store(T0, L, n, K, K);
        double* dk = di + (size_t)K * CB * CB;
        for (int e = tid; e < CB * CB; e += blockDim.x) __stcg(dk + e, T1[e / CB][e % CB]);
      }
    }
    grid.sync();
    if (*(volatile int*)bad) return;
    // ---- panel: L_IK = A_IK DI_K^T, I > K
    const double* dk = di + (size_t)K * CB * CB;
    // (two CTAs per tile, one per half of its rows: a row of L_IK needs only that row of A_IK)
    for (int t = r; t < 2 * (nt - K - 1); t += P) {
      const int I = K + 1 + t / 2, h = (t % 2) * (CB / 2);
      for (int e = tid; e < CB * CB; e += blockDim.x) T1[e / CB][e % CB] = __ldcg(dk + e);
      tile_load(T0, L, n, I, K);
      for (int e = tid; e < CB * CB; e += blockDim.x) T2[e / CB][e % CB] = 0.0;
      __syncthreads();
      tile_acc_part(T2, T0, T1, true, 1.0, h, CB / 2, 0, CB);
      __syncthreads();
      tile_store_part(T2, L, n, I, K, h, CB / 2, 0, CB);
      __syncthreads();
    }
    grid.sync();
    // ---- trailing update of the lower triangle: A_IJ -= L_IK L_JK^T, K < J <= I
    {
      const int m = nt - K - 1;
      const int tiles = m * (m + 1) / 2;
      // (four CTAs per tile, one per quadrant of outputs; the operands are other tiles)
      for (int tq = r; tq < 4 * tiles; tq += P) {
        const int t = tq / 4, qr = ((tq % 4) / 2) * (CB / 2), qc = (tq % 2) * (CB / 2);
        // t -> (I, J) with J <= I: row a = I - K - 1 holds a + 1 tiles
        int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((a + 1) * (a + 2) / 2 <= t) ++a;
        while (a * (a + 1) / 2 > t) --a;
        const int I = K + 1 + a, J = K + 1 + (t - a * (a + 1) / 2);
        tile_load(T0, L, n, I, K);
        tile_load(T1, L, n, J, K);
        tile_load(T2, L, n, I, J);
        __syncthreads();
        tile_acc_part(T2, T0, T1, true, -1.0, qr, CB / 2, qc, CB / 2);
        __syncthreads();
        tile_store_part(T2, L, n, I, J, qr, CB / 2, qc, CB / 2);
        __syncthreads();
      }
    }
    grid.sync();
  }
  // L^-1: B = I in Linv; per block row K: X_K,: = DI_K B_K,: (column tiles <= K), then
  // B_I,: -= L_IK X_K,: for I > K
  for (int K = 0; K < nt; ++K) {
    const double* dk = di + (size_t)K * CB * CB;
    // (two CTAs per tile, one per half of its columns: a column of X_KJ needs only that column of B_KJ)
    for (int t = r; t < 2 * (K + 1); t += P) {
      const int J = t / 2, h = (t % 2) * (CB / 2);
      for (int e = tid; e < CB * CB; e += blockDim.x) T1[e / CB][e % CB] = __ldcg(dk + e);
      tile_load(T0, Linv, n, K, J);
      for (int e = tid; e < CB * CB; e += blockDim.x) T2[e / CB][e % CB] = 0.0;
      __syncthreads();
      tile_acc_part(T2, T1, T0, false, 1.0, 0, CB, h, CB / 2);
      __syncthreads();
      tile_store_part(T2, Linv, n, K, J, 0, CB, h, CB / 2);
      __syncthreads();
    }
    grid.sync();
    const int rows = nt - K - 1, tiles = rows * (K + 1);
    for (int tq = r; tq < 4 * tiles; tq += P) {
      const int t = tq / 4, qr = ((tq % 4) / 2) * (CB / 2), qc = (tq % 2) * (CB / 2);
      const int I = K + 1 + t / (K + 1), J = t % (K + 1);
      tile_load(T0, L, n, I, K);
      tile_load(T1, Linv, n, K, J);
      tile_load(T2, Linv, n, I, J);
      __syncthreads();
      tile_acc_part(T2, T0, T1, false, -1.0, qr, CB / 2, qc, CB / 2);
      __syncthreads();
      tile_store_part(T2, Linv, n, I, J, qr, CB / 2, qc, CB / 2);
      __syncthreads();
    }
    grid.sync();
  }
  if (r == 0 && tid == 0) *info = 0;
}

// ------------------------------------------------------------------ Householder tridiagonalisation
// M (n x n, column-major, full symmetric storage, destroyed).  Outputs: d (n), e (n-1), the
// Householder vectors H(:, k) = v_k (rows k+1 .. n-1, v_k(k+1) = 1) and tau (n-1), so that
// Q = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^T, and Q^T M Q = tridiag(e, d, e).
// p: n doubles of scratch.  Column c of the trailing matrix is owned by CTA c mod P.
template <bool CLUSTER>
__global__ void __launch_bounds__(EIG_THREADS) tridiag_kernel(int n, double* M, double* H, double* d, double* e,
                                                              double* tau, double* p) {
  extern __shared__ double sm[];
  double* v = sm;          // n
  double* w = sm + n;      // n
  double* red = sm + 2 * n;  // 33
  const int P = gridDim.x, r = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const int rr = n - k - 1;  // order of the trailing block
    const double* mk = M + (int64_t)k * n + k + 1;
    for (int i = tid; i < rr; i += blockDim.x) v[i] = __ldcg(mk + i);
    __syncthreads();
    const double alpha = v[0];
    double s = 0.0;
    for (int i = 1 + tid; i < rr; i += blockDim.x) s += v[i] * v[i];
    const double xn2 = block_sum(s, red);
    double beta = alpha, t = 0.0;
    if (xn2 > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      t = (beta - alpha) / beta;
      const double sc = 1.0 / (alpha - beta);
      for (int i = 1 + tid; i < rr; i += blockDim.x) v[i] *= sc;
    }
    __syncthreads();
    if (tid == 0) v[0] = 1.0;
    __syncthreads();
    if (r == 0) {
      if (tid == 0) {
        d[k] = __ldcg(M + (int64_t)k * n + k);
        e[k] = beta;
        tau[k] = t;
      }
      for (int i = tid; i < rr; i += blockDim.x) H[(int64_t)k * n + k + 1 + i] = v[i];
    }
    if (t == 0.0) continue;  // H_k = I: nothing to update (every CTA takes the same branch)
    // p_c = t * M(k+1:, c) . v for the owned columns c >= k + 1
    const int c0 = k + 1 + ((r - (k + 1)) % P + P) % P;
    for (int c = c0 + warp * P; c < n; c += nw * P) {
      const double* mc = M + (int64_t)c * n + k + 1;
      double acc = 0.0;
      for (int i = lane; i < rr; i += 32) acc += mc[i] * v[i];
      acc = warp_sum(acc);
      if (lane == 0) __stcg(p + c, t * acc);
    }
    all_sync<CLUSTER>();
    for (int i = tid; i < rr; i += blockDim.x) w[i] = __ldcg(p + k + 1 + i);
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < rr; i += blockDim.x) pv += w[i] * v[i];
    const double K = -0.5 * t * block_sum(pv, red);
    for (int i = tid; i < rr; i += blockDim.x) w[i] += K * v[i];
    __syncthreads();
    // M(k+1:, c) -= v w_c + w v_c on the owned columns
    for (int c = c0 + warp * P; c < n; c += nw * P) {
      double* mc = M + (int64_t)c * n + k + 1;
      const double wc = w[c - k - 1], vc = v[c - k - 1];
      for (int i = lane; i < rr; i += 32) mc[i] = fma(-w[i], vc, fma(-v[i], wc, mc[i]));
    }
    all_sync<CLUSTER>();
  }
  if (r == 0 && tid == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(M + (int64_t)(n - 2) * n + n - 2);
      e[n - 2] = __ldcg(M + (int64_t)(n - 2) * n + n - 1);
    }
    d[n - 1] = __ldcg(M + (int64_t)(n - 1) * n + n - 1);
  }
}

// Same reduction with the owned columns resident in shared memory (nq = ceil(n / P) columns of n
// doubles per CTA).  Per step only the pivot column (xch: rows k+1.., then M(k,k) at xch[n]) and the
// product p travel through L2; the owner of column k+1 publishes it at the end of step k, so each
// step needs two barriers.
constexpr int TRI_THREADS = 256;

template <bool CLUSTER>
__global__ void __launch_bounds__(TRI_THREADS) tridiag_smem_kernel(int n, const double* __restrict__ Min, double* H,
                                                                   double* d, double* e, double* tau, double* xch,
                                                                   double* xp) {
  extern __shared__ double sm[];
  const int P = gridDim.x, r = blockIdx.x;
  const int nq = (n - r + P - 1) / P;  // owned columns c = r + q P, q < nq
  double* cols = sm;                   // nq x n
  double* v = cols + (size_t)nq * n;   // n
  double* w = v + n;                   // n
  double* red = w + n;                 // 33
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int q = 0; q < nq; ++q)
    for (int i = tid; i < n; i += blockDim.x) cols[(size_t)q * n + i] = Min[(size_t)(r + q * P) * n + i];
  __syncthreads();
  if (r == 0) {  // column 0 is owned by CTA 0
    for (int i = 1 + tid; i < n; i += blockDim.x) __stcg(xch + i - 1, cols[i]);
    if (tid == 0) __stcg(xch + n, cols[0]);
  }
  all_sync<CLUSTER>();
  for (int k = 0; k + 2 < n; ++k) {
    const int rr = n - k - 1;
    for (int i = tid; i < rr; i += blockDim.x) v[i] = __ldcg(xch + i);
    __syncthreads();
    const double alpha = v[0];
    double s = 0.0;
    for (int i = 1 + tid; i < rr; i += blockDim.x) s += v[i] * v[i];
    const double xn2 = block_sum(s, red);
    double beta = alpha, t = 0.0;
    if (xn2 > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      // t = (beta - alpha) / beta and sc = 1 / (alpha - beta) from one reciprocal
      const double g = alpha - beta, rcp = 1.0 / (beta * g);
      t = -(g * g) * rcp;
      const double sc = beta * rcp;
      for (int i = 1 + tid; i < rr; i += blockDim.x) v[i] *= sc;
    }
    __syncthreads();
    if (tid == 0) v[0] = 1.0;
    __syncthreads();
    if (r == 0) {
      if (tid == 0) {
        d[k] = __ldcg(xch + n);
        e[k] = beta;
        tau[k] = t;
      }
      for (int i = tid; i < rr; i += blockDim.x) H[(int64_t)k * n + k + 1 + i] = v[i];
    }
    // owned columns c >= k + 1: q from qa on
    const int qa = (k + 1 - r + P - 1) / P > 0 ? (k + 1 - r + P - 1) / P : 0;
    if (t != 0.0) {
      for (int q = qa + warp; q < nq; q += nw) {
        const double* mc = cols + (size_t)q * n + k + 1;
        double acc0 = 0.0, acc1 = 0.0;
        int i = lane;
        for (; i + 32 < rr; i += 64) {
          acc0 = fma(mc[i], v[i], acc0);
          acc1 = fma(mc[i + 32], v[i + 32], acc1);
        }
        if (i < rr) acc0 = fma(mc[i], v[i], acc0);
        const double acc = warp_sum(acc0 + acc1);
        if (lane == 0) __stcg(xp + r + q * P, t * acc);
      }
    }
    all_sync<CLUSTER>();
    if (t != 0.0) {
      for (int i = tid; i < rr; i += blockDim.x) w[i] = __ldcg(xp + k + 1 + i);
      __syncthreads();
      double pv = 0.0;
      for (int i = tid; i < rr; i += blockDim.x) pv += w[i] * v[i];
      const double K = -0.5 * t * block_sum(pv, red);
      for (int i = tid; i < rr; i += blockDim.x) w[i] += K * v[i];
      __syncthreads();
      for (int q = qa + warp; q < nq; q += nw) {
        const int c = r + q * P;
        double* mc = cols + (size_t)q * n + k + 1;
        const double wc = w[c - k - 1], vc = v[c - k - 1];
        for (int i = lane; i < rr; i += 32) mc[i] = fma(-w[i], vc, fma(-v[i], wc, mc[i]));
      }
      __syncthreads();
    }
    // publish column k + 1 (rows k+2.., then its diagonal) for the next step
    if ((k + 1) % P == r) {
      const double* mc = cols + (size_t)((k + 1 - r) / P) * n;
      for (int i = k + 2 + tid; i < n; i += blockDim.x) __stcg(xch + i - (k + 2), mc[i]);
      if (tid == 0) __stcg(xch + n, mc[k + 1]);
    }
    all_sync<CLUSTER>();
  }
  // last 2 x 2 block
  if (n >= 2 && (n - 2) % P == r && tid == 0) {
    const double* mc = cols + (size_t)((n - 2 - r) / P) * n;
    d[n - 2] = mc[n - 2];
    e[n - 2] = mc[n - 1];
  }
  if ((n - 1) % P == r && tid == 0) d[n - 1] = cols[(size_t)((n - 1 - r) / P) * n + n - 1];
}

// The same reduction for one thread-block cluster, with every exchange through distributed shared
// memory instead of L2.  All CTAs use one layout (nqm = ceil(n / P) column slots), so a remote
// address is the local one in another rank.  The owner of column k + 1 updates that column first
// (warp 0) and, while its other warps finish the rank-2 update, computes the Householder scalars of
// the next step (alpha, beta, tau and the scale 1 / (alpha - beta)) and keeps them with the column;
// the other CTAs read them after the barrier instead of each recomputing the norm, the square root
// and the divide.  Step k: read pivot column k and its scalars from the owner -> own products
// t (A v)_c -> barrier -> read the products p_c of all CTAs -> rank-2 update -> barrier.  The loop
// writes nothing to global memory (a barrier's release then has no stores to wait for); H, d, e
// and tau are written at the end from the owned columns and their scalars.
constexpr int TRI_DS_SLOTS = 8;  // per owned column: beta, tau, scale, diagonal (4 used)

size_t tridiag_dsmem_smem(int n, int P) {
  const size_t nqm = ((size_t)n + P - 1) / P;
  return (nqm * n + 2 * (size_t)n + nqm * (1 + TRI_DS_SLOTS) + 40) * sizeof(double);
}

// Householder scalars of x = column c rows c+1.. (alpha = x_0, xn2 = |x_1..|^2), as in tridiag_smem_kernel.
__device__ __forceinline__ void house_scalars(double alpha, double xn2, double* beta, double* t, double* sc) {
  *beta = alpha;
  *t = 0.0;
  *sc = 1.0;
  if (xn2 > 0.0) {
    const double b = -copysign(sqrt(alpha * alpha + xn2), alpha);
    const double g = alpha - b, rcp = 1.0 / (b * g);
    *beta = b;
    *t = -(g * g) * rcp;
    *sc = b * rcp;
  }
}

__global__ void __launch_bounds__(TRI_THREADS) tridiag_dsmem_kernel(int n, const double* __restrict__ Min, double* H,
                                                                    double* d, double* e, double* tau) {
  extern __shared__ double sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int P = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
  const int nqm = (n + P - 1) / P;
  const int nq = (n - r + P - 1) / P;  // owned columns c = r + q P, q < nq
  double* cols = sm;                          // nqm x n
  double* v = cols + (size_t)nqm * n;         // n
  double* w = v + n;                          // n
  double* prod = w + n;                       // nqm: t (A v)_c of the owned columns
  double* hs = prod + nqm;                    // nqm x TRI_DS_SLOTS: beta, tau, scale, diagonal
  double* red = hs + (size_t)nqm * TRI_DS_SLOTS;  // 33
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int q = 0; q < nq; ++q)
    for (int i = tid; i < n; i += blockDim.x) cols[(size_t)q * n + i] = Min[(size_t)(r + q * P) * n + i];
  __syncthreads();
  // scalars of pivot column 0 (owner: rank 0)
  if (r == 0 && warp == 0 && n > 2) {
    double s2 = 0.0;
    for (int i = 2 + lane; i < n; i += 32) s2 += cols[i] * cols[i];
    s2 = warp_sum(s2);
    if (lane == 0) {
      house_scalars(cols[1], s2, hs + 0, hs + 1, hs + 2);
      hs[3] = cols[0];
    }
  }
  cluster.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int rr = n - k - 1;
    const int ok_ = k % P, oq = k / P;  // owner of the pivot column and its slot
    const double* pc = cluster.map_shared_rank(cols + (size_t)oq * n, ok_);
    const double* ph = cluster.map_shared_rank(hs + (size_t)oq * TRI_DS_SLOTS, ok_);
    // v = (1, x_1 sc, x_2 sc, ...) from the owner's column (the loads are issued together)
    double xv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = tid + (int)blockDim.x * u;
      xv[u] = (i > 0 && i < rr) ? pc[k + 1 + i] : 0.0;
    }
    const double t = ph[1], sc = ph[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = tid + (int)blockDim.x * u;
      if (i < rr) v[i] = i == 0 ? 1.0 : xv[u] * sc;
    }
    for (int i = tid + 2 * (int)blockDim.x; i < rr; i += blockDim.x) v[i] = pc[k + 1 + i] * sc;
    __syncthreads();
    const int qa = (k + 1 - r + P - 1) / P > 0 ? (k + 1 - r + P - 1) / P : 0;
    if (t != 0.0) {
      // owned columns in pairs per warp, the two reductions interleaved
      for (int q = qa + warp; q < nq; q += 2 * nw) {
        const int q2 = q + nw;
        double a = dot_part(cols + (size_t)q * n + k + 1, v, rr, lane);
        double b = q2 < nq ? dot_part(cols + (size_t)q2 * n + k + 1, v, rr, lane) : 0.0;
        warp_sum2(a, b);
        if (lane == 0) {
          prod[q] = t * a;
          if (q2 < nq) prod[q2] = t * b;
        }
      }
    }
    cluster.sync();
    // the owner of column k + 1 computes the next scalars; its warp 0 updates only that column
    const bool next_owner = (k + 1) % P == r && k + 3 < n;
    if (t != 0.0) {
      for (int i = tid; i < rr; i += blockDim.x) {
        const int c = k + 1 + i;
        w[i] = cluster.map_shared_rank(prod, c % P)[c / P];
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = tid; i < rr; i += blockDim.x) pv += w[i] * v[i];
      const double K = -0.5 * t * block_sum(pv, red);
      for (int i = tid; i < rr; i += blockDim.x) w[i] += K * v[i];
      __syncthreads();
      if (next_owner && warp == 0) {
        const int q = qa;  // column k + 1
        double* col = cols + (size_t)q * n;
        double s2 = rank2_part<true>(col + k + 1, v, w, v[0], w[0], rr, lane);
        s2 = warp_sum(s2);
        __syncwarp();
        if (lane == 0) {
          double* h = hs + (size_t)q * TRI_DS_SLOTS;
          house_scalars(col[k + 2], s2, h + 0, h + 1, h + 2);
          h[3] = col[k + 1];
        }
      } else {
        const int q0 = next_owner ? qa + 1 : qa, w0 = next_owner ? 1 : 0, ws = nw - w0;
        for (int q = q0 + (warp - w0); q < nq; q += ws) {
          const int c = r + q * P;
          rank2_part<false>(cols + (size_t)q * n + k + 1, v, w, v[c - k - 1], w[c - k - 1], rr, lane);
        }
      }
    } else if (next_owner && warp == 0) {
      // no update this step: column k + 1 as it stands
      const int q = qa;
      const double* col = cols + (size_t)q * n;
      double s2 = 0.0;
      for (int i = k + 3 + lane; i < n; i += 32) s2 += col[i] * col[i];
      s2 = warp_sum(s2);
      if (lane == 0) {
        double* h = hs + (size_t)q * TRI_DS_SLOTS;
        house_scalars(col[k + 2], s2, h + 0, h + 1, h + 2);
        h[3] = col[k + 1];
      }
    }
    cluster.sync();
  }
  // outputs of the owned pivot columns k < n - 2: d, e, tau and H(:, k) = (1, x sc)
  for (int q = 0; q < nq; ++q) {
    const int k = r + q * P;
    if (k + 2 >= n) break;
    const double* col = cols + (size_t)q * n;
    const double* h = hs + (size_t)q * TRI_DS_SLOTS;
    const double sc = h[2];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) H[(int64_t)k * n + i] = i == k + 1 ? 1.0 : col[i] * sc;
    if (tid == 0) {
      d[k] = h[3];
      e[k] = h[0];
      tau[k] = h[1];
    }
  }
  // last 2 x 2 block
  if (n >= 2 && (n - 2) % P == r && tid == 0) {
    const double* mc = cols + (size_t)((n - 2 - r) / P) * n;
    d[n - 2] = mc[n - 2];
    e[n - 2] = mc[n - 1];
  }
  if ((n - 1) % P == r && tid == 0) d[n - 1] = cols[(size_t)((n - 1 - r) / P) * n + n - 1];
}

// ------------------------------------------------------------------ tridiagonal eigenvalues
// Number of eigenvalues of T below x: sign changes of the Sturm sequence of leading principal
// minors p_i = det(T_i - x I), by the three-term recurrence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}
// (p_{-1} = 1) on T scaled by 1 / tnorm (ds = d / tnorm, e2s[i] = (e_{i-1} / tnorm)^2, e2s[0] = 0).
// The recurrence needs no division (an FP64 divide costs ~9 dependent FMAs on this GPU), so its
// critical chain is one FMA per step; the pair (p_i, p_{i-1}) is rescaled by a power of two every
// 8 steps.  A zero minor between two nonzero ones of opposite sign counts one sign change either
// way; an exact zero is replaced by a tiny value of the sign opposite to its predecessor.
__device__ __forceinline__ bool neg_bits(double v) { return __double_as_longlong(v) < 0; }

template <int K>
__device__ void sturm_count_k(int n, const double* ds, const double* e2s, const double* xs, int* cnt) {
  // K independent sequences interleaved, so their dependent FMAs overlap
  double pm[K], p[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    pm[c] = 1.0;
    p[c] = ds[0] - xs[c];
    if ((__double_as_longlong(p[c]) << 1) == 0) p[c] = -DBL_MIN;
    cnt[c] = neg_bits(p[c]);
  }
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double d = ds[i + u], e2 = e2s[i + u];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        double pn = fma(d - xs[c], p[c], -e2 * pm[c]);
        if ((__double_as_longlong(pn) << 1) == 0) pn = neg_bits(p[c]) ? DBL_MIN : -DBL_MIN;
        cnt[c] += neg_bits(pn) != neg_bits(p[c]);
        pm[c] = p[c];
        p[c] = pn;
      }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const long long bp = __double_as_longlong(p[c]) & 0x7fffffffffffffffLL;
      const long long bq = __double_as_longlong(pm[c]) & 0x7fffffffffffffffLL;
      const long long ex = ((bp > bq ? bp : bq) >> 52) - 1023;
      const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
      p[c] *= sc;
      pm[c] *= sc;
    }
  }
  for (; i < n; ++i) {
    const double d = ds[i], e2 = e2s[i];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double pn = fma(d - xs[c], p[c], -e2 * pm[c]);
      if ((__double_as_longlong(pn) << 1) == 0) pn = neg_bits(p[c]) ? DBL_MIN : -DBL_MIN;
      cnt[c] += neg_bits(pn) != neg_bits(p[c]);
      pm[c] = p[c];
      p[c] = pn;
    }
  }
}

// Sturm sequences per lane.  One: on this GPU a warp-wide FP64 instruction occupies the SM's FP64
// pipe for ~12 clocks, so more sequences per lane trade latency for pipe time at a loss (measured).
constexpr int kChains = 1;

// The same count without the per-step zero substitution, so that the dependency chain from one
// minor to the next is the FMA alone: sign changes are read from the high words and accumulated
// off the chain, and *zero is set when a minor came out exactly zero (or with a zero high word, a
// subnormal below 2^-1042), the one case in which the substitution would have changed the count.
// The caller then recounts that shift with sturm_count_k.
__device__ __forceinline__ int sturm_count_fast(int n, const double* ds, const double* e2s, double xs, bool* zero) {
  double pm = 1.0, p = ds[0] - xs;
  uint32_t hp = (uint32_t)__double2hiint(p);
  int cnt = (int)(hp >> 31);
  uint32_t zmin = hp << 1;  // zero iff some minor had a zero high word (sign bit dropped)
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double pn = fma(ds[i + u] - xs, p, -e2s[i + u] * pm);
      const uint32_t hn = (uint32_t)__double2hiint(pn);
      cnt += (int)((hn ^ hp) >> 31);
      zmin = min(zmin, hn << 1);
      pm = p;
      p = pn;
      hp = hn;
    }
    // rescale the pair by a power of two (signs and ratios unchanged)
    const uint32_t ep = ((uint32_t)__double2hiint(p) >> 20) & 0x7ffu, eq = ((uint32_t)__double2hiint(pm) >> 20) & 0x7ffu;
    const int ex = (int)(ep > eq ? ep : eq) - 1023;
    const double sc = __hiloint2double((1023 - ex) << 20, 0);
    p *= sc;
    pm *= sc;
  }
  for (; i < n; ++i) {
    const double pn = fma(ds[i] - xs, p, -e2s[i] * pm);
    const uint32_t hn = (uint32_t)__double2hiint(pn);
    cnt += (int)((hn ^ hp) >> 31);
    zmin = min(zmin, hn << 1);
    pm = p;
    p = pn;
    hp = hn;
  }
  *zero = zmin == 0u;
  return cnt;
}

// Eigenvalue j (ascending) of T = tridiag(e, d, e): one warp (one CTA), 32 kChains trial points per step.
__global__ void __launch_bounds__(32) bisect_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                                                    double* lam, double* tnorm_out) {
  extern __shared__ double sm[];
  double* ds = sm;       // n
  double* e2s = sm + n;  // n
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int i = lane; i < n; i += 32) {
    const double a = i + 1 < n ? fabs(e[i]) : 0.0, b = i > 0 ? fabs(e[i - 1]) : 0.0;
    lo = fmin(lo, d[i] - a - b);
    hi = fmax(hi, d[i] + a + b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const double inv_tn = tnorm > 0.0 ? 1.0 / tnorm : 1.0;
  for (int i = lane; i < n; i += 32) {
    ds[i] = d[i] * inv_tn;
    const double b = i > 0 ? e[i - 1] * inv_tn : 0.0;
    e2s[i] = b * b;
  }
  __syncwarp();
  const double tiny = DBL_MIN * 4.0;
  lo -= 2.0 * DBL_EPSILON * tnorm + tiny;
  hi += 2.0 * DBL_EPSILON * tnorm + tiny;
  constexpr int NP = 32 * kChains;  // trial points per step; point q = c * 32 + lane
  for (int it = 0; it < 64; ++it) {
    // relative accuracy, but no finer than the eps ||T|| that the Sturm counts resolve
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 0.5 * DBL_EPSILON * tnorm + tiny) break;
    const double w = (hi - lo) / (double)(NP + 1);
    double x[kChains], xs[kChains];
    int cnt[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      x[c] = lo + w * (double)(c * 32 + lane + 1);
      xs[c] = x[c] * inv_tn;
    }
    bool zero = false;
    cnt[0] = sturm_count_fast(n, ds, e2s, xs[0], &zero);
    if (zero) sturm_count_k<1>(n, ds, e2s, xs, cnt);
    // counts grow with x, so the first point with count > j bounds the eigenvalue from above
    int q = -1;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const unsigned ge = __ballot_sync(0xffffffffu, cnt[c] >= j + 1);
      if (q < 0 && ge != 0u) q = c * 32 + __ffs(ge) - 1;
    }
    if (q < 0) {
      lo = lo + w * (double)NP;
    } else {
      const double nlo = q > 0 ? lo + w * (double)q : lo;
      hi = lo + w * (double)(q + 1);
      lo = nlo;
    }
  }
  if (lane == 0) {
    lam[j] = 0.5 * (lo + hi);
    if (j == 0) *tnorm_out = tnorm;
  }
}

// ------------------------------------------------------------------ tridiagonal eigenvectors
// LU factorisation with partial pivoting of T - lam I (one thread).  Row i of U holds u0 (diagonal),
// u1, u2 (first and second superdiagonals); mult/sw record the elimination of row i + 1.
__device__ void tri_lu(int n, const double* d, const double* e, double lam, double small, double* u0, double* u1,
                       double* u2, double* mult, int* sw) {
  for (int i = 0; i < n; ++i) {
    u0[i] = d[i] - lam;
    u1[i] = i + 1 < n ? e[i] : 0.0;
    u2[i] = 0.0;
  }
  for (int i = 0; i + 1 < n; ++i) {
    const double c = e[i];  // subdiagonal entry (i + 1, i)
    if (fabs(u0[i]) >= fabs(c)) {
      if (u0[i] == 0.0) u0[i] = small;
      const double m = c / u0[i];
      mult[i] = m;
      sw[i] = 0;
      u0[i + 1] -= m * u1[i];
    } else {
      // exchange rows i and i + 1, then eliminate
      const double m = u0[i] / c;
      mult[i] = m;
      sw[i] = 1;
      const double r0 = u1[i];   // old row i: (u0, u1, 0) at columns i, i+1, i+2
      const double a1 = u0[i + 1], b1 = u1[i + 1];
      u0[i] = c;
      u1[i] = a1;
      u2[i] = b1;
      u0[i + 1] = r0 - m * a1;
      u1[i + 1] = -m * b1;
    }
  }
  if (u0[n - 1] == 0.0) u0[n - 1] = small;
  // keep the reciprocals of the pivots (clamped away from zero) so the solves need no divide
  for (int i = 0; i < n; ++i) {
    double u = u0[i];
    if (fabs(u) < small) u = u >= 0.0 ? small : -small;
    u0[i] = 1.0 / u;
  }
}

// y <- (T - lam I)^-1 y with the factors of tri_lu (one thread; u0 holds the pivot reciprocals).
__device__ void tri_solve(int n, const double* u0, const double* u1, const double* u2, const double* mult,
                          const int* sw, double* y) {
  for (int i = 0; i + 1 < n; ++i) {
    if (sw[i]) {
      const double t = y[i];
      y[i] = y[i + 1];
      y[i + 1] = t - mult[i] * y[i];
    } else {
      y[i + 1] -= mult[i] * y[i];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    if (i + 1 < n) s -= u1[i] * y[i + 1];
    if (i + 2 < n) s -= u2[i] * y[i + 2];
    y[i] = s * u0[i];
  }
}

// One warp (one CTA) per cluster of eigenvalues, a cluster being a run of eigenvalues with
// consecutive gaps <= 1e-9 ||T|| (numerically degenerate, e.g. the pairs of a complex problem's
// real embedding): inverse iteration for each member in turn, with Gram-Schmidt (twice) against the
// members already done.  Eigenvectors of better separated eigenvalues come out orthogonal to
// O(eps ||T|| / gap); the caller removes that residue with one Newton-Schulz step.  The LU factors
// and the iterate live in shared memory (6 n doubles).  Z (n x n, column-major) receives the unit
// eigenvectors of T.  A cluster larger than maxc sets *flag (the caller then uses another solver).
__global__ void __launch_bounds__(32) inviter_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                                                     const double* __restrict__ lam, const double* __restrict__ tnorm_p,
                                                     double* Z, int maxc, int* flag) {
  extern __shared__ double sm[];
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  const double tnorm = *tnorm_p;
  const double ortol = 1e-9 * tnorm;
  if (j > 0 && lam[j] - lam[j - 1] <= ortol) return;  // not the first member of its cluster
  int k = j + 1;
  while (k < n && lam[k] - lam[k - 1] <= ortol) ++k;
  if (k - j > maxc) {
    if (lane == 0) atomicExch(flag, 1);
    return;
  }
  const double small = DBL_EPSILON * fmax(tnorm, DBL_MIN);
  double* u0 = sm;
  double* u1 = u0 + n;
  double* u2 = u1 + n;
  double* mult = u2 + n;
  double* y = mult + n;
  int* sw = reinterpret_cast<int*>(y + n);
  double* dd = reinterpret_cast<double*>(sw) + (n + 1) / 2;  // copies of d and e (n each)
  double* ee = dd + n;
  for (int m = lane; m < n; m += 32) {
    dd[m] = d[m];
    ee[m] = m + 1 < n ? e[m] : 0.0;
  }
  __syncwarp();
  for (int i = j; i < k; ++i) {
    if (lane == 0) tri_lu(n, dd, ee, lam[i], small, u0, u1, u2, mult, sw);
    // deterministic start vector with no structure shared with T
    double nr = 0.0;
    for (int m = lane; m < n; m += 32) {
      const double v = cos(0.7548776662 * m + 1.3247179572 * (i - j) + 0.5) + 0.1;
      y[m] = v;
      nr += v * v;
    }
    nr = warp_sum(nr);
    for (int m = lane; m < n; m += 32) y[m] *= rsqrt(nr);
    __syncwarp();
    // the shift is accurate to a few ulps, so two solves already give the eigenvector to round-off
    for (int it = 0; it < 2; ++it) {
      if (lane == 0) tri_solve(n, u0, u1, u2, mult, sw, y);
      __syncwarp();
      for (int rep = 0; rep < 2; ++rep) {
        for (int l = j; l < i; ++l) {
          const double* zl = Z + (size_t)l * n;
          double dt = 0.0;
          for (int m = lane; m < n; m += 32) dt += zl[m] * y[m];
          dt = warp_sum(dt);
          for (int m = lane; m < n; m += 32) y[m] -= dt * zl[m];
          __syncwarp();
        }
      }
      nr = 0.0;
      for (int m = lane; m < n; m += 32) nr += y[m] * y[m];
      nr = warp_sum(nr);
      const double sc = 1.0 / sqrt(nr);
      for (int m = lane; m < n; m += 32) y[m] *= sc;
      __syncwarp();
    }
    double* zi = Z + (size_t)i * n;
    for (int m = lane; m < n; m += 32) zi[m] = y[m];
    __syncwarp();
  }
}

size_t inviter_smem(int n) { return (8 * (size_t)n + 1) * sizeof(double); }

// V = Q Z = H_0 H_1 ... H_{n-3} Z, one warp per column (in place on V), the column held in registers
// (rows lane + 32 t, t < R) and the next Householder vector prefetched while the current one is
// applied.  For n <= 32 R.
template <int R>
__global__ void __launch_bounds__(64) backtransform_reg_kernel(int n, const double* __restrict__ H,
                                                               const double* __restrict__ tau, double* V) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= n) return;
  double* zc = V + (size_t)col * n;
  double z[R], hc[R], hn[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int i = lane + 32 * t;
    z[t] = i < n ? zc[i] : 0.0;
  }
  int k = n - 3;
  if (k < 0) return;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int i = lane + 32 * t;
    hc[t] = (i > k && i < n) ? H[(size_t)k * n + i] : 0.0;
  }
  for (; k >= 0; --k) {
    if (k > 0) {
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const int i = lane + 32 * t;
        hn[t] = (i > k - 1 && i < n) ? H[(size_t)(k - 1) * n + i] : 0.0;
      }
    }
    const double tk = tau[k];
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < R; ++t) s += hc[t] * z[t];
    s = warp_sum(s) * tk;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      z[t] -= s * hc[t];
      hc[t] = hn[t];
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int i = lane + 32 * t;
    if (i < n) zc[i] = z[t];
  }
}

// V = Q Z = H_0 H_1 ... H_{n-3} Z, one warp per column (in place on V).
__global__ void __launch_bounds__(64) backtransform_kernel(int n, const double* __restrict__ H,
                                                           const double* __restrict__ tau, double* V) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= n) return;
  double* z = V + (size_t)col * n;
  for (int k = n - 3; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    const double* h = H + (size_t)k * n;
    double s = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) s += h[i] * z[i];
    s = warp_sum(s) * t;
    for (int i = k + 1 + lane; i < n; i += 32) z[i] -= s * h[i];
    __syncwarp();
  }
}

// C = val * I (n x n, column-major)
// S = 1.5 I - 0.5 S (n x n): the Newton-Schulz factor from the Gram matrix Z^T Z.
__global__ void ns_shift_kernel(int n, double* S) {
  const int64_t tot = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / n, i = t - j * n;
    S[t] = fma(-0.5, S[t], i == j ? 1.5 : 0.0);
  }
}

__global__ void diag_fill_kernel(int n, double* C, double val) {
  const int64_t tot = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    C[t] = (t / n == t % n) ? val : 0.0;
}

}  // namespace

// ------------------------------------------------------------------ launchers
namespace {

constexpr int CLUSTER_MAX_N = 1024;     // global-memory variants: above this the cooperative grid is used
constexpr int INV_MAX_CLUSTER = 256;    // inverse iteration handles clusters up to this size
constexpr size_t SMEM_CAP = 220 * 1024; // dynamic shared memory of the resident variants

size_t multi_smem(int n) { return (2 * (size_t)n + 33) * sizeof(double); }

// Shared memory of a resident kernel (owned columns + two n-vectors + reduction slots) for P CTAs.
size_t resident_smem(int n, int P) {
  const size_t nq = ((size_t)n + P - 1) / P;
  return (nq * n + 2 * (size_t)n + 40) * sizeof(double);
}

cudaLaunchConfig_t cluster_cfg(int cs, int threads, size_t smem, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Largest cluster size (16, else 8, else 0) with which `kernel` can be resident.
int cluster_size_for(const void* kernel, int threads, size_t smem) {
  RC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP));
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    cudaGetLastError();
  for (int cs : {16, 8}) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(cs, threads, smem, nullptr, at);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, kernel, &cfg) == cudaSuccess && num >= 1) return cs;
    cudaGetLastError();
  }
  return 0;
}

// Launch a multi-CTA kernel pair (cluster / cooperative grid variants) with 2 n + 33 doubles of
// shared memory.
template <typename... Args>
void launch_multi(cudaStream_t s, void (*kc)(Args...), void (*kg)(Args...), int n, int num_sms, Args... args) {
  const size_t smem = multi_smem(n);
  if (n <= CLUSTER_MAX_N) {
    // one query per kernel (per instantiation), at the largest shared-memory size of this path
    static const int csz = cluster_size_for(reinterpret_cast<const void*>(kc), EIG_THREADS,
                                            multi_smem(CLUSTER_MAX_N));
    if (csz > 0) {
      cudaLaunchAttribute at[1];
      cudaLaunchConfig_t cfg = cluster_cfg(csz, EIG_THREADS, smem, s, at);
      RC_CUDA(cudaLaunchKernelEx(&cfg, kc, args...));
      RC_LAUNCH();
      return;
    }
  }
  RC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(kg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_CAP));
  int per_sm = 0;
  RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kg, EIG_THREADS, smem));
  RC_CHECK(per_sm >= 1, RCHFSI_ERR_UNSUPPORTED, "eigensolver kernel does not fit on an SM");
  const int ctas = std::max(1, std::min(num_sms, std::max(8, n / 16)));
  void* argv[] = {(void*)&args...};
  RC_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kg), dim3(ctas), dim3(EIG_THREADS), argv, smem,
                                      s));
  RC_LAUNCH();
}

// Launch a shared-memory-resident kernel pair (256 threads): one cluster when its CTAs can hold the
// owned columns, else a cooperative grid of one CTA per SM; false when neither fits.
template <typename... Args>
bool launch_resident(cudaStream_t s, void (*kc)(Args...), void (*kg)(Args...), int n, int num_sms, Args... args) {
  static const int csz = cluster_size_for(reinterpret_cast<const void*>(kc), TRI_THREADS, SMEM_CAP);
  if (csz > 0 && resident_smem(n, csz) <= SMEM_CAP) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(csz, TRI_THREADS, resident_smem(n, csz), s, at);
    RC_CUDA(cudaLaunchKernelEx(&cfg, kc, args...));
    RC_LAUNCH();
    return true;
  }
  const int P = num_sms;
  const size_t smem = resident_smem(n, P);
  if (smem > SMEM_CAP) return false;
  RC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(kg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_CAP));
  int per_sm = 0;
  RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kg, TRI_THREADS, smem));
  if (per_sm < 1) return false;
  void* argv[] = {(void*)&args...};
  RC_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kg), dim3(P), dim3(TRI_THREADS), argv, smem, s));
  RC_LAUNCH();
  return true;
}

// Above this order the tridiagonalisation runs on a cooperative grid of one CTA per SM: its rank-2
// updates, O(n^2) FP64 work per column, then outweigh the grid barrier's cost over the cluster's
// (measured per Rayleigh-Ritz step: n = 240 cluster 4.10 ms / grid 4.52 ms, n = 600 18.8 / 16.3 ms;
// a n^3 + b n fits put the crossover near 380).
constexpr int kTriClusterMaxN = 384;

// tridiag_smem_kernel on a cooperative grid of one CTA per SM when the owned columns fit in shared
// memory; false otherwise.
bool launch_tridiag_grid(cudaStream_t s, int n, int num_sms, const double* M, double* H, double* d, double* e,
                         double* tau, double* xch, double* p) {
  const int P = num_sms;
  const size_t smem = resident_smem(n, P);
  if (smem > SMEM_CAP) return false;
  static const bool attr = [] {
    RC_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(tridiag_smem_kernel<false>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP));
    return true;
  }();
  (void)attr;
  int per_sm = 0;
  RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_smem_kernel<false>, TRI_THREADS, smem));
  if (per_sm < 1) return false;
  int nn = n;
  void* argv[] = {(void*)&nn, (void*)&M, (void*)&H, (void*)&d, (void*)&e, (void*)&tau, (void*)&xch, (void*)&p};
  RC_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(tridiag_smem_kernel<false>), dim3(P),
                                      dim3(TRI_THREADS), argv, smem, s));
  RC_LAUNCH();
  return true;
}

// One cluster of tridiag_dsmem_kernel when its CTAs hold the owned columns; false otherwise.
bool launch_tridiag_dsmem(cudaStream_t s, int n, const double* M, double* H, double* d, double* e, double* tau) {
  static const int csz = cluster_size_for(reinterpret_cast<const void*>(tridiag_dsmem_kernel), TRI_THREADS, SMEM_CAP);
  if (csz <= 0 || tridiag_dsmem_smem(n, csz) > SMEM_CAP) return false;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(csz, TRI_THREADS, tridiag_dsmem_smem(n, csz), s, at);
  RC_CUDA(cudaLaunchKernelEx(&cfg, tridiag_dsmem_kernel, n, M, H, d, e, tau));
  RC_LAUNCH();
  return true;
}

template <int R>
void launch_backtransform(cudaStream_t s, int n, const double* H, const double* tau, double* V) {
  backtransform_reg_kernel<R><<<cdiv(n, 2), 64, 0, s>>>(n, H, tau, V);
  RC_LAUNCH();
}

}  // namespace

int cholesky_inverse_f64(cudaStream_t s, int n, double* A, double* L, double* Linv, int* d_info, int num_sms,
                         DevBuf<double>& scratch) {
  RC_CHECK(n >= 1 && n <= 6144, RCHFSI_ERR_UNSUPPORTED, "cholesky_inverse: order out of [1, 6144]");
  // blocked on a cooperative grid (5 grid barriers per 32 columns, FP64 work on every SM)
  {
    const int nt = (n + CB - 1) / CB;
    const size_t need = (size_t)nt * CB * CB + 8;
    double* di = scratch.ensure(std::max(need, 3 * (size_t)n));
    int* bad = reinterpret_cast<int*>(di + (size_t)nt * CB * CB);
    int per_sm = 0;
    RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_inv_blocked_kernel, 256, 0));
    if (per_sm >= 1) {
      const int P = std::max(1, std::min(num_sms, 2 * nt * (nt + 1)));
      const double* Ac = A;
      void* argv[] = {(void*)&n, (void*)&Ac, (void*)&L, (void*)&Linv, (void*)&di, (void*)&bad, (void*)&d_info};
      RC_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(chol_inv_blocked_kernel), dim3(P), dim3(256),
                                          argv, 0, s));
      RC_LAUNCH();
      return 0;
    }
  }
  double* xch = scratch.ensure(3 * (size_t)n);
  double* dinv = xch + 2 * (size_t)n;
  if (n <= 4096 && launch_resident(s, chol_inv_smem_kernel<true>, chol_inv_smem_kernel<false>, n, num_sms, n,
                                   (const double*)A, L, Linv, xch, dinv, d_info))
    return 0;
  launch_multi(s, chol_inv_kernel<true>, chol_inv_kernel<false>, n, num_sms, n, A, L, Linv, d_info);
  return 0;
}

bool sym_eig_f64(cudaStream_t s, int n, double* M, double* V, double* evals, DevBuf<double>& ws, int* d_flag,
                 int num_sms, const OzScratch* oz) {
  if (n < 1 || n > 3072) return false;
  // workspace: H, S, V2 (n^2 each), d, e, tau, p (n each), xch (n + 8), tnorm
  const size_t nn = (size_t)n * n;
  double* H = ws.ensure(3 * nn + 6 * (size_t)n + 16);
  double* S = H + nn;
  double* V2 = S + nn;
  double* d = V2 + nn;
  double* e = d + n;
  double* tau = e + n;
  double* p = tau + n;
  double* xch = p + n;
  double* tnorm = xch + n + 8;
  if (n == 1) {
    RC_CUDA(cudaMemcpyAsync(evals, M, sizeof(double), cudaMemcpyDeviceToDevice, s));
    const double one = 1.0;
    RC_CUDA(cudaMemcpyAsync(V, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaStreamSynchronize(s));
    return true;
  }
  RC_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  RC_CUDA(cudaMemsetAsync(tau, 0, sizeof(double) * n, s));
  // 1. Q^T M Q = T
  if (!(n <= kTriClusterMaxN ? launch_tridiag_dsmem(s, n, M, H, d, e, tau)
                             : launch_tridiag_grid(s, n, num_sms, M, H, d, e, tau, xch, p)) &&
      !launch_resident(s, tridiag_smem_kernel<true>, tridiag_smem_kernel<false>, n, num_sms, n, (const double*)M, H,
                       d, e, tau, xch, p))
    launch_multi(s, tridiag_kernel<true>, tridiag_kernel<false>, n, num_sms, n, M, H, d, e, tau, p);
  // 2. eigenvalues of T
  bisect_kernel<<<n, 32, 2 * (size_t)n * sizeof(double), s>>>(n, d, e, evals, tnorm);
  RC_LAUNCH();
  // 3. eigenvectors of T (into V2)
  RC_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  set_smem_limit(reinterpret_cast<const void*>(inviter_kernel), (int)SMEM_CAP);
  inviter_kernel<<<n, 32, inviter_smem(n), s>>>(n, d, e, evals, tnorm, V2, INV_MAX_CLUSTER, d_flag);
  RC_LAUNCH();
  int flag = 0;
  RC_CUDA(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  RC_CUDA(cudaStreamSynchronize(s));
  if (flag) return false;
  // 4. one Newton-Schulz step towards the orthogonal factor: Z <- Z (3 I - Z^T Z) / 2
  if (oz) {
    // FP64-accurate products from BF16 slices: G = Z^T Z (symmetric), S = 1.5 I - 0.5 G, V = Z S
    oz_slice(s, n, n, V2, n, 1, *oz->a);  // row i = column i of Z
    oz_gemm(s, oz->num_sms, *oz->a, *oz->a, S, n, *oz->ws, oz->err, true);
    ns_shift_kernel<<<cdiv((int64_t)n * n, 256) < 1216 ? cdiv((int64_t)n * n, 256) : 1216, 256, 0, s>>>(n, S);
    RC_LAUNCH();
    oz_slice(s, n, n, V2, 1, n, *oz->b);  // row i of Z
    oz_slice(s, n, n, S, n, 1, *oz->a);   // column j of S as row j
    oz_gemm(s, oz->num_sms, *oz->b, *oz->a, V, n, *oz->ws, oz->err);
  } else {
  diag_fill_kernel<<<cdiv((int64_t)n * n, 256) < 1216 ? cdiv((int64_t)n * n, 256) : 1216, 256, 0, s>>>(n, S, 1.5);
  RC_LAUNCH();
  EpiArgs g;
  g.kind = EPI_STORE;
  g.C = S;
  g.ldc = n;
  g.alpha = -0.5;
  g.beta = 1.0;
  g.prof_cls = RCHFSI_KERNEL_EIG;
  gemm_f64(s, n, n, n, V2, n, true, V2, n, true, g);
  EpiArgs z;
  z.kind = EPI_STORE;
  z.C = V;
  z.ldc = n;
  z.prof_cls = RCHFSI_KERNEL_EIG;
  gemm_f64(s, n, n, n, V2, n, false, S, n, true, z);
  }
  // 5. V = Q Z
  const int R = (n + 31) / 32;
  if (R <= 2) launch_backtransform<2>(s, n, H, tau, V);
  else if (R <= 4) launch_backtransform<4>(s, n, H, tau, V);
  else if (R <= 8) launch_backtransform<8>(s, n, H, tau, V);
  else if (R <= 16) launch_backtransform<16>(s, n, H, tau, V);
  else if (R <= 32) launch_backtransform<32>(s, n, H, tau, V);
  else {
    backtransform_kernel<<<cdiv(n, 2), 64, 0, s>>>(n, H, tau, V);
    RC_LAUNCH();
  }
  return true;
}

}  // namespace rchfsi
