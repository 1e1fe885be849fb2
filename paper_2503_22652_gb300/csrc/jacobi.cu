// Symmetric eigensolver for the N x N projected matrix of the Rayleigh-Ritz step (FP64):
// parallel cyclic Jacobi.
//
// One cooperative kernel runs whole sweeps.  A sweep is N'-1 rounds (N' = N rounded up to even) of
// the round-robin ("circle") pairing, in which the N'/2 index pairs are disjoint, so their plane
// rotations commute: each round computes the rotation (c, s) of every pair from the current 2 x 2
// block, then applies all row rotations (M <- J^T M), then all column rotations (M <- M J, V <- V J),
// with a grid-wide barrier between phases.  The rotation is the textbook symmetric Schur 2 x 2
// (tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2),
// s = t c), which zeroes a_pq.  After each sweep the off-diagonal Frobenius norm is compared with
// tol * ||M||_F.  The projected matrices of subspace iteration become nearly diagonal as the
// iteration converges, where Jacobi needs one or two sweeps.  Eigenvalues are returned ascending with
// the eigenvector columns permuted to match.
#include <cooperative_groups.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rchfsi {
namespace {

struct JacobiArgs {
  int n, np;          // size, size rounded up to even
  double* M;          // n x n, column-major, destroyed (diagonal = eigenvalues at exit)
  double* V;          // n x n eigenvectors (column-major)
  double* rot;        // np/2 x 4 scratch: p, q, c, s
  double* red;        // 4 doubles: off-diagonal sum, total sum, sweeps done, converged flag
  double tol;
  int max_sweeps;
};

__device__ __forceinline__ void pair_of(int r, int k, int np, int& p, int& q) {
  // circle method: index np-1 fixed, the others rotate
  if (k == 0) {
    p = np - 1;
    q = r;
  } else {
    p = (r + k) % (np - 1);
    q = (r - k + np - 1) % (np - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

__global__ void __launch_bounds__(512) jacobi_kernel(JacobiArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int n = a.n, np = a.np, half = np / 2;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  double* M = a.M;
  double* V = a.V;
  // V = I
  for (int64_t e = tid; e < (int64_t)n * n; e += nth) V[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
  if (tid == 0) {
    a.red[2] = 0.0;
    a.red[3] = 0.0;
  }
  grid.sync();
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      // rotations of this round's pairs
      for (int64_t k = tid; k < half; k += nth) {
        int p, q;
        pair_of(r, (int)k, np, p, q);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = M[(int64_t)q * n + p];
          if (apq != 0.0) {
            const double app = M[(int64_t)p * n + p], aqq = M[(int64_t)q * n + q];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        a.rot[4 * k + 0] = p;
        a.rot[4 * k + 1] = q;
        a.rot[4 * k + 2] = c;
        a.rot[4 * k + 3] = s;
      }
      grid.sync();
      // rows: M <- J^T M   (rows p, q of every pair, all columns)
      for (int64_t e = tid; e < (int64_t)half * n; e += nth) {
        const int64_t k = e / n, j = e - k * n;
        const int p = (int)a.rot[4 * k], q = (int)a.rot[4 * k + 1];
        const double s = a.rot[4 * k + 3];
        if (q >= n || s == 0.0) continue;
        const double c = a.rot[4 * k + 2];
        const double mp = M[j * n + p], mq = M[j * n + q];
        M[j * n + p] = c * mp - s * mq;
        M[j * n + q] = s * mp + c * mq;
      }
      grid.sync();
      // columns: M <- M J, V <- V J   (columns p, q of every pair, all rows)
      for (int64_t e = tid; e < (int64_t)half * n; e += nth) {
        const int64_t k = e / n, i = e - k * n;
        const int p = (int)a.rot[4 * k], q = (int)a.rot[4 * k + 1];
        const double s = a.rot[4 * k + 3];
        if (q >= n || s == 0.0) continue;
        const double c = a.rot[4 * k + 2];
        const double mp = M[(int64_t)p * n + i], mq = M[(int64_t)q * n + i];
        M[(int64_t)p * n + i] = c * mp - s * mq;
        M[(int64_t)q * n + i] = s * mp + c * mq;
        const double vp = V[(int64_t)p * n + i], vq = V[(int64_t)q * n + i];
        V[(int64_t)p * n + i] = c * vp - s * vq;
        V[(int64_t)q * n + i] = s * vp + c * vq;
      }
      grid.sync();
    }
    // convergence: off-diagonal vs total Frobenius norm
    if (tid == 0) {
      a.red[0] = 0.0;
      a.red[1] = 0.0;
    }
    grid.sync();
    double off = 0.0, tot = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += nth) {
      const double v = M[e];
      tot += v * v;
      if ((e / n) != (e % n)) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&a.red[0], off);
      atomicAdd(&a.red[1], tot);
    }
    grid.sync();
    const bool done = a.red[0] <= a.tol * a.tol * a.red[1];
    if (tid == 0) a.red[2] = sweep + 1;
    grid.sync();
    if (done) {
      if (tid == 0) a.red[3] = 1.0;
      break;
    }
  }
}

__global__ void permute_kernel(int n, const double* __restrict__ M, const double* __restrict__ V,
                               const int* __restrict__ perm, double* __restrict__ evals, double* __restrict__ Vout) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const int pj = perm[j];
    Vout[e] = V[(int64_t)pj * n + i];
    if (i == 0) evals[j] = M[(int64_t)pj * n + pj];
  }
}

}  // namespace

// Eigen-decomposition of the symmetric n x n matrix M (column-major, destroyed): eigenvalues
// ascending in evals (device), eigenvectors in V (device, column-major).  Returns the number of
// sweeps; throws NUMERIC if the off-diagonal norm did not fall below tol * ||M||_F in max_sweeps.
int jacobi_eig_f64(cudaStream_t s, int n, double* M, double* V, double* evals, DevBuf<double>& ws, double tol,
                   int max_sweeps) {
  RC_CHECK(n >= 1, RCHFSI_ERR_INVALID_ARG, "jacobi: empty matrix");
  const int np = n + (n & 1);
  const size_t need = (size_t)n * n + 2 * (size_t)np + 8 + (size_t)n;
  double* w = ws.ensure(need);
  double* Vtmp = w;
  double* rot = w + (size_t)n * n;
  double* red = rot + 2 * (size_t)np;
  int* perm = reinterpret_cast<int*>(red + 8);
  int dev = 0, sms = 0, per_sm = 0;
  RC_CUDA(cudaGetDevice(&dev));
  RC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, 512, 0));
  RC_CHECK(per_sm >= 1, RCHFSI_ERR_CUDA, "jacobi kernel cannot be resident");
  // enough threads for one phase of a round, at most one wave of co-resident blocks
  const int64_t work = (int64_t)(np / 2) * n;
  int blocks = (int)std::min<int64_t>((work + 511) / 512, (int64_t)sms * per_sm);
  blocks = std::max(blocks, 1);
  JacobiArgs a{n, np, M, Vtmp, rot, red, tol, max_sweeps};
  void* args[] = {&a};
  RC_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(512), args, 0, s));
  RC_LAUNCH();
  // order: ascending eigenvalues
  std::vector<double> diag(n), flags(4);
  RC_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), M, sizeof(double) * (n + 1), sizeof(double), n,
                            cudaMemcpyDeviceToHost, s));
  RC_CUDA(cudaMemcpyAsync(flags.data(), red, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  RC_CUDA(cudaStreamSynchronize(s));
  RC_CHECK(flags[3] == 1.0, RCHFSI_ERR_NUMERIC, "Jacobi eigensolver did not converge");
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return diag[x] < diag[y]; });
  RC_CUDA(cudaMemcpyAsync(perm, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  const unsigned pb = (unsigned)std::min<int64_t>(((int64_t)n * n + 255) / 256, 152 * 8);
  permute_kernel<<<pb, 256, 0, s>>>(n, M, Vtmp, perm, evals, V);
  RC_LAUNCH();
  RC_CUDA(cudaStreamSynchronize(s));  // idx must outlive the copy
  return (int)flags[2];
}

}  // namespace rchfsi
