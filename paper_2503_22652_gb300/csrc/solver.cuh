// Internal solver state shared by the C ABI, the filter and the Rayleigh-Ritz drivers.
#pragma once
#include <cusolverDn.h>

#include <memory>

#include "common.cuh"
#include "fe.cuh"
#include "oz_gemm.cuh"
#include "prof.cuh"

struct rchfsi_ctx;

namespace rchfsi {

// Device buffers of one solve (column-major m x N blocks and N x N matrices).
struct Work {
  int64_t m = 0;
  int N = 0;
  DevBuf<double> X, AX, BX, W, Y, AY, BY, T1;  // m x N
  DevBuf<double> GA, GB, Z, Zt, Lb, Li;        // N x N (Lb: Cholesky factor, Li: its inverse)
  DevBuf<double> eigws;                        // workspace of the projected eigensolver
  DevBuf<double> evals, nrm, rabs, xnrm, lamtab;
  DevBuf<float> lamtab_f;                      // FP32 copy of lamtab for the fused FE step
  DevBuf<float> R32a, R32b, W32;               // low-precision filter buffers (col-major or row-major)
  DevBuf<__nv_bfloat16> R16a, R16b, W16;
  DevBuf<float> split;                         // split-K partial sums of the tensor-core product
  DevBuf<int> info;
  DevBuf<double> lz_v, lz_w, lz_vp, lz_t, lz_ab;  // Lanczos vectors and scalars
  DevBuf<double> syev_work;
  DevBuf<double> coefd;                        // Chebyshev coefficient table of the batched filter
  DevBuf<double> stage_in, stage_out;          // host <-> device staging (row-major)
  OzOperand ozL, ozR, ozE;                     // FP64-emulation slices of the current operands
  DevBuf<double> ozws;                         // split-K partials of the emulated FP64 GEMM
  void ensure(int64_t m_, int N_);
};

struct DenseOp {
  DevBuf<double> A, B, Dinv, Dinv_dense;  // exact FP64 operators (A, B row-major = symmetric)
  DevBuf<double> AD64, DA64;              // filter operators A~ D^-1 and D^-1 A~, row-major
  DevBuf<float> AD32, DA32, ADtf, DAtf;   // FP32 copies (plain and TF32-rounded)
  DevBuf<__nv_bfloat16> AD16, DA16;       // BF16 copies
  OzOperand ozA, ozB;                     // FP64-emulation slices of A and B (made on first use)
  bool has_B = false, has_dinv = false, has_dinv_dense = false;
  void reset() {
    A.release(); B.release(); Dinv.release(); Dinv_dense.release(); AD64.release(); DA64.release();
    AD32.release(); DA32.release(); ADtf.release(); DAtf.release(); AD16.release(); DA16.release();
    ozA.sl.release(); ozA.ex.release(); ozB.sl.release(); ozB.ex.release(); ozA.R = ozB.R = 0;
    has_B = has_dinv = has_dinv_dense = false;
  }
};

}  // namespace rchfsi

struct rchfsi_ctx {
  rchfsi_params p{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = 0;
  int num_sms = 152;
  cusolverDnHandle_t solver = nullptr;
  std::string err;
  bool has_op = false;
  int op_kind = -1;
  rchfsi::DenseOp dense;
  std::unique_ptr<rchfsi::FeOp> fe;
  rchfsi::Work w;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // statistics of the last filter
  int64_t last_applies = 0;
  double last_flops = 0.0;
  bool is_server = false;
  void* server = nullptr;
  // complex Hermitian problems run as their real embedding (p holds the embedded sizes 2m, 2N,
  // 2 nev); the caller-facing sizes are kept here
  bool cplx = false;
  int64_t mc = 0;
  int Nc = 0, nevc = 0;
  rchfsi::DevBuf<double> cstage;  // complex staging (m x N interleaved)
  rchfsi::DevBuf<int> ccols;      // embedded columns selected for complex outputs
  rchfsi::DevBuf<double> cdot;    // complex inner product scratch
  bool rr_paired = false;         // the last Rayleigh-Ritz already kept one Ritz vector per complex pair
  int rr_retries = 0;             // the last Rayleigh-Ritz needed the shifted Cholesky QR step
  rchfsi::prof::Profiler prof;
};

namespace rchfsi {

// Operator applications in FP64 on column-major m x n blocks.
void apply_A_f64(rchfsi_ctx& c, const double* X, double* Y, int n);
void apply_B_f64(rchfsi_ctx& c, const double* X, double* Y, int n);  // Y = B X (copy when B = I)
void apply_AB_f64(rchfsi_ctx& c, const double* X, double* AX, double* BX, int n);  // both, one pass over X
bool has_B(const rchfsi_ctx& c);
const double* dinv_diag(const rchfsi_ctx& c);

// Algorithm 3 / Algorithm 2 on column-major inputs; Y is column-major FP64.
void filter_internal(rchfsi_ctx& c, const double* X, const double* lam_host, const double* W, double lmin,
                     double lT, double lmax, int p, double* Y, bool chfsi);

// Rayleigh-Ritz on column-major Y (scaled in place): X, AX, BX, evals (device) are outputs.
int rayleigh_ritz(rchfsi_ctx& c, double* Y, double* X, double* AX, double* BX, double* evals);

// Lanczos bounds (host results).
void lanczos(rchfsi_ctx& c, const double* v0_dev, int k, double* lmax, double* normA);

size_t device_bytes(const rchfsi_ctx& c);

// Batched FE filter (Algorithm 3 for several problems at once): every degree step runs the
// recurrence terms of each problem and one persistent tensor-core launch over all problems' cells,
// the whole degree loop replayed from a CUDA graph (re-captured when the set of problems changes).
struct FeFilterJob {
  rchfsi_ctx* c;
  const double* X;    // column-major block (first N columns are filtered; complex: N = Nc)
  const double* lam;  // host Ritz values (N)
  const double* W;    // column-major residual block
  double lmin, lT, lmax;
  double* Y;          // output, column-major
};
struct FeBatchPlan {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
  int kernels = 0;
  int64_t replays = 0;
  ~FeBatchPlan();
};
bool fe_batchable(const rchfsi_ctx& c, int degree);
void filter_fe_batch(cudaStream_t s, int num_sms, std::vector<FeFilterJob>& jobs, FeBatchPlan& plan);

}  // namespace rchfsi
