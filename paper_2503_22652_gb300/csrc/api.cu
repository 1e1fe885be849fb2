// C ABI of the R-ChFSI library and the host-side drivers of Algorithms 1-3.
//
// Host code computes the O(p) Chebyshev scalars and the O(pN) table of Lambda_k (the eigenvalue
// recurrence of Proposition 3.3) in FP64 and uploads them once per filter, so the whole degree
// loop is enqueued on the stream without host round trips.  Everything that touches an m-sized
// array runs in this library's kernels.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "solver.cuh"
#include "tc_gemm.cuh"
#include "fe_tc.cuh"
#include "fe_step.cuh"

#include <map>
#include <tuple>

using namespace rchfsi;

namespace rchfsi {

void Work::ensure(int64_t m_, int N_) {
  if (m_ == m && N_ == N && X.p) return;
  m = m_;
  N = N_;
  const size_t blk = (size_t)m * N;
  X.ensure(blk); AX.ensure(blk); BX.ensure(blk); W.ensure(blk); Y.ensure(blk); AY.ensure(blk); BY.ensure(blk);
  T1.ensure(blk);
  GA.ensure((size_t)N * N); GB.ensure((size_t)N * N); Z.ensure((size_t)N * N); Zt.ensure((size_t)N * N);
  Lb.ensure((size_t)N * N); Li.ensure((size_t)N * N);
  evals.ensure(N); nrm.ensure(N); rabs.ensure(N); xnrm.ensure(N);
  info.ensure(4);
  RC_CUDA(cudaMemset(info.p, 0, 4 * sizeof(int)));
}

bool has_B(const rchfsi_ctx& c) {
  if (c.op_kind == RCHFSI_OP_DENSE) return c.dense.has_B;
  return true;
}

const double* dinv_diag(const rchfsi_ctx& c) {
  if (c.op_kind == RCHFSI_OP_DENSE) return c.dense.has_dinv ? c.dense.Dinv.p : nullptr;
  return c.fe->Dinv.p;
}

static EpiArgs epi_store(void* C, int64_t ldc) {
  EpiArgs e;
  e.kind = EPI_STORE;
  e.C = C;
  e.ldc = ldc;
  return e;
}

// FE applies on column-major solver blocks: the FP64-accurate tensor-core products take them as
// they are (both products from one slicing of X); the DFMA path works on row-major copies.
static void fe_apply_cols(rchfsi_ctx& c, const double* X, double* AX, double* BX, int n) {
  const int64_t m = c.p.m;
  double* s0 = c.w.stage_in.ensure((size_t)m * n);
  double* s1 = c.w.stage_out.ensure((size_t)m * n);
  if (c.p.rr_mode == RCHFSI_RR_FP64_EMULATED) {
    fe_apply_f64_cols_tc(c.s, *c.fe, X, AX, BX, n, c.num_sms, s0, s1);
    return;
  }
  transpose_f64(c.s, n, m, X, m, s0, n);  // X col-major = n x m row-major view -> m x n row-major
  for (int which = 0; which < 2; ++which) {
    double* out = which ? BX : AX;
    if (!out) continue;
    fe_apply_f64_rows(c.s, *c.fe, which == 1, s0, s1, n);
    transpose_f64(c.s, m, n, s1, n, out, m);
  }
}

void apply_A_f64(rchfsi_ctx& c, const double* X, double* Y, int n) {
  const int64_t m = c.p.m;
  if (c.op_kind == RCHFSI_OP_DENSE) {
    gemm_f64(c.s, m, n, m, c.dense.A.p, m, true, X, m, true, epi_store(Y, m));
  } else {
    fe_apply_cols(c, X, Y, nullptr, n);
  }
}

void apply_B_f64(rchfsi_ctx& c, const double* X, double* Y, int n) {
  const int64_t m = c.p.m;
  if (c.op_kind == RCHFSI_OP_DENSE) {
    if (c.dense.has_B)
      gemm_f64(c.s, m, n, m, c.dense.B.p, m, true, X, m, true, epi_store(Y, m));
    else
      RC_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * m * n, cudaMemcpyDeviceToDevice, c.s));
  } else {
    fe_apply_cols(c, X, nullptr, Y, n);
  }
}

void apply_AB_f64(rchfsi_ctx& c, const double* X, double* AX, double* BX, int n) {
  if (c.op_kind == RCHFSI_OP_DENSE) {
    apply_A_f64(c, X, AX, n);
    apply_B_f64(c, X, BX, n);
  } else {
    fe_apply_cols(c, X, AX, BX, n);
  }
}

size_t device_bytes(const rchfsi_ctx& c) {
  size_t t = 0;
  const DenseOp& d = c.dense;
  t += d.A.bytes() + d.B.bytes() + d.Dinv.bytes() + d.Dinv_dense.bytes() + d.AD64.bytes() + d.DA64.bytes();
  t += d.AD32.bytes() + d.DA32.bytes() + d.ADtf.bytes() + d.DAtf.bytes() + d.AD16.bytes() + d.DA16.bytes();
  if (c.fe) {
    const FeOp& f = *c.fe;
    t += f.dofs.bytes() + f.A64.bytes() + f.B64.bytes() + f.Dinv.bytes() + f.A32.bytes() + f.Atf.bytes() +
         f.A16.bytes() + f.Dinv32.bytes();
  }
  const Work& w = c.w;
  t += w.X.bytes() * 8 + w.GA.bytes() * 4 + w.R32a.bytes() * 3 + w.R16a.bytes() * 3 + w.split.bytes() +
       w.stage_in.bytes() + w.stage_out.bytes() + w.lamtab.bytes();
  return t;
}

static void check_budget(rchfsi_ctx& c) {
  if (c.p.hbm_budget_bytes && device_bytes(c) > c.p.hbm_budget_bytes)
    throw Error(RCHFSI_ERR_OOM, "device footprint " + std::to_string(device_bytes(c)) +
                                    " bytes exceeds hbm_budget_bytes " + std::to_string(c.p.hbm_budget_bytes));
}

// ------------------------------------------------------------------ low-precision operator copies
// Reduced-precision dense operands use a row pitch padded to a multiple of 8 elements, so that
// every row starts on a 16-byte boundary (a TMA requirement); padding is zero-filled.
static inline int64_t padded(int64_t m) { return (m + 7) / 8 * 8; }

static const float* dense_op32(rchfsi_ctx& c, bool chfsi, bool tf32) {
  DenseOp& d = c.dense;
  const int64_t m = c.p.m, mp = padded(m);
  DevBuf<float>& buf = chfsi ? (tf32 ? d.DAtf : d.DA32) : (tf32 ? d.ADtf : d.AD32);
  if (!buf.p) {
    buf.ensure((size_t)m * mp);
    fill_zero(c.s, buf.p, buf.bytes());
    cast2d_f64_to_f32(c.s, m, m, chfsi ? d.DA64.p : d.AD64.p, m, buf.p, mp, 1.0, tf32 ? 1 : 0);
    check_budget(c);
  }
  return buf.p;
}

static const __nv_bfloat16* dense_op16(rchfsi_ctx& c, bool chfsi) {
  DenseOp& d = c.dense;
  const int64_t m = c.p.m, mp = padded(m);
  DevBuf<__nv_bfloat16>& buf = chfsi ? d.DA16 : d.AD16;
  if (!buf.p) {
    buf.ensure((size_t)m * mp);
    fill_zero(c.s, buf.p, buf.bytes());
    cast2d_f64_to_bf16(c.s, m, m, chfsi ? d.DA64.p : d.AD64.p, m, buf.p, mp, 1.0);
    check_budget(c);
  }
  return buf.p;
}

// ------------------------------------------------------------------ the filters
struct Coef {
  double a, b, c;
};

static void filter_scalars(double lmin, double lT, double lmax, int p, double& e, double& cc, double& s1,
                           std::vector<Coef>& co) {
  // Algorithms 2/3, first line: e, c, sigma_1, gamma; loop k = 2..p: sigma_2 = 1/(gamma - sigma)
  e = 0.5 * (lmax - lT);
  cc = 0.5 * (lmax + lT);
  s1 = e / (lmin - cc);
  const double gamma = 2.0 / s1;
  double sigma = s1;
  co.clear();
  for (int k = 2; k <= p; ++k) {
    const double s2 = 1.0 / (gamma - sigma);
    const double a = 2.0 * s2 / e;
    co.push_back({a, -a * cc, -sigma * s2});
    sigma = s2;
  }
}

// Lambda_d = C_d(Lambda) for d = 0..p (Proposition 3.3), row d of the (p+1) x N table.
static void lambda_table(const double* lam, int N, double e, double cc, double s1, const std::vector<Coef>& co,
                         std::vector<double>& tab) {
  const int p = (int)co.size() + 1;
  tab.assign((size_t)(p + 1) * N, 0.0);
  for (int j = 0; j < N; ++j) {
    double lx = 1.0, ly = (s1 / e) * (lam[j] - cc);
    tab[j] = 1.0;
    tab[(size_t)N + j] = ly;
    for (int k = 0; k < p - 1; ++k) {
      const double a = co[k].a;
      const double nx = a * ly * lam[j] - a * cc * ly + co[k].c * lx;
      lx = ly;
      ly = nx;
      tab[(size_t)(k + 2) * N + j] = ly;
    }
  }
}

// Scales s_k of the iterates S_k = s_k R_k of the fused FE step (s_1 = s_2 = 1, s_k = s_{k-2} / c_k,
// so that S_{k-2} enters step k with coefficient 1); false when one leaves [2^-60, 2^60] (the
// unfused step is used then).
static bool fused_scales(const std::vector<Coef>& co, std::vector<double>& sc) {
  const int p = (int)co.size() + 1;
  sc.assign((size_t)p + 1, 1.0);
  for (int k = 3; k <= p; ++k) {
    sc[k] = sc[k - 2] / co[k - 2].c;
    if (!std::isfinite(sc[k]) || std::fabs(sc[k]) > 0x1p60 || std::fabs(sc[k]) < 0x1p-60) return false;
  }
  return true;
}

// (alpha, beta, omega) of the fused step producing degree k (k >= 2): S_k = S_{k-2} + alpha A D^-1
// S_{k-1} + beta S_{k-1} + omega W Lambda_{k-1}.
static void fused_coefs(const std::vector<Coef>& co, const std::vector<double>& sc, int k, double* out) {
  const Coef& q = co[k - 2];
  out[0] = sc[k] * q.a / sc[k - 1];
  out[1] = sc[k] * q.b / sc[k - 1];
  out[2] = sc[k] * q.a;
}

static void check_bounds(double lmin, double lT, double lmax, int p) {
  RC_CHECK(p >= 1, RCHFSI_ERR_INVALID_ARG, "degree must be >= 1");
  RC_CHECK(std::isfinite(lmin) && std::isfinite(lT) && std::isfinite(lmax), RCHFSI_ERR_INVALID_ARG,
           "bounds must be finite");
  RC_CHECK(lmax > lT, RCHFSI_ERR_INVALID_ARG, "need lmax > lT");
  RC_CHECK(lmin < lT, RCHFSI_ERR_INVALID_ARG, "need lmin < lT");
}

// Dense filter product step for the reduced precisions on column-major FP32/BF16 blocks of pitch mp.
static void dense_step_lowp(rchfsi_ctx& c, bool chfsi, int prec, const void* Ry, const void* Rx, const void* W,
                            const double* lam, const Coef& k, void* out) {
  const int64_t m = c.p.m, mp = padded(m);
  const int N = c.p.block;
  if (prec == RCHFSI_FP32) {
    EpiArgs e;
    e.kind = EPI_RECUR;
    e.C = out;
    e.ldc = mp;
    e.a = k.a;
    e.b = k.b;
    e.c = k.c;
    e.Ry = Ry;
    e.Rx = Rx;
    e.W = W;
    e.lam = lam;
    e.prof_cls = RCHFSI_KERNEL_FILTER_SIMT;
    gemm_f32(c.s, m, N, m, dense_op32(c, chfsi, false), mp, true, (const float*)Ry, mp, true, e);
  } else if (prec == RCHFSI_TF32) {
    TcRecur r{(float)k.a, (float)k.b, (float)k.c, (const float*)Ry, (const float*)Rx, (const float*)W, lam,
              (float*)out};
    tc_gemm_tf32_recur(c.s, c.num_sms, m, N, m, dense_op32(c, chfsi, true), mp, (const float*)Ry, mp, c.w.split,
                       r, mp, c.w.info.p + 2);
  } else {
    TcRecur16 r{(float)k.a, (float)k.b, (float)k.c, (const __nv_bfloat16*)Ry, (const __nv_bfloat16*)Rx,
                (const __nv_bfloat16*)W, lam, (__nv_bfloat16*)out};
    tc_gemm_bf16_recur(c.s, c.num_sms, m, N, m, dense_op16(c, chfsi), mp, (const __nv_bfloat16*)Ry, mp, c.w.split,
                       r, mp, c.w.info.p + 2);
  }
}

static void filter_dense(rchfsi_ctx& c, const double* X, const double* W, int p, const double* lamtab, double e,
                         double cc, double s1, const std::vector<Coef>& co, double* Y, bool chfsi) {
  const int64_t m = c.p.m;
  const int N = c.p.block;
  const size_t blk = (size_t)m * N;
  const int prec = c.p.precision;
  DenseOp& d = c.dense;
  const double* lam_p = lamtab + (size_t)p * N;
  if (prec == RCHFSI_FP64) {
    double* RX = c.w.AY.p;
    double* RY = c.w.BY.p;
    const double* op = chfsi ? d.DA64.p : d.AD64.p;
    if (!chfsi) {
      scaled_copy_f64(c.s, blk, W, RY, s1 / e);
    } else {
      // Algorithm 2: Y_0 = X, Y_1 = (sigma_1/e)(H - cI) X
      RC_CUDA(cudaMemcpyAsync(RX, X, blk * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
      EpiArgs e1;
      e1.kind = EPI_RECUR;
      e1.C = RY;
      e1.ldc = m;
      e1.a = s1 / e;
      e1.b = -(s1 / e) * cc;
      e1.c = 0.0;
      e1.Ry = X;
      e1.prof_cls = RCHFSI_KERNEL_FILTER_SIMT;
      gemm_f64(c.s, m, N, m, op, m, true, X, m, true, e1);
    }
    for (size_t k = 0; k < co.size(); ++k) {
      EpiArgs ep;
      ep.kind = EPI_RECUR;
      ep.C = RX;
      ep.ldc = m;
      ep.a = co[k].a;
      ep.b = co[k].b;
      ep.c = co[k].c;
      ep.Ry = RY;
      ep.Rx = (chfsi || k > 0) ? RX : nullptr;  // R_X = 0 before the first step of Algorithm 3
      ep.W = chfsi ? nullptr : W;
      ep.lam = chfsi ? nullptr : lamtab + (k + 1) * N;
      ep.prof_cls = RCHFSI_KERNEL_FILTER_SIMT;
      gemm_f64(c.s, m, N, m, op, m, true, RY, m, true, ep);
      std::swap(RX, RY);
    }
    if (chfsi) {
      RC_CUDA(cudaMemcpyAsync(Y, RY, blk * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    } else if (d.has_dinv_dense) {
      EpiArgs ep;
      ep.kind = EPI_AXPY_DIAG;
      ep.C = Y;
      ep.ldc = m;
      ep.Xadd = X;
      ep.ldx = m;
      ep.lam = lam_p;
      gemm_f64(c.s, m, N, m, d.Dinv_dense.p, m, true, RY, m, true, ep);
    } else {
      reconstruct_f64(c.s, m, N, RY, m, d.has_dinv ? d.Dinv.p : nullptr, X, lam_p, Y);
    }
    c.last_applies = (int64_t)co.size() + (chfsi ? 1 : 0);
    return;
  }
  // reduced precision: FP32 / TF32 storage in float, BF16 storage in bfloat16, pitch mp
  const int64_t mp = padded(m);
  const size_t pblk = (size_t)mp * N;
  const bool bf = prec == RCHFSI_BF16;
  void *RX, *RY, *Wl;
  if (bf) {
    const bool fresh = c.w.R16a.n < pblk;
    RX = c.w.R16a.ensure(pblk);
    RY = c.w.R16b.ensure(pblk);
    Wl = c.w.W16.ensure(pblk);
    if (fresh) {
      fill_zero(c.s, RX, pblk * 2);
      fill_zero(c.s, RY, pblk * 2);
      fill_zero(c.s, Wl, pblk * 2);
    }
  } else {
    const bool fresh = c.w.R32a.n < pblk;
    RX = c.w.R32a.ensure(pblk);
    RY = c.w.R32b.ensure(pblk);
    Wl = c.w.W32.ensure(pblk);
    if (fresh) {
      fill_zero(c.s, RX, pblk * 4);
      fill_zero(c.s, RY, pblk * 4);
      fill_zero(c.s, Wl, pblk * 4);
    }
  }
  check_budget(c);
  // column-major m x N (pitch m) -> pitch mp: N "rows" of m contiguous entries
  auto cast = [&](const double* in, void* out, double scale) {
    if (bf) cast2d_f64_to_bf16(c.s, N, m, in, m, (__nv_bfloat16*)out, mp, scale);
    else cast2d_f64_to_f32(c.s, N, m, in, m, (float*)out, mp, scale, 0);
  };
  auto recon = [&](const void* R, const double* dv, const double* lam, double* out) {
    if (bf) reconstruct_bf16(c.s, m, N, (const __nv_bfloat16*)R, mp, dv, X, lam, out);
    else reconstruct_f32(c.s, m, N, (const float*)R, mp, dv, X, lam, out);
  };
  if (!chfsi) {
    cast(W, RY, s1 / e);
    cast(W, Wl, 1.0);
  } else {
    cast(X, RX, 1.0);
    dense_step_lowp(c, true, prec, RX, nullptr, nullptr, nullptr, Coef{s1 / e, -(s1 / e) * cc, 0.0}, RY);
  }
  for (size_t k = 0; k < co.size(); ++k) {
    dense_step_lowp(c, chfsi, prec, RY, (chfsi || k > 0) ? RX : nullptr, chfsi ? nullptr : Wl,
                    chfsi ? nullptr : lamtab + (k + 1) * N, co[k], RX);
    std::swap(RX, RY);
  }
  if (chfsi) {
    recon(RY, nullptr, c.w.nrm.p, Y);  // nrm holds zeros: plain upcast
  } else if (d.has_dinv_dense) {
    recon(RY, nullptr, c.w.nrm.p, c.w.T1.p);
    EpiArgs ep;
    ep.kind = EPI_AXPY_DIAG;
    ep.C = Y;
    ep.ldc = m;
    ep.Xadd = X;
    ep.ldx = m;
    ep.lam = lam_p;
    gemm_f64(c.s, m, N, m, d.Dinv_dense.p, m, true, c.w.T1.p, m, true, ep);
  } else {
    recon(RY, d.has_dinv ? d.Dinv.p : nullptr, lam_p, Y);
  }
  c.last_applies = (int64_t)co.size() + (chfsi ? 1 : 0);
}

static void filter_fe(rchfsi_ctx& c, const double* X, const double* W, int p, const double* lamtab, double e,
                      double cc, double s1, const std::vector<Coef>& co, double* Y, bool chfsi) {
  const int64_t m = c.p.m;
  const int N = c.p.block;
  const size_t blk = (size_t)m * N;
  const int prec = c.p.precision;
  FeOp& f = *c.fe;
  if (prec == RCHFSI_FP64) {
    // row-major working copy of the input block (W for Algorithm 3, X for Algorithm 2)
    double* Wr = c.w.stage_out.ensure(blk);
    transpose_f64(c.s, N, m, chfsi ? X : W, m, Wr, N);
    double* RX = c.w.AY.p;
    double* RY = c.w.BY.p;
    if (!chfsi) {
      scaled_copy_f64(c.s, blk, Wr, RY, s1 / e);
    } else {
      RC_CUDA(cudaMemcpyAsync(RX, Wr, blk * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
      recur_terms_rows_f64(c.s, m, N, RX, RY, nullptr, nullptr, 0.0, -(s1 / e) * cc, 0.0);
      fe_filter_product_f64(c.s, f, RX, RY, N, s1 / e, 2);
    }
    for (size_t k = 0; k < co.size(); ++k) {
      if (!chfsi && k == 0) fill_zero(c.s, RX, blk * sizeof(double));
      recur_terms_rows_f64(c.s, m, N, RY, RX, chfsi ? nullptr : Wr, chfsi ? nullptr : lamtab + (k + 1) * N,
                           co[k].a, co[k].b, co[k].c);
      fe_filter_product_f64(c.s, f, RY, RX, N, co[k].a, chfsi ? 2 : 1);
      std::swap(RX, RY);
    }
    // back to column-major, then Y = D^-1 R_Y + X Lambda_p (or Y = R_Y for ChFSI)
    transpose_f64(c.s, m, N, RY, N, Y, m);
    if (!chfsi) reconstruct_f64(c.s, m, N, Y, m, f.Dinv.p, X, lamtab + (size_t)p * N, Y);
    c.last_applies = (int64_t)co.size() + (chfsi ? 1 : 0);
    return;
  }
  RC_CHECK(prec == RCHFSI_FP32 || prec == RCHFSI_TF32 || prec == RCHFSI_BF16, RCHFSI_ERR_INVALID_ARG,
           "bad precision");
  std::vector<double> sc;
  if (!chfsi && fe_step_supported(f, N, prec) && fused_scales(co, sc)) {
    // fused degree steps on scaled iterates: one tensor-core launch per step does the cell products,
    // the recurrence terms and the update of R_X
    float* RX = c.w.R32a.ensure(blk);
    float* RY = c.w.R32b.ensure(blk);
    float* Wl = c.w.W32.ensure(blk);
    check_budget(c);
    // S_1 = R_1 = (sigma_1 / e) W and W, row-major FP32, in one pass over the column-major W
    cols_to_rows_f32x2(c.s, m, N, W, s1 / e, 1.0, RY, Wl);
    fill_zero(c.s, RX, blk * sizeof(float));  // S_0 = R_0 = 0
    if (!co.empty()) {
      float* lamf = c.w.lamtab_f.ensure((size_t)(p + 1) * N);  // the Lambda table in FP32 for the kernel
      cast_f64_to_f32(c.s, (int64_t)(p + 1) * N, lamtab, lamf, 1.0, 0);
      const int BN = fe_step_tune(c.s, c.num_sms, f, N, RY, Wl, lamf + N);
      for (int k = 2; k <= p; ++k) {
        double cf[3];
        fused_coefs(co, sc, k, cf);
        FeStepPart parts[4];
        const int np = fe_step_parts(f, RY, Wl, RX, lamf + (size_t)(k - 1) * N, N, (float)cf[0], (float)cf[1],
                                     (float)cf[2], nullptr, parts);
        fe_step_batch(c.s, parts, np, BN, c.num_sms);
        std::swap(RX, RY);
      }
    }
    // Y = D^-1 R_p + X Lambda_p with R_p = S_p / s_p, in one pass back to column-major
    rows_to_cols_recon(c.s, m, N, RY, 1.0 / sc[p], f.Dinv.p, X, lamtab + (size_t)p * N, Y);
    c.last_applies = (int64_t)co.size();
    return;
  }
  float* RX = c.w.R32a.ensure(blk);
  float* RY = c.w.R32b.ensure(blk);
  float* Wl = c.w.W32.ensure(blk);
  check_budget(c);
  if (!chfsi) {
    cols_to_rows_f32x2(c.s, m, N, W, s1 / e, 1.0, RY, Wl);
  } else {
    cols_to_rows_f32x2(c.s, m, N, X, 1.0, 1.0, RX, RX);
    recur_terms_rows_f32(c.s, m, N, RX, RY, nullptr, nullptr, 0.0, -(s1 / e) * cc, 0.0);
    fe_filter_product_f32(c.s, f, prec, RX, RY, N, (float)(s1 / e), 2);
  }
  for (size_t k = 0; k < co.size(); ++k) {
    if (!chfsi && k == 0) fill_zero(c.s, RX, blk * sizeof(float));
    recur_terms_rows_f32(c.s, m, N, RY, RX, chfsi ? nullptr : Wl, chfsi ? nullptr : lamtab + (k + 1) * N,
                         co[k].a, co[k].b, co[k].c);
    fe_filter_product_f32(c.s, f, prec, RY, RX, N, (float)co[k].a, chfsi ? 2 : 1);
    std::swap(RX, RY);
  }
  // Y = D^-1 R_p + X Lambda_p (Algorithm 3), or Y = R_p (Algorithm 2: no D^-1, zero Lambda)
  rows_to_cols_recon(c.s, m, N, RY, 1.0, chfsi ? nullptr : f.Dinv.p, X, chfsi ? c.w.nrm.p : lamtab + (size_t)p * N, Y);
  c.last_applies = (int64_t)co.size() + (chfsi ? 1 : 0);
}

void filter_internal(rchfsi_ctx& c, const double* X, const double* lam_host, const double* W, double lmin, double lT,
                     double lmax, int p, double* Y, bool chfsi) {
  check_bounds(lmin, lT, lmax, p);
  const int N = c.p.block;
  double e, cc, s1;
  std::vector<Coef> co;
  filter_scalars(lmin, lT, lmax, p, e, cc, s1, co);
  std::vector<double> tab;
  if (!chfsi) {
    lambda_table(lam_host, N, e, cc, s1, co, tab);
  } else {
    tab.assign((size_t)(p + 1) * N, 0.0);
  }
  double* dtab = c.w.lamtab.ensure(tab.size());
  RC_CUDA(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  // zero "lambda" vector used by reconstructions that only upcast
  RC_CUDA(cudaMemsetAsync(c.w.nrm.p, 0, sizeof(double) * N, c.s));
  if (c.op_kind == RCHFSI_OP_DENSE)
    filter_dense(c, X, W, p, dtab, e, cc, s1, co, Y, chfsi);
  else
    filter_fe(c, X, W, p, dtab, e, cc, s1, co, Y, chfsi);
  // the host table must outlive the async copy; then read the kernels' timeout flag
  int flag = 0;
  RC_CUDA(cudaMemcpyAsync(&flag, c.w.info.p + 2, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  if (flag) {
    RC_CUDA(cudaMemsetAsync(c.w.info.p + 2, 0, sizeof(int), c.s));
    throw Error(RCHFSI_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel ran out");
  }
  // (a complex FE product is four real cell products; the dense embedding already counts 4x)
  const double flops_per = (c.op_kind == RCHFSI_OP_DENSE)
                               ? 2.0 * (double)c.p.m * (double)c.p.m * N
                               : 2.0 * (double)c.fe->nc * c.fe->nc * (double)c.fe->n_cells * N *
                                     (c.fe->cplx ? 4.0 : 1.0);
  c.last_flops = flops_per * (double)c.last_applies;
}

// ------------------------------------------------------------------ batched FE filter
namespace {

// Column tile of the batched cell-matrix product, picked by timing candidate tiles on the problem's
// own data (into a scratch output) the first time a shape is met; cached per shape.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int64_t, int>, int> g_tune_cache;

int tune_bn(cudaStream_t s, int num_sms, FeOp& op, int prec, int n, const float* Ry) {
  const auto key = std::make_tuple(prec, n, op.nc, (int64_t)op.n_cells, op.cplx ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  const int bmax = fe_tc_bn_max(prec);
  const int nr = (n + 15) / 16 * 16;
  std::vector<int> cand;
  for (int bn : {32, 48, 64, 96, 128, 160, 208})
    if (bn <= bmax && bn <= std::max(nr, 32)) cand.push_back(bn);
  if (cand.empty()) cand.push_back(16);
  DevBuf<float> scratch;
  float* out = scratch.ensure((size_t)op.m * n);
  cudaEvent_t e0, e1;
  RC_CUDA(cudaEventCreate(&e0));
  RC_CUDA(cudaEventCreate(&e1));
  int best = cand[0];
  float best_ms = 1e30f;
  for (int bn : cand) {
    FeTcPart parts[4];
    const int np = fe_tc_parts(op, Ry, out, n, 1.f, nullptr, 1, bn, parts);
    fe_tc_batch(s, prec, parts, np, num_sms);  // warm-up
    RC_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 2; ++r) fe_tc_batch(s, prec, parts, np, num_sms);
    RC_CUDA(cudaEventRecord(e1, s));
    RC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return best;
}

}  // namespace

FeBatchPlan::~FeBatchPlan() {
  if (exec) cudaGraphExecDestroy(exec);
}

bool fe_batchable(const rchfsi_ctx& c, int degree) {
  return c.op_kind == RCHFSI_OP_FE_CELL && c.fe && (c.p.precision == RCHFSI_TF32 || c.p.precision == RCHFSI_BF16) &&
         c.p.method == RCHFSI_METHOD_RCHFSI && c.p.degree == degree && c.p.degree >= 2;
}

void filter_fe_batch(cudaStream_t s, int num_sms, std::vector<FeFilterJob>& jobs, FeBatchPlan& plan) {
  RC_CHECK(!jobs.empty(), RCHFSI_ERR_INVALID_ARG, "empty batch");
  const int p = jobs[0].c->p.degree;
  const int prec = jobs[0].c->p.precision;
  for (auto& j : jobs)
    RC_CHECK(fe_batchable(*j.c, p) && j.c->p.precision == prec, RCHFSI_ERR_UNSUPPORTED,
             "batched filter: FE operators, R-ChFSI, one TF32/BF16 precision and degree");
  const int nj = (int)jobs.size();
  std::vector<std::vector<double>> tabs(nj), coefs(nj), scales(nj);
  std::vector<float*> RX(nj), RY(nj), WL(nj);
  std::vector<int> nn(nj), bn(nj);
  std::vector<double*> dtab(nj), dcoef(nj);
  std::vector<std::vector<Coef>> cos(nj);
  // fused degree steps (scaled iterates, one tensor-core launch per step) when every problem allows
  bool fused = true;
  for (int q = 0; q < nj; ++q) {
    rchfsi_ctx& c = *jobs[q].c;
    const int n = c.cplx ? c.Nc : c.p.block;
    double e, cc, s1;
    filter_scalars(jobs[q].lmin, jobs[q].lT, jobs[q].lmax, p, e, cc, s1, cos[q]);
    fused = fused && fe_step_supported(*c.fe, n, prec) && fused_scales(cos[q], scales[q]);
  }
  // 1. per problem: scalars, Lambda table and coefficient table on the device, initial blocks
  for (int q = 0; q < nj; ++q) {
    FeFilterJob& J = jobs[q];
    rchfsi_ctx& c = *J.c;
    check_bounds(J.lmin, J.lT, J.lmax, p);
    const int n = c.cplx ? c.Nc : c.p.block;  // a complex block is filtered on its first N columns
    const int64_t m = c.p.m;
    const size_t blk = (size_t)m * n;
    nn[q] = n;
    double e, cc, s1;
    std::vector<Coef> co;
    filter_scalars(J.lmin, J.lT, J.lmax, p, e, cc, s1, co);
    lambda_table(J.lam, n, e, cc, s1, co, tabs[q]);
    coefs[q].resize(3 * co.size());
    for (size_t k = 0; k < co.size(); ++k) {
      if (fused) {
        fused_coefs(co, scales[q], (int)k + 2, &coefs[q][3 * k]);
        continue;
      }
      coefs[q][3 * k] = co[k].a;
      coefs[q][3 * k + 1] = co[k].b;
      coefs[q][3 * k + 2] = co[k].c;
    }
    dtab[q] = c.w.lamtab.ensure(tabs[q].size());
    dcoef[q] = c.w.coefd.ensure(coefs[q].size());
    RC_CUDA(cudaMemcpyAsync(dtab[q], tabs[q].data(), tabs[q].size() * sizeof(double), cudaMemcpyHostToDevice, s));
    RC_CUDA(cudaMemcpyAsync(dcoef[q], coefs[q].data(), coefs[q].size() * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    RX[q] = c.w.R32a.ensure(blk);
    RY[q] = c.w.R32b.ensure(blk);
    WL[q] = c.w.W32.ensure(blk);
    cols_to_rows_f32x2(s, m, n, J.W, s1 / e, 1.0, RY[q], WL[q]);
    fill_zero(s, RX[q], blk * sizeof(float));
    if (fused) {
      fe_step_prepare(s, *c.fe);
      float* lf = c.w.lamtab_f.ensure(tabs[q].size());  // the Lambda table in FP32 for the kernel
      cast_f64_to_f32(s, (int64_t)tabs[q].size(), dtab[q], lf, 1.0, 0);
    } else {
      fe_tc_parts_prepare(s, *c.fe, prec);
    }
  }
  // 2. column tiles (autotuned once per shape); the fused launch takes one tile for all problems,
  //    the one tuned for the problem with the most cells
  int bn_fused = 0;
  int64_t most = -1;
  for (int q = 0; q < nj; ++q) {
    FeOp& op = *jobs[q].c->fe;
    bn[q] = fused ? fe_step_tune(s, num_sms, op, nn[q], RY[q], WL[q], jobs[q].c->w.lamtab_f.p + nn[q])
                  : tune_bn(s, num_sms, op, prec, nn[q], RY[q]);
    if (op.n_cells * (op.cplx ? 4 : 1) > most) {
      most = op.n_cells * (op.cplx ? 4 : 1);
      bn_fused = bn[q];
    }
  }
  // 3. the degree loop as one CUDA graph: per step one persistent tensor-core launch over every
  //    problem's cells (at most 64 parts per launch); the unfused form runs the recurrence terms of
  //    every problem first
  std::vector<uintptr_t> key = {(uintptr_t)p, (uintptr_t)prec, (uintptr_t)fused};
  for (int q = 0; q < nj; ++q)
    for (uintptr_t v : {(uintptr_t)jobs[q].c, (uintptr_t)RX[q], (uintptr_t)RY[q], (uintptr_t)WL[q],
                        (uintptr_t)dtab[q], (uintptr_t)dcoef[q], (uintptr_t)nn[q], (uintptr_t)bn[q],
                        (uintptr_t)jobs[q].c->w.lamtab_f.p})
      key.push_back(v);
  if (!plan.exec || plan.key != key) {
    if (plan.exec) {
      cudaGraphExecDestroy(plan.exec);
      plan.exec = nullptr;
    }
    prof::Profiler* saved = prof::current();
    prof::current() = nullptr;  // no timing events inside a capture
    int kernels = 0;
    RC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      std::vector<float*> rx = RX, ry = RY;
      for (int k = 0; fused && k + 1 < p; ++k) {
        std::vector<FeStepPart> parts;
        for (int q = 0; q < nj; ++q) {
          rchfsi_ctx& c = *jobs[q].c;
          FeStepPart pp[4];
          const int np = fe_step_parts(*c.fe, ry[q], WL[q], rx[q], c.w.lamtab_f.p + (size_t)(k + 1) * nn[q], nn[q],
                                       0.f, 0.f, 0.f, dcoef[q] + 3 * k, pp);
          parts.insert(parts.end(), pp, pp + np);
        }
        for (size_t o = 0; o < parts.size(); o += 64) {
          fe_step_batch(s, parts.data() + o, (int)std::min<size_t>(64, parts.size() - o), bn_fused, num_sms);
          ++kernels;
        }
        std::swap(rx, ry);
      }
      for (int k = 0; !fused && k + 1 < p; ++k) {
        std::vector<FeTcPart> parts;
        for (int q = 0; q < nj; ++q) {
          rchfsi_ctx& c = *jobs[q].c;
          recur_terms_rows_f32_dev(s, c.p.m, nn[q], ry[q], rx[q], WL[q], dtab[q] + (size_t)(k + 1) * nn[q],
                                   dcoef[q] + 3 * k);
          ++kernels;
          FeTcPart pp[4];
          const int np = fe_tc_parts(*c.fe, ry[q], rx[q], nn[q], 0.f, dcoef[q] + 3 * k, 1, bn[q], pp);
          parts.insert(parts.end(), pp, pp + np);
        }
        for (size_t o = 0; o < parts.size(); o += 64) {
          fe_tc_batch(s, prec, parts.data() + o, (int)std::min<size_t>(64, parts.size() - o), num_sms);
          ++kernels;
        }
        std::swap(rx, ry);
      }
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      prof::current() = saved;
      throw;
    }
    cudaGraph_t g = nullptr;
    RC_CUDA(cudaStreamEndCapture(s, &g));
    prof::current() = saved;
    const cudaError_t ie = cudaGraphInstantiate(&plan.exec, g, 0);
    cudaGraphDestroy(g);
    RC_CUDA(ie);
    plan.key = key;
    plan.kernels = kernels;
    plan.replays = 0;
  }
  {
    // algorithmic work of the replayed degree loop: per step and problem the cell products and the
    // four block streams (R_Y, R_X read and written, W) plus the cell matrices of every real part
    double fl = 0.0, by = 0.0;
    for (int q = 0; q < nj; ++q) {
      const FeOp& op = *jobs[q].c->fe;
      const double parts = op.cplx ? 4.0 : 1.0;
      fl += 2.0 * op.nc * op.nc * (double)op.n_cells * nn[q] * parts * (p - 1);
      by += (16.0 * (double)jobs[q].c->p.m * nn[q] + 4.0 * op.nc * op.nc * (double)op.n_cells * parts) * (p - 1);
    }
    prof::Scope ps(s, RCHFSI_KERNEL_FE_CELL, fl, by);
    RC_CUDA(cudaGraphLaunch(plan.exec, s));
  }
  // launches inside the capture were counted once; count every later replay too
  if (plan.replays++ > 0) __atomic_add_fetch(&launch_counter(), (int64_t)plan.kernels, __ATOMIC_RELAXED);
  // 4. per problem: Y = D^-1 R_Y + X Lambda_p, back in FP64 column-major (+ the J half for complex)
  for (int q = 0; q < nj; ++q) {
    FeFilterJob& J = jobs[q];
    rchfsi_ctx& c = *J.c;
    const int n = nn[q];
    const int64_t m = c.p.m;
    float* ryf = ((p - 1) % 2 == 0) ? RY[q] : RX[q];
    // fused: R_p = S_p / s_p
    rows_to_cols_recon(s, m, n, ryf, fused ? 1.0 / scales[q][p] : 1.0, c.fe->Dinv.p, J.X, dtab[q] + (size_t)p * n,
                       J.Y);
    if (c.cplx) cplx_rebuild(s, c.mc, c.Nc, J.Y, nullptr, J.Y);
    c.last_applies = p - 1;
    c.last_flops = 2.0 * c.fe->nc * c.fe->nc * (double)c.fe->n_cells * n * (c.fe->cplx ? 4.0 : 1.0) * (p - 1);
  }
  RC_CUDA(cudaStreamSynchronize(s));  // the host tables must outlive their copies
  for (int q = 0; q < nj; ++q) {
    rchfsi_ctx& c = *jobs[q].c;
    int flag = 0;
    RC_CUDA(cudaMemcpy(&flag, c.w.info.p + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      RC_CUDA(cudaMemset(c.w.info.p + 2, 0, sizeof(int)));
      throw Error(RCHFSI_ERR_TIMEOUT, "a bounded wait in the batched tensor-core kernel ran out");
    }
  }
}

// ------------------------------------------------------------------ Rayleigh-Ritz (FP64)
[[maybe_unused]] static void syevd(rchfsi_ctx& c, int n, double* A, double* w) {
  if (!c.solver) {
    RC_CHECK(cusolverDnCreate(&c.solver) == CUSOLVER_STATUS_SUCCESS, RCHFSI_ERR_CUDA, "cusolverDnCreate failed");
  }
  RC_CHECK(cusolverDnSetStream(c.solver, c.s) == CUSOLVER_STATUS_SUCCESS, RCHFSI_ERR_CUDA, "cusolverDnSetStream");
  int lwork = 0;
  RC_CHECK(cusolverDnDsyevd_bufferSize(c.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w,
                                       &lwork) == CUSOLVER_STATUS_SUCCESS,
           RCHFSI_ERR_CUDA, "syevd buffer query failed");
  double* work = c.w.syev_work.ensure((size_t)std::max(lwork, 1));
  RC_CHECK(cusolverDnDsyevd(c.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w, work, lwork,
                            c.w.info.p + 1) == CUSOLVER_STATUS_SUCCESS,
           RCHFSI_ERR_CUDA, "syevd failed");
}

int rayleigh_ritz(rchfsi_ctx& c, double* Y, double* X, double* AX, double* BX, double* evals) {
  const int64_t m = c.p.m;
  const int N = c.p.block;
  Work& w = c.w;
  // column scaling to unit 2-norm (span unchanged)
  {
    prof::Scope ps(c.s, RCHFSI_KERNEL_RR_AUX, 2.0 * m * N, 8.0 * m * N);
    col_norms_f64(c.s, m, N, Y, m, w.nrm.p);
  }
  // invert norms on device: reuse scale kernel through a tiny copy
  {
    std::vector<double> hn(N);
    RC_CUDA(cudaMemcpyAsync(hn.data(), w.nrm.p, N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
    for (int j = 0; j < N; ++j) {
      RC_CHECK(std::isfinite(hn[j]), RCHFSI_ERR_NUMERIC, "non-finite column in the filtered block");
      RC_CHECK(hn[j] > 0.0, RCHFSI_ERR_ILL_CONDITIONED, "zero column in the filtered block");
      hn[j] = 1.0 / hn[j];
    }
    RC_CUDA(cudaMemcpyAsync(w.nrm.p, hn.data(), N * sizeof(double), cudaMemcpyHostToDevice, c.s));
    prof::Scope ps(c.s, RCHFSI_KERNEL_RR_AUX, (double)m * N, 16.0 * m * N);
    scale_cols_f64(c.s, m, N, Y, m, w.nrm.p);
    RC_CUDA(cudaStreamSynchronize(c.s));
  }
  double* AY = w.AY.p;
  double* BY = w.BY.p;
  const bool emu = c.p.rr_mode == RCHFSI_RR_FP64_EMULATED;
  int* eflag = w.info.p + 2;
  // A complex problem's block is Y = [Y1, J Y1] (J = multiplication by i) and A, B commute with J:
  // the operator products are formed on the first Nc columns and completed by J, which halves the
  // FP64 operator work.
  const int Na = c.cplx ? c.Nc : N;
  auto jcomplete = [&](double* Z) {
    if (c.cplx) cplx_rebuild(c.s, c.mc, c.Nc, Z, nullptr, Z);
  };
  // A Y, B Y and the Gram matrices G_A = Y^T A Y, G_B = Y^T B Y of the current Y
  auto grams = [&]() {
    if (emu) {
      // FP64-accurate products from BF16 slices: Y as N logical rows of length m
      oz_slice(c.s, Na, m, Y, m, 1, w.ozL);
      if (c.op_kind == RCHFSI_OP_DENSE) {
        DenseOp& d = c.dense;
        if (d.ozA.R != m) oz_slice(c.s, m, m, d.A.p, m, 1, d.ozA);
        oz_gemm(c.s, c.num_sms, d.ozA, w.ozL, AY, m, w.ozws, eflag);
        jcomplete(AY);
        if (d.has_B) {
          if (d.ozB.R != m) oz_slice(c.s, m, m, d.B.p, m, 1, d.ozB);
          oz_gemm(c.s, c.num_sms, d.ozB, w.ozL, BY, m, w.ozws, eflag);
          jcomplete(BY);
        } else {
          RC_CUDA(cudaMemcpyAsync(BY, Y, sizeof(double) * m * N, cudaMemcpyDeviceToDevice, c.s));
        }
      } else {
        apply_AB_f64(c, Y, AY, BY, Na);
        jcomplete(AY);
        jcomplete(BY);
      }
      if (Na != N) oz_slice(c.s, N, m, Y, m, 1, w.ozL);  // every column for the Gram matrices
      // G_A = Y^T A Y, G_B = Y^T B Y (complex: the left N x Na half; the rest follows from J)
      // (real problems: both are symmetric, only the tiles reaching the upper triangle are formed)
      oz_slice(c.s, Na, m, AY, m, 1, w.ozR);
      oz_gemm(c.s, c.num_sms, w.ozL, w.ozR, w.GA.p, N, w.ozws, eflag, Na == N);
      oz_slice(c.s, Na, m, BY, m, 1, w.ozR);
      oz_gemm(c.s, c.num_sms, w.ozL, w.ozR, w.GB.p, N, w.ozws, eflag, Na == N);
    } else {
      apply_AB_f64(c, Y, AY, BY, Na);
      jcomplete(AY);
      jcomplete(BY);
      // G_A = Y^T A Y, G_B = Y^T B Y  (N x Na, column-major)
      gemm_f64(c.s, N, Na, m, Y, m, true, AY, m, true, epi_store(w.GA.p, N));
      gemm_f64(c.s, N, Na, m, Y, m, true, BY, m, true, epi_store(w.GB.p, N));
    }
    if (c.cplx) {
      cplx_gram_complete(c.s, c.Nc, w.GA.p);
      cplx_gram_complete(c.s, c.Nc, w.GB.p);
    }
  };
  // G_B = L L^T and L^-1 (one cluster / cooperative kernel); G_B is kept in Zt for a retry
  auto factor = [&]() {
    prof::Scope ps(c.s, RCHFSI_KERNEL_SMALL_DENSE, 2.0 * N * N * N / 3.0, 8.0 * N * N * 3);
    symmetrize_f64(c.s, N, w.GA.p, N);
    symmetrize_f64(c.s, N, w.GB.p, N);
    RC_CUDA(cudaMemcpyAsync(w.Zt.p, w.GB.p, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.s));
    cholesky_inverse_f64(c.s, N, w.GB.p, w.Lb.p, w.Li.p, w.info.p, c.num_sms, w.eigws);
    int inf = 0;
    RC_CUDA(cudaMemcpyAsync(&inf, w.info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
    return inf;
  };
  grams();
  int info = factor();
  c.rr_retries = 0;
  if (info != 0 && !c.cplx) {
    // The basis is numerically rank deficient for the Cholesky factorisation of its Gram matrix
    // (Section 2.1 Rayleigh-Ritz of a non-orthogonal basis): precondition it by one shifted
    // Cholesky QR step in the B inner product, Y <- Y L_s^-T with L_s L_s^T = G_B + s I and
    // s = 11 (m N + N (N + 1)) u tr(G_B) (the shift of Fukaya et al.'s shifted CholeskyQR, with the
    // trace bounding ||B^1/2 Y||_2^2), then form the products and Gram matrices of the new basis
    // again; the Cholesky factorisation of that Gram matrix is the second CholeskyQR pass.
    const double u = std::ldexp(1.0, -53);
    shift_diag_by_trace_f64(c.s, N, w.Zt.p, N, 11.0 * ((double)m * N + (double)N * (N + 1)) * u);
    cholesky_inverse_f64(c.s, N, w.Zt.p, w.Lb.p, w.Li.p, w.info.p, c.num_sms, w.eigws);
    RC_CUDA(cudaMemcpyAsync(&info, w.info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
    if (info != 0) return RCHFSI_ERR_ILL_CONDITIONED;
    // Y <- Y L_s^-T (column-major m x N times the transpose of the lower-triangular inverse)
    gemm_f64(c.s, m, N, N, Y, m, false, w.Li.p, N, false, epi_store(w.T1.p, m));
    RC_CUDA(cudaMemcpyAsync(Y, w.T1.p, sizeof(double) * m * N, cudaMemcpyDeviceToDevice, c.s));
    grams();
    info = factor();
    c.rr_retries = 1;
  }
  if (info != 0) return RCHFSI_ERR_ILL_CONDITIONED;
  // M = L^-1 G_A L^-T: two FP64-accurate products (BF16 slices on the tensor cores, the Gram
  // slices no longer needed) or two FP64 GEMMs on all SMs
  if (emu) {
    oz_slice(c.s, N, N, w.Li.p, 1, N, w.ozR);   // L^-1, row i = L^-1(i, :)
    oz_slice(c.s, N, N, w.GA.p, N, 1, w.ozE);   // column j of G_A as row j
    oz_gemm(c.s, c.num_sms, w.ozR, w.ozE, w.Zt.p, N, w.ozws, eflag);
    oz_slice(c.s, N, N, w.Zt.p, 1, N, w.ozE);   // L^-1 G_A by rows
    oz_gemm(c.s, c.num_sms, w.ozE, w.ozR, w.Z.p, N, w.ozws, eflag);
  } else {
    EpiArgs e1 = epi_store(w.Zt.p, N), e2 = epi_store(w.Z.p, N);
    e1.prof_cls = e2.prof_cls = RCHFSI_KERNEL_SMALL_DENSE;
    gemm_f64(c.s, N, N, N, w.Li.p, N, false, w.GA.p, N, true, e1);
    gemm_f64(c.s, N, N, N, w.Zt.p, N, false, w.Li.p, N, false, e2);
  }
  {
    prof::Scope ps(c.s, RCHFSI_KERNEL_SMALL_DENSE, 0.0, 8.0 * N * N * 2);
    symmetrize_f64(c.s, N, w.Z.p, N);
  }
  // eigenpairs of the projected matrix M (in Z, destroyed); eigenvectors land in `vec`
  double* vec = w.Z.p;
  {
    prof::Scope ps(c.s, RCHFSI_KERNEL_EIG, 4.0 * N * N * N, 8.0 * N * N * 2);
    if (c.p.eig_mode == RCHFSI_EIG_JACOBI) {
      jacobi_eig_f64(c.s, N, w.Z.p, w.Zt.p, evals, w.syev_work, 1e-14, 60);
      vec = w.Zt.p;
    } else if (c.p.eig_mode == RCHFSI_EIG_TRIDIAG) {
      // keep a copy of M for the library fallback (a cluster of close eigenvalues too large)
      RC_CUDA(cudaMemcpyAsync(w.Lb.p, w.Z.p, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.s));
      const OzScratch oz{&w.ozR, &w.ozE, &w.ozws, eflag, c.num_sms};
      if (sym_eig_f64(c.s, N, w.Z.p, w.Zt.p, evals, w.eigws, w.info.p + 3, c.num_sms, emu ? &oz : nullptr)) {
        vec = w.Zt.p;
      } else {
        RC_CUDA(cudaMemcpyAsync(w.Z.p, w.Lb.p, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.s));
        syevd(c, N, w.Z.p, evals);
      }
    } else {
      syevd(c, N, w.Z.p, evals);
    }
  }
  // E = L^-T V
  double* Ep = vec == w.Z.p ? w.Zt.p : w.Z.p;
  if (emu) {
    oz_slice(c.s, N, N, w.Li.p, N, 1, w.ozR);  // L^-T, row i = column i of L^-1
    oz_slice(c.s, N, N, vec, N, 1, w.ozE);     // column j of V as row j
    oz_gemm(c.s, c.num_sms, w.ozR, w.ozE, Ep, N, w.ozws, eflag);
  } else {
    EpiArgs e3 = epi_store(Ep, N);
    e3.prof_cls = RCHFSI_KERNEL_SMALL_DENSE;
    gemm_f64(c.s, N, N, N, w.Li.p, N, true, vec, N, true, e3);
  }
  // X = Y E, AX = AY E, BX = BY E.  Complex problems: each complex Ritz pair appears twice; when
  // every cluster of equal Ritz values is a pair, the first member of each is kept and only those
  // Nc columns are rotated, then completed by J ([X_s, J X_s]); otherwise all columns are rotated
  // and the caller selects (with complex Gram-Schmidt inside larger clusters).
  int ncol = N;
  const double* Erot = Ep;
  c.rr_paired = false;
  if (c.cplx) {
    std::vector<double> ev(N);
    RC_CUDA(cudaMemcpyAsync(ev.data(), evals, N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
    double scale = 1e-300;
    for (double v : ev) scale = std::max(scale, std::fabs(v));
    const double thr = 1e-9 * scale;
    std::vector<int> sel;
    bool pairs = true;
    for (int k = 0; k < N && pairs;) {
      int e = k + 1;
      while (e < N && std::fabs(ev[e] - ev[k]) <= thr) ++e;
      if (e - k == 2) sel.push_back(k);
      else pairs = false;
      k = e;
    }
    if (pairs && (int)sel.size() == c.Nc) {
      int* dcols = c.ccols.ensure(c.Nc);
      RC_CUDA(cudaMemcpyAsync(dcols, sel.data(), sizeof(int) * c.Nc, cudaMemcpyHostToDevice, c.s));
      double* Es = (Ep == w.Z.p) ? w.Zt.p : w.Z.p;  // the eigenvectors V are no longer needed
      gather_cols_f64(c.s, N, c.Nc, Ep, dcols, Es);
      std::vector<double> e2(N);
      for (int j = 0; j < c.Nc; ++j) e2[j] = e2[c.Nc + j] = ev[sel[j]];
      RC_CUDA(cudaMemcpyAsync(evals, e2.data(), N * sizeof(double), cudaMemcpyHostToDevice, c.s));
      RC_CUDA(cudaStreamSynchronize(c.s));  // sel and e2 must outlive their copies
      ncol = c.Nc;
      Erot = Es;
      c.rr_paired = true;
    }
  }
  // FE operators: A X and B X are applied directly (a cell product costs 2 n_c^2 C per column,
  // below the 2 m N of rotating A Y and B Y, and gives the residual of X itself); dense operators
  // rotate A Y and B Y (2 m N per column against 2 m^2)
  bool direct = false;
  if (c.op_kind == RCHFSI_OP_FE_CELL) {
    // per column: a (complex: four) cell product(s), 2 n_c^2 C each, against the rotation's 2 m N
    const double cell = (double)c.fe->nc * c.fe->nc * (double)c.fe->n_cells * (c.fe->cplx ? 4.0 : 1.0);
    direct = cell < (double)m * N;
  }
  if (emu) {
    // E^T as ncol logical rows (row j = column j of E, contiguous); blocks as m logical rows (dofs)
    oz_slice(c.s, ncol, N, Erot, N, 1, w.ozE);
    oz_slice(c.s, m, N, Y, 1, m, w.ozL);
    oz_gemm(c.s, c.num_sms, w.ozL, w.ozE, X, m, w.ozws, eflag);
    if (!direct) {
      oz_slice(c.s, m, N, AY, 1, m, w.ozL);
      oz_gemm(c.s, c.num_sms, w.ozL, w.ozE, AX, m, w.ozws, eflag);
      oz_slice(c.s, m, N, BY, 1, m, w.ozL);
      oz_gemm(c.s, c.num_sms, w.ozL, w.ozE, BX, m, w.ozws, eflag);
    }
    int flag = 0;
    RC_CUDA(cudaMemcpyAsync(&flag, eflag, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
    if (flag) {
      RC_CUDA(cudaMemsetAsync(eflag, 0, sizeof(int), c.s));
      throw Error(RCHFSI_ERR_TIMEOUT, "a bounded wait in the emulated FP64 GEMM ran out");
    }
  } else {
    gemm_f64(c.s, m, ncol, N, Y, m, false, Erot, N, true, epi_store(X, m));
    if (!direct) {
      gemm_f64(c.s, m, ncol, N, AY, m, false, Erot, N, true, epi_store(AX, m));
      gemm_f64(c.s, m, ncol, N, BY, m, false, Erot, N, true, epi_store(BX, m));
    }
  }
  if (c.rr_paired) jcomplete(X);
  if (direct) {
    apply_AB_f64(c, X, AX, BX, ncol);
    if (c.rr_paired) {
      jcomplete(AX);
      jcomplete(BX);
    }
  } else if (c.rr_paired) {
    jcomplete(AX);
    jcomplete(BX);
  }
  RC_CUDA(cudaMemcpyAsync(&info, w.info.p + 1, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  if (info != 0) return RCHFSI_ERR_NUMERIC;
  return RCHFSI_OK;
}

// ------------------------------------------------------------------ Lanczos
// Eigenvalues of the symmetric tridiagonal T (alpha, beta) by Sturm-sequence bisection.
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    q = (a[i] - x) - (i ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) ++cnt;
  }
  return cnt;
}

static double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int idx) {
  double lo = 1e300, hi = -1e300;
  const size_t k = a.size();
  for (size_t i = 0; i < k; ++i) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(a, b, mid) > idx) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

namespace {
__global__ void lz_scale_kernel(int64_t n, const double* x, const double* d, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = d ? x[i] * sqrt(d[i]) : x[i];
}
// w <- w - alpha v - beta_prev vp   (beta_prev given as its square; null on the first step)
__global__ void lz_update_kernel(int64_t n, double* w, const double* v, const double* vp, const double* alpha,
                                 const double* beta_prev_sq) {
  const double a = *alpha, b = beta_prev_sq ? sqrt(*beta_prev_sq) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    w[i] = w[i] - a * v[i] - b * vp[i];
}
// vp <- v, v <- w / sqrt(beta_sq)
__global__ void lz_next_kernel(int64_t n, double* vp, double* v, const double* w, const double* beta_sq) {
  const double b = sqrt(*beta_sq);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    vp[i] = v[i];
    v[i] = w[i] / b;
  }
}
}  // namespace

// k Lanczos steps on S = D^1/2 A D^1/2 (dinv = diagonal of the approximate inverse D^-1, or null for
// S = A).  Returns alpha[0..k) and beta[0..k) (beta_j = ||w_j||).
static void lanczos_run(rchfsi_ctx& c, const double* v0, int k, const double* dinv, std::vector<double>& al,
                        std::vector<double>& be) {
  const int64_t m = c.p.m;
  Work& w = c.w;
  double* v = w.lz_v.ensure(m);
  double* wv = w.lz_w.ensure(m);
  double* vp = w.lz_vp.ensure(m);
  double* t = w.lz_t.ensure(m);
  double* ab = w.lz_ab.ensure(2 * (size_t)k + 2);  // alpha[0..k), beta^2[0..k), ||v0||^2
  const unsigned nb = std::min<unsigned>(cdiv(m, 256), 1024);
  dot_f64(c.s, m, v0, v0, ab + 2 * k);
  RC_CUDA(cudaMemcpyAsync(wv, v0, m * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  lz_next_kernel<<<nb, 256, 0, c.s>>>(m, vp, v, wv, ab + 2 * k);  // v = v0 / ||v0||
  RC_LAUNCH();
  RC_CUDA(cudaMemsetAsync(vp, 0, m * sizeof(double), c.s));
  for (int j = 0; j < k; ++j) {
    lz_scale_kernel<<<nb, 256, 0, c.s>>>(m, v, dinv, t);
    RC_LAUNCH();
    apply_A_f64(c, t, wv, 1);
    lz_scale_kernel<<<nb, 256, 0, c.s>>>(m, wv, dinv, wv);
    RC_LAUNCH();
    dot_f64(c.s, m, v, wv, ab + j);
    lz_update_kernel<<<nb, 256, 0, c.s>>>(m, wv, v, vp, ab + j, j ? ab + k + j - 1 : nullptr);
    RC_LAUNCH();
    dot_f64(c.s, m, wv, wv, ab + k + j);
    lz_next_kernel<<<nb, 256, 0, c.s>>>(m, vp, v, wv, ab + k + j);
    RC_LAUNCH();
  }
  std::vector<double> h(2 * (size_t)k);
  RC_CUDA(cudaMemcpyAsync(h.data(), ab, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  al.assign(h.begin(), h.begin() + k);
  be.resize(k);
  for (int j = 0; j < k; ++j) be[j] = std::sqrt(h[k + j]);
}

void lanczos(rchfsi_ctx& c, const double* v0, int k, double* lmax, double* normA) {
  RC_CHECK(k >= 2 && k <= c.p.m, RCHFSI_ERR_INVALID_ARG, "lanczos_steps must be in [2, m]");
  std::vector<double> al, be;
  if (lmax) {
    lanczos_run(c, v0, k, dinv_diag(c), al, be);
    *lmax = tridiag_eig(al, be, k - 1) + be[k - 1];
  }
  if (normA) {
    lanczos_run(c, v0, k, nullptr, al, be);
    *normA = std::max(std::fabs(tridiag_eig(al, be, 0)), std::fabs(tridiag_eig(al, be, k - 1)));
  }
}

}  // namespace rchfsi
