// extern "C" entry points (include/rchfsi.h): argument checks, host/device staging and the
// outer loop of Algorithm 1.  Every C++ exception is turned into a status code here.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <set>
#include <thread>
#include <tuple>

#include "solver.cuh"

using namespace rchfsi;

namespace rchfsi {
void resid_form_f64(cudaStream_t s, int64_t m, int64_t n, const double* AX, const double* BX, const double* lam,
                    double* W);
}

namespace rchfsi {
namespace prof {
Profiler*& current() {
  static thread_local Profiler* p = nullptr;
  return p;
}
}  // namespace prof
int64_t& launch_counter() {
  static int64_t n = 0;
  return n;
}

void set_smem_limit(const void* kernel, int bytes) {
  int dev = 0;
  RC_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> done;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(kernel, dev, bytes);
  if (done.count(key)) return;
  RC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert(key);
}
}  // namespace rchfsi

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace rchfsi {
// Message returned by rchfsi_last_error(NULL, ...) on this thread.
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace rchfsi

namespace {

struct ProfBind {
  prof::Profiler* prev;
  explicit ProfBind(rchfsi_ctx* h) : prev(prof::current()) { prof::current() = h ? &h->prof : nullptr; }
  ~ProfBind() { prof::current() = prev; }
};

template <class F>
int guarded(rchfsi_ctx* h, F&& f) {
  ProfBind pb(h);
  try {
    return f();
  } catch (const Error& e) {
    if (h) h->err = e.what();
    g_last_error = e.what();
    if (h && h->s) {
      cudaStreamSynchronize(h->s);
      cudaGetLastError();
    }
    return e.code;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    g_last_error = e.what();
    return RCHFSI_ERR_CUDA;
  }
}

void validate_params(const rchfsi_params* p) {
  RC_CHECK(p, RCHFSI_ERR_INVALID_ARG, "params is NULL");
  RC_CHECK(p->m > 0, RCHFSI_ERR_INVALID_ARG, "m must be positive");
  RC_CHECK(p->block >= 1 && p->block <= p->m, RCHFSI_ERR_INVALID_ARG, "block must be in [1, m]");
  RC_CHECK(p->nev >= 1 && p->nev <= p->block, RCHFSI_ERR_INVALID_ARG, "nev must be in [1, block]");
  RC_CHECK(p->degree >= 1 && p->degree <= 4096, RCHFSI_ERR_INVALID_ARG, "degree must be in [1, 4096]");
  RC_CHECK(p->precision >= RCHFSI_FP64 && p->precision <= RCHFSI_BF16, RCHFSI_ERR_INVALID_ARG, "bad precision");
  RC_CHECK(p->method == RCHFSI_METHOD_RCHFSI || p->method == RCHFSI_METHOD_CHFSI, RCHFSI_ERR_INVALID_ARG,
           "bad method");
  RC_CHECK(p->field == RCHFSI_REAL || p->field == RCHFSI_COMPLEX, RCHFSI_ERR_INVALID_ARG, "bad field");
  RC_CHECK(p->max_iter >= 0 && p->min_iter >= 0, RCHFSI_ERR_INVALID_ARG, "iteration counts must be >= 0");
  RC_CHECK(p->lanczos_steps >= 2 && p->lanczos_steps <= p->m, RCHFSI_ERR_INVALID_ARG,
           "lanczos_steps must be in [2, m]");
  RC_CHECK(p->tol >= 0.0, RCHFSI_ERR_INVALID_ARG, "tol must be >= 0");
  RC_CHECK(p->block * (p->field == RCHFSI_COMPLEX ? 2 : 1) <= 6144, RCHFSI_ERR_UNSUPPORTED,
           "block larger than 6144 (3072 for complex problems)");
  RC_CHECK(p->rr_mode == RCHFSI_RR_FP64 || p->rr_mode == RCHFSI_RR_FP64_EMULATED, RCHFSI_ERR_INVALID_ARG,
           "bad rr_mode");
  RC_CHECK(p->eig_mode >= RCHFSI_EIG_SYEVD && p->eig_mode <= RCHFSI_EIG_TRIDIAG, RCHFSI_ERR_INVALID_ARG,
           "bad eig_mode");
}

void need_op(rchfsi_ctx* h) {
  RC_CHECK(h, RCHFSI_ERR_INVALID_ARG, "handle is NULL");
  RC_CHECK(h->has_op, RCHFSI_ERR_NO_OPERATOR, "rchfsi_set_operator has not been called");
}

// Copy n doubles (host or device) to a device buffer.
void to_device(rchfsi_ctx& c, const double* src, double* dst, size_t n) {
  RC_CHECK(src, RCHFSI_ERR_INVALID_ARG, "NULL input array");
  const auto kind = is_device_pointer(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  RC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, c.s));
}

void from_device(rchfsi_ctx& c, const double* src, double* dst, size_t n) {
  if (!dst) return;
  const auto kind = is_device_pointer(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  RC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, c.s));
}

// Row-major m x N caller block -> column-major device block.
void load_block(rchfsi_ctx& c, const double* src, double* dst_col) {
  RC_CHECK(src, RCHFSI_ERR_INVALID_ARG, "NULL block argument");
  const int64_t m = c.p.m;
  const int N = c.p.block;
  const double* d = src;
  if (!is_device_pointer(src)) {
    double* st = c.w.stage_in.ensure((size_t)m * N);
    RC_CUDA(cudaMemcpyAsync(st, src, sizeof(double) * m * N, cudaMemcpyHostToDevice, c.s));
    d = st;
  }
  transpose_f64(c.s, m, N, d, N, dst_col, m);
}

// Column-major device block -> row-major m x N caller block.
void store_block(rchfsi_ctx& c, const double* src_col, double* dst) {
  if (!dst) return;
  const int64_t m = c.p.m;
  const int N = c.p.block;
  if (is_device_pointer(dst)) {
    transpose_f64(c.s, N, m, src_col, m, dst, N);
  } else {
    double* st = c.w.stage_out.ensure((size_t)m * N);
    transpose_f64(c.s, N, m, src_col, m, st, N);
    RC_CUDA(cudaMemcpyAsync(dst, st, sizeof(double) * m * N, cudaMemcpyDeviceToHost, c.s));
  }
}

std::vector<double> host_vec(rchfsi_ctx& c, const double* src, size_t n) {
  RC_CHECK(src, RCHFSI_ERR_INVALID_ARG, "NULL vector argument");
  std::vector<double> v(n);
  const auto kind = is_device_pointer(src) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  RC_CUDA(cudaMemcpyAsync(v.data(), src, n * sizeof(double), kind, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  return v;
}

// ------------------------------------------------------------------ complex problems (real embedding)
// Caller block (real m x N row-major, or complex m x N interleaved) -> internal column-major block.
void load_any(rchfsi_ctx& c, const double* src, double* dst_col) {
  if (!c.cplx) {
    load_block(c, src, dst_col);
    return;
  }
  RC_CHECK(src, RCHFSI_ERR_INVALID_ARG, "NULL block argument");
  const size_t n = 2 * (size_t)c.mc * c.Nc;
  double* st = c.cstage.ensure(n);
  const auto kind = is_device_pointer(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  RC_CUDA(cudaMemcpyAsync(st, src, n * sizeof(double), kind, c.s));
  cplx_embed_block(c.s, c.mc, c.Nc, st, dst_col);
}

// Eigenvalue-like vectors: N caller values -> the internal block's (duplicated for complex).
std::vector<double> lam_any(rchfsi_ctx& c, const double* Lambda) {
  if (!c.cplx) return host_vec(c, Lambda, c.p.block);
  std::vector<double> v = host_vec(c, Lambda, c.Nc);
  v.insert(v.end(), v.begin(), v.end());
  return v;
}

// Internal column-major block -> caller block; for complex problems the embedded columns `cols`
// become the caller's complex columns (default: the first Nc, the embedding of the input block).
void store_any(rchfsi_ctx& c, const double* src_col, double* dst, const std::vector<int>* cols = nullptr) {
  if (!dst) return;
  if (!c.cplx) {
    store_block(c, src_col, dst);
    return;
  }
  std::vector<int> idx(c.Nc);
  for (int j = 0; j < c.Nc; ++j) idx[j] = cols ? (*cols)[j] : j;
  int* dcols = c.ccols.ensure(c.Nc);
  RC_CUDA(cudaMemcpyAsync(dcols, idx.data(), sizeof(int) * c.Nc, cudaMemcpyHostToDevice, c.s));
  const size_t n = 2 * (size_t)c.mc * c.Nc;
  if (is_device_pointer(dst)) {
    cplx_extract_cols(c.s, c.mc, c.Nc, src_col, dcols, dst);
  } else {
    double* st = c.cstage.ensure(n);
    cplx_extract_cols(c.s, c.mc, c.Nc, src_col, dcols, st);
    RC_CUDA(cudaMemcpyAsync(dst, st, n * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  }
  RC_CUDA(cudaStreamSynchronize(c.s));  // idx must outlive the copy
}

// Choose, among the 2N embedded Ritz vectors (ascending eigenvalues ev), N that represent distinct
// complex eigenvectors.  Each complex eigenpair appears as two real ones with equal eigenvalues,
// spanning {x, i x}; for an isolated pair the first member is taken.  A cluster of more than two
// equal eigenvalues (a complex eigenvalue of multiplicity > 1) is orthonormalised in the complex
// B inner product (Gram-Schmidt on the device, using B X), dropping members that depend on the ones
// already kept.  X, AX and BX (column-major, 2m rows; AX may be null) receive the same column
// operations, so they stay consistent.
std::vector<int> select_complex(rchfsi_ctx& c, const std::vector<double>& ev, double* X, double* AX, double* BX) {
  const int n2 = (int)ev.size();
  double scale = 1e-300;
  for (double v : ev) scale = std::max(scale, std::fabs(v));
  const double thr = 1e-9 * scale;
  std::vector<int> out;
  double* d = c.cdot.ensure(2);
  int k = 0;
  while (k < n2 && (int)out.size() < c.Nc) {
    int e = k + 1;
    while (e < n2 && std::fabs(ev[e] - ev[k]) <= thr) ++e;
    const int size = e - k;
    if (size <= 2) {
      out.push_back(k);
    } else {
      std::vector<int> kept;
      for (int j = k; j < e && (int)kept.size() < size / 2; ++j) {
        for (int l : kept) {
          double h[2];
          cplx_dot(c.s, c.mc, X, BX, l, j, d);
          RC_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c.s));
          RC_CUDA(cudaStreamSynchronize(c.s));
          cplx_axpy(c.s, c.mc, X, AX, BX, l, j, h[0], h[1], 1.0);
        }
        double h[2];
        cplx_dot(c.s, c.mc, X, BX, j, j, d);
        RC_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c.s));
        RC_CUDA(cudaStreamSynchronize(c.s));
        if (h[0] > 0.25) {
          cplx_axpy(c.s, c.mc, X, AX, BX, j, j, 0.0, 0.0, 1.0 / std::sqrt(h[0]));
          kept.push_back(j);
        }
      }
      for (int j : kept)
        if ((int)out.size() < c.Nc) out.push_back(j);
    }
    k = e;
  }
  RC_CHECK((int)out.size() == c.Nc, RCHFSI_ERR_NUMERIC, "complex eigenpairs could not be paired");
  return out;
}

// After a Rayleigh-Ritz step of a complex problem: keep one real representative of each complex
// Ritz pair and rebuild X, AX, BX as [X_s, J X_s] (J = multiplication by i), so that the first N
// columns carry the complex block and the filter needs to run on them only.  ev (2N ascending
// values) becomes [ev_s, ev_s], also on the device.
void pair_complex(rchfsi_ctx& c, std::vector<double>& ev) {
  Work& w = c.w;
  const std::vector<int> sel = select_complex(c, ev, w.X.p, w.AX.p, w.BX.p);
  int* dcols = c.ccols.ensure(c.Nc);
  RC_CUDA(cudaMemcpyAsync(dcols, sel.data(), sizeof(int) * c.Nc, cudaMemcpyHostToDevice, c.s));
  const size_t blk = (size_t)c.p.m * c.p.block;
  for (double* b : {w.X.p, w.AX.p, w.BX.p}) {
    cplx_rebuild(c.s, c.mc, c.Nc, b, dcols, w.T1.p);
    RC_CUDA(cudaMemcpyAsync(b, w.T1.p, blk * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  }
  std::vector<double> e2(2 * c.Nc);
  for (int j = 0; j < c.Nc; ++j) e2[j] = e2[c.Nc + j] = ev[sel[j]];
  ev = e2;
  RC_CUDA(cudaMemcpyAsync(w.evals.p, ev.data(), ev.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));  // sel and ev must outlive the copies
}

// Filter of the caller-facing block.  A complex block's embedding [[Xr, -Xi], [Xi, Xr]] is closed
// under J, and the embedded A, B, D^-1 commute with J, so only its first N columns are filtered;
// `complete` fills the other N with J times them.
void filter_any(rchfsi_ctx& c, const double* X, const double* lam, const double* W, double lmin, double lT,
                double lmax, int p, double* Y, bool chfsi, bool complete) {
  if (!c.cplx) {
    filter_internal(c, X, lam, W, lmin, lT, lmax, p, Y, chfsi);
    return;
  }
  const int saved = c.p.block;
  c.p.block = c.Nc;
  try {
    filter_internal(c, X, lam, W, lmin, lT, lmax, p, Y, chfsi);
  } catch (...) {
    c.p.block = saved;
    throw;
  }
  c.p.block = saved;
  if (complete) cplx_rebuild(c.s, c.mc, c.Nc, Y, nullptr, Y);
}

void set_dense(rchfsi_ctx& c, const rchfsi_operator* op) {
  const int64_t m = c.p.m;
  const size_t mm = (size_t)m * m;
  DenseOp& d = c.dense;
  RC_CHECK(op->A, RCHFSI_ERR_INVALID_ARG, "dense operator needs A");
  RC_CHECK(!(op->Dinv && op->Dinv_dense), RCHFSI_ERR_INVALID_ARG, "give Dinv or Dinv_dense, not both");
  d.AD32.release(); d.DA32.release(); d.ADtf.release(); d.DAtf.release(); d.AD16.release(); d.DA16.release();
  d.ozA.R = 0;  // slices of the previous operator are stale
  d.ozB.R = 0;
  to_device(c, op->A, d.A.ensure(mm), mm);
  d.has_B = op->B != nullptr;
  if (d.has_B) to_device(c, op->B, d.B.ensure(mm), mm);
  else d.B.release();
  d.has_dinv = op->Dinv != nullptr;
  d.has_dinv_dense = op->Dinv_dense != nullptr;
  if (d.has_dinv) to_device(c, op->Dinv, d.Dinv.ensure(m), m);
  else d.Dinv.release();
  if (d.has_dinv_dense) to_device(c, op->Dinv_dense, d.Dinv_dense.ensure(mm), mm);
  else d.Dinv_dense.release();
  // F = the matrix used inside the filter
  const double* F = d.A.p;
  DevBuf<double> fbuf;
  if (op->A_filter) {
    to_device(c, op->A_filter, fbuf.ensure(mm), mm);
    F = fbuf.p;
  }
  double* AD = d.AD64.ensure(mm);
  double* DA = d.DA64.ensure(mm);
  if (d.has_dinv) {
    scale_rows_f64(c.s, m, m, F, AD, d.Dinv.p, true);   // A~ D^-1: column scaling
    scale_rows_f64(c.s, m, m, F, DA, d.Dinv.p, false);  // D^-1 A~: row scaling
  } else if (d.has_dinv_dense) {
    DevBuf<double> tmp;
    tmp.ensure(mm);
    EpiArgs e;
    e.kind = EPI_STORE;
    e.C = tmp.p;
    e.ldc = m;
    gemm_f64(c.s, m, m, m, F, m, true, d.Dinv_dense.p, m, false, e);  // col-major (F D)
    transpose_f64(c.s, m, m, tmp.p, m, AD, m);
    gemm_f64(c.s, m, m, m, d.Dinv_dense.p, m, true, F, m, false, e);  // col-major (D F)
    transpose_f64(c.s, m, m, tmp.p, m, DA, m);
    RC_CUDA(cudaStreamSynchronize(c.s));
  } else {
    RC_CUDA(cudaMemcpyAsync(AD, F, mm * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    RC_CUDA(cudaMemcpyAsync(DA, F, mm * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
  }
  RC_CUDA(cudaStreamSynchronize(c.s));
}

void set_fe(rchfsi_ctx& c, const rchfsi_operator* op) {
  RC_CHECK(op->n_cells > 0 && op->n_c > 0 && op->n_c <= 128, RCHFSI_ERR_INVALID_ARG,
           "FE operator needs n_cells > 0 and 0 < n_c <= 128");
  RC_CHECK(op->cell_dofs && op->A_cells && op->B_cells && op->Dinv, RCHFSI_ERR_INVALID_ARG,
           "FE operator needs cell_dofs, A_cells, B_cells and Dinv");
  RC_CHECK(!op->A_filter && !op->Dinv_dense, RCHFSI_ERR_UNSUPPORTED,
           "A_filter / Dinv_dense are for dense operators");
  // a new operator takes over the previous one's allocations: those set_fe rewrites, the per-product
  // scratch and the packed images (repacked from the new matrices on first use); the rest is freed
  std::unique_ptr<FeOp> old = std::move(c.fe);
  c.fe.reset(new FeOp());
  FeOp& f = *c.fe;
  if (old) {
    f.dofs.take(old->dofs);
    f.A64.take(old->A64);
    f.B64.take(old->B64);
    f.Dinv.take(old->Dinv);
    f.own_pos.take(old->own_pos);
    f.imgADtf.take(old->imgADtf);
    f.ozA.take(old->ozA);
    f.ozB.take(old->ozB);
    f.ozAe.take(old->ozAe);
    f.ozBe.take(old->ozBe);
    f.ozArow.take(old->ozArow);
    f.ozBrow.take(old->ozBrow);
    f.ozcexp.take(old->ozcexp);
    f.ozplanes.take(old->ozplanes);
    old.reset();
  }
  const int64_t mc = c.cplx ? c.mc : c.p.m;  // dofs of the (complex) problem
  f.m = c.p.m;
  f.n_cells = op->n_cells;
  f.nc = op->n_c;
  f.B_shared = op->B_cells_shared != 0;
  const size_t nd = (size_t)f.n_cells * f.nc;
  const size_t na = nd * f.nc;
  int* dofs = f.dofs.ensure(nd);
  const auto kind = is_device_pointer(op->cell_dofs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  RC_CUDA(cudaMemcpyAsync(dofs, op->cell_dofs, nd * sizeof(int), kind, c.s));
  // validate the connectivity on the host before any kernel indexes with it
  std::vector<int> hd(nd);
  RC_CUDA(cudaMemcpyAsync(hd.data(), dofs, nd * sizeof(int), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  for (size_t i = 0; i < nd; ++i)
    RC_CHECK(hd[i] >= 0 && hd[i] < mc, RCHFSI_ERR_INVALID_ARG, "cell_dofs entry out of [0, m)");
  // owner of each dof, balanced over the cells: dofs in increasing order, each to the cell that
  // contains it and owns the fewest dofs so far (the lowest cell index among equals); own_pos[c][k]
  // = position of node k among the dofs cell c owns (node order), -1 when not owned
  {
    const size_t C = (size_t)f.n_cells;
    std::vector<int> start((size_t)mc + 1, 0), cells(C * f.nc);
    for (size_t i = 0; i < C * f.nc; ++i) ++start[(size_t)hd[i] + 1];
    for (size_t d = 0; d < (size_t)mc; ++d) start[d + 1] += start[d];
    {
      std::vector<int> fill(start.begin(), start.end() - 1);
      for (size_t cl = 0; cl < C; ++cl)
        for (int k = 0; k < f.nc; ++k) cells[(size_t)fill[hd[cl * f.nc + k]]++] = (int)cl;
    }
    int mult = 1;
    for (size_t d = 0; d < (size_t)mc; ++d) mult = std::max(mult, start[d + 1] - start[d]);
    f.max_mult = mult;
    std::vector<int> cnt(C, 0), owner((size_t)mc, -1);
    for (size_t d = 0; d < (size_t)mc; ++d) {
      int best = -1;
      for (int e = start[d]; e < start[d + 1]; ++e) {
        const int cl = cells[(size_t)e];
        if (best < 0 || cnt[cl] < cnt[best] || (cnt[cl] == cnt[best] && cl < best)) best = cl;
      }
      if (best >= 0) {
        owner[d] = best;
        ++cnt[best];
      }
    }
    std::vector<int8_t> pos(C * 128, -1);
    int most = 0;
    for (size_t cl = 0; cl < C; ++cl) {
      int n = 0;
      for (int k = 0; k < f.nc; ++k) {
        const int d = hd[cl * f.nc + k];
        if (owner[d] == (int)cl) {
          owner[d] = -2;  // a dof listed twice in one cell is owned once
          pos[cl * 128 + k] = (int8_t)n++;
        }
      }
      most = std::max(most, n);
    }
    f.own_max = most;
    RC_CUDA(cudaMemcpyAsync(f.own_pos.ensure(pos.size()), pos.data(), pos.size(), cudaMemcpyHostToDevice, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
  }
  const size_t nb = f.B_shared ? (size_t)f.nc * f.nc : na;
  to_device(c, op->B_cells, f.B64.ensure(nb), nb);
  f.err = c.w.info.p + 2;
  if (!c.cplx) {
    to_device(c, op->A_cells, f.A64.ensure(na), na);
    to_device(c, op->Dinv, f.Dinv.ensure(c.p.m), c.p.m);
  } else {
    // complex cell matrices: real parts in this operator, imaginary parts in f.imag
    f.cplx = true;
    f.mc = mc;
    f.imag.reset(new FeOp());
    FeOp& g = *f.imag;
    g.m = c.p.m;
    g.mc = mc;
    g.n_cells = f.n_cells;
    g.nc = f.nc;
    g.err = f.err;
    DevBuf<double> tmp;
    to_device(c, op->A_cells, tmp.ensure(2 * na), 2 * na);
    cplx_deinterleave(c.s, na, tmp.p, f.A64.ensure(na), g.A64.ensure(na));
    RC_CUDA(cudaMemcpyAsync(g.dofs.ensure(nd), dofs, nd * sizeof(int), cudaMemcpyDeviceToDevice, c.s));
    RC_CUDA(cudaMemcpyAsync(g.own_pos.ensure(f.own_pos.n), f.own_pos.p, f.own_pos.bytes(), cudaMemcpyDeviceToDevice, c.s));
    g.own_max = f.own_max;
    g.max_mult = f.max_mult;
    // D^-1 of the embedding: [D^-1; D^-1]
    double* dv = f.Dinv.ensure(2 * mc);
    to_device(c, op->Dinv, dv, mc);
    RC_CUDA(cudaMemcpyAsync(dv + mc, dv, mc * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    RC_CUDA(cudaMemcpyAsync(g.Dinv.ensure(2 * mc), dv, 2 * mc * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    RC_CUDA(cudaStreamSynchronize(c.s));
  }
  RC_CUDA(cudaStreamSynchronize(c.s));
}

// Complex Hermitian dense operator: build the real embedding on the device and set it.
void set_dense_complex(rchfsi_ctx& c, const rchfsi_operator* op) {
  const int64_t mc = c.mc, m2 = 2 * mc;
  RC_CHECK(op->A, RCHFSI_ERR_INVALID_ARG, "dense operator needs A");
  RC_CHECK(!op->A_filter && !op->Dinv_dense, RCHFSI_ERR_UNSUPPORTED,
           "A_filter / Dinv_dense are not available for complex operators");
  DevBuf<double> ac, ae, bc, be, de;
  to_device(c, op->A, ac.ensure(2 * (size_t)mc * mc), 2 * (size_t)mc * mc);
  cplx_embed_dense(c.s, mc, ac.p, ae.ensure((size_t)m2 * m2));
  ac.release();
  rchfsi_operator e{};
  e.kind = RCHFSI_OP_DENSE;
  e.field = RCHFSI_REAL;
  e.m = m2;
  e.A = ae.p;
  if (op->B) {
    to_device(c, op->B, bc.ensure((size_t)mc * mc), (size_t)mc * mc);
    cplx_embed_blockdiag(c.s, mc, bc.p, be.ensure((size_t)m2 * m2));
    e.B = be.p;
  }
  if (op->Dinv) {
    double* dv = de.ensure(m2);
    to_device(c, op->Dinv, dv, mc);
    RC_CUDA(cudaMemcpyAsync(dv + mc, dv, mc * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    e.Dinv = dv;
  }
  RC_CUDA(cudaStreamSynchronize(c.s));
  set_dense(c, &e);
}

}  // namespace

namespace rchfsi {
// W = AX - BX diag(lam), column-major
namespace {
__global__ void resid_form_kernel(int64_t m, int64_t n, const double* AX, const double* BX, const double* lam,
                                  double* W) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int64_t j = e / m;
    W[e] = AX[e] - BX[e] * lam[j];
  }
}
}  // namespace
void resid_form_f64(cudaStream_t s, int64_t m, int64_t n, const double* AX, const double* BX, const double* lam,
                    double* W) {
  int64_t b = (m * n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  resid_form_kernel<<<(unsigned)std::max<int64_t>(b, 1), 256, 0, s>>>(m, n, AX, BX, lam, W);
  RC_LAUNCH();
}
}  // namespace rchfsi

namespace {

// State of one rchfsi_solve (Algorithm 1), split into phases so that several problems can be
// advanced together (rchfsi_solve_batch): begin (initial block, Lanczos bounds, first
// Rayleigh-Ritz), check (residuals, convergence test, filter bounds), filter, Rayleigh-Ritz, end.
struct SolveRun {
  rchfsi_ctx* h;
  double* X_inout;
  double* evals;
  double* resid;
  rchfsi_stats* st;
  double* hist;
  int N = 0, nev = 0, Nout = 0;
  double lmax = 0.0, normA = 1.0;
  std::vector<double> ev, ra, xn;
  int rc = RCHFSI_OK, it = 0, best_it = 0, retries = 0;
  double best = INFINITY, maxrel = INFINITY, maxabs = INFINITY;
  int64_t applies = 0;
  double flops = 0.0, t_filter = 0.0, t_rr = 0.0;
  double lmin = 0.0, lT = 0.0, lmx = 0.0;  // bounds of the next filter
  std::chrono::steady_clock::time_point t0;
  SolveRun(rchfsi_ctx* h_, double* X, double* e, double* r, rchfsi_stats* s)
      : h(h_), X_inout(X), evals(e), resid(r), st(s), hist(s ? s->history : nullptr) {}
};

double ms_since(std::chrono::steady_clock::time_point a) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
}

// After a Rayleigh-Ritz step of a complex problem: one Ritz vector per complex pair.
void pair_after_rr(SolveRun& r) {
  rchfsi_ctx& c = *r.h;
  if (r.rc != RCHFSI_OK || !c.cplx) return;
  RC_CUDA(cudaMemcpyAsync(r.ev.data(), c.w.evals.p, r.N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  if (!c.rr_paired) pair_complex(c, r.ev);
}

void run_begin(SolveRun& r) {
  rchfsi_ctx& c = *r.h;
  const rchfsi_params& p = c.p;
  RC_CHECK(r.X_inout, RCHFSI_ERR_INVALID_ARG, "X_inout is NULL");
  r.t0 = std::chrono::steady_clock::now();
  r.N = p.block;
  // complex problems: convergence and outputs over the first Nc columns (one per complex pair)
  r.nev = c.cplx ? c.nevc : p.nev;
  r.Nout = c.cplx ? c.Nc : r.N;
  r.ev.assign(r.N, 0.0);
  r.ra.assign(r.N, 0.0);
  r.xn.assign(r.N, 1.0);
  load_any(c, r.X_inout, c.w.Y.p);
  // bounds: Lanczos from the first column of the initial block (contiguous in column-major)
  r.lmax = p.lmax;
  lanczos(c, c.w.Y.p, p.lanczos_steps, p.fixed_bounds ? nullptr : &r.lmax, &r.normA);
  RC_CHECK(r.normA > 0.0 && std::isfinite(r.normA), RCHFSI_ERR_NUMERIC, "||A|| estimate is not positive");
  const auto tr = std::chrono::steady_clock::now();
  r.rc = rayleigh_ritz(c, c.w.Y.p, c.w.X.p, c.w.AX.p, c.w.BX.p, c.w.evals.p);
  r.retries += c.rr_retries;
  pair_after_rr(r);
  r.t_rr += ms_since(tr);
}

// Residuals and the convergence test; true when another filter + Rayleigh-Ritz pass is needed
// (the filter bounds are then in r.lmin, r.lT, r.lmx).
bool run_check(SolveRun& r) {
  if (r.rc != RCHFSI_OK) return false;
  rchfsi_ctx& c = *r.h;
  const rchfsi_params& p = c.p;
  const int64_t m = p.m;
  const int N = r.N;
  Work& w = c.w;
  const auto tr = std::chrono::steady_clock::now();
  // a complex problem's block is [X_s, J X_s]: its residuals are those of the first Nc columns
  const int Nr = c.cplx ? c.Nc : N;
  resid_form_f64(c.s, m, Nr, w.AX.p, w.BX.p, w.evals.p, w.W.p);
  resid_rel_norms(c.s, m, Nr, w.W.p, w.X.p, w.rabs.p, w.xnrm.p);
  RC_CUDA(cudaMemcpyAsync(r.ev.data(), w.evals.p, N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaMemcpyAsync(r.ra.data(), w.rabs.p, N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaMemcpyAsync(r.xn.data(), w.xnrm.p, N * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  RC_CUDA(cudaStreamSynchronize(c.s));
  r.t_rr += ms_since(tr);
  r.maxrel = 0.0;
  r.maxabs = 0.0;
  bool finite = true;
  for (int j = 0; j < r.nev; ++j) {
    finite = finite && std::isfinite(r.ra[j]) && std::isfinite(r.ev[j]);
    r.maxrel = std::max(r.maxrel, r.ra[j] / (r.normA * r.xn[j]));
    r.maxabs = std::max(r.maxabs, r.ra[j]);
  }
  if (r.hist && r.it <= p.max_iter) r.hist[r.it] = r.maxrel;
  if (!finite) {
    r.rc = RCHFSI_ERR_NUMERIC;
    return false;
  }
  if (r.maxrel <= p.tol && r.it >= p.min_iter) return false;
  if (r.it >= p.max_iter) {
    r.rc = RCHFSI_ERR_NOT_CONVERGED;
    return false;
  }
  if (r.maxrel < 0.5 * r.best) {
    r.best = r.maxrel;
    r.best_it = r.it;
  } else if (p.stall_iters > 0 && r.it - r.best_it >= p.stall_iters) {
    r.rc = RCHFSI_ERR_STAGNATED;
    return false;
  }
  r.lmin = p.fixed_bounds ? p.lmin : r.ev[0];
  r.lT = p.fixed_bounds ? p.lT : r.ev[N - 1];
  r.lmx = p.fixed_bounds ? p.lmax : r.lmax;
  return true;
}

void run_filter_single(SolveRun& r) {
  rchfsi_ctx& c = *r.h;
  const auto tf = std::chrono::steady_clock::now();
  filter_any(c, c.w.X.p, r.ev.data(), c.w.W.p, r.lmin, r.lT, r.lmx, c.p.degree, c.w.Y.p,
             c.p.method == RCHFSI_METHOD_CHFSI, true);
  r.t_filter += ms_since(tf);
  r.applies += c.last_applies;
  r.flops += c.last_flops;
}

void run_rr(SolveRun& r) {
  rchfsi_ctx& c = *r.h;
  const auto tr = std::chrono::steady_clock::now();
  r.rc = rayleigh_ritz(c, c.w.Y.p, c.w.X.p, c.w.AX.p, c.w.BX.p, c.w.evals.p);
  r.retries += c.rr_retries;
  pair_after_rr(r);
  r.t_rr += ms_since(tr);
  ++r.it;
}

void run_end(SolveRun& r) {
  rchfsi_ctx& c = *r.h;
  store_any(c, c.w.X.p, r.X_inout);
  from_device(c, c.w.evals.p, r.evals, r.Nout);
  std::vector<double> rel(r.Nout);
  if (r.resid) {
    for (int j = 0; j < r.Nout; ++j) rel[j] = r.ra[j] / (r.normA * r.xn[j]);
    const auto kind = is_device_pointer(r.resid) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    RC_CUDA(cudaMemcpyAsync(r.resid, rel.data(), r.Nout * sizeof(double), kind, c.s));
  }
  RC_CUDA(cudaStreamSynchronize(c.s));
  if (r.st) {
    r.st->iterations = r.it;
    r.st->status = r.rc;
    r.st->max_rel_residual = r.maxrel;
    r.st->max_abs_residual = r.maxabs;
    r.st->lmax = r.lmax;
    r.st->normA = r.normA;
    r.st->t_total_ms = ms_since(r.t0);
    r.st->t_filter_ms = r.t_filter;
    r.st->t_rr_ms = r.t_rr;
    r.st->filter_flops = r.flops;
    r.st->operator_applies = r.applies;
    r.st->cholqr_retries = r.retries;
  }
}

// Meeting point of the workers of rchfsi_solve_batch before each filter: the last worker to
// arrive runs the batched filter for every worker that asked for one, then releases all; workers
// that are done leave the group.
struct Rendezvous {
  std::mutex mu;
  std::condition_variable cv;
  int expected = 0, arrived = 0, leaving = 0;
  uint64_t gen = 0;
  std::vector<int> want;
  template <class F>
  void arrive(int id, bool needs_filter, F&& run) {
    std::unique_lock<std::mutex> lk(mu);
    if (needs_filter) want.push_back(id);
    else ++leaving;
    const uint64_t g = gen;
    if (++arrived == expected) {
      std::vector<int> act;
      act.swap(want);
      std::sort(act.begin(), act.end());
      lk.unlock();
      if (!act.empty()) run(act);
      lk.lock();
      expected -= leaving;
      leaving = 0;
      arrived = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return gen != g; });
    }
  }
};

}  // namespace

extern "C" {

int rchfsi_solve_batch(struct rchfsi_ctx** handles, int count, double** X_inout, double** evals, double** resid,
                       rchfsi_stats* stats) {
  if (!handles || count < 1 || !X_inout) return RCHFSI_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !X_inout[i]) return RCHFSI_ERR_INVALID_ARG;
    if (!handles[i]->has_op) return RCHFSI_ERR_NO_OPERATOR;
    for (int k = 0; k < i; ++k)
      if (handles[k] == handles[i]) return RCHFSI_ERR_INVALID_ARG;
  }
  std::vector<SolveRun> runs;
  runs.reserve(count);
  for (int i = 0; i < count; ++i)
    runs.emplace_back(handles[i], X_inout[i], evals ? evals[i] : nullptr, resid ? resid[i] : nullptr,
                      stats ? stats + i : nullptr);
  // one batch stream for the shared filter launches
  cudaStream_t bs = nullptr;
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return RCHFSI_ERR_CUDA;
  int num_sms = handles[0]->num_sms;
  FeBatchPlan plan;
  Rendezvous rv;
  rv.expected = count;
  std::vector<int> rcs(count, RCHFSI_OK);
  auto fail = [&](int i, const std::exception& e, int code) {
    handles[i]->err = e.what();
    runs[i].rc = code;
  };
  // the batched filter, run by the last worker to arrive
  auto batch_filter = [&](const std::vector<int>& act) {
    std::vector<int> batched, single;
    const int deg = handles[act[0]]->p.degree, prec = handles[act[0]]->p.precision;
    for (int i : act)
      (fe_batchable(*handles[i], deg) && handles[i]->p.precision == prec ? batched : single).push_back(i);
    if (batched.size() < 2) {
      single.insert(single.end(), batched.begin(), batched.end());
      batched.clear();
    }
    if (!batched.empty()) {
      std::vector<FeFilterJob> jobs;
      for (int i : batched) {
        rchfsi_ctx& c = *handles[i];
        jobs.push_back(FeFilterJob{&c, c.w.X.p, runs[i].ev.data(), c.w.W.p, runs[i].lmin, runs[i].lT, runs[i].lmx,
                                   c.w.Y.p});
      }
      const auto tf = std::chrono::steady_clock::now();
      try {
        ProfBind pb(handles[batched[0]]);
        filter_fe_batch(bs, num_sms, jobs, plan);
        const double ms = ms_since(tf);
        for (int i : batched) {
          runs[i].t_filter += ms;
          runs[i].applies += handles[i]->last_applies;
          runs[i].flops += handles[i]->last_flops;
        }
      } catch (const Error& e) {
        for (int i : batched) fail(i, e, e.code);
      } catch (const std::exception& e) {
        for (int i : batched) fail(i, e, RCHFSI_ERR_CUDA);
      }
    }
    for (int i : single) {
      try {
        ProfBind pb(handles[i]);
        run_filter_single(runs[i]);
      } catch (const Error& e) {
        fail(i, e, e.code);
      } catch (const std::exception& e) {
        fail(i, e, RCHFSI_ERR_CUDA);
      }
    }
  };
  auto worker = [&](int i) {
    SolveRun& r = runs[i];
    ProfBind pb(handles[i]);
    bool ok = true;
    try {
      run_begin(r);
    } catch (const Error& e) {
      fail(i, e, e.code);
      ok = false;
    } catch (const std::exception& e) {
      fail(i, e, RCHFSI_ERR_CUDA);
      ok = false;
    }
    for (;;) {
      bool more = false;
      if (ok) {
        try {
          more = run_check(r);
        } catch (const Error& e) {
          fail(i, e, e.code);
        } catch (const std::exception& e) {
          fail(i, e, RCHFSI_ERR_CUDA);
        }
      }
      rv.arrive(i, more, batch_filter);
      if (!more || r.rc != RCHFSI_OK) break;
      try {
        run_rr(r);
      } catch (const Error& e) {
        fail(i, e, e.code);
        break;
      } catch (const std::exception& e) {
        fail(i, e, RCHFSI_ERR_CUDA);
        break;
      }
    }
    try {
      run_end(r);
    } catch (const Error& e) {
      if (r.rc == RCHFSI_OK) fail(i, e, e.code);
    } catch (const std::exception& e) {
      if (r.rc == RCHFSI_OK) fail(i, e, RCHFSI_ERR_CUDA);
    }
    rcs[i] = r.rc;
  };
  {
    std::vector<std::thread> th;
    th.reserve(count);
    for (int i = 0; i < count; ++i) th.emplace_back(worker, i);
    for (auto& t : th) t.join();
  }
  cudaStreamSynchronize(bs);
  cudaStreamDestroy(bs);
  for (int i = 0; i < count; ++i)
    if (rcs[i] != RCHFSI_OK) return rcs[i];
  return RCHFSI_OK;
}


int rchfsi_params_default(rchfsi_params* p) {
  if (!p) return RCHFSI_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->nev = 1;
  p->block = 1;
  p->degree = 20;
  p->precision = RCHFSI_FP64;
  p->method = RCHFSI_METHOD_RCHFSI;
  p->field = RCHFSI_REAL;
  p->max_iter = 100;
  p->min_iter = 0;
  p->lanczos_steps = 10;
  p->stall_iters = 0;
  p->fixed_bounds = 0;
  p->rr_mode = RCHFSI_RR_FP64_EMULATED;
  p->eig_mode = RCHFSI_EIG_TRIDIAG;
  p->tol = 1e-8;
  return RCHFSI_OK;
}

int rchfsi_create(rchfsi_ctx** out, const rchfsi_params* p, void* cuda_stream) {
  if (!out) return RCHFSI_ERR_INVALID_ARG;
  *out = nullptr;
  rchfsi_ctx* h = new rchfsi_ctx();
  const int rc = guarded(h, [&] {
    validate_params(p);
    h->p = *p;
    if (p->field == RCHFSI_COMPLEX) {
      // the real embedding: twice the rows, twice the block, twice the wanted pairs
      h->cplx = true;
      h->mc = p->m;
      h->Nc = p->block;
      h->nevc = p->nev;
      h->p.m = 2 * p->m;
      h->p.block = 2 * p->block;
      h->p.nev = 2 * p->nev;
      h->p.field = RCHFSI_REAL;
    }
    RC_CUDA(cudaGetDevice(&h->device));
    RC_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    if (cuda_stream) {
      h->s = (cudaStream_t)cuda_stream;
    } else {
      RC_CUDA(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    for (auto& e : h->ev) RC_CUDA(cudaEventCreate(&e));
    h->w.ensure(h->p.m, h->p.block);
    return RCHFSI_OK;
  });
  if (rc != RCHFSI_OK) {
    rchfsi_destroy(h);
    return rc;
  }
  *out = h;
  return RCHFSI_OK;
}

int rchfsi_destroy(rchfsi_ctx* h) {
  if (!h) return RCHFSI_OK;
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->solver) cusolverDnDestroy(h->solver);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  cudaStream_t s = h->s;
  bool own = h->own_stream;
  delete h;
  if (own && s) cudaStreamDestroy(s);
  return RCHFSI_OK;
}

int rchfsi_set_params(rchfsi_ctx* h, const rchfsi_params* p) {
  if (!h) return RCHFSI_ERR_INVALID_ARG;
  return guarded(h, [&] {
    validate_params(p);
    const bool cp = p->field == RCHFSI_COMPLEX;
    const int64_t m0 = h->cplx ? h->mc : h->p.m;
    const int n0 = h->cplx ? h->Nc : h->p.block;
    RC_CHECK(p->m == m0 && p->block == n0 && cp == h->cplx, RCHFSI_ERR_INVALID_ARG,
             "m, block and field cannot change on an existing handle");
    h->p = *p;
    if (cp) {
      h->nevc = p->nev;
      h->p.m = 2 * p->m;
      h->p.block = 2 * p->block;
      h->p.nev = 2 * p->nev;
      h->p.field = RCHFSI_REAL;
    }
    return RCHFSI_OK;
  });
}

int rchfsi_set_operator(rchfsi_ctx* h, const rchfsi_operator* op) {
  if (!h) return RCHFSI_ERR_INVALID_ARG;
  return guarded(h, [&] {
    RC_CHECK(op, RCHFSI_ERR_INVALID_ARG, "operator is NULL");
    RC_CHECK(op->m == (h->cplx ? h->mc : h->p.m), RCHFSI_ERR_INVALID_ARG, "operator m differs from params m");
    RC_CHECK((op->field == RCHFSI_COMPLEX) == h->cplx, RCHFSI_ERR_INVALID_ARG,
             "operator field differs from the handle's field");
    h->has_op = false;
    if (op->kind == RCHFSI_OP_DENSE && h->cplx) {
      h->fe.reset();
      set_dense_complex(*h, op);
    } else if (op->kind == RCHFSI_OP_DENSE) {
      h->fe.reset();
      set_dense(*h, op);
    } else if (op->kind == RCHFSI_OP_FE_CELL) {
      h->dense.reset();
      set_fe(*h, op);
    } else {
      throw Error(RCHFSI_ERR_INVALID_ARG, "unknown operator kind");
    }
    h->op_kind = op->kind;
    h->has_op = true;
    if (h->p.hbm_budget_bytes && device_bytes(*h) > h->p.hbm_budget_bytes) {
      h->has_op = false;
      throw Error(RCHFSI_ERR_OOM, "operator does not fit in hbm_budget_bytes");
    }
    return RCHFSI_OK;
  });
}

int rchfsi_filter(rchfsi_ctx* h, const double* X, const double* Lambda, const double* W, double lmin, double lT,
                  double lmax, int degree, double* Yp) {
  return guarded(h, [&] {
    need_op(h);
    RC_CHECK(Yp, RCHFSI_ERR_INVALID_ARG, "Yp is NULL");
    rchfsi_ctx& c = *h;
    const std::vector<double> lam = lam_any(c, Lambda);
    load_any(c, X, c.w.X.p);
    load_any(c, W, c.w.W.p);
    filter_any(c, c.w.X.p, lam.data(), c.w.W.p, lmin, lT, lmax, degree, c.w.Y.p, false, false);
    store_any(c, c.w.Y.p, Yp);
    RC_CUDA(cudaStreamSynchronize(c.s));
    return RCHFSI_OK;
  });
}

int rchfsi_chfsi_filter(rchfsi_ctx* h, const double* X, double lmin, double lT, double lmax, int degree,
                        double* Yp) {
  return guarded(h, [&] {
    need_op(h);
    RC_CHECK(Yp, RCHFSI_ERR_INVALID_ARG, "Yp is NULL");
    rchfsi_ctx& c = *h;
    load_any(c, X, c.w.X.p);
    filter_any(c, c.w.X.p, nullptr, nullptr, lmin, lT, lmax, degree, c.w.Y.p, true, false);
    store_any(c, c.w.Y.p, Yp);
    RC_CUDA(cudaStreamSynchronize(c.s));
    return RCHFSI_OK;
  });
}

int rchfsi_residual(rchfsi_ctx* h, const double* X, const double* Lambda, double* W, double* rnorm) {
  return guarded(h, [&] {
    need_op(h);
    rchfsi_ctx& c = *h;
    const int64_t m = c.p.m;
    // a complex block needs only the first N embedded columns
    const int N = c.cplx ? c.Nc : c.p.block;
    load_any(c, X, c.w.X.p);
    const std::vector<double> lam = lam_any(c, Lambda);
    RC_CUDA(cudaMemcpyAsync(c.w.evals.p, lam.data(), N * sizeof(double), cudaMemcpyHostToDevice, c.s));
    apply_AB_f64(c, c.w.X.p, c.w.AX.p, c.w.BX.p, N);
    resid_form_f64(c.s, m, N, c.w.AX.p, c.w.BX.p, c.w.evals.p, c.w.W.p);
    store_any(c, c.w.W.p, W);
    if (rnorm) {
      resid_rel_norms(c.s, m, N, c.w.W.p, c.w.X.p, c.w.rabs.p, c.w.xnrm.p);
      from_device(c, c.w.rabs.p, rnorm, N);
    }
    RC_CUDA(cudaStreamSynchronize(c.s));
    return RCHFSI_OK;
  });
}

int rchfsi_rayleigh_ritz(rchfsi_ctx* h, const double* Y, double* X, double* evals) {
  return guarded(h, [&] {
    need_op(h);
    rchfsi_ctx& c = *h;
    load_any(c, Y, c.w.Y.p);
    const int rc = rayleigh_ritz(c, c.w.Y.p, c.w.X.p, c.w.AX.p, c.w.BX.p, c.w.evals.p);
    if (rc != RCHFSI_OK) return rc;
    if (c.cplx && !c.rr_paired) {
      std::vector<double> ev = host_vec(c, c.w.evals.p, c.p.block);
      pair_complex(c, ev);
    }
    store_any(c, c.w.X.p, X);
    from_device(c, c.w.evals.p, evals, c.cplx ? c.Nc : c.p.block);
    RC_CUDA(cudaStreamSynchronize(c.s));
    return RCHFSI_OK;
  });
}

int rchfsi_lanczos_bounds(rchfsi_ctx* h, const double* v0, int steps, double* lmax, double* normA) {
  return guarded(h, [&] {
    need_op(h);
    rchfsi_ctx& c = *h;
    double* v = c.w.T1.p;
    if (c.cplx) {
      // complex start vector (interleaved) -> [v_r; v_i]
      double* st = c.cstage.ensure(2 * c.mc);
      to_device(c, v0, st, 2 * c.mc);
      cplx_deinterleave(c.s, c.mc, st, v, v + c.mc);
    } else {
      to_device(c, v0, v, c.p.m);
    }
    lanczos(c, v, steps, lmax, normA);
    return RCHFSI_OK;
  });
}

int rchfsi_solve(rchfsi_ctx* h, double* X_inout, double* evals, double* resid, rchfsi_stats* st) {
  return guarded(h, [&] {
    need_op(h);
    SolveRun r(h, X_inout, evals, resid, st);
    run_begin(r);
    while (run_check(r)) {
      run_filter_single(r);
      run_rr(r);
    }
    run_end(r);
    return r.rc;
  });
}

int rchfsi_profile(rchfsi_ctx* h, int enable) {
  if (!h) return RCHFSI_ERR_INVALID_ARG;
  return guarded(h, [&] {
    if (h->s) RC_CUDA(cudaStreamSynchronize(h->s));
    h->prof.clear();
    h->prof.on = enable != 0;
    h->prof.launch_base = __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED);
    return RCHFSI_OK;
  });
}

int rchfsi_profile_read(rchfsi_ctx* h, int cls, double* total_ms, int64_t* launches, double* flops, double* bytes) {
  if (!h) return RCHFSI_ERR_INVALID_ARG;
  return guarded(h, [&] {
    RC_CHECK(cls >= 0 && cls <= RCHFSI_KERNEL_CLASSES, RCHFSI_ERR_INVALID_ARG, "bad kernel class");
    if (h->s) RC_CUDA(cudaStreamSynchronize(h->s));
    if (cls == RCHFSI_KERNEL_CLASSES) {
      // all kernel launches of this library (every thread) since the last rchfsi_profile(h, .)
      if (launches) *launches = __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED) - h->prof.launch_base;
      if (total_ms) *total_ms = 0.0;
      if (flops) *flops = 0.0;
      if (bytes) *bytes = 0.0;
      return RCHFSI_OK;
    }
    double t = 0.0, fl = 0.0, by = 0.0;
    int64_t n = 0;
    for (const auto& r : h->prof.recs) {
      if (r.cls != cls) continue;
      float ms = 0.f;
      RC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      t += ms;
      fl += r.flops;
      by += r.bytes;
      ++n;
    }
    if (total_ms) *total_ms = t;
    if (launches) *launches = n;
    if (flops) *flops = fl;
    if (bytes) *bytes = by;
    return RCHFSI_OK;
  });
}

const char* rchfsi_strerror(int code) {
  switch (code) {
    case RCHFSI_OK: return "ok";
    case RCHFSI_PENDING: return "pending";
    case RCHFSI_ERR_INVALID_ARG: return "invalid argument";
    case RCHFSI_ERR_OOM: return "out of device memory or over the HBM budget";
    case RCHFSI_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case RCHFSI_ERR_STAGNATED: return "residual stagnated";
    case RCHFSI_ERR_ILL_CONDITIONED: return "Gram matrix not positive definite";
    case RCHFSI_ERR_NUMERIC: return "non-finite value";
    case RCHFSI_ERR_TIMEOUT: return "bounded device wait timed out";
    case RCHFSI_ERR_CUDA: return "CUDA error";
    case RCHFSI_ERR_NO_OPERATOR: return "no operator set";
    case RCHFSI_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int rchfsi_last_error(rchfsi_ctx* h, char* buf, size_t len) {
  if (!buf || len == 0) return RCHFSI_ERR_INVALID_ARG;
  const std::string& s = h ? h->err : g_last_error;
  const size_t n = std::min(len - 1, s.size());
  std::memcpy(buf, s.data(), n);
  buf[n] = 0;
  return RCHFSI_OK;
}

}  // extern "C"
