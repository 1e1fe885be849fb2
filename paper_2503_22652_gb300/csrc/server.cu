// Request loop for repeated eigensolves (rchfsi_server_* / rchfsi_submit / rchfsi_poll).
//
// Continuous batching: `slots` worker threads each own a CUDA stream; a request is admitted, in
// arrival order, as soon as a slot is free and its estimated device footprint fits in the HBM
// budget next to the requests already running, so requests that arrive while others are on the
// GPU start while those are still running and their kernels overlap on the device.  Each request
// is an independent rchfsi_solve on its own handle.  Warm starts: the Ritz vectors of the last
// finished request of a warm_key stay in device memory and seed the next request with that key
// (the subspace reuse of an outer self-consistent loop, where each operator is a small
// perturbation of the previous one).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "solver.cuh"

using namespace rchfsi;

namespace {

using Clock = std::chrono::steady_clock;

struct HostOp {
  rchfsi_operator op{};
  std::vector<double> A, B, A_filter, Dinv, Dinv_dense, A_cells, B_cells;
  std::vector<int32_t> dofs;
};

struct Job {
  uint64_t ticket = 0;
  HostOp hop;
  rchfsi_params params{};
  std::vector<double> X0;
  uint64_t warm_key = 0;
  size_t footprint = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool done = false;
  int status = RCHFSI_PENDING;
  int iterations = 0;
  double max_rel = 0.0;
  std::vector<double> evals, X;
  std::string error;  // text of the failure (empty on success)
};

struct Warm {
  int64_t m = 0;
  int N = 0;
  int field = RCHFSI_REAL;
  DevBuf<double> X;  // row-major m x N on the device (complex: interleaved)
};

struct Server {
  int slots = 1;
  uint64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::map<uint64_t, std::unique_ptr<Warm>> warm;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

template <typename T>
void copy_in(std::vector<T>& dst, const T* src, size_t n) {
  dst.clear();
  if (!src) return;
  dst.resize(n);
  cudaPointerAttributes a{};
  bool dev = cudaPointerGetAttributes(&a, src) == cudaSuccess &&
             (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (dev) {
    RC_CUDA(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst.data(), src, n * sizeof(T));
  }
}

// Values per entry of the caller's blocks and A: 2 for complex problems (interleaved re, im).
size_t field_factor(const rchfsi_params& p) { return p.field == RCHFSI_COMPLEX ? 2 : 1; }

size_t estimate_footprint(const rchfsi_operator& op, const rchfsi_params& p) {
  // a complex problem runs as its real embedding of twice the rows and block columns
  const size_t cf = field_factor(p);
  const size_t m = (size_t)p.m * cf, N = (size_t)p.block * cf;
  size_t t = 0;
  if (op.kind == RCHFSI_OP_DENSE) {
    t += m * m * 8 * (op.B ? 5 : 4);  // A, (B), A D^-1, D^-1 A, low-precision copy
  } else {
    const size_t na = (size_t)op.n_cells * op.n_c * op.n_c;
    t += na * 8 * (op.B_cells_shared ? 1 : 2) * cf + na * 4 * cf + (size_t)op.n_cells * op.n_c * 4 + m * 8;
  }
  t += m * N * 8 * 12 + m * N * 4 * 3 + N * N * 8 * 5;
  return t;
}

void run_job(Server& S, Job& j) {
  rchfsi_ctx* h = nullptr;
  int rc = rchfsi_create(&h, &j.params, nullptr);
  if (rc == RCHFSI_OK) rc = rchfsi_set_operator(h, &j.hop.op);
  const size_t blk = (size_t)j.params.m * j.params.block * field_factor(j.params);
  const double* x0 = j.X0.empty() ? nullptr : j.X0.data();
  Warm* wp = nullptr;
  if (rc == RCHFSI_OK && j.warm_key) {
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.warm.find(j.warm_key);
    if (it != S.warm.end() && it->second->m == j.params.m && it->second->N == j.params.block &&
        it->second->field == j.params.field)
      wp = it->second.get();
  }
  DevBuf<double> xdev;
  if (rc == RCHFSI_OK) {
    try {
      xdev.ensure(blk);
      if (wp) {
        std::lock_guard<std::mutex> lk(S.mu);
        RC_CUDA(cudaMemcpy(xdev.p, wp->X.p, blk * sizeof(double), cudaMemcpyDeviceToDevice));
      } else if (x0) {
        RC_CUDA(cudaMemcpy(xdev.p, x0, blk * sizeof(double), cudaMemcpyHostToDevice));
      } else {
        rc = RCHFSI_ERR_INVALID_ARG;
      }
    } catch (const Error& e) {
      rc = e.code;
    }
  }
  rchfsi_stats st{};
  if (rc == RCHFSI_OK) {
    j.evals.resize(j.params.block);
    rc = rchfsi_solve(h, xdev.p, j.evals.data(), nullptr, &st);
    j.iterations = st.iterations;
    j.max_rel = st.max_rel_residual;
    if (rc == RCHFSI_OK || rc == RCHFSI_ERR_NOT_CONVERGED) {
      j.X.resize(blk);
      cudaMemcpy(j.X.data(), xdev.p, blk * sizeof(double), cudaMemcpyDeviceToHost);
      if (j.warm_key && rc == RCHFSI_OK) {
        std::lock_guard<std::mutex> lk(S.mu);
        auto& w = S.warm[j.warm_key];
        if (!w) w.reset(new Warm());
        w->m = j.params.m;
        w->N = j.params.block;
        w->field = j.params.field;
        try {
          w->X.ensure(blk);
          cudaMemcpy(w->X.p, xdev.p, blk * sizeof(double), cudaMemcpyDeviceToDevice);
        } catch (const Error&) {
          S.warm.erase(j.warm_key);
        }
      }
    }
  }
  if (rc != RCHFSI_OK) {
    char buf[160] = {0};
    rchfsi_last_error(h, buf, sizeof(buf));
    j.error = buf;
  }
  rchfsi_destroy(h);
  j.status = rc;
}

void worker(Server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        const size_t need = S->queue.front()->footprint;
        // admit the head of the queue when it fits next to the running requests; a request
        // larger than the whole budget runs alone
        return S->budget == 0 || S->in_use + need <= S->budget || S->running == 0;
      });
      if (S->stop && S->queue.empty()) return;
      if (S->queue.empty()) continue;
      job = S->queue.front();
      S->queue.pop_front();
      S->in_use += job->footprint;
      S->running++;
      job->t_admit = Clock::now();
    }
    run_job(*S, *job);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= job->footprint;
      S->running--;
      job->t_done = Clock::now();
      job->done = true;
      // free the operator copies now; only results stay until polled
      job->hop = HostOp();
      job->X0.clear();
    }
    S->cv.notify_all();
  }
}

Server* as_server(rchfsi_ctx* h) {
  if (!h || !h->is_server || !h->server) return nullptr;
  return (Server*)h->server;
}

}  // namespace

extern "C" {

int rchfsi_server_create(rchfsi_ctx** out, int slots, uint64_t hbm_budget_bytes) {
  if (!out || slots < 1 || slots > 64) return RCHFSI_ERR_INVALID_ARG;
  rchfsi_ctx* h = new rchfsi_ctx();
  Server* S = new Server();
  S->slots = slots;
  S->budget = hbm_budget_bytes;
  cudaGetDevice(&S->device);
  h->is_server = true;
  h->server = S;
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S);
  *out = h;
  return RCHFSI_OK;
}

int rchfsi_server_destroy(rchfsi_ctx* h) {
  Server* S = as_server(h);
  if (!S) return h ? RCHFSI_ERR_INVALID_ARG : RCHFSI_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->queue.clear();
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  h->server = nullptr;
  h->is_server = false;
  delete h;
  return RCHFSI_OK;
}

int rchfsi_submit(rchfsi_ctx* h, const rchfsi_request* rq, uint64_t* ticket) {
  Server* S = as_server(h);
  if (!S || !rq || !ticket) return RCHFSI_ERR_INVALID_ARG;
  auto job = std::make_shared<Job>();
  try {
    const rchfsi_operator& op = rq->op;
    const rchfsi_params& p = rq->params;
    if (op.m != p.m || p.m <= 0 || p.block <= 0) return RCHFSI_ERR_INVALID_ARG;
    const size_t cf = field_factor(p);
    const size_t m = (size_t)p.m, blk = m * p.block * cf;
    HostOp& ho = job->hop;
    ho.op = op;
    if (op.kind == RCHFSI_OP_DENSE) {
      copy_in(ho.A, op.A, m * m * cf);
      copy_in(ho.B, op.B, m * m);
      copy_in(ho.A_filter, op.A_filter, m * m);
      copy_in(ho.Dinv, op.Dinv, m);
      copy_in(ho.Dinv_dense, op.Dinv_dense, m * m);
      ho.op.A = ho.A.empty() ? nullptr : ho.A.data();
      ho.op.B = ho.B.empty() ? nullptr : ho.B.data();
      ho.op.A_filter = ho.A_filter.empty() ? nullptr : ho.A_filter.data();
      ho.op.Dinv = ho.Dinv.empty() ? nullptr : ho.Dinv.data();
      ho.op.Dinv_dense = ho.Dinv_dense.empty() ? nullptr : ho.Dinv_dense.data();
    } else if (op.kind == RCHFSI_OP_FE_CELL) {
      if (op.n_cells <= 0 || op.n_c <= 0) return RCHFSI_ERR_INVALID_ARG;
      const size_t nd = (size_t)op.n_cells * op.n_c, na = nd * op.n_c;
      copy_in(ho.dofs, op.cell_dofs, nd);
      copy_in(ho.A_cells, op.A_cells, na * cf);
      copy_in(ho.B_cells, op.B_cells, op.B_cells_shared ? (size_t)op.n_c * op.n_c : na);
      copy_in(ho.Dinv, op.Dinv, m);
      ho.op.cell_dofs = ho.dofs.data();
      ho.op.A_cells = ho.A_cells.data();
      ho.op.B_cells = ho.B_cells.data();
      ho.op.Dinv = ho.Dinv.data();
    } else {
      return RCHFSI_ERR_INVALID_ARG;
    }
    job->params = p;
    copy_in(job->X0, rq->X0, rq->X0 ? blk : 0);
    job->warm_key = rq->warm_key;
    job->footprint = estimate_footprint(op, p);
  } catch (const Error& e) {
    return e.code;
  } catch (const std::exception&) {
    return RCHFSI_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    job->ticket = S->next_ticket++;
    job->t_submit = Clock::now();
    S->jobs[job->ticket] = job;
    S->queue.push_back(job);
    *ticket = job->ticket;
  }
  S->cv.notify_all();
  return RCHFSI_OK;
}

int rchfsi_poll(rchfsi_ctx* h, uint64_t ticket, rchfsi_result* out) {
  Server* S = as_server(h);
  if (!S || !out) return RCHFSI_ERR_INVALID_ARG;
  std::shared_ptr<Job> job;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return RCHFSI_ERR_INVALID_ARG;
    if (!it->second->done) return RCHFSI_PENDING;
    job = it->second;
    S->jobs.erase(it);
  }
  out->status = job->status;
  out->iterations = job->iterations;
  out->max_rel_residual = job->max_rel;
  out->latency_ms = std::chrono::duration<double, std::milli>(job->t_done - job->t_submit).count();
  out->queue_ms = std::chrono::duration<double, std::milli>(job->t_admit - job->t_submit).count();
  std::memset(out->error, 0, sizeof(out->error));
  std::strncpy(out->error, job->error.c_str(), sizeof(out->error) - 1);
  auto put = [](double* dst, const std::vector<double>& v) {
    if (!dst || v.empty()) return;
    cudaPointerAttributes a{};
    bool dev = cudaPointerGetAttributes(&a, dst) == cudaSuccess &&
               (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) cudaMemcpy(dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
    else std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  put(out->evals, job->evals);
  put(out->X, job->X);
  return RCHFSI_OK;
}

}  // extern "C"
