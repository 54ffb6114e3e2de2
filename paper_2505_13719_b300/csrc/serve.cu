// Serving engine: continuous batching of whole HALLaR solves.
//
// A FIFO of requests feeds up to max_inflight worker threads.  A worker takes
// the head request when the HBM budget has room for its estimated footprint,
// builds a handle on a stream of its own (hallar_create with no stream), runs
// hallar_solve, copies the solution to host memory the engine owns and
// destroys the handle, which returns the footprint to the budget.  Handles
// allocate with the stream-ordered allocator and never synchronise the
// device, so the solves in flight overlap on the GPU; their kernels are
// deterministic and share no device state, so a result is the same whether
// the request ran alone or among others.  The paper solves one problem at a
// time; this layer has no counterpart there.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hallar.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket = 0;
  // the request, copied at submit
  int64_t n = 0, n1 = 0, m = 0, m_pairs = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  double C_J = 0.0, C_I = 0.0;
  int32_t family = 0, has_trace = 0, r0 = 0;
  std::vector<int32_t> ci, cj;
  std::vector<double> b;
  double tau2 = 0.0;
  std::vector<unsigned char> U0;
  hallar_options opt{};
  int64_t footprint = 0;
  size_t elem = 8;
  // timing and results
  Clock::time_point t_submit, t_done;
  bool done = false;
  hallar_status status = HALLAR_OK;
  hallar_result res{};
  std::vector<unsigned char> U;  // n x rank, leading dimension rank
  int32_t rank = 0;
  std::vector<double> p;
  std::string error;
};

int64_t padded(int64_t r, int64_t v) { return (r + v - 1) / v * v; }

}  // namespace

struct hallar_server {
  hallar_server_options opt{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<int64_t, std::shared_ptr<Job>> jobs;  // submitted, not yet waited for
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_ticket = 1;
  double bytes_inflight = 0.0, peak_bytes = 0.0;
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, inflight = 0;
  int64_t max_inflight_seen = 0;
  std::vector<double> latencies;
  bool have_first = false;
  Clock::time_point t_first, t_last_done;
  std::string last_error;
};

namespace {

// one solve, outside the lock
void run_job(Job& j) {
  hallar_options o = j.opt;
  o.stream = nullptr;  // a stream of the handle's own
  hallar_t h = nullptr;
  hallar_status st = hallar_create(
      j.n, j.n1, j.rowptr.empty() ? nullptr : j.rowptr.data(),
      j.col.empty() ? nullptr : j.col.data(), j.val.empty() ? nullptr : j.val.data(), j.C_J,
      j.C_I, j.family, j.m_pairs, j.ci.empty() ? nullptr : j.ci.data(),
      j.cj.empty() ? nullptr : j.cj.data(), j.has_trace, j.b.data(), j.tau2, &o, &h);
  if (st != HALLAR_OK) {
    j.status = st;
    j.error = hallar_last_error(nullptr);
    return;
  }
  st = hallar_solve(h, j.U0.data(), j.r0, nullptr, &j.res);
  j.status = st;
  if (st == HALLAR_OK || st == HALLAR_ENOTCONV || st == HALLAR_ETIMEOUT) {
    int32_t rank = 0;
    hallar_status g = hallar_get_solution(h, nullptr, 0, nullptr, &rank);
    if (g == HALLAR_OK) {
      j.rank = rank;
      j.U.assign((size_t)j.n * (size_t)std::max(rank, 1) * j.elem, 0);
      j.p.assign((size_t)j.m, 0.0);
      g = hallar_get_solution(h, j.U.data(), std::max(rank, 1), j.p.data(), nullptr);
    }
    if (g != HALLAR_OK) {
      j.status = g;
      j.error = hallar_last_error(h);
    }
  } else {
    j.error = hallar_last_error(h);
  }
  hallar_destroy(h);
}

void worker_loop(hallar_server* s) {
  cudaSetDevice(s->opt.device);
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // strict FIFO: the head request waits until the budget has room for it
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        if (s->queue.empty()) return false;
        const double need = (double)s->queue.front()->footprint;
        return s->bytes_inflight + need <= s->opt.hbm_budget_bytes;
      });
      if (s->stop) return;
      j = s->queue.front();
      s->queue.pop_front();
      s->bytes_inflight += (double)j->footprint;
      s->peak_bytes = std::max(s->peak_bytes, s->bytes_inflight);
      ++s->inflight;
      ++s->admitted;
      s->max_inflight_seen = std::max(s->max_inflight_seen, s->inflight);
    }
    run_job(*j);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      j->t_done = Clock::now();
      j->done = true;
      s->bytes_inflight -= (double)j->footprint;
      --s->inflight;
      ++s->completed;
      if (j->status != HALLAR_OK) ++s->failed;
      s->latencies.push_back(std::chrono::duration<double>(j->t_done - j->t_submit).count());
      s->t_last_done = j->t_done;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  // linear interpolation between closest ranks
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)std::floor(pos), hi = (size_t)std::ceil(pos);
  return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

int64_t hallar_solve_footprint(const hallar_request* q) {
  if (!q) return -1;
  const int64_t n = std::max<int64_t>(q->n, 1);
  const bool mixed = q->opt.precision == HALLAR_MIXED;
  const int64_t es = mixed ? 4 : 8;
  const int64_t m = q->family == HALLAR_DIAG ? n : q->m_pairs + (q->has_trace_row ? 1 : 0);
  const int64_t nnz_c = q->C_rowptr ? std::max<int64_t>(q->C_nnz, 0) : 0;
  const int64_t nnz = nnz_c + (q->family == HALLAR_DIAG ? 0 : 2 * q->m_pairs);
  int64_t b = 0;
  // problem: rowptr, col, code, values (double and float), diagonal, b
  b += 4 * (n + 1) + 4 * nnz + 4 * nnz + 12 * nnz + 12 * n + 12 * m;
  // handle: grid-reduction partials and small scalars
  b += 4096LL * (2 * 256 + 2) * 8 + 64 * 1024;
  // solver: ten factor-sized buffers, vectors of length m and n, Gram matrix
  const int64_t rcap = std::max(q->opt.r_cap, 1);
  const int64_t ld = padded(rcap + 1, mixed ? 4 : 2);
  // a mixed solve that goes on in FP64 (opt.promote) holds 8-byte factors then
  const int64_t esf = mixed && q->opt.promote ? 8 : es;
  b += 10 * n * ld * esf + m * (8 + 4 + 3 * esf + 8) + 24 * n + ld * ld * 8;
  // Lanczos: row-major basis, two vectors, per-block partial rows
  int64_t k = std::min<int64_t>(std::min<int64_t>(std::max(q->opt.lanczos_kmax, 2), 512), n);
  const int64_t kcap = padded(k, 4);
  b += n * kcap * 8 + 16 * n + 1184 * kcap * 8;
  // staging of the start factor and of the solution, constraint values
  b += 2 * n * ld * es + 8 * m;
  // Gram partials of the rank trim
  b += 512 * ld * ld * 8;
  return (int64_t)((double)b * 1.05) + (64LL << 20);
}

hallar_status hallar_server_create(const hallar_server_options* opt, hallar_server_t* out) {
  if (!out) return HALLAR_EINVAL;
  *out = nullptr;
  if (!opt || !(opt->hbm_budget_bytes > 0.0) || opt->max_inflight < 1 ||
      opt->max_inflight > 256 || opt->device < 0)
    return HALLAR_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || opt->device >= count) {
    cudaGetLastError();
    return HALLAR_ECUDA;
  }
  hallar_server* s = new (std::nothrow) hallar_server();
  if (!s) return HALLAR_ENOMEM;
  s->opt = *opt;
  try {
    for (int i = 0; i < opt->max_inflight; ++i) s->workers.emplace_back(worker_loop, s);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    return HALLAR_ENOMEM;
  }
  *out = s;
  return HALLAR_OK;
}

hallar_status hallar_server_submit(hallar_server_t s, const hallar_request* q, int64_t* ticket) {
  if (!s) return HALLAR_EINVAL;
  auto bad = [&](const char* msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->last_error = msg;
    return HALLAR_EINVAL;
  };
  if (!q || !ticket) return bad("hallar_server_submit: NULL request or ticket");
  if (q->n <= 0 || q->n >= (int64_t)INT32_MAX) return bad("request: n out of range");
  if (!q->b || !q->U0 || q->r0 < 1 || q->r0 > 256) return bad("request: b, U0 or r0 invalid");
  if (q->family < 0 || q->family > 2) return bad("request: unknown family");
  if (q->m_pairs < 0 || (q->m_pairs > 0 && (!q->cons_i || !q->cons_j)))
    return bad("request: constraint pairs invalid");
  if (q->C_rowptr && (q->C_nnz < 0 || q->C_rowptr[q->n] != q->C_nnz ||
                      (q->C_nnz > 0 && (!q->C_col || !q->C_val))))
    return bad("request: C_nnz does not match C_rowptr[n] or C arrays NULL");
  const int64_t fp = hallar_solve_footprint(q);
  if ((double)fp > s->opt.hbm_budget_bytes) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->last_error = "request footprint exceeds the HBM budget";
    return HALLAR_ENOMEM;
  }
  std::shared_ptr<Job> j;
  try {
    j = std::make_shared<Job>();
    j->n = q->n;
    j->n1 = q->n1;
    j->family = q->family;
    j->m_pairs = q->m_pairs;
    j->has_trace = q->has_trace_row;
    j->m = q->family == HALLAR_DIAG ? q->n : q->m_pairs + (q->has_trace_row ? 1 : 0);
    if (q->C_rowptr) {
      j->rowptr.assign(q->C_rowptr, q->C_rowptr + q->n + 1);
      j->col.assign(q->C_col, q->C_col + q->C_nnz);
      j->val.assign(q->C_val, q->C_val + q->C_nnz);
    }
    j->C_J = q->C_J;
    j->C_I = q->C_I;
    if (q->m_pairs > 0) {
      j->ci.assign(q->cons_i, q->cons_i + q->m_pairs);
      j->cj.assign(q->cons_j, q->cons_j + q->m_pairs);
    }
    j->b.assign(q->b, q->b + std::max<int64_t>(j->m, 0));
    j->tau2 = q->tau2;
    j->opt = q->opt;
    j->elem = q->opt.precision == HALLAR_MIXED ? 4 : 8;
    j->r0 = q->r0;
    const unsigned char* u0 = static_cast<const unsigned char*>(q->U0);
    j->U0.assign(u0, u0 + (size_t)q->n * q->r0 * j->elem);
    j->footprint = fp;
  } catch (const std::bad_alloc&) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->last_error = "host allocation failed";
    return HALLAR_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j->ticket = s->next_ticket++;
    j->t_submit = Clock::now();
    if (!s->have_first) {
      s->have_first = true;
      s->t_first = j->t_submit;
    }
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    ++s->submitted;
    *ticket = j->ticket;
  }
  s->cv_work.notify_all();
  return HALLAR_OK;
}

hallar_status hallar_server_wait(hallar_server_t s, int64_t ticket, double timeout_s,
                                 hallar_result* res, void* U, int32_t U_capacity, double* p,
                                 int32_t* rank, double* latency_s) {
  // errors of the call itself (and a wait that timed out) leave rank and
  // latency at -1; a completed ticket reports its solve's status
  if (rank) *rank = -1;
  if (latency_s) *latency_s = -1.0;
  if (!s) return HALLAR_EINVAL;
  std::shared_ptr<Job> j;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) {
      s->last_error = "unknown ticket";
      return HALLAR_EINVAL;
    }
    j = it->second;
    auto ready = [&] { return j->done; };
    if (timeout_s < 0.0) {
      s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
      return HALLAR_ETIMEOUT;  // still queued or running (rank and latency -1)
    }
    if (U && j->rank > U_capacity) {
      s->last_error = "U_capacity below the solution rank";
      return HALLAR_EINVAL;
    }
    s->jobs.erase(it);
    if (j->status != HALLAR_OK) s->last_error = j->error;
  }
  if (res) *res = j->res;
  if (rank) *rank = j->rank;
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  if (U && j->rank > 0 && !j->U.empty()) {
    unsigned char* dst = static_cast<unsigned char*>(U);
    const size_t row = (size_t)j->rank * j->elem;
    for (int64_t i = 0; i < j->n; ++i)
      std::memcpy(dst + (size_t)i * U_capacity * j->elem, j->U.data() + (size_t)i * row, row);
  }
  if (p && !j->p.empty()) std::memcpy(p, j->p.data(), j->p.size() * sizeof(double));
  return j->status;
}

hallar_status hallar_server_get_stats(hallar_server_t s, hallar_server_stats* st) {
  if (!s || !st) return HALLAR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->admitted = s->admitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->queued = (int64_t)s->queue.size();
  st->inflight = s->inflight;
  st->max_inflight_seen = s->max_inflight_seen;
  st->bytes_inflight = s->bytes_inflight;
  st->peak_bytes_inflight = s->peak_bytes;
  st->p50_latency_s = percentile(s->latencies, 0.50);
  st->p99_latency_s = percentile(s->latencies, 0.99);
  if (!s->latencies.empty()) {
    double sum = 0.0, mx = 0.0;
    for (double v : s->latencies) {
      sum += v;
      mx = std::max(mx, v);
    }
    st->mean_latency_s = sum / (double)s->latencies.size();
    st->max_latency_s = mx;
  }
  if (s->have_first && s->completed > 0)
    st->first_submit_to_last_done_s =
        std::chrono::duration<double>(s->t_last_done - s->t_first).count();
  return HALLAR_OK;
}

void hallar_server_destroy(hallar_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

const char* hallar_server_last_error(hallar_server_t s) {
  // a copy per calling thread: the server's own string may change as soon as
  // the lock is released (workers and other callers write it)
  static thread_local std::string copy;
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  copy = s->last_error;
  return copy.c_str();
}

}  // extern "C"
