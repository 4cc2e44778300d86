// Continuous batching of solve requests (dm_submit, dm_submit_system, dm_poll).
//
// A process-wide server owns `slots` worker threads, each with its own
// non-blocking CUDA stream.  Requests enter a FIFO queue; a free worker takes
// the oldest request whose plan has no request in flight, points the plan at
// its stream and runs it (factor and/or solve with float64 residual and, for
// mixed precision, refinement).  Requests on different plans therefore run
// concurrently on the device, and requests that arrive while others run are
// admitted as soon as a slot frees up.  A plan serves one request at a time
// (its factors and right-hand-side workspace are single-occupancy), so
// repeated right-hand sides on one plan are applied in arrival order.
//
// Narrow requests (dm_submit_cols: fewer columns than the plan's nrhs) that
// queue up on one plan are merged: the worker that takes the oldest one also
// takes the plan's next queued solve-only requests, in order, while their
// columns fit in the plan's nrhs, packs their columns side by side into the
// plan's right-hand side (zero columns pad the rest), runs one solve and
// unpacks each request's columns.  The solve sweeps cost nearly the same for
// one column as for sixteen, so merged repeat right-hand sides share one.
//
// Admission by latency budget (dm_serve_budget): the server keeps, per plan,
// a moving average of the measured service time of a factor + solve and of a
// solve; a new request whose predicted latency -- the queued and running work
// spread over the slots, but at least its own plan's serial backlog, plus its
// own service time -- exceeds the budget is refused with DM_EAGAIN.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dm.h"
#include "dm_plan.h"

namespace dm {
namespace {

// Columns [c0, c0 + nc) of a [rows][R] array (wide) to or from a [rows][nc]
// array (narrow): pack = true writes wide from narrow, else narrow from wide.
__global__ void k_cols_move(double* __restrict__ wide, double* __restrict__ narrow, long long rows, int R, int c0,
                            int nc, bool pack) {
  const long long n = rows * nc, stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long row = i / nc;
    const long long w = row * R + c0 + (i - row * nc);
    if (pack)
      wide[w] = narrow[i];
    else
      narrow[i] = wide[w];
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

struct Request {
  uint64_t ticket;
  dm_plan_t plan;
  bool factor;
  const double *A, *B, *C, *b;
  double* x;
  int ncols;   // right-hand-side columns of b and x ([N][m][ncols]); 0: the plan's nrhs
  double cost; // predicted service time at submission (seconds; 0 while unmeasured)
};

// Moving averages of one plan's measured service times (seconds).
struct Estimate {
  double factor_s = 0, solve_s = 0;
  bool has_factor = false, has_solve = false;
};

struct Outcome {
  bool done = false;
  int status = DM_PENDING;
  double relres = 0.0;
  double t_submit = 0, t_start = 0, t_done = 0;  // steady clock, seconds
  std::string msg;  // the worker's error text for a failed request
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

class Server {
 public:
  static Server& get() {
    static Server* s = new Server();  // lives until exit; workers are detached at exit
    return *s;
  }

  int submit(const Request& r0, uint64_t* ticket) {
    std::unique_lock<std::mutex> lk(mu_);
    if (!started_) start_locked();
    if ((int)queue_.size() >= kMaxQueue) {
      ++n_refused_;
      return set_error(DM_EAGAIN, "serving queue full (%d requests)", kMaxQueue);
    }
    Request r = r0;
    r.cost = cost_locked(r);
    if (budget_s_ > 0) {
      const double lat = predicted_wait_locked(r.plan) + r.cost;
      if (lat > budget_s_) {
        ++n_refused_;
        return set_error(DM_EAGAIN, "latency budget: predicted %.4f s > %.4f s", lat, budget_s_);
      }
    }
    ++n_admitted_;
    r.ticket = ++next_ticket_;
    queue_.push_back(r);
    outcomes_[r.ticket] = Outcome();
    outcomes_[r.ticket].t_submit = now_s();
    pending_[r.plan] += 1;
    *ticket = r.ticket;
    cv_.notify_one();
    return DM_OK;
  }

  int poll(uint64_t ticket, int* status, double* relres, double* times) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = outcomes_.find(ticket);
    if (it == outcomes_.end()) return set_error(DM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second.done) {
      *status = DM_PENDING;
      return DM_OK;
    }
    *status = it->second.status;
    // hand the worker's error text to the polling thread's dm_last_error
    if (it->second.status != DM_OK && !it->second.msg.empty()) set_error(it->second.status, "%s", it->second.msg.c_str());
    if (relres) *relres = it->second.relres;
    if (times) {
      times[0] = it->second.t_submit;
      times[1] = it->second.t_start;
      times[2] = it->second.t_done;
    }
    outcomes_.erase(it);
    return DM_OK;
  }

  // Wait until no queued or running request refers to `plan`.
  void drain(dm_plan_t plan) {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] {
      auto it = pending_.find(plan);
      return it == pending_.end() || it->second == 0;
    });
    pending_.erase(plan);
    est_.erase(plan);  // the handle may be reused by a later plan
  }

  int set_budget(double seconds) {
    std::lock_guard<std::mutex> lk(mu_);
    budget_s_ = seconds;
    return DM_OK;
  }

  void stats(long long* out) {
    std::lock_guard<std::mutex> lk(mu_);
    out[0] = n_admitted_;
    out[1] = n_refused_;
    out[2] = n_solves_;
    out[3] = n_merged_;
  }

  int configure(int slots) {
    std::lock_guard<std::mutex> lk(mu_);
    if (started_) return set_error(DM_ESTATE, "the server is already running");
    if (slots < 1 || slots > 64) return set_error(DM_EINVAL, "slots must be in 1..64");
    slots_ = slots;
    return DM_OK;
  }

 private:
  static constexpr int kMaxQueue = 1 << 16;

  void start_locked() {
    started_ = true;
    for (int i = 0; i < slots_; ++i) std::thread([this] { worker(); }).detach();
  }

  // Service time of a request predicted from its plan's measured averages: a
  // narrow solve is charged its share of a full-width solve (it is merged).
  double cost_locked(const Request& r) {
    auto it = est_.find(r.plan);
    if (it == est_.end()) return 0.0;
    if (r.factor) return it->second.factor_s;
    const int R = r.plan->plan.top.spec[0].r;
    return it->second.solve_s * (r.ncols > 0 && r.ncols < R ? (double)r.ncols / R : 1.0);
  }

  // Predicted time until a new request on `plan` starts: all queued and the
  // remaining running work spread over the slots, and at least the work queued
  // or running on its own plan (which runs serially).
  double predicted_wait_locked(dm_plan_t plan) {
    const double t = now_s();
    double all = 0, own = 0;
    for (const Request& q : queue_) {
      all += q.cost;
      if (q.plan == plan) own += q.cost;
    }
    for (const auto& kv : running_) {
      const double rem = std::max(0.0, kv.second - t);
      all += rem;
      if (kv.first == plan) own += rem;
    }
    return std::max(all / slots_, own);
  }

  void record_locked(dm_plan_t plan, bool factor, double seconds) {
    Estimate& e = est_[plan];
    double& v = factor ? e.factor_s : e.solve_s;
    bool& has = factor ? e.has_factor : e.has_solve;
    v = has ? 0.7 * v + 0.3 * seconds : seconds;
    has = true;
  }

  // Run a group on the plan's stream: one request as submitted, or narrow
  // requests packed into the plan's right-hand-side columns.
  static int run_group(Plan& p, const std::vector<Request>& g, std::vector<double>& rel) {
    rel.assign(g.size(), 0.0);
    const Request& r0 = g[0];
    int rc = DM_OK;
    if (r0.factor) rc = p.factor(r0.A, r0.B, r0.C);
    if (rc != DM_OK) return rc;
    const int R = p.top.spec[0].r;
    if (g.size() == 1 && (r0.ncols == 0 || r0.ncols == R)) {
      std::vector<double> rr(std::max(1, p.top.nsys));
      rc = p.solve(r0.b, r0.x, rr.data());
      for (double v : rr) rel[0] = std::max(rel[0], v);
      return rc;
    }
    if (!p.factored) return set_error(DM_ESTATE, "solve before a successful factorisation");
    // each request's [N][m][ncols] columns go through the residual buffer
    // (free outside a solve; it holds N m nrhs doubles) to their place in F
    const SysSpec& sp = p.top.spec[0];
    const long long rows = (long long)sp.N * sp.m;
    cudaStream_t st = p.stream;
    int used = 0;
    for (const Request& q : g) used += q.ncols;
    if (used < R) DM_CUDA(cudaMemsetAsync(p.top.F, 0, rows * R * sizeof(double), st));
    int c0 = 0;
    for (const Request& q : g) {
      if ((rc = copy_in(p.R, q.b, rows * q.ncols * sizeof(double), st))) return rc;
      k_cols_move<<<grid_for(rows * q.ncols), 256, 0, st>>>(p.top.F, p.R, rows, R, c0, q.ncols, true);
      DM_CUDA(cudaGetLastError());
      c0 += q.ncols;
    }
    rc = p.solve_device(p.top.F, p.top.X);
    if (rc != DM_OK && rc != DM_ENOTCONV) return rc;
    c0 = 0;
    for (size_t i = 0; i < g.size(); ++i) {
      const Request& q = g[i];
      k_cols_move<<<grid_for(rows * q.ncols), 256, 0, st>>>(p.top.X, p.R, rows, R, c0, q.ncols, false);
      DM_CUDA(cudaGetLastError());
      const int rc2 = copy_out(q.x, p.R, rows * q.ncols * sizeof(double), st);
      if (rc2) return rc2;
      rel[i] = p.column_relres(c0, q.ncols);
      c0 += q.ncols;
    }
    DM_CUDA(cudaStreamSynchronize(st));
    return rc;
  }

  void worker() {
    // one stream per device this worker has served; the plan's device is
    // made current before any of its work (plans may live on any device)
    std::unordered_map<int, cudaStream_t> streams;
    for (;;) {
      std::vector<Request> g;
      double t_start = 0;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return pick_locked(&g); });
        t_start = now_s();
        double cost = 0;
        for (const Request& q : g) {
          outcomes_[q.ticket].t_start = t_start;
          cost += q.cost;
        }
        running_[g[0].plan] = t_start + cost;
        ++n_solves_;
        if (g.size() > 1) n_merged_ += (long long)g.size();
      }
      const Request& r = g[0];
      Plan& p = r.plan->plan;
      int rc = DM_OK;
      cudaStream_t st = nullptr;
      cudaError_t e = cudaSetDevice(p.device);
      if (e == cudaSuccess) {
        auto it = streams.find(p.device);
        if (it == streams.end()) {
          e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
          if (e == cudaSuccess) streams[p.device] = st;
        } else {
          st = it->second;
        }
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(DM_ECUDA, "serving worker: device %d: %s", p.device, cudaGetErrorString(e));
      }
      cudaStream_t keep = p.stream;
      std::vector<double> rel(g.size(), 0.0);
      if (rc == DM_OK) {
        p.stream = st;
        rc = run_group(p, g, rel);
      }
      p.stream = keep;
      {
        std::lock_guard<std::mutex> lk(mu_);
        const double t_done = now_s();
        if (rc == DM_OK || rc == DM_ENOTCONV) record_locked(r.plan, r.factor, t_done - t_start);
        for (size_t i = 0; i < g.size(); ++i) {
          Outcome& o = outcomes_[g[i].ticket];
          o.done = true;
          o.status = rc;
          if (rc != DM_OK) o.msg = g_last_error;
          o.relres = rel[i];
          o.t_done = t_done;
        }
        busy_.erase(r.plan);
        running_.erase(r.plan);
        pending_[r.plan] -= (int)g.size();
      }
      cv_.notify_all();
      done_cv_.notify_all();
    }
  }

  // Oldest queued request whose plan is idle, and after it, when it is narrow,
  // the same plan's next queued solve-only narrow requests while their columns
  // fit in the plan's nrhs (stopping at the first that does not: order kept).
  bool pick_locked(std::vector<Request>* out) {
    for (auto it = queue_.begin(); it != queue_.end(); ++it) {
      if (busy_.count(it->plan)) continue;
      out->assign(1, *it);
      busy_.insert({it->plan, true});
      const dm_plan_t plan = it->plan;
      const int R = plan->plan.top.spec[0].r;
      int cols = it->ncols;
      it = queue_.erase(it);
      if (cols > 0 && cols < R) {
        while (it != queue_.end()) {
          if (it->plan != plan) {
            ++it;
            continue;
          }
          if (it->factor || it->ncols == 0 || cols + it->ncols > R) break;
          cols += it->ncols;
          out->push_back(*it);
          it = queue_.erase(it);
        }
      }
      return true;
    }
    return false;
  }

  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::deque<Request> queue_;
  std::unordered_map<uint64_t, Outcome> outcomes_;
  std::unordered_map<dm_plan_t, bool> busy_;
  std::unordered_map<dm_plan_t, int> pending_;
  std::unordered_map<dm_plan_t, double> running_;  // predicted end of the plan's running group
  std::unordered_map<dm_plan_t, Estimate> est_;
  uint64_t next_ticket_ = 0;
  bool started_ = false;
  int slots_ = 8;
  double budget_s_ = 0;  // 0: no latency budget
  long long n_admitted_ = 0, n_refused_ = 0, n_solves_ = 0, n_merged_ = 0;
};

}  // namespace

void serve_drain(dm_plan_t plan) { Server::get().drain(plan); }

}  // namespace dm

using namespace dm;

extern "C" {

int dm_submit(dm_plan_t plan, const double* b, double* x, uint64_t* ticket) {
  if (!plan || !b || !x || !ticket) return set_error(DM_EINVAL, "NULL argument to dm_submit");
  Request r{0, plan, false, nullptr, nullptr, nullptr, b, x, 0, 0.0};
  return Server::get().submit(r, ticket);
}

int dm_submit_cols(dm_plan_t plan, const double* b, double* x, int ncols, uint64_t* ticket) {
  if (!plan || !b || !x || !ticket) return set_error(DM_EINVAL, "NULL argument to dm_submit_cols");
  const Plan& p = plan->plan;
  if (p.cplx || p.top.nsys != 1) return set_error(DM_EINVAL, "dm_submit_cols needs a real single-system plan");
  const int R = p.top.spec[0].r;
  if (ncols < 1 || ncols > R) return set_error(DM_EINVAL, "ncols = %d outside 1..%d (the plan's nrhs)", ncols, R);
  Request r{0, plan, false, nullptr, nullptr, nullptr, b, x, ncols, 0.0};
  return Server::get().submit(r, ticket);
}

int dm_submit_system(dm_plan_t plan, const double* A, const double* B, const double* C, const double* b, double* x,
                     uint64_t* ticket) {
  if (!plan || !A || !B || !C || !b || !x || !ticket)
    return set_error(DM_EINVAL, "NULL argument to dm_submit_system");
  Request r{0, plan, true, A, B, C, b, x, 0, 0.0};
  return Server::get().submit(r, ticket);
}

int dm_serve_budget(double seconds) {
  if (!(seconds >= 0) || seconds > 1e6) return set_error(DM_EINVAL, "budget must be in [0, 1e6] seconds");
  return Server::get().set_budget(seconds);
}

int dm_serve_stats(long long* out) {
  if (!out) return set_error(DM_EINVAL, "NULL stats");
  Server::get().stats(out);
  return DM_OK;
}

int dm_poll(uint64_t ticket, int* status, double* relres_out) {
  if (!status) return set_error(DM_EINVAL, "NULL status");
  return Server::get().poll(ticket, status, relres_out, nullptr);
}

int dm_poll_times(uint64_t ticket, int* status, double* relres_out, double* times) {
  if (!status || !times) return set_error(DM_EINVAL, "NULL status or times");
  return Server::get().poll(ticket, status, relres_out, times);
}

int dm_serve_slots(int slots) { return Server::get().configure(slots); }

}  // extern "C"
