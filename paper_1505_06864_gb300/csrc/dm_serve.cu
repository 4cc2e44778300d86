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
#include <cuda_runtime.h>

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

struct Request {
  uint64_t ticket;
  dm_plan_t plan;
  bool factor;
  const double *A, *B, *C, *b;
  double* x;
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
    if ((int)queue_.size() >= kMaxQueue) return set_error(DM_EAGAIN, "serving queue full (%d requests)", kMaxQueue);
    Request r = r0;
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

  void worker() {
    // one stream per device this worker has served; the plan's device is
    // made current before any of its work (plans may live on any device)
    std::unordered_map<int, cudaStream_t> streams;
    for (;;) {
      Request r;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return pick_locked(&r); });
        outcomes_[r.ticket].t_start = now_s();
      }
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
      if (rc == DM_OK) p.stream = st;
      if (rc == DM_OK && r.factor) rc = p.factor(r.A, r.B, r.C);
      double rel = 0.0;
      if (rc == DM_OK) {
        std::vector<double> rr(std::max(1, p.top.nsys));
        rc = p.solve(r.b, r.x, rr.data());
        rel = rr[0];
        for (double v : rr) rel = std::max(rel, v);
      }
      p.stream = keep;
      {
        std::lock_guard<std::mutex> lk(mu_);
        Outcome& o = outcomes_[r.ticket];
        o.done = true;
        o.status = rc;
        if (rc != DM_OK) o.msg = g_last_error;
        o.relres = rel;
        o.t_done = now_s();
        busy_.erase(r.plan);
        pending_[r.plan] -= 1;
      }
      cv_.notify_all();
      done_cv_.notify_all();
    }
  }

  // Oldest queued request whose plan is idle.
  bool pick_locked(Request* out) {
    for (auto it = queue_.begin(); it != queue_.end(); ++it) {
      if (busy_.count(it->plan)) continue;
      *out = *it;
      busy_.insert({it->plan, true});
      queue_.erase(it);
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
  uint64_t next_ticket_ = 0;
  bool started_ = false;
  int slots_ = 8;
};

}  // namespace

void serve_drain(dm_plan_t plan) { Server::get().drain(plan); }

}  // namespace dm

using namespace dm;

extern "C" {

int dm_submit(dm_plan_t plan, const double* b, double* x, uint64_t* ticket) {
  if (!plan || !b || !x || !ticket) return set_error(DM_EINVAL, "NULL argument to dm_submit");
  Request r{0, plan, false, nullptr, nullptr, nullptr, b, x};
  return Server::get().submit(r, ticket);
}

int dm_submit_system(dm_plan_t plan, const double* A, const double* B, const double* C, const double* b, double* x,
                     uint64_t* ticket) {
  if (!plan || !A || !B || !C || !b || !x || !ticket)
    return set_error(DM_EINVAL, "NULL argument to dm_submit_system");
  Request r{0, plan, true, A, B, C, b, x};
  return Server::get().submit(r, ticket);
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
