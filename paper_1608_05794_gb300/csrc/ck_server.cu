// Request server: continuous batching of reactor batches on one GPU.
//
// Requests (a batch of reactors on one mechanism, ROS4 or RKF45) are admitted
// in arrival order while their device footprint fits the HBM budget; an
// admitted request is split into chunks of reactors, and a dispatcher thread
// launches chunks on a pool of streams, each free stream taking the next
// chunk of the admitted request with the least estimated remaining work
// (reactors left x FP64 cost of one step of its method, from ck_count_work):
// short requests overtake long ones, which cuts the median latency; a request
// admitted more than STARVE_S seconds ago goes first, so none waits forever.
// A request that arrives while others run therefore starts at once, its
// kernels overlap those of earlier requests on the device, and finished
// requests release memory for queued ones.  Every reactor is integrated
// independently of its neighbours, so a request's results do not depend on
// what else is in flight.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ck.h"
#include "ck_internal.h"

namespace {

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_COPYBACK = 2, Q_DONE = 3, Q_FAILED = 4, Q_CANCELLED = 5 };

struct Request {
  uint64_t ticket = 0;
  const ck_mech* mech = nullptr;
  int method = 0;
  int64_t n = 0;
  const double* p = nullptr;
  double* y = nullptr;
  const double* dt = nullptr;
  int32_t* status = nullptr;
  int32_t* steps = nullptr;
  ck_solver_opts opts{};
  bool host = false;
  size_t bytes = 0;
  void* block = nullptr;  // staging allocation (host requests)
  const double* dp = nullptr;
  double* dy = nullptr;
  const double* ddt = nullptr;
  int32_t* dst = nullptr;
  int32_t* dsteps = nullptr;
  int64_t next = 0;        // first reactor of the next chunk
  int chunks_total = 0, chunks_launched = 0, chunks_done = 0;
  double step_cost = 0.0;  // FP64 instructions of one step of one reactor
  std::chrono::steady_clock::time_point admitted;
  int state = Q_QUEUED;
  int err = CK_OK;
  std::string msg;
  cudaEvent_t ready = nullptr;  // inputs on the device
  cudaEvent_t back = nullptr;   // outputs copied back
  cudaStream_t home = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int32_t* queue = nullptr;  // device work-queue counter of this slot
  double* scratch = nullptr; // ROS4 per-CTA matrices of this slot's launches
  size_t scratch_bytes = 0;
  Request* req = nullptr;
};

bool host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

size_t per_reactor_bytes(int nn) { return (size_t)nn * 8 + 8 + 8 + 4 + 8; }

// A request admitted longer ago than this is served before shorter ones.
constexpr double STARVE_S = 30.0;

}  // namespace

struct ck_server {
  int device = 0;
  size_t budget = 0, in_use = 0, reserved = 0;  // in_use includes the reserved slot scratch
  int64_t chunk = 8192;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;     // wakes the dispatcher
  std::condition_variable done_cv;  // wakes waiters
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int64_t completed = 0;
};

namespace {

int srv_fail(int code, const std::string& msg);

void fail_req(ck_server* s, Request* r, int code, const std::string& m) {
  r->err = code;
  r->msg = m;
  r->state = Q_FAILED;
  s->done_cv.notify_all();
}

// Admit queued requests in arrival order while they fit the budget.
void admit(ck_server* s) {
  while (!s->queue.empty()) {
    Request* r = s->queue.front();
    if (r->state == Q_CANCELLED) {
      s->queue.pop_front();
      continue;
    }
    if (s->in_use + r->bytes > s->budget) break;
    s->queue.pop_front();
    s->in_use += r->bytes;
    const int nn = r->mech->hm.d.n;
    cudaError_t e = cudaSuccess;
    if (r->host) {
      e = cudaMallocAsync(&r->block, r->bytes, r->home);
      if (e == cudaSuccess) {
        unsigned char* b = static_cast<unsigned char*>(r->block);
        r->dy = reinterpret_cast<double*>(b);
        b += (size_t)r->n * nn * 8;
        r->dp = reinterpret_cast<double*>(b);
        b += (size_t)r->n * 8;
        r->ddt = reinterpret_cast<double*>(b);
        b += (size_t)r->n * 8;
        r->dsteps = reinterpret_cast<int32_t*>(b);
        b += (size_t)r->n * 8;
        r->dst = reinterpret_cast<int32_t*>(b);
        e = cudaMemcpyAsync(r->dy, r->y, (size_t)r->n * nn * 8, cudaMemcpyHostToDevice, r->home);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(const_cast<double*>(r->dp), r->p, (size_t)r->n * 8, cudaMemcpyHostToDevice, r->home);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(const_cast<double*>(r->ddt), r->dt, (size_t)r->n * 8, cudaMemcpyHostToDevice,
                              r->home);
      }
    } else {
      r->dy = r->y;
      r->dp = r->p;
      r->ddt = r->dt;
      r->dst = r->status;
      r->dsteps = r->steps;
    }
    if (e == cudaSuccess) e = cudaEventRecord(r->ready, r->home);
    if (e != cudaSuccess) {
      if (r->block) {
        cudaFreeAsync(r->block, r->home);
        r->block = nullptr;
      }
      s->in_use -= r->bytes;
      fail_req(s, r, CK_ECUDA, std::string("admission: ") + cudaGetErrorString(e));
      continue;
    }
    r->chunks_total = (int)((r->n + s->chunk - 1) / s->chunk);
    r->state = Q_RUNNING;
    r->admitted = std::chrono::steady_clock::now();
    s->active.push_back(r);
  }
}

void launch_chunk(ck_server* s, Slot& sl, Request* r) {
  const int64_t start = r->next;
  const int64_t cnt = std::min<int64_t>(s->chunk, r->n - start);
  r->next += cnt;
  r->chunks_launched++;
  sl.req = r;
  const ck::HostMech& hm = r->mech->hm;
  const int nn = hm.d.n;
  ck::SolverParams sp{r->opts.rtol, r->opts.atol, r->opts.h0, r->opts.fixed_h, r->opts.max_steps, r->opts.jac};
  ck::LaunchCfg cfg;
  cfg.precision = r->opts.precision;
  cfg.grid_side = r->opts.team;
  if (r->opts.variant > 0) cfg.ctas_per_sm = r->opts.variant;
  cudaError_t e = cudaStreamWaitEvent(sl.stream, r->ready, 0);
  if (e == cudaSuccess) {
    const double* pp = r->dp + start;
    double* yy = r->dy + start * nn;
    const double* tt = r->ddt + start;
    int32_t* ss = r->dsteps ? r->dsteps + 2 * start : nullptr;
    int32_t* st = r->dst + start;
    if (r->method == 0)
      e = ck::launch_ros4(hm, cnt, pp, yy, tt, nullptr, sp, ss, st, sl.queue, sl.stream, cfg, sl.scratch,
                          sl.scratch_bytes, false);
    else if (r->opts.form == 1)
      e = ck::launch_rkf45(hm, cnt, pp, yy, tt, nullptr, sp, ss, st, sl.queue, sl.stream, cfg);
    else
      e = ck::launch_rkf45_team(hm, cnt, pp, yy, tt, nullptr, sp, ss, st, sl.queue, sl.stream, cfg);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
  if (e != cudaSuccess) fail_req(s, r, CK_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
}

void finish_request(ck_server* s, Request* r) {
  const int nn = r->mech->hm.d.n;
  cudaError_t e = cudaSuccess;
  if (r->host) {
    e = cudaMemcpyAsync(r->y, r->dy, (size_t)r->n * nn * 8, cudaMemcpyDeviceToHost, r->home);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->status, r->dst, (size_t)r->n * 4, cudaMemcpyDeviceToHost, r->home);
    if (e == cudaSuccess && r->steps)
      e = cudaMemcpyAsync(r->steps, r->dsteps, (size_t)r->n * 8, cudaMemcpyDeviceToHost, r->home);
    if (e == cudaSuccess) {
      e = cudaFreeAsync(r->block, r->home);
      r->block = nullptr;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(r->back, r->home);
  if (e != cudaSuccess) {
    fail_req(s, r, CK_ECUDA, std::string("copy-back: ") + cudaGetErrorString(e));
    return;
  }
  r->state = Q_COPYBACK;
}

void dispatcher(ck_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    admit(s);
    // retire finished chunks
    for (auto& sl : s->slots) {
      if (!sl.req) continue;
      cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      Request* r = sl.req;
      sl.req = nullptr;
      progress = true;
      if (q != cudaSuccess) {
        cudaGetLastError();
        fail_req(s, r, CK_ECUDA, std::string("chunk: ") + cudaGetErrorString(q));
        continue;
      }
      if (r->state == Q_RUNNING && ++r->chunks_done == r->chunks_total) finish_request(s, r);
    }
    // launch chunks: least remaining work first, starving requests before all
    const auto now = std::chrono::steady_clock::now();
    for (auto& sl : s->slots) {
      if (sl.req) continue;
      Request* pick = nullptr;
      bool pick_old = false;
      double pick_work = 0.0;
      for (Request* r : s->active) {
        if (r->state != Q_RUNNING || r->chunks_launched >= r->chunks_total) continue;
        const bool old = std::chrono::duration<double>(now - r->admitted).count() > STARVE_S;
        const double work = (double)(r->n - r->next) * r->step_cost;
        const bool better = !pick || (old && !pick_old) ||
                            (old == pick_old && (old ? r->admitted < pick->admitted
                                                     : work < pick_work || (work == pick_work && r->ticket < pick->ticket)));
        if (better) {
          pick = r;
          pick_old = old;
          pick_work = work;
        }
      }
      if (!pick) break;
      launch_chunk(s, sl, pick);
      progress = true;
    }
    // completed copy-backs release their memory
    for (size_t k = 0; k < s->active.size();) {
      Request* r = s->active[k];
      bool drop = false;
      if (r->state == Q_COPYBACK) {
        cudaError_t q = cudaEventQuery(r->back);
        if (q == cudaSuccess) {
          r->state = Q_DONE;
          s->completed++;
          drop = true;
        } else if (q != cudaErrorNotReady) {
          cudaGetLastError();
          fail_req(s, r, CK_ECUDA, std::string("copy-back: ") + cudaGetErrorString(q));
          drop = true;
        }
      } else if (r->state == Q_FAILED || r->state == Q_CANCELLED) {
        bool busy = false;
        for (auto& sl : s->slots) busy |= (sl.req == r);
        drop = !busy;
        if (drop && r->block) {
          // a failed host request still holds its staging block
          cudaFreeAsync(r->block, r->home);
          r->block = nullptr;
        }
      }
      if (drop) {
        s->in_use -= r->bytes;
        s->active.erase(s->active.begin() + k);
        s->done_cv.notify_all();
        progress = true;
      } else {
        ++k;
      }
    }
    if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

int srv_fail(int code, const std::string& msg) { return ck::set_error(code, msg.c_str()); }

}  // namespace

extern "C" {

int ck_server_create(size_t hbm_budget_bytes, int32_t streams, int64_t chunk_reactors, ck_server** out) {
  if (!out) return srv_fail(CK_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return srv_fail(CK_EINVAL, "hbm_budget_bytes must be positive");
  if (streams < 1 || streams > 64) return srv_fail(CK_ERANGE, "streams must be in [1, 64]");
  // every slot holds the ROS4 scratch of its launches for the server's
  // lifetime (the largest any mechanism can need), inside the budget
  const size_t per_slot = ck::ros4_scratch_bytes_max();
  const size_t reserved = per_slot * (size_t)streams;
  if (per_slot == 0) return srv_fail(CK_ECUDA, "no current CUDA device");
  if (hbm_budget_bytes <= reserved)
    return srv_fail(CK_ERANGE, "hbm_budget_bytes must exceed the " + std::to_string(reserved) +
                                   " bytes of solver scratch that " + std::to_string(streams) +
                                   " streams reserve (" + std::to_string(per_slot) + " each)");
  ck_server* s = new ck_server;
  s->budget = hbm_budget_bytes;
  s->reserved = reserved;
  s->in_use = reserved;
  if (chunk_reactors > 0) s->chunk = chunk_reactors;
  cudaGetDevice(&s->device);
  s->slots.resize(streams);
  for (auto& sl : s->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.queue, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&sl.scratch, per_slot);
    sl.scratch_bytes = per_slot;
    if (e != cudaSuccess) {
      for (auto& q : s->slots) {
        if (q.stream) cudaStreamDestroy(q.stream);
        if (q.ev) cudaEventDestroy(q.ev);
        if (q.queue) cudaFree(q.queue);
        if (q.scratch) cudaFree(q.scratch);
      }
      delete s;
      return srv_fail(e == cudaErrorMemoryAllocation ? CK_ENOMEM : CK_ECUDA,
                      std::string("server streams: ") + cudaGetErrorString(e));
    }
  }
  s->worker = std::thread(dispatcher, s);
  *out = s;
  return CK_OK;
}

int ck_submit(ck_server* s, const ck_mech* mech, int32_t method, int64_t n, const double* p, double* y,
              const double* dt, const ck_solver_opts* opts, int32_t* status, int32_t* steps,
              uint64_t* ticket) {
  if (n < 1 || n > CK_MAX_REACTORS) return srv_fail(CK_ERANGE, "n must be in [1, CK_MAX_REACTORS = 2^30]");
  if (!s || !mech || !ticket) return srv_fail(CK_EINVAL, "server, mech and ticket are required");
  if (method != 0 && method != 1) return srv_fail(CK_EINVAL, "method must be 0 (ROS4) or 1 (RKF45)");
  if (!p || !y || !dt || !status) return srv_fail(CK_EINVAL, "p, y, dt and status are required");
  Request* r = new Request;
  r->mech = mech;
  r->method = method;
  r->n = n;
  r->p = p;
  r->y = y;
  r->dt = dt;
  r->status = status;
  r->steps = steps;
  if (opts) r->opts = *opts;
  else ck_default_opts(&r->opts);
  if ((r->opts.precision != 0 || r->opts.jac != 0) && method != 0) {
    delete r;
    return srv_fail(CK_EINVAL, "opts.precision and opts.jac apply to ROS4 only");
  }
  if (r->opts.jac < 0 || r->opts.jac > 1) {
    delete r;
    return srv_fail(CK_EINVAL, "opts.jac must be 0 or 1");
  }
  const bool h = host_ptr(p) || host_ptr(y) || host_ptr(dt) || host_ptr(status) || host_ptr(steps);
  const bool d = !host_ptr(p) && !host_ptr(y) && !host_ptr(dt) && !host_ptr(status) && !host_ptr(steps);
  if (!h == !d) {
    delete r;
    return srv_fail(CK_EINVAL, "a request's arrays must be all host or all device memory");
  }
  r->host = h;
  r->bytes = per_reactor_bytes(mech->hm.d.n) * (size_t)n;
  ck_work_counts wc;
  ck_count_work(mech, &wc);
  r->step_cost = method == 0 ? wc.ros4_step_fp64 : wc.rkf45_step_fp64;
  if (r->bytes > s->budget - s->reserved) {
    delete r;
    return srv_fail(CK_AGAIN, "request needs " + std::to_string(per_reactor_bytes(mech->hm.d.n) * n) +
                                  " bytes, more than the server's HBM budget leaves beside its reserved scratch");
  }
  cudaError_t e = cudaStreamCreateWithFlags(&r->home, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->back, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (r->home) cudaStreamDestroy(r->home);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
    return srv_fail(CK_ECUDA, std::string("submit: ") + cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv.notify_one();
  return CK_OK;
}

int ck_poll(ck_server* s, uint64_t ticket, int32_t* state) {
  if (!s || !state) return srv_fail(CK_EINVAL, "server and state are required");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(CK_EINVAL, "unknown ticket");
  Request* r = it->second;
  *state = r->state == Q_DONE ? 1 : (r->state == Q_FAILED ? 2 : (r->state == Q_CANCELLED ? 3 : 0));
  if (r->state == Q_FAILED) return srv_fail(r->err, r->msg);
  return CK_OK;
}

int ck_wait(ck_server* s, uint64_t ticket, double timeout_s) {
  if (!s) return srv_fail(CK_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(CK_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state != Q_DONE && r->state != Q_FAILED && r->state != Q_CANCELLED) {
    if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout &&
        std::chrono::steady_clock::now() >= until)
      return srv_fail(CK_TIMEOUT, "request not finished within the timeout");
  }
  if (r->state == Q_FAILED) return srv_fail(r->err, r->msg);
  return CK_OK;
}

int ck_cancel(ck_server* s, uint64_t ticket) {
  if (!s) return srv_fail(CK_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(CK_EINVAL, "unknown ticket");
  if (it->second->state != Q_QUEUED) return srv_fail(CK_AGAIN, "only queued requests can be cancelled");
  it->second->state = Q_CANCELLED;
  s->done_cv.notify_all();
  return CK_OK;
}

int ck_release(ck_server* s, uint64_t ticket) {
  if (!s) return srv_fail(CK_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(CK_EINVAL, "unknown ticket");
  Request* r = it->second;
  if (r->state != Q_DONE && r->state != Q_FAILED && r->state != Q_CANCELLED)
    return srv_fail(CK_AGAIN, "request still in flight");
  for (auto& sl : s->slots)
    if (sl.req == r) return srv_fail(CK_AGAIN, "request still in flight");
  for (auto* a : s->active)
    if (a == r) return srv_fail(CK_AGAIN, "request still in flight");
  cudaStreamDestroy(r->home);
  cudaEventDestroy(r->ready);
  cudaEventDestroy(r->back);
  s->all.erase(it);
  delete r;
  return CK_OK;
}

int ck_server_stats(ck_server* s, ck_server_info* out) {
  if (!s || !out) return srv_fail(CK_EINVAL, "server and out are required");
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int64_t)s->queue.size();
  out->active = (int64_t)s->active.size();
  out->completed = s->completed;
  out->bytes_in_use = s->in_use;
  out->budget = s->budget;
  out->reserved = s->reserved;
  return CK_OK;
}

int ck_server_destroy(ck_server* s) {
  if (!s) return CK_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->worker.join();
  for (auto& sl : s->slots) cudaStreamSynchronize(sl.stream);
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->home) {
      cudaStreamSynchronize(r->home);
      if (r->block) cudaFree(r->block);
      cudaStreamDestroy(r->home);
    }
    if (r->ready) cudaEventDestroy(r->ready);
    if (r->back) cudaEventDestroy(r->back);
    delete r;
  }
  for (auto& sl : s->slots) {
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.ev);
    cudaFree(sl.queue);
    cudaFree(sl.scratch);
  }
  delete s;
  return CK_OK;
}

}  // extern "C"
