// Mixed batches: several groups of reactors, each on its own mechanism, in
// one call.  Every group runs as its own persistent work-queue kernel on a
// branch forked from the caller's stream, launched heaviest first at full
// occupancy: the CTAs of the next group take over SMs as soon as those of
// the previous one drain, so the tail of one group overlaps the start of the
// next instead of leaving SMs idle.  A caller may instead cap a group's
// resident CTAs per SM (opts.variant) to run groups side by side.  The fork /
// kernels / join sequence is captured once into a CUDA graph and replayed on
// later calls with the same arguments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <list>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ck.h"
#include "ck_internal.h"

namespace {

struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  int32_t* queues = nullptr;  // one work-queue counter per group
  int device = -1;
};

std::mutex g_mu;
std::list<GraphEntry> g_cache;  // most recently used first
constexpr size_t CACHE_MAX = 8;

void destroy(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  for (auto s : e.streams) cudaStreamDestroy(s);
  for (auto v : e.events) cudaEventDestroy(v);
  if (e.queues) cudaFree(e.queues);
}

std::vector<unsigned char> make_key(int method, int ng, const ck_group* g, int device, int flags) {
  std::vector<unsigned char> k(sizeof(int) * 4 + sizeof(ck_group) * ng);
  int head[4] = {method, ng, device, flags};
  std::memcpy(k.data(), head, sizeof(head));
  std::memcpy(k.data() + sizeof(head), g, sizeof(ck_group) * ng);
  return k;
}

// Estimated FP64 work of a group: reactors x cost of one step of the method.
double group_work(int method, const ck_group& g) {
  if (g.work_weight > 0.0) return g.work_weight;
  ck_work_counts w;
  ck_count_work(g.mech, &w);
  return (double)g.n * (method == 0 ? w.ros4_step_fp64 : w.rkf45_step_fp64);
}

cudaError_t launch_group(int method, const ck_group& g, int32_t* queue, cudaStream_t st, int ctas_per_sm) {
  const ck::HostMech& hm = g.mech->hm;
  const ck_solver_opts& o = g.opts;
  ck::SolverParams sp{o.rtol, o.atol, o.h0, o.fixed_h, o.max_steps, o.jac};
  ck::LaunchCfg cfg;
  cfg.precision = o.precision;
  cfg.ctas_per_sm = ctas_per_sm;
  cfg.grid_side = o.team;
  if (method == 0)
    return ck::launch_ros4(hm, g.n, g.p, g.y, g.dt, g.h_inout, sp, g.steps, g.status, queue, st, cfg, nullptr, 0,
                           true);
  const bool team = o.form == 2 || (o.form == 0 && (hm.S > 32 || g.n < (int64_t)4 * 128 * ck::sm_count()));
  if (team) return ck::launch_rkf45_team(hm, g.n, g.p, g.y, g.dt, g.h_inout, sp, g.steps, g.status, queue, st, cfg);
  return ck::launch_rkf45(hm, g.n, g.p, g.y, g.dt, g.h_inout, sp, g.steps, g.status, queue, st, cfg);
}

// Record the fork / kernels / join sequence on `st` (captured or not), in
// the given launch order; sequential: the kernels one after another on `st`.
cudaError_t record(int method, int ng, const ck_group* g, GraphEntry& e, cudaStream_t st,
                   const std::vector<int>& caps, const std::vector<int>& order, bool sequential) {
  if (sequential) {
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < ng && err == cudaSuccess; ++k)
      err = launch_group(method, g[order[k]], e.queues + order[k], st, caps[order[k]]);
    return err;
  }
  cudaError_t err = cudaEventRecord(e.events[0], st);
  for (int k = 0; k < ng && err == cudaSuccess; ++k) {
    const int i = order[k];
    err = cudaStreamWaitEvent(e.streams[i], e.events[0], 0);
    if (err == cudaSuccess) err = launch_group(method, g[i], e.queues + i, e.streams[i], caps[i]);
    if (err == cudaSuccess) err = cudaEventRecord(e.events[1 + i], e.streams[i]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, e.events[1 + i], 0);
  }
  return err;
}

}  // namespace

extern "C" {

int ck_integrate_groups(int32_t method, int32_t n_groups, const ck_group* groups, int32_t flags,
                        void* stream) {
  const bool use_graph = (flags & CK_GROUPS_GRAPH) != 0;
  const bool sequential = (flags & CK_GROUPS_SEQUENTIAL) != 0;
  if (flags & ~(CK_GROUPS_GRAPH | CK_GROUPS_SEQUENTIAL)) return ck::set_error(CK_EINVAL, "unknown flags");
  if (method != 0 && method != 1) return ck::set_error(CK_EINVAL, "method must be 0 (ROS4) or 1 (RKF45)");
  if (n_groups < 1 || n_groups > 16) return ck::set_error(CK_ERANGE, "n_groups must be in [1, 16]");
  if (!groups) return ck::set_error(CK_EINVAL, "groups is NULL");
  for (int i = 0; i < n_groups; ++i)
    if (groups[i].n < 1 || groups[i].n > CK_MAX_REACTORS)
      return ck::set_error(CK_ERANGE, "group " + std::to_string(i) + ": n must be in [1, CK_MAX_REACTORS = 2^30]");
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n_groups; ++i) {
    const ck_group& g = groups[i];
    if (!g.mech || !g.p || !g.y || !g.dt || !g.status)
      return ck::set_error(CK_EINVAL, "group " + std::to_string(i) + ": mech, p, y, dt, status required");
    if (g.mech->hm.device != dev) return ck::set_error(CK_EINVAL, "group mechanism loaded on another device");
    const ck_solver_opts& o = g.opts;
    if (!(o.rtol > 0.0) || !(o.atol > 0.0) || o.max_steps < 1 || o.precision < 0 || o.precision > 2 ||
        (o.precision && method != 0) || o.jac < 0 || o.jac > 1 || (o.jac && method != 0) || o.form < 0 || o.form > 2 || !(o.team == 0 || o.team == 8 || o.team == 16))
      return ck::set_error(CK_EINVAL, "group " + std::to_string(i) + ": invalid options");
    for (const void* ptr : {(const void*)g.p, (const void*)g.y, (const void*)g.dt, (const void*)g.status,
                            (const void*)g.steps, (const void*)g.h_inout}) {
      if (!ptr) continue;
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return ck::set_error(CK_EINVAL, "ck_integrate_groups takes device pointers only");
      }
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // heaviest group first; full occupancy unless the caller caps a group
  std::vector<double> w(n_groups);
  std::vector<int> caps(n_groups), order(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    w[i] = group_work(method, groups[i]);
    caps[i] = groups[i].opts.variant > 0 ? groups[i].opts.variant : 0;
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<unsigned char> key = make_key(method, n_groups, groups, dev, flags);
  auto it = g_cache.begin();
  for (; it != g_cache.end(); ++it)
    if (it->key == key) break;
  if (it != g_cache.end()) {
    g_cache.splice(g_cache.begin(), g_cache, it);
  } else {
    GraphEntry e;
    e.key = key;
    e.device = dev;
    cudaError_t err = cudaMalloc(&e.queues, sizeof(int32_t) * n_groups);
    e.streams.resize(n_groups, nullptr);
    e.events.resize(n_groups + 1, nullptr);
    for (int i = 0; i < n_groups && err == cudaSuccess; ++i)
      err = cudaStreamCreateWithFlags(&e.streams[i], cudaStreamNonBlocking);
    for (int i = 0; i <= n_groups && err == cudaSuccess; ++i)
      err = cudaEventCreateWithFlags(&e.events[i], cudaEventDisableTiming);
    if (err != cudaSuccess) {
      destroy(e);
      return ck::set_error(CK_ECUDA, std::string("ck_integrate_groups: ") + cudaGetErrorString(err));
    }
    g_cache.push_front(std::move(e));
    if (g_cache.size() > CACHE_MAX) {
      cudaDeviceSynchronize();
      destroy(g_cache.back());
      g_cache.pop_back();
    }
  }
  GraphEntry& e = g_cache.front();
  cudaError_t err = cudaSuccess;
  if (!use_graph) {
    err = record(method, n_groups, groups, e, st, caps, order, sequential);
  } else {
    if (!e.exec) {
      // capture on a private stream, so the caller's stream may be the legacy default
      cudaStream_t cap;
      err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (err == cudaSuccess) err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (err == cudaSuccess) {
        cudaError_t rec = record(method, n_groups, groups, e, cap, caps, order, sequential);
        err = cudaStreamEndCapture(cap, &e.graph);
        if (rec != cudaSuccess) err = rec;
      }
      if (err == cudaSuccess) err = cudaGraphInstantiate(&e.exec, e.graph, 0);
      cudaStreamDestroy(cap);
      if (err != cudaSuccess) {
        cudaGetLastError();
        return ck::set_error(CK_ECUDA, std::string("graph capture: ") + cudaGetErrorString(err));
      }
    }
    err = cudaGraphLaunch(e.exec, st);
  }
  if (err != cudaSuccess) return ck::set_error(CK_ECUDA, std::string("ck_integrate_groups: ") + cudaGetErrorString(err));
  return CK_OK;
}

int ck_graph_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  for (auto& e : g_cache) destroy(e);
  g_cache.clear();
  return CK_OK;
}

}  // extern "C"
