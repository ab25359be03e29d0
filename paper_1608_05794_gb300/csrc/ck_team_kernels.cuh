// Device code and launch helpers shared by the team-per-reactor kernels
// (one CTA per reactor): shared-memory carving, the reactor work queue, the
// forward-difference Jacobian, the error norm and the starting step of the
// integrators, and the occupancy-sized persistent grid.
#pragma once
#include <cuda_runtime.h>

#include "ck_internal.h"
#include "ck_team.cuh"

namespace ck {

static __host__ __device__ __forceinline__ int team_bufs_doubles(int S, int chunk) { return 9 * S + (3 + JP) * chunk + 48; }

static __device__ __forceinline__ TeamBufs carve_bufs(double* base, int S, int CH) {
  TeamBufs b;
  b.X = base;
  b.Gp = b.X + S;
  b.hRT = b.Gp + S;
  b.cpR = b.hRT + S;
  b.Gm = b.cpR + S;
  b.wd = b.Gm + S;
  b.aT = b.wd + S;
  b.E = b.aT + S;
  b.u = b.E + S;
  b.cs = b.Gp;  // column sums reuse Gp (free after the reaction passes)
  b.q = b.u + S;
  b.dqT = b.q + CH;
  b.D = b.dqT + CH;
  b.P = b.D + CH;
  b.red = b.P + (size_t)JP * CH;
  return b;
}

// Next reactor index for this CTA from the global queue (same in every thread).
static __device__ __forceinline__ int team_next(int32_t* queue, int* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
  __syncthreads();
  const int r = *slot;
  __syncthreads();
  return r;
}

// Forward-difference Jacobian (the paper's choice for ROS4, Sec. 5), with
// the increments of CVODE's dense difference quotients: unit roundoff U,
// weights w_i = 1/(atol + rtol |y_i|), fnorm = WRMS_w(f(y)), floor
// s0 = 1000 |h| U n fnorm (1 when fnorm = 0), and column j =
// (f(y + s_j e_j) - f(y)) / s_j with s_j = max(sqrt(U) |y_j|, s0 / w_j).
// f0 = f(y) is computed here (unless have_f0: the caller already holds it
// for this y) and reused as the first stage's f; the n columns cost n team
// RHS evaluations.  Yt, F: n-vector scratch.
static __device__ __noinline__ void team_jacobian_fd(const DevMech& d, const double* tab, double p,
                                                     const double* y, double h, double rtol, double atol,
                                                     double* f0, double* J, double* Yt, double* F, TeamBufs b,
                                                     bool have_f0 = false) {
  const int n = d.n;
  if (!have_f0) team_rhs(d, tab, p, y, f0, b);
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = f0[i] / (atol + rtol * fabs(y[i]));
    s = fma(v, v, s);
    Yt[i] = y[i];
  }
  const double fn = sqrt(team_sum(s, b.red) / n);
  const double U = 2.220446049250313080847e-16;  // 2^-52
  const double srur = 1.490116119384765625e-8;   // 2^-26 = sqrt(U)
  const double s0 = (fn != 0.0) ? 1000.0 * fabs(h) * U * n * fn : 1.0;
  for (int j = 0; j < n; ++j) {
    const double sj = fmax(srur * fabs(y[j]), s0 * (atol + rtol * fabs(y[j])));
    if (threadIdx.x == 0) Yt[j] = y[j] + sj;
    team_sync();
    team_rhs(d, tab, p, Yt, F, b);
    for (int i = threadIdx.x; i < n; i += blockDim.x) J[(size_t)i * n + j] = (F[i] - f0[i]) / sj;
    if (threadIdx.x == 0) Yt[j] = y[j];
    team_sync();
  }
}

// x^q, the step-size controller's power, by the first warp alone and handed
// to the others through red[37]: pow is long, and every warp that runs it
// pays all of its FP64 instructions.  x is the same in every thread; every
// thread must call it.
static __device__ __forceinline__ double team_pow(double x, double q, double* red) {
  if (blockDim.x == 32) return pow(x, q);
  if (threadIdx.x == 0) red[37] = pow(x, q);
  __syncthreads();
  return red[37];
}

// ------------------------------------------------------------------ ROS4
// Weighted RMS norm over the team (reading shared with the oracle:
// sqrt(mean (e_i / (atol + rtol max(|y_i|, |ynew_i|)))^2)).
static __device__ __forceinline__ double team_wrms(int n, const double* e, const double* y0,
                                            const double* y1, double rtol, double atol, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double sc = atol + rtol * fmax(fabs(y0[i]), fabs(y1[i]));
    const double v = e[i] / sc;
    s = fma(v, v, s);
  }
  s = team_sum(s, red);
  return sqrt(s / n);
}

// Initial step, Hairer-Norsett-Wanner starting-step algorithm (order 4).
static __device__ double team_h0(const DevMech& d, const double* tab, double p, const double* y0, double tspan,
                          double rtol, double atol, double* f0, double* y1, double* f1, TeamBufs& b,
                          Mix& x) {
  const int n = d.n;
  team_rhs(d, tab, p, y0, f0, b);
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double sc = atol + rtol * fabs(y0[i]);
    s0 = fma(y0[i] / sc, y0[i] / sc, s0);
    s1 = fma(f0[i] / sc, f0[i] / sc, s1);
  }
  const double d0 = sqrt(team_sum(s0, b.red) / n);
  const double d1 = sqrt(team_sum(s1, b.red) / n);
  const double ha = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y1[i] = fma(ha, f0[i], y0[i]);
  team_sync();
  team_rhs(d, tab, p, y1, f1, b);
  double s2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double sc = atol + rtol * fabs(y0[i]);
    const double v = (f1[i] - f0[i]) / sc;
    s2 = fma(v, v, s2);
  }
  const double d2 = sqrt(team_sum(s2, b.red) / n) / ha;
  const double dm = fmax(d1, d2);
  const double hb = (dm <= 1e-15) ? fmax(1e-6, ha * 1e-3) : pow(0.01 / dm, 0.2);
  return fmin(fmin(100.0 * ha, hb), tspan);
}

// ------------------------------------------------------------------ launch helpers
// Persistent grid: as many CTAs of `kernel` as fit on every SM (or the
// caller's cap), at most one per work item.
template <class K>
static inline int team_grid(K kernel, int threads, size_t smem, int64_t work, const LaunchCfg& cfg) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
  int64_t g = (int64_t)per_sm * sm_count();
  if (work < g) g = work;
  return (int)(g < 1 ? 1 : g);
}

// Shared memory of one k_ros4 CTA for a mechanism of n = S + 1.
inline size_t ros4_smem_bytes(int n, int S, int chunk) {
  return sizeof(double) * ((size_t)n * n + 9 * (size_t)n + (n + 1) / 2 + team_bufs_doubles(S, chunk));
}

}  // namespace ck
