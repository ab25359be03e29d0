// Team-per-reactor kernels: analytic and forward-difference Jacobians,
// batched dense LU / solve and RKF45 with one CTA per reactor, and the
// dispatch of the ROS4 integrator (its kernels live in ck_ros4_*.cu).  CTAs
// pull reactors from a global atomic counter (dynamic scheduling,
// granularity one reactor).
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "ck_team_kernels.cuh"

namespace ck {

// ------------------------------------------------------------------ Jacobian
__global__ void k_jacobian(const __grid_constant__ DevMech d, int64_t N, const double* __restrict__ p,
                           const double* __restrict__ y, double* __restrict__ jac) {
  extern __shared__ __align__(16) double sm[];
  const int n = d.n;
  double* J = sm;
  double* ys = J + (size_t)n * n;
  double* fs = ys + n;
  TeamBufs b = carve_bufs(fs + n, d.S, d.chunk);
  Mix x;
  for (int64_t r = blockIdx.x; r < N; r += gridDim.x) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = y[r * n + i];
    __syncthreads();
    team_jacobian(d, d.tab, p[r], ys, fs, J, b, x);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) jac[r * (int64_t)n * n + e] = J[e];
    __syncthreads();
  }
}

// Forward-difference Jacobians (one CTA per reactor), as ROS4 builds them
// with the forward-difference option at step size h[r].
__global__ void k_jacobian_fd(const __grid_constant__ DevMech d, int64_t N, const double* __restrict__ p,
                              const double* __restrict__ y, const double* __restrict__ h, double rtol,
                              double atol, double* __restrict__ jac) {
  extern __shared__ __align__(16) double sm[];
  const int n = d.n;
  double* J = sm;
  double* ys = J + (size_t)n * n;
  double* fs = ys + n;
  double* yt = fs + n;
  double* ft = yt + n;
  TeamBufs b = carve_bufs(ft + n, d.S, d.chunk);
  for (int64_t r = blockIdx.x; r < N; r += gridDim.x) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = y[r * n + i];
    __syncthreads();
    team_jacobian_fd(d, d.tab, p[r], ys, h[r], rtol, atol, fs, J, yt, ft, b);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) jac[r * (int64_t)n * n + e] = J[e];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ batched LU
template <int G, int T>
__global__ void __launch_bounds__(G * G, 1) k_lu_factor(int64_t batch, int dim, double* __restrict__ a,
                                                      int32_t* __restrict__ piv, int32_t* __restrict__ info) {
  extern __shared__ __align__(16) double sm[];
  double* A = sm;
  double* invd = A + (size_t)dim * dim;
  int* pv = reinterpret_cast<int*>(invd + dim);
  double* scratch = invd + 2 * dim;  // lu_scratch_words<G, T>() doubles
  const int64_t nn = (int64_t)dim * dim;
  for (int64_t m = blockIdx.x; m < batch; m += gridDim.x) {
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) A[e] = a[m * nn + e];
    __syncthreads();
    const int inf = lu_reg<G, T>(A, dim, pv, invd, scratch);
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) a[m * nn + e] = A[e];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) piv[m * dim + i] = pv[i];
    if (threadIdx.x == 0) info[m] = inf;
    __syncthreads();
  }
}

__global__ void k_lu_solve(int64_t batch, int dim, const double* __restrict__ lu,
                           const int32_t* __restrict__ piv, double* __restrict__ bvec) {
  extern __shared__ __align__(16) double sm[];
  double* A = sm;
  double* invd = A + (size_t)dim * dim;
  int* pv = reinterpret_cast<int*>(invd + dim);
  double* x = invd + 2 * dim;
  const int64_t nn = (int64_t)dim * dim;
  for (int64_t m = blockIdx.x; m < batch; m += gridDim.x) {
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) A[e] = lu[m * nn + e];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      pv[i] = piv[m * dim + i];
      x[i] = bvec[m * dim + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < dim; i += blockDim.x) invd[i] = rcp_rn(A[(size_t)i * dim + i]);
    __syncthreads();
    if (threadIdx.x < 32) warp_lu_solve(A, dim, pv, invd, x);
    __syncthreads();
    for (int i = threadIdx.x; i < dim; i += blockDim.x) bvec[m * dim + i] = x[i];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ RKF45 (team)
// RKF45 with one CTA per reactor (the paper's "deep" form): the six stage
// right-hand sides are evaluated by the team, so a reactor's working set
// (8 n-vectors and one chunk of reaction scratch) stays in shared memory and
// the number of steps of one reactor never holds back another.
__global__ void __launch_bounds__(64) k_rkf45_team(const __grid_constant__ DevMech d, int64_t N, const double* __restrict__ p,
                                                   double* __restrict__ y, const double* __restrict__ dt,
                                                   double* h_io, SolverParams sp, int32_t* steps,
                                                   int32_t* status, int32_t* queue) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int slot;
  const int n = d.n;
  double* yv = sm;
  double* yt = yv + n;
  double* kk = yt + n;  // six stages, n each
  TeamBufs b = carve_bufs(kk + 6 * n, d.S, d.chunk);
  Mix x;
  const bool fixed = sp.fixed_h > 0.0;
  const int tid = threadIdx.x, P = blockDim.x;
  double* k0 = kk;
  double* k1 = kk + n;
  double* k2 = kk + 2 * n;
  double* k3 = kk + 3 * n;
  double* k4 = kk + 4 * n;
  double* k5 = kk + 5 * n;
  for (;;) {
    const int r = team_next(queue, &slot);
    if (r >= N) break;
    for (int i = tid; i < n; i += P) yv[i] = y[(int64_t)r * n + i];
    const double pr = p[r];
    const double tf = dt[r];
    __syncthreads();
    int bad = 0;
    for (int i = tid; i < n; i += P) bad |= !isfinite(yv[i]);
    bad = __syncthreads_or(bad);
    bad |= !(pr > 0.0) || !isfinite(pr) || !(yv[0] > 0.0) || !isfinite(tf) || !(tf >= 0.0);
    int st = ST_OK, acc = 0, rej = 0;
    double h = 0.0;
    if (bad) {
      st = ST_BADINPUT;
    } else if (tf > 0.0) {
      if (fixed) h = sp.fixed_h;
      else if (h_io && h_io[r] > 0.0) h = h_io[r];
      else if (sp.h0 > 0.0) h = sp.h0;
      else h = team_h0(d, d.tab, pr, yv, tf, sp.rtol, sp.atol, k0, yt, k1, b, x);
      const double hmin = 1e-15 * tf;
      double t = 0.0;
      bool last_rej = false, last_nf = false;
      while (t < tf) {
        if (acc + rej >= sp.max_steps) { st = ST_MAXSTEPS; break; }
        const bool clamped = h >= tf - t;
        const double hh = clamped ? tf - t : h;
        if (hh < hmin) { st = last_nf ? ST_NONFINITE : ST_HMIN; break; }
        // k_s = hh f(y + sum_j a_sj k_j)
        team_rhs(d, d.tab, pr, yv, k0, b);
        for (int i = tid; i < n; i += P) {
          k0[i] *= hh;
          yt[i] = fma(RK_A21, k0[i], yv[i]);
        }
        team_sync();
        team_rhs(d, d.tab, pr, yt, k1, b);
        for (int i = tid; i < n; i += P) {
          k1[i] *= hh;
          yt[i] = fma(RK_A32, k1[i], fma(RK_A31, k0[i], yv[i]));
        }
        team_sync();
        team_rhs(d, d.tab, pr, yt, k2, b);
        for (int i = tid; i < n; i += P) {
          k2[i] *= hh;
          yt[i] = fma(RK_A43, k2[i], fma(RK_A42, k1[i], fma(RK_A41, k0[i], yv[i])));
        }
        team_sync();
        team_rhs(d, d.tab, pr, yt, k3, b);
        for (int i = tid; i < n; i += P) {
          k3[i] *= hh;
          yt[i] = fma(RK_A54, k3[i], fma(RK_A53, k2[i], fma(RK_A52, k1[i], fma(RK_A51, k0[i], yv[i]))));
        }
        team_sync();
        team_rhs(d, d.tab, pr, yt, k4, b);
        for (int i = tid; i < n; i += P) {
          k4[i] *= hh;
          yt[i] = fma(RK_A65, k4[i],
                      fma(RK_A64, k3[i], fma(RK_A63, k2[i], fma(RK_A62, k1[i], fma(RK_A61, k0[i], yv[i])))));
        }
        team_sync();
        team_rhs(d, d.tab, pr, yt, k5, b);
        // y* = y + sum b k (into yt), e = sum (bh - b) k (into k1, whose weights are 0)
        int nf = 0;
        for (int i = tid; i < n; i += P) {
          k5[i] *= hh;
          const double yn =
              fma(RK_B5, k4[i], fma(RK_B4, k3[i], fma(RK_B3, k2[i], fma(RK_B1, k0[i], yv[i]))));
          k1[i] = fma(RK_D6, k5[i], fma(RK_D5, k4[i], fma(RK_D4, k3[i], fma(RK_D3, k2[i], RK_D1 * k0[i]))));
          yt[i] = yn;
          nf |= !isfinite(yn);
        }
        nf = __syncthreads_or(nf);
        if (fixed) {
          for (int i = tid; i < n; i += P) yv[i] = yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          continue;
        }
        const double e = team_wrms(n, k1, yv, yt, sp.rtol, sp.atol, b.red);
        if (nf || !isfinite(e)) {
          ++rej;
          h = FAC_MIN * hh;
          last_rej = true;
          last_nf = true;
          continue;
        }
        last_nf = false;
        const double pe = (e == 0.0) ? 0.0 : team_pow(e, -0.2, b.red);
        if (e < 1.0) {
          for (int i = tid; i < n; i += P) yv[i] = yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          double fac = (e == 0.0) ? FAC_MAX : fmin(FAC_MAX, fmax(FAC_MIN, SAFETY * pe));
          if (last_rej) fac = fmin(1.0, fac);
          h = hh * fac;
          last_rej = false;
        } else {
          ++rej;
          h = hh * fmax(FAC_MIN, SAFETY * pe);
          last_rej = true;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += P) y[(int64_t)r * n + i] = yv[i];
    if (tid == 0) {
      if (h_io && st != ST_BADINPUT && tf > 0.0) h_io[r] = h;
      if (steps) {
        steps[2 * (int64_t)r] = acc;
        steps[2 * (int64_t)r + 1] = rej;
      }
      status[r] = st;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ launchers
static int team_threads(int n, const LaunchCfg& cfg) {
  int w = cfg.team_warps;
  if (w <= 0) w = (n <= 24) ? 1 : (n <= 64 ? 2 : 4);
  if (w > 8) w = 8;
  return 32 * w;
}


// Thread grid of the register-tiled LU for dimension n: G x G threads with
// T x T tiles (n <= G T).
template <class F>
static cudaError_t with_grid(int n, F f, int side = 0) {
  if (side == 16 && n <= 112) return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 7>{});
  if (n <= 56) return f(std::integral_constant<int, 8>{}, std::integral_constant<int, 7>{});
  if (n <= 112) return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 7>{});
  if (n <= 144) return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 9>{});
  return cudaErrorInvalidValue;
}
cudaError_t launch_jacobian(const HostMech& hm, int64_t n, const double* p, const double* y,
                            double* jac, cudaStream_t st, const LaunchCfg& cfg) {
  if (n <= 0) return cudaSuccess;
  const int nn = hm.d.n;
  const size_t smem = sizeof(double) * ((size_t)nn * nn + 2 * nn + team_bufs_doubles(hm.S, hm.d.chunk));
  const int threads = hm.d.chunk;
  const int grid = team_grid(k_jacobian, threads, smem, n, cfg);
  k_jacobian<<<grid, threads, smem, st>>>(hm.d, n, p, y, jac);
  return cudaGetLastError();
}

cudaError_t launch_jacobian_fd(const HostMech& hm, int64_t n, const double* p, const double* y, const double* h,
                               double rtol, double atol, double* jac, cudaStream_t st, const LaunchCfg& cfg) {
  if (n <= 0) return cudaSuccess;
  const int nn = hm.d.n;
  const size_t smem = sizeof(double) * ((size_t)nn * nn + 4 * nn + team_bufs_doubles(hm.S, hm.d.chunk));
  const int threads = hm.d.chunk;
  const int grid = team_grid(k_jacobian_fd, threads, smem, n, cfg);
  k_jacobian_fd<<<grid, threads, smem, st>>>(hm.d, n, p, y, h, rtol, atol, jac);
  return cudaGetLastError();
}

cudaError_t launch_lu_factor(int64_t batch, int dim, double* a, int32_t* piv, int32_t* info,
                             cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  LaunchCfg cfg;
  return with_grid(dim, [&](auto Gc, auto Tc) {
    constexpr int G = decltype(Gc)::value, T = decltype(Tc)::value;
    const size_t smem = sizeof(double) * ((size_t)dim * dim + 2 * dim + lu_scratch_words<G, T>());
    auto kern = k_lu_factor<G, T>;
    const int grid = team_grid(kern, G * G, smem, batch, cfg);
    kern<<<grid, G * G, smem, st>>>(batch, dim, a, piv, info);
    return cudaGetLastError();
  });
}

cudaError_t launch_lu_solve(int64_t batch, int dim, const double* lu, const int32_t* piv,
                            double* b, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * ((size_t)dim * dim + 3 * dim);
  LaunchCfg cfg;
  const int threads = team_threads(dim, cfg);
  const int grid = team_grid(k_lu_solve, threads, smem, batch, cfg);
  k_lu_solve<<<grid, threads, smem, st>>>(batch, dim, lu, piv, b);
  return cudaGetLastError();
}

size_t ros4_scratch_bytes_max() {
  static size_t cached[NOALLOC_MAX_DEVICES] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return 0;
  if (!cached[dev]) {
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // grid * (n^2 + n) * 8 <= grid * (shared memory of a CTA) <= SMs * (shared memory of an SM)
    cached[dev] = (size_t)sm_count() * (size_t)smem_sm;
  }
  return cached[dev];
}


cudaError_t launch_ros4(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                        double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                        int32_t* queue, cudaStream_t st, const LaunchCfg& cfg, double* scratch,
                        size_t scratch_bytes, bool may_alloc) {
  if (n <= 0) return cudaSuccess;
  const int nn = hm.d.n;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  auto* fn = (cfg.grid_side == 16 && nn <= 112) ? launch_ros4_16x7
             : nn <= 56                         ? launch_ros4_8x7
             : nn <= 112                        ? launch_ros4_16x7
             : nn <= 144                        ? launch_ros4_16x9
                                                : nullptr;
  if (!fn) return cudaErrorInvalidValue;
  return fn(hm, n, p, y, dt, h_io, sp, steps, status, queue, st, cfg, scratch, scratch_bytes, may_alloc);
}

cudaError_t launch_rkf45_team(const HostMech& hm, int64_t n, const double* p, double* y,
                              const double* dt, double* h_io, const SolverParams& sp, int32_t* steps,
                              int32_t* status, int32_t* queue, cudaStream_t st, const LaunchCfg& cfg) {
  if (n <= 0) return cudaSuccess;
  const int nn = hm.d.n;
  const size_t smem = sizeof(double) * (8 * (size_t)nn + team_bufs_doubles(hm.S, hm.d.chunk));
  const int grid = team_grid(k_rkf45_team, 64, smem, n, cfg);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_rkf45_team<<<grid, 64, smem, st>>>(hm.d, n, p, y, dt, h_io, sp, steps, status, queue);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ allocation-free ROS4
// Scratch of ck_integrate_ros4_noalloc: the work-queue counter that
// launch_ros4 otherwise receives from a per-call stream-ordered allocation.
// Every GPU that loads the library holds these 256 bytes until the process
// exits; all calls on a device share them.
static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_SCRATCH_INTS];

namespace {
std::mutex g_noalloc_mu;
int32_t* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

// Device address of g_noalloc_scratch on the current device.  The name is
// only a host-side stand-in, so the address is looked up once per device,
// with that device current, and cached.
cudaError_t noalloc_scratch(int32_t** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_ros4_noalloc(const HostMech& hm, int64_t n, const double* p, double* y,
                                const double* dt, double* h_io, const SolverParams& sp,
                                int32_t* steps, int32_t* status, cudaStream_t st,
                                const LaunchCfg& cfg) {
  if (cfg.precision) return cudaErrorNotSupported;  // its FP64 matrices need an allocation
  int32_t* queue = nullptr;
  cudaError_t e = noalloc_scratch(&queue);
  if (e != cudaSuccess) return e;
  // launch_ros4 zeroes the counter on the stream before the kernel starts;
  // no Jacobian copies (a rejected step recomputes J at the same state)
  return launch_ros4(hm, n, p, y, dt, h_io, sp, steps, status, queue, st, cfg, nullptr, 0, false);
}

}  // namespace ck
