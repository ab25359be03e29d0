// Thread-per-reactor kernels: the right-hand side (Sec. 5.1 benchmark: many
// independent RHS evaluations) and the RKF45 integrator (Sec. 2, App. B,
// Algorithm 1 per lane).  Every lane reads the same reaction record at the
// same time (broadcast).  Where that costs no residency (stage_pays) the
// mechanism tables are staged once per CTA into shared memory with a bulk
// TMA copy (cp.async.bulk + mbarrier); otherwise they are read through L1.
#include <cuda_runtime.h>

#include "ck_internal.h"
#include "ck_thread.cuh"

namespace ck {

// ------------------------------------------------------------------ staging
constexpr long long STAGE_SPIN_LIMIT = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Copy the table block into shared memory with bulk TMA copies completing on
// an mbarrier.  Waits are bounded: on timeout the error word is set and the
// CTA returns false (after a second bounded wait for its own copies).
__device__ bool stage_tables(unsigned char* dst, const unsigned char* src, uint32_t bytes,
                             uint64_t* mbar, int32_t* err) {
  const uint32_t bar = smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    const uint32_t CH = 32768;
    for (uint32_t off = 0; off < bytes; off += CH) {
      const uint32_t sz = (bytes - off) < CH ? (bytes - off) : CH;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(dst + off)),
          "l"(src + off), "r"(sz), "r"(bar)
          : "memory");
    }
  }
  __syncthreads();
  uint32_t ok = 0;
  for (long long it = 0; it < STAGE_SPIN_LIMIT && !ok; ++it) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
  }
  const int all_ok = __syncthreads_and(ok);
  if (!all_ok) {
    if (threadIdx.x == 0) atomicOr(err, DEVERR_STAGE_TIMEOUT);
    for (long long it = 0; it < STAGE_SPIN_LIMIT && !ok; ++it) {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
          : "=r"(ok)
          : "r"(bar)
          : "memory");
    }
    __syncthreads();
    return false;
  }
  return true;
}

__device__ __forceinline__ MechView view_of(const DevMech& d, const StageLayout& L,
                                            const unsigned char* base) {
  MechView m;
  m.S = d.S;
  m.R = d.R;
  m.rx = reinterpret_cast<const RxnRec*>(base + L.rx);
  m.th = reinterpret_cast<const double*>(base + L.th);
  m.tmid = reinterpret_cast<const double*>(base + L.tmid);
  m.W = reinterpret_cast<const double*>(base + L.W);
  m.invW = reinterpret_cast<const double*>(base + L.invW);
  m.eff_sp = reinterpret_cast<const int16_t*>(base + L.eff_sp);
  m.eff_m1 = reinterpret_cast<const double*>(base + L.eff_m1);
  m.tab = reinterpret_cast<const double*>(base + L.tab);
  m.revp = reinterpret_cast<const double*>(base + L.revp);
  m.cv = d.cv;
  return m;
}

// Shared-memory layout of the thread kernels: [mbarrier (16 B) | tables].
constexpr uint32_t STAGE_HDR = 16;

// ------------------------------------------------------------------ RHS
// R reactors a thread (rhs_thread_r); the last group of a batch repeats
// reactor N - 1 in its missing places (the same thread writes the same
// values there).
template <int MAXS, int R>
__global__ void __launch_bounds__(128) k_rhs(DevMech d, StageLayout L, int staged, int64_t N,
                                             const double* __restrict__ p,
                                             const double* __restrict__ y, double* __restrict__ f,
                                             int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned char* base = reinterpret_cast<const unsigned char*>(d.rxn);
  if (staged) {
    if (!stage_tables(smem + STAGE_HDR, base, L.bytes, reinterpret_cast<uint64_t*>(smem), err)) return;
    base = smem + STAGE_HDR;
  }
  const MechView m = view_of(d, L, base);
  double X[R * MAXS], G[2 * R * MAXS], wd[R * MAXS];
  const int n = d.n;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * R; r < N;
       r += (int64_t)gridDim.x * blockDim.x * R) {
    if constexpr (R == 1) {
      rhs_thread(m, p[r], y + r * n, 1, f + r * n, 1, X, G, wd);
    } else {
      double pr[R];
      const double* yr[R];
      double* fr[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int64_t rj = r + j < N ? r + j : N - 1;
        pr[j] = p[rj];
        yr[j] = y + rj * n;
        fr[j] = f + rj * n;
      }
      rhs_thread_r<R>(m, pr, yr, fr, X, G, wd);
    }
  }
}

// ------------------------------------------------------------------ RKF45
__device__ __forceinline__ double wrms_thread(int n, const double* e, const double* y0,
                                              const double* y1, double rtol, double atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double sc = atol + rtol * fmax(fabs(y0[i]), fabs(y1[i]));
    const double v = e[i] / sc;
    s = fma(v, v, s);
  }
  return sqrt(s / n);
}

// Initial step (reading: Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4,
// order 4, weights atol + rtol |y0|).  f0, y1, f1 are scratch vectors.
__device__ double h0_thread(const MechView& m, int n, double p, const double* y0, double tspan,
                            double rtol, double atol, double* f0, double* y1, double* f1, double* X,
                            double* G, double* wd) {
  rhs_thread(m, p, y0, 1, f0, 1, X, G, wd);
  double d0 = 0.0, d1 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double sc = atol + rtol * fabs(y0[i]);
    d0 = fma(y0[i] / sc, y0[i] / sc, d0);
    d1 = fma(f0[i] / sc, f0[i] / sc, d1);
  }
  d0 = sqrt(d0 / n);
  d1 = sqrt(d1 / n);
  const double ha = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  for (int i = 0; i < n; ++i) y1[i] = fma(ha, f0[i], y0[i]);
  rhs_thread(m, p, y1, 1, f1, 1, X, G, wd);
  double d2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double sc = atol + rtol * fabs(y0[i]);
    const double v = (f1[i] - f0[i]) / sc;
    d2 = fma(v, v, d2);
  }
  d2 = sqrt(d2 / n) / ha;
  const double dm = fmax(d1, d2);
  const double hb = (dm <= 1e-15) ? fmax(1e-6, ha * 1e-3) : pow(0.01 / dm, 0.2);
  return fmin(fmin(100.0 * ha, hb), tspan);
}

// One lane integrates one reactor at a time and fetches the next reactor
// from a global atomic counter as soon as it finishes (dynamic scheduling
// with granularity one, per lane), so lanes of a warp never wait for a
// slower neighbour beyond one step.
template <int MAXS>
__global__ void __launch_bounds__(128) k_rkf45(DevMech d, StageLayout L, int staged, int64_t N,
                                               const double* __restrict__ p, double* __restrict__ y,
                                               const double* __restrict__ dt, double* h_io,
                                               SolverParams sp, int32_t* steps, int32_t* status,
                                               int32_t* queue, int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned char* base = reinterpret_cast<const unsigned char*>(d.rxn);
  if (staged) {
    if (!stage_tables(smem + STAGE_HDR, base, L.bytes, reinterpret_cast<uint64_t*>(smem), err)) return;
    base = smem + STAGE_HDR;
  }
  const MechView m = view_of(d, L, base);
  constexpr int MAXN = MAXS + 1;
  double X[MAXS], G[2 * MAXS], wd[MAXS];
  double yv[MAXN], yt[MAXN], k[6][MAXN];
  const int n = d.n;
  const bool fixed = sp.fixed_h > 0.0;
  int64_t r = -1;
  double t = 0.0, tf = 0.0, h = 0.0, pr = 0.0;
  int acc = 0, rej = 0, st = ST_OK;
  bool last_rej = false, last_nf = false;
  for (;;) {
    bool finish = false;
    if (r < 0) {
      r = atomicAdd(queue, 1);
      if (r >= N) break;
      for (int i = 0; i < n; ++i) yv[i] = y[r * n + i];
      pr = p[r];
      tf = dt[r];
      t = 0.0;
      acc = rej = 0;
      st = ST_OK;
      last_rej = last_nf = false;
      bool bad = !(pr > 0.0) || !isfinite(pr) || !(yv[0] > 0.0) || !isfinite(tf) || !(tf >= 0.0);
      for (int i = 0; i < n; ++i) bad |= !isfinite(yv[i]);
      if (bad) {
        st = ST_BADINPUT;
        finish = true;
      } else if (tf == 0.0) {
        finish = true;
      } else if (fixed) {
        h = sp.fixed_h;
      } else if (h_io && h_io[r] > 0.0) {
        h = h_io[r];
      } else if (sp.h0 > 0.0) {
        h = sp.h0;
      } else {
        h = h0_thread(m, n, pr, yv, tf, sp.rtol, sp.atol, k[0], yt, k[1], X, G, wd);
      }
    }
    if (!finish) {
      const bool clamped = h >= tf - t;
      const double hh = clamped ? tf - t : h;
      if (acc + rej >= sp.max_steps) {
        st = ST_MAXSTEPS;
        finish = true;
      } else if (hh < 1e-15 * tf) {
        st = last_nf ? ST_NONFINITE : ST_HMIN;
        finish = true;
      } else {
        // stages k_s = hh f(y + sum_j a_sj k_j)
        rhs_thread(m, pr, yv, 1, k[0], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[0][i] *= hh;
        for (int i = 0; i < n; ++i) yt[i] = fma(RK_A21, k[0][i], yv[i]);
        rhs_thread(m, pr, yt, 1, k[1], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[1][i] *= hh;
        for (int i = 0; i < n; ++i) yt[i] = fma(RK_A32, k[1][i], fma(RK_A31, k[0][i], yv[i]));
        rhs_thread(m, pr, yt, 1, k[2], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[2][i] *= hh;
        for (int i = 0; i < n; ++i)
          yt[i] = fma(RK_A43, k[2][i], fma(RK_A42, k[1][i], fma(RK_A41, k[0][i], yv[i])));
        rhs_thread(m, pr, yt, 1, k[3], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[3][i] *= hh;
        for (int i = 0; i < n; ++i)
          yt[i] = fma(RK_A54, k[3][i],
                      fma(RK_A53, k[2][i], fma(RK_A52, k[1][i], fma(RK_A51, k[0][i], yv[i]))));
        rhs_thread(m, pr, yt, 1, k[4], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[4][i] *= hh;
        for (int i = 0; i < n; ++i)
          yt[i] = fma(RK_A65, k[4][i],
                      fma(RK_A64, k[3][i],
                          fma(RK_A63, k[2][i], fma(RK_A62, k[1][i], fma(RK_A61, k[0][i], yv[i])))));
        rhs_thread(m, pr, yt, 1, k[5], 1, X, G, wd);
        for (int i = 0; i < n; ++i) k[5][i] *= hh;
        // y* = y + sum b k (into yt), e = sum (bh - b) k (into k[1], whose b is 0)
        bool nf = false;
        for (int i = 0; i < n; ++i) {
          const double yn =
              fma(RK_B5, k[4][i], fma(RK_B4, k[3][i], fma(RK_B3, k[2][i], fma(RK_B1, k[0][i], yv[i]))));
          const double e = fma(RK_D6, k[5][i],
                               fma(RK_D5, k[4][i], fma(RK_D4, k[3][i], fma(RK_D3, k[2][i], RK_D1 * k[0][i]))));
          yt[i] = yn;
          k[1][i] = e;
          nf |= !isfinite(yn);
        }
        if (fixed) {
          for (int i = 0; i < n; ++i) yv[i] = yt[i];
          t = clamped ? tf : t + hh;
          ++acc;
        } else {
          const double e = wrms_thread(n, k[1], yv, yt, sp.rtol, sp.atol);
          if (nf || !isfinite(e)) {
            ++rej;
            h = FAC_MIN * hh;
            last_rej = true;
            last_nf = true;
          } else if (e < 1.0) {
            last_nf = false;
            for (int i = 0; i < n; ++i) yv[i] = yt[i];
            t = clamped ? tf : t + hh;
            ++acc;
            double fac = (e == 0.0) ? FAC_MAX : fmin(FAC_MAX, fmax(FAC_MIN, SAFETY * pow(e, -0.2)));
            if (last_rej) fac = fmin(1.0, fac);
            h = hh * fac;
            last_rej = false;
          } else {
            last_nf = false;
            ++rej;
            h = hh * fmax(FAC_MIN, SAFETY * pow(e, -0.2));
            last_rej = true;
          }
        }
        if (t >= tf) finish = true;
      }
    }
    if (finish) {
      for (int i = 0; i < n; ++i) y[r * n + i] = yv[i];
      if (h_io && st != ST_BADINPUT) h_io[r] = h;
      if (steps) {
        steps[2 * r] = acc;
        steps[2 * r + 1] = rej;
      }
      status[r] = st;
      r = -1;
    }
  }
}

// ------------------------------------------------------------------ launchers
int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

static bool stage_fits(const HostMech& hm, size_t* smem) {
  *smem = STAGE_HDR + hm.L.bytes;
  return *smem <= 200 * 1024;
}

// Stage the tables in shared memory (one bulk copy a CTA) only when the
// copy costs the grid no resident blocks.  Every lane reads the same record
// at the same time, so L1 serves the tables nearly as well; on GB300 the
// staged copy of the 53- and 111-species mechanisms cut the residency, and
// reading them through L1 instead made the RHS 15 and 37 % faster and the
// thread-per-reactor RKF45 43 and 38 %.  The 10-species tables (3 KB) stay
// staged.  Returns the dynamic shared memory to launch with.
template <class K>
static int stage_pays(const HostMech& hm, K kernel, int threads, size_t* smem) {
  if (!stage_fits(hm, smem)) {
    *smem = 0;
    return 0;
  }
  if (*smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  int with = 0, without = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&with, kernel, threads, *smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&without, kernel, threads, 0);
  if (with < without) {
    *smem = 0;
    return 0;
  }
  return 1;
}

template <class K>
static int blocks_for(K kernel, int threads, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sm_count();
}

// Reactors a thread of k_rhs, for mechanisms above and up to 32 species.
// Two and four (rhs_thread_r, each table record read once for all of them)
// measured slower on GB300: 33.2 and 22.7 M evaluations/s against 38.1 M on
// the 53-species mechanism, 9.4 and 5.2 M against 13.4 M on the 111-species
// one, 392 and 383 M against 440 M on the 10-species one (twice and four
// times the per-lane scratch in local memory, and fewer resident threads).
constexpr int RHS_REACTORS = 1;
constexpr int RHS_REACTORS_SMALL = 1;

template <int MAXS, int R>
static cudaError_t rhs_impl(const HostMech& hm, int64_t n, const double* p, const double* y,
                            double* f, cudaStream_t st) {
  auto kern = k_rhs<MAXS, R>;
  const int threads = 128;
  size_t smem = 0;
  const int staged = stage_pays(hm, kern, threads, &smem);
  int64_t want = (n + (int64_t)threads * R - 1) / ((int64_t)threads * R);
  int64_t cap = blocks_for(kern, threads, smem);
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  kern<<<blocks, threads, smem, st>>>(hm.d, hm.L, staged, n, p, y, f, hm.dev_err);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const HostMech& hm, int64_t n, const double* p, const double* y, double* f,
                       cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (hm.S <= 32) return rhs_impl<32, RHS_REACTORS_SMALL>(hm, n, p, y, f, st);
  return rhs_impl<128, RHS_REACTORS>(hm, n, p, y, f, st);
}

template <int MAXS>
static cudaError_t rkf45_impl(const HostMech& hm, int64_t n, const double* p, double* y,
                              const double* dt, double* h_io, const SolverParams& sp,
                              int32_t* steps, int32_t* status, int32_t* queue, cudaStream_t st,
                              const LaunchCfg& cfg) {
  auto kern = k_rkf45<MAXS>;
  const int threads = 128;
  size_t smem = 0;
  const int staged = stage_pays(hm, kern, threads, &smem);
  int64_t want = (n + threads - 1) / threads;
  int64_t cap = blocks_for(kern, threads, smem);
  if (cfg.ctas_per_sm > 0) cap = (int64_t)cfg.ctas_per_sm * sm_count();
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  kern<<<blocks, threads, smem, st>>>(hm.d, hm.L, staged, n, p, y, dt, h_io, sp, steps, status,
                                      queue, hm.dev_err);
  return cudaGetLastError();
}

cudaError_t launch_rkf45(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                         double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                         int32_t* queue, cudaStream_t st, const LaunchCfg& cfg) {
  if (n <= 0) return cudaSuccess;
  if (hm.S <= 32) return rkf45_impl<32>(hm, n, p, y, dt, h_io, sp, steps, status, queue, st, cfg);
  return rkf45_impl<128>(hm, n, p, y, dt, h_io, sp, steps, status, queue, st, cfg);
}

}  // namespace ck
