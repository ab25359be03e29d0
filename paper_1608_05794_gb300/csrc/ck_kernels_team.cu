// Team-per-reactor kernels: analytic Jacobian, batched dense LU / solve and
// the ROS4 Rosenbrock integrator (Sec. 2 transformed form, App. C, driven by
// Algorithm 1).  One CTA owns one reactor at a time and keeps its iteration
// matrix I/(h gamma) - J in shared memory; CTAs pull reactors from a global
// atomic counter (dynamic scheduling, granularity one reactor).
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "ck_internal.h"
#include "ck_team.cuh"

namespace ck {

__host__ __device__ __forceinline__ int team_bufs_doubles(int S, int chunk) { return 9 * S + (3 + JP) * chunk + 48; }

__device__ __forceinline__ TeamBufs carve_bufs(double* base, int S, int CH) {
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
__device__ __forceinline__ int team_next(int32_t* queue, int* slot) {
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
    for (int i = threadIdx.x; i < dim; i += blockDim.x) invd[i] = 1.0 / A[(size_t)i * dim + i];
    __syncthreads();
    if (threadIdx.x < 32) warp_lu_solve(A, dim, pv, invd, x);
    __syncthreads();
    for (int i = threadIdx.x; i < dim; i += blockDim.x) bvec[m * dim + i] = x[i];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ ROS4
// Weighted RMS norm over the team (reading shared with the oracle:
// sqrt(mean (e_i / (atol + rtol max(|y_i|, |ynew_i|)))^2)).
__device__ __forceinline__ double team_wrms(int n, const double* e, const double* y0,
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
__device__ double team_h0(const DevMech& d, const double* tab, double p, const double* y0, double tspan,
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

// Stage solve of the precision form: the iteration matrix is factored in
// FP32 (M32, piv, invd32) and each solve is refined against the FP64 matrix
// M64 (the CTA's copy in global memory, L2-resident): x = LU32^-1 b, then
// REFINE times r = b - M64 x (FP64), x += LU32^-1 r.
// b (in u) is overwritten with x; xf (n floats) and x (n doubles) are scratch
// that must not hold anything the caller still needs (stage 4 reuses the
// third stage's f, so the first three solves take u4's buffer as xf).
__device__ void refined_solve(const double* M64, const float* M32, int n, const int* piv,
                              const float* invd32, double* u, float* xf, double* x, int refine) {
  const int tid = threadIdx.x, P = blockDim.x;
  for (int i = tid; i < n; i += P) xf[i] = (float)u[i];
  __syncthreads();
  if (tid < 32) warp_lu_solve<true>(M32, n, piv, invd32, xf);
  __syncthreads();
  for (int i = tid; i < n; i += P) x[i] = (double)xf[i];
  __syncthreads();
  for (int it = 0; it < refine; ++it) {
    for (int i = tid; i < n; i += P) {
      const double* row = M64 + (size_t)i * n;
      double s0 = u[i], s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 4 <= n; j += 4) {
        s0 = fma(-row[j], x[j], s0);
        s1 = fma(-row[j + 1], x[j + 1], s1);
        s2 = fma(-row[j + 2], x[j + 2], s2);
        s3 = fma(-row[j + 3], x[j + 3], s3);
      }
      for (; j < n; ++j) s0 = fma(-row[j], x[j], s0);
      xf[i] = (float)((s0 + s1) + (s2 + s3));
    }
    __syncthreads();
    if (tid < 32) warp_lu_solve<true>(M32, n, piv, invd32, xf);
    __syncthreads();
    for (int i = tid; i < n; i += P) x[i] += (double)xf[i];
    __syncthreads();
  }
  for (int i = tid; i < n; i += P) u[i] = x[i];
  __syncthreads();
}

// PREC 0: FP64 LU and solves.  PREC 1 / 2: FP32 LU and solves with one /
// two steps of FP64 iterative refinement (the rates, K_c, the temperature
// equation, the error norm and the step control stay FP64).
//
// m64g (may be NULL for PREC 0) holds ros4_scratch_doubles(n) doubles per
// CTA, m64g[blockIdx.x][.]: global memory, 23 KB a CTA at n = 54 (21 MB for
// the 912 CTAs of the medium workload), so it stays in L2.  Its first n*n
// doubles hold J of the current state, its last n (precision form) the
// diagonal J_ii.
//
// The matrix factored is A = J - I/(h gamma) = -M rather than the iteration
// matrix M itself: partial pivoting picks the same rows, the multipliers and
// the pre-divided upper factor come out identical, and every solve returns
// exactly -u, so the stage vectors are kept as v_i = -u_i and the method's
// coefficients enter with their signs flipped.  The results are bitwise those
// of factoring M, without negating the n^2 entries of each new J.
//   - After a rejected step (error test, singular matrix or non-finite trial
//     state) y is unchanged, so J and f(y) are reused rather than recomputed
//     (only the analytic J: the forward-difference increments depend on h);
//     the new matrix J - I/(h gamma) is rebuilt from the copy.  With
//     m64g NULL (the allocation-free entry point) J is recomputed at the same
//     state instead, which gives the same values.
//   - The precision form keeps its FP64 iteration matrix, which the
//     refinement reads, in the first n*n doubles (the diagonal rebuilt from
//     the last n for each h) and its FP32 factors in the first half of the
//     shared FP64 matrix, so both forms need the same shared memory and
//     residency.
template <int G, int T, int PREC>
__global__ void __launch_bounds__(G * G, G == 8 ? 6 : 1) k_ros4(const __grid_constant__ DevMech d, int64_t N, const double* __restrict__ p,
                                                 double* __restrict__ y, const double* __restrict__ dt,
                                                 double* h_io, SolverParams sp, int32_t* steps,
                                                 int32_t* status, int32_t* queue, double* __restrict__ m64g) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int slot;
  const int n = d.n;
  const double* tab = d.tab;  // 2 KB, stays in L1
  double* M = sm;
  double* yv = M + (size_t)n * n;
  double* F0 = yv + n;
  double* F = F0 + n;
  double* Yt = F + n;
  double* u1 = Yt + n;
  double* u2 = u1 + n;
  double* u3 = u2 + n;
  double* u4 = u3 + n;
  double* invd = u4 + n;
  int* piv = reinterpret_cast<int*>(invd + n);
  // the LU's scratch (lu_scratch_words: at most 578 doubles) reuses the
  // team buffers, free while factoring (9 S + 10 chunk + 48 >= 688 doubles)
  TeamBufs b = carve_bufs(invd + n + (n + 1) / 2, d.S, d.chunk);
  float* M32 = reinterpret_cast<float*>(M);  // PREC >= 1: FP32 factors over the FP64 matrix
  double* Mg = m64g ? m64g + (size_t)blockIdx.x * ros4_scratch_doubles(n) : nullptr;
  const bool keep_j = Mg != nullptr && sp.jac == 0;
  Mix x;
  const bool fixed = sp.fixed_h > 0.0;
  const int tid = threadIdx.x, P = blockDim.x;
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
      else h = team_h0(d, tab, pr, yv, tf, sp.rtol, sp.atol, F0, Yt, F, b, x);
      const double hmin = 1e-15 * tf;
      double t = 0.0;
      bool last_rej = false, last_nf = false;
      int sing_run = 0;
      bool have_j = false;   // J of yv in Mg (analytic form with a copy only)
      bool have_f = false;   // F0 = f(yv)
      while (t < tf) {
        if (acc + rej >= sp.max_steps) { st = ST_MAXSTEPS; break; }
        const bool clamped = h >= tf - t;
        const double hh = clamped ? tf - t : h;
        if (hh < hmin) { st = last_nf ? ST_NONFINITE : ST_HMIN; break; }
        // J and f at y (or the copy kept since a rejected attempt at the
        // same y); A = J - I/(hh gamma) = -M; LU of A
        const int nn = n * n;
        if (!have_j) {
          if (sp.jac == 1) team_jacobian_fd(d, tab, pr, yv, hh, sp.rtol, sp.atol, F0, M, Yt, F, b, have_f);
          else team_jacobian(d, tab, pr, yv, F0, M, b, x);
          team_sync();
          if (Mg && (keep_j || PREC)) {
            for (int e = tid; e < nn; e += P) Mg[e] = M[e];
            if (PREC)
              for (int i = tid; i < n; i += P) Mg[nn + i] = M[(size_t)i * n + i];
            __syncthreads();
          }
          have_j = keep_j;
          have_f = true;
        } else if (PREC == 0) {
          for (int e = tid; e < nn; e += P) M[e] = Mg[e];
          team_sync();
        }
        const double dg = 1.0 / (hh * ROS_GAMMA);
        int info;
        if (PREC == 0) {
          for (int i = tid; i < n; i += P) M[(size_t)i * n + i] -= dg;
          team_sync();
          info = lu_reg<G, T, true>(M, n, piv, invd, b.X);
        } else {
          for (int i = tid; i < n; i += P) Mg[(size_t)i * n + i] = Mg[nn + i] - dg;
          __syncthreads();
          for (int e = tid; e < nn; e += P) M32[e] = (float)Mg[e];
          __syncthreads();
          info = lu_reg<G, T, true>(M32, n, piv, reinterpret_cast<float*>(invd), reinterpret_cast<float*>(b.X));
        }
        if (info) {
          ++rej;
          if (++sing_run >= SINGULAR_LIMIT) { st = ST_SINGULAR; break; }
          h = 0.5 * hh;
          last_rej = true;
          continue;
        }
        sing_run = 0;
        const double ih = 1.0 / hh;
        // stage 1: M u1 = f(y), solved as A v1 = f(y) with v = -u (A = -M)
        for (int i = tid; i < n; i += P) u1[i] = F0[i];
        team_sync();
        if (PREC == 0) {
          if (tid < 32) warp_lu_solve<true>(M, n, piv, invd, u1);
          __syncthreads();
        } else {
          refined_solve(Mg, M32, n, piv, reinterpret_cast<const float*>(invd), u1, reinterpret_cast<float*>(u4), Yt, PREC);
        }
        // stage 2: M u2 = f(y + a21 u1) + (c21/h) u1
        for (int i = tid; i < n; i += P) Yt[i] = fma(-ROS_A21, u1[i], yv[i]);
        team_sync();
        team_rhs(d, tab, pr, Yt, F, b);
        for (int i = tid; i < n; i += P) u2[i] = fma(-ROS_C21 * ih, u1[i], F[i]);
        team_sync();
        if (PREC == 0) {
          if (tid < 32) warp_lu_solve<true>(M, n, piv, invd, u2);
          __syncthreads();
        } else {
          refined_solve(Mg, M32, n, piv, reinterpret_cast<const float*>(invd), u2, reinterpret_cast<float*>(u4), Yt, PREC);
        }
        // stage 3: M u3 = f(y + a31 u1 + a32 u2) + (c31 u1 + c32 u2)/h
        for (int i = tid; i < n; i += P) Yt[i] = fma(-ROS_A32, u2[i], fma(-ROS_A31, u1[i], yv[i]));
        team_sync();
        team_rhs(d, tab, pr, Yt, F, b);
        for (int i = tid; i < n; i += P)
          u3[i] = fma(-ROS_C32 * ih, u2[i], fma(-ROS_C31 * ih, u1[i], F[i]));
        team_sync();
        if (PREC == 0) {
          if (tid < 32) warp_lu_solve<true>(M, n, piv, invd, u3);
          __syncthreads();
        } else {
          refined_solve(Mg, M32, n, piv, reinterpret_cast<const float*>(invd), u3, reinterpret_cast<float*>(u4), Yt, PREC);
        }
        // stage 4: same argument as stage 3 (a4j = a3j, a43 = 0), so f is reused
        for (int i = tid; i < n; i += P)
          u4[i] = fma(-ROS_C43 * ih, u3[i], fma(-ROS_C42 * ih, u2[i], fma(-ROS_C41 * ih, u1[i], F[i])));
        team_sync();
        if (PREC == 0) {
          if (tid < 32) warp_lu_solve<true>(M, n, piv, invd, u4);
          __syncthreads();
        } else {
          refined_solve(Mg, M32, n, piv, reinterpret_cast<const float*>(invd), u4, reinterpret_cast<float*>(F), Yt, PREC);
        }
        // y* = y + sum m_i u_i (into Yt), e = sum E_i u_i (into F); u_i = -v_i
        int nf = 0;
        for (int i = tid; i < n; i += P) {
          const double yn =
              fma(-ROS_M4, u4[i], fma(-ROS_M3, u3[i], fma(-ROS_M2, u2[i], fma(-ROS_M1, u1[i], yv[i]))));
          Yt[i] = yn;
          F[i] = fma(-ROS_E4, u4[i], fma(-ROS_E3, u3[i], fma(-ROS_E2, u2[i], -ROS_E1 * u1[i])));
          nf |= !isfinite(yn);
        }
        nf = __syncthreads_or(nf);
        if (fixed) {
          for (int i = tid; i < n; i += P) yv[i] = Yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          have_j = have_f = false;
          continue;
        }
        const double e = team_wrms(n, F, yv, Yt, sp.rtol, sp.atol, b.red);
        if (nf || !isfinite(e)) {
          ++rej;
          h = FAC_MIN * hh;
          last_rej = true;
          last_nf = true;
          continue;
        }
        last_nf = false;
        if (e < 1.0) {
          for (int i = tid; i < n; i += P) yv[i] = Yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          have_j = have_f = false;
          double fac = (e == 0.0) ? FAC_MAX : fmin(FAC_MAX, fmax(FAC_MIN, SAFETY * pow(e, -0.25)));
          if (last_rej) fac = fmin(1.0, fac);
          h = hh * fac;
          last_rej = false;
        } else {
          ++rej;
          h = hh * fmax(FAC_MIN, SAFETY * pow(e, -0.25));
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
        if (e < 1.0) {
          for (int i = tid; i < n; i += P) yv[i] = yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          double fac = (e == 0.0) ? FAC_MAX : fmin(FAC_MAX, fmax(FAC_MIN, SAFETY * pow(e, -0.2)));
          if (last_rej) fac = fmin(1.0, fac);
          h = hh * fac;
          last_rej = false;
        } else {
          ++rej;
          h = hh * fmax(FAC_MIN, SAFETY * pow(e, -0.2));
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

template <class K>
static int team_grid(K kernel, int threads, size_t smem, int64_t work, const LaunchCfg& cfg) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
  int64_t g = (int64_t)per_sm * sm_count();
  if (work < g) g = work;
  return (int)(g < 1 ? 1 : g);
}

size_t ros4_smem_bytes(int n, int S, int chunk) {
  return sizeof(double) * ((size_t)n * n + 9 * (size_t)n + (n + 1) / 2 + team_bufs_doubles(S, chunk));
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
  const size_t smem = ros4_smem_bytes(nn, hm.S, hm.d.chunk);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  return with_grid(nn, [&](auto Gc, auto Tc) {
    constexpr int G = decltype(Gc)::value, T = decltype(Tc)::value;
    auto kern = cfg.precision == 2 ? k_ros4<G, T, 2> : (cfg.precision == 1 ? k_ros4<G, T, 1> : k_ros4<G, T, 0>);
    const int grid = team_grid(kern, G * G, smem, n, cfg);
    // per-CTA copies of -J (every form) and the FP64 iteration matrices of
    // the precision form: the caller's scratch when it is large enough, else
    // a stream-ordered allocation around the launch, else (allocation-free
    // FP64 form) none
    const size_t need = sizeof(double) * (size_t)grid * ros4_scratch_doubles(nn);
    double* m64g = nullptr;
    bool owned = false;
    if (scratch && scratch_bytes >= need) {
      m64g = scratch;
    } else if (may_alloc) {
      cudaError_t a = cudaMallocAsync(reinterpret_cast<void**>(&m64g), need, st);
      if (a != cudaSuccess) return a;
      owned = true;
    } else if (cfg.precision) {
      return cudaErrorNotSupported;
    }
    kern<<<grid, G * G, smem, st>>>(hm.d, n, p, y, dt, h_io, sp, steps, status, queue, m64g);
    cudaError_t k = cudaGetLastError();
    if (owned) {
      cudaError_t f = cudaFreeAsync(m64g, st);
      if (k == cudaSuccess) k = f;
    }
    return k;
  }, cfg.grid_side);
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
