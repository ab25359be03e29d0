// The ROS4 integrator kernel (Sec. 2 transformed form, App. C, driven by
// Algorithm 1): one CTA per reactor, iteration matrix in shared memory,
// register-tiled LU, warp solves; and its launcher for one thread grid.
// Included by one translation unit per thread grid (ck_ros4_*.cu).
#pragma once
#include "ck_team_kernels.cuh"

namespace ck {

// Stage solve of the precision form: the iteration matrix is factored in
// FP32 (M32, piv, invd32) and each solve is refined against the FP64 matrix
// M64 (the CTA's copy in global memory, L2-resident): x = LU32^-1 b, then
// REFINE times r = b - M64 x (FP64), x += LU32^-1 r.
// b (in u) is overwritten with x; xf (n floats) and x (n doubles) are scratch
// that must not hold anything the caller still needs (stage 4 reuses the
// third stage's f, so the first three solves take u4's buffer as xf).
static __device__ void refined_solve(const double* M64, const float* M32, int n, const int* piv,
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
        const double dg = rcp_rn(hh * ROS_GAMMA);
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
        const double ih = rcp_rn(hh);
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
        const double pe = (e == 0.0) ? 0.0 : team_pow(e, -0.25, b.red);
        if (e < 1.0) {
          for (int i = tid; i < n; i += P) yv[i] = Yt[i];
          team_sync();
          t = clamped ? tf : t + hh;
          ++acc;
          have_j = have_f = false;
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

// Launch k_ros4<G, T, precision> (the body of launch_ros4 for one thread
// grid; each grid is compiled in its own translation unit).
template <int G, int T>
cudaError_t launch_ros4_tile(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                             double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                             int32_t* queue, cudaStream_t st, const LaunchCfg& cfg, double* scratch,
                             size_t scratch_bytes, bool may_alloc) {
  const int nn = hm.d.n;
  const size_t smem = ros4_smem_bytes(nn, hm.S, hm.d.chunk);
  auto kern = cfg.precision == 2 ? k_ros4<G, T, 2> : (cfg.precision == 1 ? k_ros4<G, T, 1> : k_ros4<G, T, 0>);
  const int grid = team_grid(kern, G * G, smem, n, cfg);
  // per-CTA copies of J (every form) and the FP64 iteration matrices of
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
}

}  // namespace ck
