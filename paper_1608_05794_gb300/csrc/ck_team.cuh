// Team-per-reactor device code: one CTA (1..8 warps) evaluates one reactor's
// right-hand side and analytic Jacobian, and factors and solves its
// iteration matrix I/(h gamma) - J held in shared memory (Sec. 2, ROS4).
// This is the paper's "deep" vectorisation (Sec. 4): lanes split the
// reactions and species of a single ODE system.  All sums that feed a
// control decision are reduced in a fixed order, so every thread of the CTA
// takes the same branch and results are bitwise reproducible.
#pragma once
#include "ck_common.cuh"

namespace ck {

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum returned to every thread (fixed order).  red: >= 32 doubles.
__device__ __forceinline__ double team_sum(double v, double* red) {
  v = warp_allsum(v);
  const int nw = blockDim.x >> 5;
  if (nw == 1) return v;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

__device__ __forceinline__ void team_sync() {
  if (blockDim.x == 32) __syncwarp();
  else __syncthreads();
}

// Shared-memory work arrays of one team.
struct TeamBufs {
  double *X, *g2, *hRT, *cpR, *dcpR, *wd, *aT, *E, *u, *cs;  // [S]
  double *q, *ckf, *ckr, *w, *dqT, *D;                         // [R]
  double* red;                                                // [64]
};

// Mixture quantities shared by the RHS and the Jacobian.
struct Mix {
  double T, invT, lnT, log2T, T2, T3, T4, rho, Wbar, Ctot;
};

// Species pass: rho, [X_k], Gibbs / enthalpy / heat-capacity polynomials.
__device__ __forceinline__ void team_species(const DevMech& m, double p, const double* y,
                                             TeamBufs& b, Mix& x, bool want_dcp) {
  const int S = m.S;
  x.T = y[0];
  x.invT = 1.0 / x.T;
  x.lnT = log(x.T);
  x.log2T = x.lnT * INV_LN2;
  x.T2 = x.T * x.T;
  x.T3 = x.T2 * x.T;
  x.T4 = x.T3 * x.T;
  double s = 0.0;
  for (int k = threadIdx.x; k < S; k += blockDim.x) s = fma(y[1 + k], m.invW[k], s);
  const double sumYW = team_sum(s, b.red);
  x.Wbar = 1.0 / sumYW;
  x.rho = p / (R_GAS * x.T * sumYW);
  double c = 0.0;
  for (int k = threadIdx.x; k < S; k += blockDim.x) {
    const double xk = x.rho * (y[1 + k] * m.invW[k]);
    b.X[k] = xk;
    c += xk;
    const double* a = m.thermo + k * TH_PER_SPECIES + (x.T < m.tmid[k] ? 0 : TH_STRIDE);
    double g = fma(a[11], x.lnT, a[12]);
    g = fma(a[13], x.T, g);
    g = fma(a[14], x.T2, g);
    g = fma(a[15], x.T3, g);
    g = fma(a[16], x.T4, g);
    b.g2[k] = fma(a[17], x.invT, g);
    b.cpR[k] = fma(a[4], x.T4, fma(a[3], x.T3, fma(a[2], x.T2, fma(a[1], x.T, a[0]))));
    b.hRT[k] = fma(a[10], x.invT, fma(a[9], x.T4, fma(a[8], x.T3, fma(a[7], x.T2, fma(a[6], x.T, a[5])))));
    if (want_dcp) b.dcpR[k] = fma(4.0 * a[4], x.T3, fma(3.0 * a[3], x.T2, fma(2.0 * a[2], x.T, a[1])));
  }
  x.Ctot = team_sum(c, b.red);
}

// Rates of one reaction at the mixture state.  With want_jac also the
// partial-derivative pieces used by the Jacobian (see team_jacobian).
__device__ __forceinline__ void team_reaction(const DevMech& m, const RxnRec& r, const Mix& x,
                                              const TeamBufs& b, const double* tab, int i,
                                              bool want_jac) {
  const double* X = b.X;
  const double* g2 = b.g2;
  const double l2kf = fma(-r.EoR2, x.invT, fma(r.beta, x.log2T, r.lA2));
  const double kf = ck_exp2(l2kf, tab);
  double fwd = X[r.sp[0]];
  if (r.nreac > 1) fwd *= X[r.sp[1]];
  if (r.nreac > 2) fwd *= X[r.sp[2]];
  double kr = 0.0, rv = 0.0, dlnkc = 0.0;
  if (r.rev) {
    double l2kc = (double)r.dnu * (LOG2_P0_OVER_R - x.log2T);
    l2kc += g2[r.sp[3]];
    if (r.nprod > 1) l2kc += g2[r.sp[4]];
    if (r.nprod > 2) l2kc += g2[r.sp[5]];
    l2kc -= g2[r.sp[0]];
    if (r.nreac > 1) l2kc -= g2[r.sp[1]];
    if (r.nreac > 2) l2kc -= g2[r.sp[2]];
    kr = ck_exp2(l2kf - l2kc, tab);
    rv = X[r.sp[3]];
    if (r.nprod > 1) rv *= X[r.sp[4]];
    if (r.nprod > 2) rv *= X[r.sp[5]];
    if (want_jac) {
      // d ln K_c / dT = (sum_j nu_j H_j/(R T) - dnu) / T
      double hs = b.hRT[r.sp[3]];
      if (r.nprod > 1) hs += b.hRT[r.sp[4]];
      if (r.nprod > 2) hs += b.hRT[r.sp[5]];
      hs -= b.hRT[r.sp[0]];
      if (r.nreac > 1) hs -= b.hRT[r.sp[1]];
      if (r.nreac > 2) hs -= b.hRT[r.sp[2]];
      dlnkc = (hs - (double)r.dnu) * x.invT;
    }
  }
  const double net = fma(-kr, rv, kf * fwd);
  double c = 1.0, dcdM = 0.0, dcdT = 0.0, M = 0.0;
  const double dlnkf = fma(r.EoR2 * LN2, x.invT, r.beta) * x.invT;
  if (r.type) {
    M = x.Ctot;
    for (int e = r.eff_beg; e < r.eff_beg + r.eff_cnt; ++e) M = fma(m.eff_m1[e], X[m.eff_sp[e]], M);
    if (r.type == 1) {
      c = M;
      dcdM = 1.0;
    } else {
      const double l2k0 = fma(-r.E0oR2, x.invT, fma(r.beta0, x.log2T, r.lA02));
      const double k0_kf = ck_exp2(l2k0 - l2kf, tab);
      const double Pr = k0_kf * M;
      const double inv1p = 1.0 / (1.0 + Pr);
      c = Pr * inv1p;
      dcdM = k0_kf * inv1p * inv1p;
      if (want_jac) {
        const double dlnk0 = fma(r.E0oR2 * LN2, x.invT, r.beta0) * x.invT;
        dcdT = Pr * (dlnk0 - dlnkf) * inv1p * inv1p;
      }
    }
  }
  const double q = c * net;
  b.q[i] = q;
  if (want_jac) {
    const double ckf = c * kf, ckr = c * kr;
    b.ckf[i] = ckf;
    b.ckr[i] = ckr;
    const double w = dcdM * net;
    b.w[i] = w;
    // D = sum_j dq/d[X_j] [X_j]: Euler's theorem for the mass-action
    // products (homogeneous of degree nreac / nprod) plus the [M] part.
    const double D = fma(ckf * fwd, (double)r.nreac, -(ckr * rv) * (double)r.nprod) + M * w;
    b.D[i] = D;
    // dq/dT at fixed [X], then the total derivative at fixed Y (d[X]/dT = -[X]/T)
    const double dqTX = fma(dcdT, net, ckf * fwd * dlnkf - ckr * rv * (dlnkf - dlnkc));
    b.dqT[i] = fma(-D, x.invT, dqTX);
  }
}

// f(y) for one reactor.  y, f: shared memory, n = S + 1.
__device__ void team_rhs(const DevMech& m, const double* tab, double p, const double* y, double* f,
                         TeamBufs& b, Mix& x) {
  team_species(m, p, y, b, x, false);
  team_sync();
  for (int i = threadIdx.x; i < m.R; i += blockDim.x) team_reaction(m, m.rxn[i], x, b, tab, i, false);
  team_sync();
  const double invrho = 1.0 / x.rho;
  double cpm = 0.0, hw = 0.0;
  for (int k = threadIdx.x; k < m.S; k += blockDim.x) {
    double w = 0.0;
    for (int e = m.csr_ptr[k]; e < m.csr_ptr[k + 1]; ++e) {
      const int32_t code = m.csr_rx[e];
      w = fma((double)((code & 255) - 8), b.q[code >> 8], w);
    }
    b.wd[k] = w;
    cpm = fma(y[1 + k] * m.invW[k], b.cpR[k], cpm);
    hw = fma(b.hRT[k], w, hw);
    f[1 + k] = w * (m.W[k] * invrho);
  }
  cpm = team_sum(cpm, b.red);
  hw = team_sum(hw, b.red);
  if (threadIdx.x == 0) f[0] = -x.T * hw / (x.rho * cpm);
  team_sync();
}

// Analytic Jacobian J = df/d(T, Y) at constant p, written row-major into J
// (shared memory, n x n), and f(y) into f.  Derivation (chain rule through
// rho(T, Y) and [X](rho, Y); dlnK_c/dT = (sum nu H/RT - dnu)/T):
//   A_kj   = sum_i nu_ki dq_i/d[X_j] (sparse mass-action part and the
//            (eff - 1) corrections) + u_k (dense third-body part, u_k = sum nu_ki w_i),
//   E_k    = sum_i nu_ki D_i,  a_k = sum_i nu_ki dq_i/dT,
//   J[1+k][1+j] = (W_k (A_kj + u_k) + W_k Wbar (wdot_k - E_k)/rho) / W_j,
//   J[1+k][0]   = W_k (a_k + wdot_k / T) / rho,
//   J[0][1+j]   = -(T (rho cs_j - Wbar HE)/(rho cpm) + Tdot (cp_j/cpm - Wbar)) / W_j,
//   J[0][0]     = -(sum cp_k wdot_k + T sum H_k/RT a_k)/(rho cpm) - Tdot (dcpm/cpm - 1/T),
// with cs_j = sum_k H_k/RT (A_kj + u_k), HE = sum_k H_k/RT E_k, and heat
// capacities in units of R.
__device__ void team_jacobian(const DevMech& m, const double* tab, double p, const double* y,
                              double* f, double* J, TeamBufs& b, Mix& x) {
  const int S = m.S, n = m.n;
  team_species(m, p, y, b, x, true);
  team_sync();
  for (int i = threadIdx.x; i < m.R; i += blockDim.x) team_reaction(m, m.rxn[i], x, b, tab, i, true);
  team_sync();
  // row pass: each thread owns whole species rows of A (no write conflicts)
  for (int k = threadIdx.x; k < S; k += blockDim.x) {
    double* row = J + (size_t)(1 + k) * n + 1;
    for (int j = 0; j < S; ++j) row[j] = 0.0;
    double w = 0.0, aT = 0.0, E = 0.0, u = 0.0;
    for (int e = m.csr_ptr[k]; e < m.csr_ptr[k + 1]; ++e) {
      const int32_t code = m.csr_rx[e];
      const int i = code >> 8;
      const double nu = (double)((code & 255) - 8);
      const RxnRec& r = m.rxn[i];
      w = fma(nu, b.q[i], w);
      aT = fma(nu, b.dqT[i], aT);
      E = fma(nu, b.D[i], E);
      // d(prod [X]^nu')/d[X_s] slot by slot
      const double cf = nu * b.ckf[i];
      const double x0 = b.X[r.sp[0]];
      if (r.nreac == 1) {
        row[r.sp[0]] += cf;
      } else if (r.nreac == 2) {
        const double x1 = b.X[r.sp[1]];
        row[r.sp[0]] = fma(cf, x1, row[r.sp[0]]);
        row[r.sp[1]] = fma(cf, x0, row[r.sp[1]]);
      } else {
        const double x1 = b.X[r.sp[1]], x2 = b.X[r.sp[2]];
        row[r.sp[0]] = fma(cf, x1 * x2, row[r.sp[0]]);
        row[r.sp[1]] = fma(cf, x0 * x2, row[r.sp[1]]);
        row[r.sp[2]] = fma(cf, x0 * x1, row[r.sp[2]]);
      }
      if (r.rev) {
        const double cr = -nu * b.ckr[i];
        const double y0 = b.X[r.sp[3]];
        if (r.nprod == 1) {
          row[r.sp[3]] += cr;
        } else if (r.nprod == 2) {
          const double y1 = b.X[r.sp[4]];
          row[r.sp[3]] = fma(cr, y1, row[r.sp[3]]);
          row[r.sp[4]] = fma(cr, y0, row[r.sp[4]]);
        } else {
          const double y1 = b.X[r.sp[4]], y2 = b.X[r.sp[5]];
          row[r.sp[3]] = fma(cr, y1 * y2, row[r.sp[3]]);
          row[r.sp[4]] = fma(cr, y0 * y2, row[r.sp[4]]);
          row[r.sp[5]] = fma(cr, y0 * y1, row[r.sp[5]]);
        }
      }
      if (r.type) {
        const double nw = nu * b.w[i];
        u += nw;
        for (int e2 = r.eff_beg; e2 < r.eff_beg + r.eff_cnt; ++e2)
          row[m.eff_sp[e2]] = fma(nw, m.eff_m1[e2], row[m.eff_sp[e2]]);
      }
    }
    b.wd[k] = w;
    b.aT[k] = aT;
    b.E[k] = E;
    b.u[k] = u;
  }
  team_sync();
  // column sums for the temperature row, and the RHS itself
  const double invrho = 1.0 / x.rho;
  double cpm = 0.0, hw = 0.0, he = 0.0, dcpm = 0.0, cw = 0.0, ha = 0.0;
  for (int k = threadIdx.x; k < S; k += blockDim.x) {
    const double yk = y[1 + k] * m.invW[k];
    cpm = fma(yk, b.cpR[k], cpm);
    dcpm = fma(yk, b.dcpR[k], dcpm);
    hw = fma(b.hRT[k], b.wd[k], hw);
    he = fma(b.hRT[k], b.E[k], he);
    cw = fma(b.cpR[k], b.wd[k], cw);
    ha = fma(b.hRT[k], b.aT[k], ha);
    f[1 + k] = b.wd[k] * (m.W[k] * invrho);
  }
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < S; ++k) s = fma(b.hRT[k], J[(size_t)(1 + k) * n + 1 + j] + b.u[k], s);
    b.cs[j] = s;
  }
  cpm = team_sum(cpm, b.red);
  dcpm = team_sum(dcpm, b.red);
  hw = team_sum(hw, b.red);
  he = team_sum(he, b.red);
  cw = team_sum(cw, b.red);
  ha = team_sum(ha, b.red);
  const double Tdot = -x.T * hw / (x.rho * cpm);
  team_sync();
  // species block and temperature column
  const int SS = S * S;
  for (int e = threadIdx.x; e < SS; e += blockDim.x) {
    const int k = e / S, j = e - k * S;
    double* a = J + (size_t)(1 + k) * n + 1 + j;
    const double ck = m.W[k] * x.Wbar * (b.wd[k] - b.E[k]) * invrho;
    *a = fma(m.W[k], *a + b.u[k], ck) * m.invW[j];
  }
  for (int k = threadIdx.x; k < S; k += blockDim.x)
    J[(size_t)(1 + k) * n] = m.W[k] * invrho * fma(b.wd[k], x.invT, b.aT[k]);
  const double inv_rc = 1.0 / (x.rho * cpm);
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    const double t1 = x.T * (x.rho * b.cs[j] - x.Wbar * he) * inv_rc;
    const double t2 = Tdot * (b.cpR[j] / cpm - x.Wbar);
    J[1 + j] = -(t1 + t2) * m.invW[j];
  }
  if (threadIdx.x == 0) {
    J[0] = -fma(x.T, ha, cw) * inv_rc - Tdot * (dcpm / cpm - x.invT);
    f[0] = Tdot;
  }
  team_sync();
}

// In-place LU with partial pivoting of the n x n row-major matrix A
// (shared memory).  piv[k] = row swapped with row k; the inverse pivots go
// to invd.  Returns 0, or k+1 when pivot k is zero or not finite (the value
// is the same in every thread).  Ties pick the smallest row index.
__device__ int team_lu(double* A, int n, int* piv, double* invd, double* red) {
  const int P = blockDim.x;
  const int tid = threadIdx.x;
  int* ired = reinterpret_cast<int*>(red + 32);
  for (int k = 0; k < n; ++k) {
    // pivot search over column k, rows k..n-1 (NaN counts as +inf)
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += P) {
      double v = fabs(A[(size_t)i * n + k]);
      if (v != v) v = __longlong_as_double(0x7ff0000000000000LL);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (P > 32) {
      __syncthreads();
      if ((tid & 31) == 0) { red[tid >> 5] = best; ired[tid >> 5] = bi; }
      __syncthreads();
      best = red[0];
      bi = ired[0];
      for (int w = 1; w < (P >> 5); ++w)
        if (red[w] > best || (red[w] == best && ired[w] < bi)) { best = red[w]; bi = ired[w]; }
    }
    if (!(best > 0.0) || !isfinite(best)) {
      team_sync();
      return k + 1;
    }
    if (tid == 0) piv[k] = bi;
    if (bi != k) {
      for (int j = tid; j < n; j += P) {
        const double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)bi * n + j];
        A[(size_t)bi * n + j] = t;
      }
    }
    team_sync();
    const double ip = 1.0 / A[(size_t)k * n + k];
    if (tid == 0) invd[k] = ip;
    const int mrem = n - k - 1;
    for (int i = k + 1 + tid; i < n; i += P) A[(size_t)i * n + k] *= ip;
    team_sync();
    // trailing update A[i][j] -= A[i][k] A[k][j], flattened over threads
    const int cnt = mrem * mrem;
    if (cnt > 0) {
      int e = tid;
      int ii = e / mrem, jj = e - ii * mrem;
      const int di = P / mrem, dj = P - di * mrem;
      for (; e < cnt; e += P) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        A[(size_t)i * n + j] = fma(-A[(size_t)i * n + k], A[(size_t)k * n + j], A[(size_t)i * n + j]);
        ii += di;
        jj += dj;
        if (jj >= mrem) { jj -= mrem; ++ii; }
      }
    }
    team_sync();
  }
  return 0;
}

// Solve (LU) x = b in place (b in shared memory), pivots as from team_lu.
__device__ void team_lu_solve(const double* A, int n, const int* piv, const double* invd, double* b) {
  const int P = blockDim.x, tid = threadIdx.x;
  if (tid == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
  }
  team_sync();
  // forward substitution with the unit lower triangle, column by column
  for (int j = 0; j < n - 1; ++j) {
    const double bj = b[j];
    for (int i = j + 1 + tid; i < n; i += P) b[i] = fma(-A[(size_t)i * n + j], bj, b[i]);
    team_sync();
  }
  // back substitution with U
  for (int j = n - 1; j >= 0; --j) {
    if (tid == 0) b[j] *= invd[j];
    team_sync();
    const double bj = b[j];
    for (int i = tid; i < j; i += P) b[i] = fma(-A[(size_t)i * n + j], bj, b[i]);
    team_sync();
  }
}

}  // namespace ck
