// Thread-per-reactor right-hand side ("shallow" vectorisation, Sec. 4 of
// the paper: one ODE system per SIMT lane).  Every lane walks the same
// reaction list, so table reads are uniform (broadcast) and the only
// divergence is the per-species choice of NASA-7 range (Sec. 4, "Select").
#pragma once
#include "ck_common.cuh"

namespace ck {

// Tables as seen by one kernel: shared memory when staged, else global.
struct MechView {
  int S, R;
  const RxnRec* rx;
  const double* th;
  const double* tmid;
  const double* W;
  const double* invW;
  const int16_t* eff_sp;
  const double* eff_m1;
  const double* tab;  // 2^(j/256), j = 0..255
  const double* revp; // explicit reverse rows: log2 A_r, beta_r, Ea_r / (R ln 2)
  int cv;             // 1: constant volume (p is the density)
};

// f = (dT/dt, dY_k/dt) at state y (Eqs. ydot, tdot, wdot, kfor, krev, kc,
// tfits).  y and f are strided (element k at y[k*ys]); X and wd are per-lane
// scratch of S doubles, G of 2S (the species factors 2^(g_k), 2^(-g_k)).
//   rho = p Wbar / (R T), [X_k] = rho Y_k / W_k,
//   k_f = 2^(log2 A + beta log2 T - Ea/(R T ln 2)),
//   1/K_c = (R T/p0)^dnu prod_reactants 2^(g_j) prod_products 2^(-g_j), g_j = (S/R - H/RT)_j / ln 2,
//   k_r = k_f / K_c,
//   c = 1, [M], or P_r/(1+P_r) with P_r = 2^(log2 k0 - log2 k_inf) [M],
//   q = c (k_f prod [X]^nu' - k_r prod [X]^nu''),  wdot_k = sum (nu'' - nu') q,
//   dY_k/dt = wdot_k W_k / rho, dT/dt = -T sum_k (H_k/RT) wdot_k / (rho sum_k Y_k (cp_k/R)/W_k).
// Explicit reverse rows: k_r = 2^(log2 A_r + beta_r log2 T - Ea_r/(R T ln 2)).
// Constant volume (Sec. 3): rho = p (the parameter is the density) and
// H/RT -> U/RT = H/RT - 1, cp/R -> cv/R = cp/R - 1 in dT/dt.
__device__ __forceinline__ void rhs_thread(const MechView& m, double p, const double* y, int ys,
                                           double* f, int fs, double* X, double* G, double* wd) {
  const int S = m.S;
  const double T = y[0];
  const double invT = __drcp_rn(T);
  const double lnT = log(T);
  const double log2T = lnT * INV_LN2;
  const double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  double sumYW = 0.0;
  for (int k = 0; k < S; ++k) sumYW = fma(y[(1 + k) * ys], m.invW[k], sumYW);
  const double rho = m.cv ? p : p / (R_GAS * T * sumYW);
  double Ctot = 0.0;
  for (int k = 0; k < S; ++k) {
    const double xk = rho * (y[(1 + k) * ys] * m.invW[k]);
    X[k] = xk;
    Ctot += xk;
    const double* a = m.th + k * TH_PER_SPECIES + (T < m.tmid[k] ? 0 : TH_STRIDE);
    double g = fma(a[11], lnT, a[12]);
    g = fma(a[13], T, g);
    g = fma(a[14], T2, g);
    g = fma(a[15], T3, g);
    g = fma(a[16], T4, g);
    g = fma(a[17], invT, g);
    ck_exp2_pm(g, m.tab, G[k], G[S + k]);
    wd[k] = 0.0;
  }
  const double* Gm = G + S;
  for (int i = 0; i < m.R; ++i) {
    const RxnRec& r = m.rx[i];
    const double l2kf = fma(-r.EoR2, invT, fma(r.beta, log2T, r.lA2));
    const double kf = ck_exp2(l2kf, m.tab);
    double fwd = X[r.sp[0]];
    if (r.nreac > 1) fwd *= X[r.sp[1]];
    if (r.nreac > 2) fwd *= X[r.sp[2]];
    double net = kf * fwd;
    if (r.rev == 2) {
      const double* ra = m.revp + 3 * r.rev_ix;
      const double kr = ck_exp2(fma(-ra[2], invT, fma(ra[1], log2T, ra[0])), m.tab);
      double rv = X[r.sp[3]];
      if (r.nprod > 1) rv *= X[r.sp[4]];
      if (r.nprod > 2) rv *= X[r.sp[5]];
      net = fma(-kr, rv, net);
    } else if (r.rev) {
      double kci = rt_over_p0_pow(r.dnu, T, invT) * G[r.sp[0]];
      kci *= Gm[r.sp[3]];
      if (r.nreac > 1) kci *= G[r.sp[1]];
      if (r.nprod > 1) kci *= Gm[r.sp[4]];
      if (r.nreac > 2) kci *= G[r.sp[2]];
      if (r.nprod > 2) kci *= Gm[r.sp[5]];
      const double kr = kf * kci;
      double rv = X[r.sp[3]];
      if (r.nprod > 1) rv *= X[r.sp[4]];
      if (r.nprod > 2) rv *= X[r.sp[5]];
      net = fma(-kr, rv, net);
    }
    double q = net;
    if (r.type) {
      double M = Ctot;
      for (int e = r.eff_beg; e < r.eff_beg + r.eff_cnt; ++e) M = fma(m.eff_m1[e], X[m.eff_sp[e]], M);
      if (r.type == 1) {
        q = M * net;
      } else {
        const double l2k0 = fma(-r.E0oR2, invT, fma(r.beta0, log2T, r.lA02));
        const double Pr = ck_exp2(l2k0 - l2kf, m.tab) * M;
        q = net * (Pr / (1.0 + Pr));
      }
    }
    wd[r.sp[0]] -= q;
    if (r.nreac > 1) wd[r.sp[1]] -= q;
    if (r.nreac > 2) wd[r.sp[2]] -= q;
    wd[r.sp[3]] += q;
    if (r.nprod > 1) wd[r.sp[4]] += q;
    if (r.nprod > 2) wd[r.sp[5]] += q;
  }
  const double invrho = __drcp_rn(rho);
  const double cvf = m.cv ? 1.0 : 0.0;
  double cpm = 0.0, hw = 0.0;
  for (int k = 0; k < S; ++k) {
    const double* a = m.th + k * TH_PER_SPECIES + (T < m.tmid[k] ? 0 : TH_STRIDE);
    double cp = fma(a[4], T4, fma(a[3], T3, fma(a[2], T2, fma(a[1], T, a[0])))) - cvf;
    double h = fma(a[10], invT, fma(a[9], T4, fma(a[8], T3, fma(a[7], T2, fma(a[6], T, a[5]))))) - cvf;
    const double w = wd[k];
    cpm = fma(y[(1 + k) * ys] * m.invW[k], cp, cpm);
    hw = fma(h, w, hw);
    f[(1 + k) * fs] = w * (m.W[k] * invrho);
  }
  f[0] = -T * hw / (rho * cpm);
}

// R reactors a thread: rhs_thread's arithmetic for each of them, in the
// same order, with every table record read once for all R (the several-
// reactors-a-lane form of Sec. 4, where a SIMD vector holds several ODE
// systems).  y[j], f[j]: the R states and outputs (element k at [k]); X,
// G, wd: per-lane scratch of R S, 2 R S and R S doubles, reactor j of
// species k at [k R + j].
template <int R>
__device__ __forceinline__ void rhs_thread_r(const MechView& m, const double (&p)[R], const double* const (&y)[R],
                                             double* const (&f)[R], double* X, double* G, double* wd) {
  const int S = m.S;
  double T[R], invT[R], lnT[R], log2T[R], T2[R], T3[R], T4[R], rho[R], Ctot[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    T[j] = y[j][0];
    invT[j] = __drcp_rn(T[j]);
    lnT[j] = log(T[j]);
    log2T[j] = lnT[j] * INV_LN2;
    T2[j] = T[j] * T[j];
    T3[j] = T2[j] * T[j];
    T4[j] = T3[j] * T[j];
  }
  double sumYW[R];
#pragma unroll
  for (int j = 0; j < R; ++j) sumYW[j] = 0.0;
  for (int k = 0; k < S; ++k) {
    const double iw = m.invW[k];
#pragma unroll
    for (int j = 0; j < R; ++j) sumYW[j] = fma(y[j][1 + k], iw, sumYW[j]);
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    rho[j] = m.cv ? p[j] : p[j] / (R_GAS * T[j] * sumYW[j]);
    Ctot[j] = 0.0;
  }
  for (int k = 0; k < S; ++k) {
    const double iw = m.invW[k], tm = m.tmid[k];
    const double* a0 = m.th + k * TH_PER_SPECIES;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const double xk = rho[j] * (y[j][1 + k] * iw);
      X[k * R + j] = xk;
      Ctot[j] += xk;
      const double* a = a0 + (T[j] < tm ? 0 : TH_STRIDE);
      double g = fma(a[11], lnT[j], a[12]);
      g = fma(a[13], T[j], g);
      g = fma(a[14], T2[j], g);
      g = fma(a[15], T3[j], g);
      g = fma(a[16], T4[j], g);
      g = fma(a[17], invT[j], g);
      ck_exp2_pm(g, m.tab, G[k * R + j], G[(S + k) * R + j]);
      wd[k * R + j] = 0.0;
    }
  }
  const double* Gm = G + S * R;
  for (int i = 0; i < m.R; ++i) {
    const RxnRec& r = m.rx[i];
    const int s0 = r.sp[0] * R, s1 = r.sp[1] * R, s2 = r.sp[2] * R;
    const int s3 = r.sp[3] * R, s4 = r.sp[4] * R, s5 = r.sp[5] * R;
    double net[R], l2kf[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      l2kf[j] = fma(-r.EoR2, invT[j], fma(r.beta, log2T[j], r.lA2));
      const double kf = ck_exp2(l2kf[j], m.tab);
      double fwd = X[s0 + j];
      if (r.nreac > 1) fwd *= X[s1 + j];
      if (r.nreac > 2) fwd *= X[s2 + j];
      net[j] = kf * fwd;
      if (r.rev == 2) {
        const double* ra = m.revp + 3 * r.rev_ix;
        const double kr = ck_exp2(fma(-ra[2], invT[j], fma(ra[1], log2T[j], ra[0])), m.tab);
        double rv = X[s3 + j];
        if (r.nprod > 1) rv *= X[s4 + j];
        if (r.nprod > 2) rv *= X[s5 + j];
        net[j] = fma(-kr, rv, net[j]);
      } else if (r.rev) {
        double kci = rt_over_p0_pow(r.dnu, T[j], invT[j]) * G[s0 + j];
        kci *= Gm[s3 + j];
        if (r.nreac > 1) kci *= G[s1 + j];
        if (r.nprod > 1) kci *= Gm[s4 + j];
        if (r.nreac > 2) kci *= G[s2 + j];
        if (r.nprod > 2) kci *= Gm[s5 + j];
        const double kr = kf * kci;
        double rv = X[s3 + j];
        if (r.nprod > 1) rv *= X[s4 + j];
        if (r.nprod > 2) rv *= X[s5 + j];
        net[j] = fma(-kr, rv, net[j]);
      }
    }
    double q[R];
#pragma unroll
    for (int j = 0; j < R; ++j) q[j] = net[j];
    if (r.type) {
      double M[R];
#pragma unroll
      for (int j = 0; j < R; ++j) M[j] = Ctot[j];
      for (int e = r.eff_beg; e < r.eff_beg + r.eff_cnt; ++e) {
        const double em = m.eff_m1[e];
        const int es = m.eff_sp[e] * R;
#pragma unroll
        for (int j = 0; j < R; ++j) M[j] = fma(em, X[es + j], M[j]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (r.type == 1) {
          q[j] = M[j] * net[j];
        } else {
          const double l2k0 = fma(-r.E0oR2, invT[j], fma(r.beta0, log2T[j], r.lA02));
          const double Pr = ck_exp2(l2k0 - l2kf[j], m.tab) * M[j];
          q[j] = net[j] * (Pr / (1.0 + Pr));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      wd[s0 + j] -= q[j];
      if (r.nreac > 1) wd[s1 + j] -= q[j];
      if (r.nreac > 2) wd[s2 + j] -= q[j];
      wd[s3 + j] += q[j];
      if (r.nprod > 1) wd[s4 + j] += q[j];
      if (r.nprod > 2) wd[s5 + j] += q[j];
    }
  }
  const double cvf = m.cv ? 1.0 : 0.0;
  double invrho[R], cpm[R], hw[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    invrho[j] = __drcp_rn(rho[j]);
    cpm[j] = 0.0;
    hw[j] = 0.0;
  }
  for (int k = 0; k < S; ++k) {
    const double* a0 = m.th + k * TH_PER_SPECIES;
    const double tm = m.tmid[k], Wk = m.W[k], iw = m.invW[k];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const double* a = a0 + (T[j] < tm ? 0 : TH_STRIDE);
      const double cp = fma(a[4], T4[j], fma(a[3], T3[j], fma(a[2], T2[j], fma(a[1], T[j], a[0])))) - cvf;
      const double h =
          fma(a[10], invT[j], fma(a[9], T4[j], fma(a[8], T3[j], fma(a[7], T2[j], fma(a[6], T[j], a[5]))))) - cvf;
      const double w = wd[k * R + j];
      cpm[j] = fma(y[j][1 + k] * iw, cp, cpm[j]);
      hw[j] = fma(h, w, hw[j]);
      f[j][1 + k] = w * (Wk * invrho[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) f[j][0] = -T[j] * hw[j] / (rho[j] * cpm[j]);
}

}  // namespace ck
