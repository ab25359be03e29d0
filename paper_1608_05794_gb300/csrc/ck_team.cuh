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

// K block-wide sums at once (each in the order of team_sum, so the values
// are those of K calls), with one pair of barriers.  K <= 4, blockDim <= 256.
template <int K>
__device__ __forceinline__ void team_sum_n(double (&v)[K], double* red) {
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_allsum(v[q]);
  const int nw = blockDim.x >> 5;
  if (nw == 1) return;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) red[8 * q + (threadIdx.x >> 5)] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[8 * q + i];
    v[q] = s;
  }
}

__device__ __forceinline__ void team_sync() {
  if (blockDim.x == 32) __syncwarp();
  else __syncthreads();
}

// Shared-memory work arrays of one team.
// The Jacobian processes reactions in chunks of m.chunk (64 if n <= 56, else
// 256), so the per-reaction arrays hold one chunk; the right-hand side, which
// keeps one value per reaction, uses them as one array of 10 m.chunk values
// when all reactions fit.  cs aliases Gp (free once the reaction passes are
// done).  Gp_k = 2^(g_k) and Gm_k = 2^(-g_k) with g_k = (S/R -
// H/RT)_k / ln 2, so that 1/K_c of Eq. kc is a product of species factors.
struct TeamBufs {
  double *X, *Gp, *hRT, *cpR, *Gm, *wd, *aT, *E, *u, *cs;  // [S]
  double *q, *dqT, *D;                                        // [chunk]
  double* P;                                                  // [chunk * JP] Jacobian partials
  double* red;                                                // [48]
};

// Mixture quantities shared by the RHS and the Jacobian.
struct Mix {
  double T, invT, lnT, log2T, T2, T3, T4, rho, invrho, Wbar, Ctot;
  double dcpm;  // this thread's part of sum_k Y_k/W_k d(cp_k/R)/dT (Jacobian only)
};

// Species pass: rho, [X_k], Gibbs / enthalpy / heat-capacity polynomials.
__device__ __forceinline__ void team_species(const DevMech& m, double p, const double* y,
                                             TeamBufs& b, Mix& x, bool want_dcp, const double* tab) {
  const int S = m.S;
  x.T = y[0];
  // the temperature functions are formed by the first warp alone (an FP64
  // instruction costs every warp that issues it a full slot) and handed to
  // the others through red[40..45] across the barriers of the sum below
  double* tf = b.red + 40;
  if (threadIdx.x < 32) {
    x.invT = rcp_rn(x.T);
    x.lnT = log(x.T);
    x.log2T = x.lnT * INV_LN2;
    x.T2 = x.T * x.T;
    x.T3 = x.T2 * x.T;
    x.T4 = x.T3 * x.T;
    if (threadIdx.x == 0) {
      tf[0] = x.invT;
      tf[1] = x.lnT;
      tf[2] = x.log2T;
      tf[3] = x.T2;
      tf[4] = x.T3;
      tf[5] = x.T4;
    }
  }
  double s = 0.0;
  for (int k = threadIdx.x; k < S; k += blockDim.x) s = fma(y[1 + k], m.invW[k], s);
  const double sumYW = team_sum(s, b.red);
  if (threadIdx.x >= 32) {
    x.invT = tf[0];
    x.lnT = tf[1];
    x.log2T = tf[2];
    x.T2 = tf[3];
    x.T3 = tf[4];
    x.T4 = tf[5];
  }
  // the mean molar mass, rho and 1 / rho likewise by the first warp,
  // through red[32..34]
  double* sc = b.red + 32;
  if (threadIdx.x < 32) {
    x.Wbar = rcp_rn(sumYW);
    x.rho = m.cv ? p : p / (R_GAS * x.T * sumYW);  // constant volume: p is the density
    x.invrho = rcp_rn(x.rho);
    if (threadIdx.x == 0) {
      sc[0] = x.Wbar;
      sc[1] = x.rho;
      sc[2] = x.invrho;
    }
  }
  if (blockDim.x > 32) {
    __syncthreads();
    if (threadIdx.x >= 32) {
      x.Wbar = sc[0];
      x.rho = sc[1];
      x.invrho = sc[2];
    }
  }
  double c = 0.0, dcpm = 0.0;
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
    g = fma(a[17], x.invT, g);
    ck_exp2_pm(g, tab, b.Gp[k], b.Gm[k]);
    b.cpR[k] = fma(a[4], x.T4, fma(a[3], x.T3, fma(a[2], x.T2, fma(a[1], x.T, a[0]))));
    b.hRT[k] = fma(a[10], x.invT, fma(a[9], x.T4, fma(a[8], x.T3, fma(a[7], x.T2, fma(a[6], x.T, a[5])))));
    if (want_dcp)
      dcpm = fma(y[1 + k] * m.invW[k], fma(4.0 * a[4], x.T3, fma(3.0 * a[3], x.T2, fma(2.0 * a[2], x.T, a[1]))), dcpm);
    b.wd[k] = 0.0;
    b.aT[k] = 0.0;
    b.E[k] = 0.0;
    b.u[k] = 0.0;
  }
  x.dcpm = dcpm;
  x.Ctot = team_sum(c, b.red);
}

// A 96-byte reaction record in six 16-byte loads (the fields are then read
// from registers).
__device__ __forceinline__ RxnRec load_rxn(const RxnRec* src) {
  RxnRec r;
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* t = reinterpret_cast<int4*>(&r);
#pragma unroll
  for (int q = 0; q < 6; ++q) t[q] = __ldg(s + q);
  return r;
}

// Rates of one reaction at the mixture state.  With want_jac also the
// partial-derivative pieces used by the Jacobian (see team_jacobian).
__device__ __forceinline__ void team_reaction(const DevMech& m, const RxnRec& r, const Mix& x,
                                              const TeamBufs& b, const double* tab, int i,
                                              bool want_jac) {
  // i: index of the reaction inside the current chunk
  const double* X = b.X;
  const double l2kf = fma(-r.EoR2, x.invT, fma(r.beta, x.log2T, r.lA2));
  const double kf = ck_exp2(l2kf, tab);
  double fwd = X[r.sp[0]];
  if (r.nreac > 1) fwd *= X[r.sp[1]];
  if (r.nreac > 2) fwd *= X[r.sp[2]];
  double kr = 0.0, rv = 0.0, dlnkc = 0.0;
  if (r.rev == 2) {
    // explicit reverse Arrhenius; for the Jacobian, d ln k_r/dT enters as
    // d ln k_f/dT - d ln K_c/dT, so dlnkc carries their difference
    const double* ra = m.revp + 3 * r.rev_ix;
    kr = ck_exp2(fma(-ra[2], x.invT, fma(ra[1], x.log2T, ra[0])), tab);
    rv = X[r.sp[3]];
    if (r.nprod > 1) rv *= X[r.sp[4]];
    if (r.nprod > 2) rv *= X[r.sp[5]];
    if (want_jac) {
      const double dlnkf = fma(r.EoR2 * LN2, x.invT, r.beta) * x.invT;
      dlnkc = dlnkf - fma(ra[2] * LN2, x.invT, ra[1]) * x.invT;
    }
  } else if (r.rev) {
    // 1/K_c = (R T/p0)^dnu prod_reactants Gp prod_products Gm (Eq. kc)
    double kci = rt_over_p0_pow(r.dnu, x.T, x.invT) * b.Gp[r.sp[0]];
    kci *= b.Gm[r.sp[3]];
    if (r.nreac > 1) kci *= b.Gp[r.sp[1]];
    if (r.nprod > 1) kci *= b.Gm[r.sp[4]];
    if (r.nreac > 2) kci *= b.Gp[r.sp[2]];
    if (r.nprod > 2) kci *= b.Gm[r.sp[5]];
    kr = kf * kci;
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
      dlnkc = (hs - r.dnu_d) * x.invT;
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
      const double inv1p = rcp_rn(1.0 + Pr);
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
    const double w = dcdM * net;
    // d q / d[X] slot by slot: c k_f prod of the other reactant slots, and
    // -c k_r prod of the other product slots
    double* P = b.P + (size_t)i * JP;
    const double x0 = X[r.sp[0]];
    if (r.nreac == 1) {
      P[0] = ckf;
    } else if (r.nreac == 2) {
      const double x1 = X[r.sp[1]];
      P[0] = ckf * x1;
      P[1] = ckf * x0;
    } else {
      const double x1 = X[r.sp[1]], x2 = X[r.sp[2]];
      P[0] = ckf * (x1 * x2);
      P[1] = ckf * (x0 * x2);
      P[2] = ckf * (x0 * x1);
    }
    if (r.rev) {
      const double y0 = X[r.sp[3]];
      if (r.nprod == 1) {
        P[3] = -ckr;
      } else if (r.nprod == 2) {
        const double y1 = X[r.sp[4]];
        P[3] = -ckr * y1;
        P[4] = -ckr * y0;
      } else {
        const double y1 = X[r.sp[4]], y2 = X[r.sp[5]];
        P[3] = -ckr * (y1 * y2);
        P[4] = -ckr * (y0 * y2);
        P[5] = -ckr * (y0 * y1);
      }
    }
    P[6] = w;
    // D = sum_j dq/d[X_j] [X_j]: Euler's theorem for the mass-action
    // products (homogeneous of degree nreac / nprod) plus the [M] part.
    const double D = fma(ckf * fwd, r.nreac_d, -(ckr * rv) * r.nprod_d) + M * w;
    b.D[i] = D;
    // dq/dT at fixed [X], then the total derivative at fixed Y (d[X]/dT =
    // -[X]/T at constant pressure, 0 at constant volume)
    const double dqTX = fma(dcdT, net, ckf * fwd * dlnkf - ckr * rv * (dlnkf - dlnkc));
    b.dqT[i] = m.cv ? dqTX : fma(-D, x.invT, dqTX);
  }
}

// f(y) for one reactor.  y, f: shared memory, n = S + 1.
static __device__ __noinline__ void team_rhs(const DevMech& m, const double* tab, double p,
                                             const double* y, double* f, TeamBufs b) {
  Mix x;
  team_species(m, p, y, b, x, false, tab);
  team_sync();
  const int NC = m.n_chunks, CH = m.chunk;
  if (m.R <= (3 + JP) * CH) {
    // the right-hand side needs one value per reaction, so the whole chunk
    // scratch (q, dqT, D, P are contiguous) holds every rate of progress at
    // once: one reaction pass and one gather, two barriers in all.  The
    // gather sums in the same order as the chunked form below.
    for (int i = threadIdx.x; i < m.R; i += blockDim.x) {
      const RxnRec r = load_rxn(m.rxn + i);
      team_reaction(m, r, x, b, tab, i, false);
    }
    team_sync();
    for (int kk = threadIdx.x; kk < m.S; kk += blockDim.x) {
      const int k = m.rsp[kk];
      double w = b.wd[k];
      for (int e = m.csr_ptr[k]; e < m.csr_ptr[k + 1]; ++e) {
        const CsrTerm t = m.csr[e];
        w = fma(t.nu, b.q[t.rx], w);
      }
      b.wd[k] = w;
    }
    team_sync();
  } else {
    for (int c = 0; c < NC; ++c) {
      const int base = c * CH;
      for (int li = threadIdx.x; li < CH; li += blockDim.x)
        if (base + li < m.R) {
          const RxnRec r = load_rxn(m.rxn + base + li);
          team_reaction(m, r, x, b, tab, li, false);
        }
      team_sync();
      for (int k = threadIdx.x; k < m.S; k += blockDim.x) {
        const int* cp = m.csr_cptr + k * (NC + 1) + c;
        double w = b.wd[k];
        for (int e = cp[0]; e < cp[1]; ++e) {
          const CsrTerm t = m.csr[e];
          w = fma(t.nu, b.q[t.rx - base], w);
        }
        b.wd[k] = w;
      }
      team_sync();
    }
  }
  const double invrho = x.invrho;
  const double cvf = m.cv ? 1.0 : 0.0;  // constant volume: U/RT = H/RT - 1, cv/R = cp/R - 1
  double cpm = 0.0, hw = 0.0;
  for (int k = threadIdx.x; k < m.S; k += blockDim.x) {
    const double w = b.wd[k];
    cpm = fma(y[1 + k] * m.invW[k], b.cpR[k] - cvf, cpm);
    hw = fma(b.hRT[k] - cvf, w, hw);
    f[1 + k] = w * (m.W[k] * invrho);
  }
  double sums[2] = {cpm, hw};
  team_sum_n(sums, b.red);
  cpm = sums[0];
  hw = sums[1];
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
// capacities in units of R.  Constant volume (rho fixed; u_k, c_v in Eq.
// tdot): the Wbar and 1/T terms vanish, a_k is taken at fixed [X], and H/RT,
// cp/R become U/RT = H/RT - 1 and cv/R = cp/R - 1:
//   J[1+k][1+j] = W_k (A_kj + u_k) / W_j,   J[1+k][0] = W_k a_k / rho,
//   J[0][1+j]   = -(T cs_j / cvm + Tdot cv_j / cvm) / W_j,
//   J[0][0]     = -(sum cv_k wdot_k + T sum U_k/RT a_k)/(rho cvm) - Tdot dcpm/cvm.
static __device__ void team_jacobian(const DevMech& m, const double* tab, double p, const double* y,
                              double* f, double* J, TeamBufs& b, Mix& x) {
  const int S = m.S, n = m.n;
  team_species(m, p, y, b, x, true, tab);
  // species block A starts at zero (the whole matrix is cleared: the
  // temperature row and column are written whole further down); chunk by
  // chunk, every entry touched by the chunk and every species sum (wdot,
  // d wdot/dT, E = sum nu D and the dense third-body part u) adds its
  // fixed-order sum of contributions, one thread per target, the targets in
  // one list sorted by length so that a warp's lanes do similar work
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) J[e] = 0.0;
  team_sync();
  const int NC = m.n_chunks, CH = m.chunk;
  for (int c = 0; c < NC; ++c) {
    const int base = c * CH;
    for (int li = threadIdx.x; li < CH; li += blockDim.x)
      if (base + li < m.R) {
        const RxnRec r = load_rxn(m.rxn + base + li);
        team_reaction(m, r, x, b, tab, li, true);
      }
    team_sync();
    // every target of the chunk (species-block entries and the per-species
    // sums wdot, a, E, u, whose arrays wd, aT, E, u are contiguous) adds its
    // fixed-order sum of terms; one thread per target, no conflicts
    for (int e = m.jc_ptr[c] + threadIdx.x; e < m.jc_ptr[c + 1]; e += blockDim.x) {
      const JcEntry h = m.jc[e];
      double* tgt = h.idx < n * n ? J + h.idx : b.wd + (h.idx - n * n);
      double a = *tgt;
      for (int t = h.beg; t < h.end; ++t) {
        const JcTerm ct = m.jt[t];
        a = fma(ct.coef, b.q[ct.pidx], a);
      }
      *tgt = a;
    }
    team_sync();
  }
  // column sums for the temperature row, and the RHS itself.  Constant
  // volume: rho is fixed, so every term that comes from d rho/dT or
  // d rho/dY (cpf) drops out, and U/RT = H/RT - 1, cv/R = cp/R - 1 take the
  // places of H/RT and cp/R (cvf).  The contributions were pre-scaled by
  // W_k/W_j, so J holds A'_kj = W_k A_kj / W_j here.
  const double invrho = x.invrho;
  const double cvf = m.cv ? 1.0 : 0.0, cpf = 1.0 - cvf;
  double cpm = 0.0, hw = 0.0, he = 0.0, dcpm = x.dcpm, cw = 0.0, ha = 0.0, eu = 0.0;
  for (int k = threadIdx.x; k < S; k += blockDim.x) {
    const double yk = y[1 + k] * m.invW[k];
    const double e = b.hRT[k] - cvf, c = b.cpR[k] - cvf;
    cpm = fma(yk, c, cpm);
    hw = fma(e, b.wd[k], hw);
    he = fma(b.hRT[k], b.E[k], he);
    cw = fma(c, b.wd[k], cw);
    ha = fma(e, b.aT[k], ha);
    eu = fma(e, b.u[k], eu);
    f[1 + k] = b.wd[k] * (m.W[k] * invrho);
    // per row: e_k / W_k for the column sums, and the dense part of the
    // species block, W_k u_k + W_k Wbar (wdot_k - E_k) / rho (constant p)
    b.hRT[k] = e * m.invW[k];
    b.u[k] = m.W[k] * fma(cpf * x.Wbar * invrho, b.wd[k] - b.E[k], b.u[k]);
  }
  double s4[4] = {cpm, dcpm, hw, he}, s3[3] = {cw, ha, eu};
  team_sum_n(s4, b.red);
  team_sum_n(s3, b.red);
  cpm = s4[0];
  dcpm = s4[1];
  hw = s4[2];
  he = s4[3];
  cw = s3[0];
  ha = s3[1];
  eu = s3[2];
  // Tdot and 1 / cpm by the first warp, handed over through red[35..36]
  // across the barrier below
  double Tdot = 0.0, inv_cpm = 0.0;
  double* sc = b.red + 32;
  if (threadIdx.x < 32) {
    Tdot = -x.T * hw / (x.rho * cpm);
    inv_cpm = rcp_rn(cpm);
    if (threadIdx.x == 0) {
      sc[3] = Tdot;
      sc[4] = inv_cpm;
    }
  }
  // cs_j = sum_k e_k (A_kj + u_k) = W_j sum_k (e_k / W_k) A'_kj + sum_k e_k u_k
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < S; ++k) s = fma(b.hRT[k], J[(size_t)(1 + k) * n + 1 + j], s);
    b.cs[j] = fma(m.W[j], s, eu);
  }
  team_sync();
  if (threadIdx.x >= 32) {
    Tdot = sc[3];
    inv_cpm = sc[4];
  }
  // species block (J_kj = A'_kj + dense_k / W_j) and temperature column
  // entries e = k S + j of the species block, (k, j) advanced without
  // dividing by the runtime S
  {
    const int P = blockDim.x, dk = P / S, dj = P - (P / S) * S;
    int k = threadIdx.x / S, j = threadIdx.x - k * S;
    for (; k < S;) {
      double* a = J + (size_t)(1 + k) * n + 1 + j;
      *a = fma(b.u[k], m.invW[j], *a);
      k += dk;
      j += dj;
      if (j >= S) {
        j -= S;
        ++k;
      }
    }
  }
  for (int k = threadIdx.x; k < S; k += blockDim.x)
    J[(size_t)(1 + k) * n] = m.W[k] * invrho * fma(cpf * b.wd[k], x.invT, b.aT[k]);
  const double inv_rc = invrho * inv_cpm;
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    const double t1 = x.T * (x.rho * b.cs[j] - cpf * x.Wbar * he) * inv_rc;
    const double t2 = Tdot * fma(b.cpR[j] - cvf, inv_cpm, -cpf * x.Wbar);
    J[1 + j] = -(t1 + t2) * m.invW[j];
  }
  if (threadIdx.x == 0) {
    J[0] = -fma(x.T, ha, cw) * inv_rc - Tdot * fma(dcpm, inv_cpm, -cpf * x.invT);
    f[0] = Tdot;
  }
  team_sync();
}

// LU with partial pivoting, register-tiled.  The CTA is a G x G grid of
// threads laid out column-major: thread t = tc G + tr holds the elements
// (tr + G r, tc + G c), r, c < T, of the n x n row-major matrix A (shared
// memory, n <= G T) in registers, so the G owners of a matrix column are G
// consecutive lanes of one warp.  An FP64 instruction costs a full warp slot
// of the FP64 pipe however few lanes are active, and the non-FP64 work
// around it sets how densely those slots fill, so step k (slot row and
// column kq = k / G, position kt = k % G):
//   1. the owners of column k pick the pivot among rows i >= k (magnitudes
//      compared as integers: the bit pattern of |v| orders like |v|, NaN
//      above +inf; ties take the smallest row) with shuffles of (magnitude,
//      row) inside their group, fetch the pivot's value from the lane that
//      holds its row, form 1 / pivot, and write the column below the
//      diagonal, as it stands after the exchange of rows k and p (row p
//      takes row k's entry), to lb; their whole warp scales it into the
//      multipliers;
//   2. barrier; the owners of rows k and p exchange the two rows through
//      shared memory, which also publishes the new row k (the pivot row) in
//      ub; barrier;
//   3. every thread applies A_ij -= l_i u_j to its tile; column k below the
//      diagonal becomes the multipliers.
// Two barriers a step.  The slot bounds of a step are compile-time
// constants (the step is instantiated for every kq), so the update carries
// no per-element predicates: rows and columns beyond n are zero and lb / ub
// are zero-padded there, and only slot row and column kq need per-thread
// tests.  lb is double-buffered because the next pivot's owners write it
// while other warps may still read the current one.
// PRE = false: piv[k] receives the row swapped with row k (LAPACK order) and
// A the factors.  PRE = true (the form the stage solves of ROS4 take): piv
// receives the composite row permutation (row i of PA is row piv[i] of A),
// and the strict upper triangle of U is stored pre-divided by its diagonal,
// so that a solve gathers b once and needs no division in back
// substitution.  On return A holds the unit lower factor below the diagonal
// and the upper factor on and above it; invd[k] = 1 / U_kk.  Returns 0, or
// k+1 when pivot k is zero or not finite (the same in every thread).
// scratch: lu_scratch_words<G, T>() doubles of shared memory.
// Bits of |v| as an unsigned integer (orders like |v|; NaN above +inf).
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned long long abs_key(float v) {
  return (unsigned long long)((unsigned)__float_as_int(v) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long inf_key(double) { return 0x7ff0000000000000ULL; }
__device__ __forceinline__ unsigned long long inf_key(float) { return 0x7f800000ULL; }

template <int G, int T>
__host__ __device__ constexpr int lu_scratch_words() { return 4 * G * T + 2; }


// Slot row ps (>= KQ; the same in every thread) of a tile out to / in from
// a shared row buffer.  The switch is on a CTA-uniform value, so only the
// taken case executes, instead of a predicated copy of every slot row.
template <int G, int T, int KQ, class F>
__device__ __forceinline__ void lu_slot_row_out(const F (&a)[T][T], int ps, int tn, F* row) {
  const int tc = threadIdx.x / G;
  if constexpr (KQ < T) {
    if (ps == KQ) {
#pragma unroll
      for (int c = 0; c < T; ++c)
        if (c < tn) row[tc + G * c] = a[KQ][c];
    } else {
      lu_slot_row_out<G, T, KQ + 1>(a, ps, tn, row);
    }
  }
}
template <int G, int T, int KQ, class F>
__device__ __forceinline__ void lu_slot_row_in(F (&a)[T][T], int ps, int tn, const F* row) {
  const int tc = threadIdx.x / G;
  if constexpr (KQ < T) {
    if (ps == KQ) {
#pragma unroll
      for (int c = 0; c < T; ++c)
        if (c < tn) a[KQ][c] = row[tc + G * c];
    } else {
      lu_slot_row_in<G, T, KQ + 1>(a, ps, tn, row);
    }
  }
}

// Pivot search of step k = KQ G + kt in its branch-free form, run by every
// lane of the warp that holds column k: each group of G lanes searches its
// own column, so the warp stays converged, and the group of column k alone
// stores the multipliers (column k below the diagonal, as it stands after
// the exchange of rows k and p, times 1 / pivot, each lane scaling its own
// rows) in lb.  Returns the pivot row, or -1 when the pivot is zero or not
// finite; ip receives 1 / pivot.  The results are bitwise those of the
// owner-group form in lu_step.
template <int G, int T, int KQ, bool FULL, class F>
__device__ __forceinline__ int lu_pivot(const F (&a)[T][T], int n, int kt, F* scratch, F& ip) {
  constexpr int GT = G * T;
  const int tid = threadIdx.x, tr = tid % G, tc = tid / G;
  const int k = KQ * G + kt;
  const int tn = FULL ? T : (n + G - 1) / G;
  F* lb = scratch + (k & 1) * GT;
  const unsigned long long INFB = inf_key(F(0));
  unsigned long long best = 0;
  F bv = F(0);
  int bi = n;
#pragma unroll
  for (int r = KQ; r < T; ++r) {
    if (r >= tn) break;
    const int i = tr + G * r;
    const bool ok = (r > KQ || tr >= kt) && i < n;
    const unsigned long long key = abs_key(a[r][KQ]);
    const bool take = ok && key > best;
    best = take ? key : best;
    bv = take ? a[r][KQ] : bv;
    bi = take ? i : bi;
  }
#pragma unroll
  for (int off = 1; off < G; off <<= 1) {
    const unsigned long long ok_ = __shfl_xor_sync(0xffffffffu, best, off, G);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off, G);
    const bool take = ok_ > best || (ok_ == best && oi < bi);
    best = take ? ok_ : best;
    bi = take ? oi : bi;
  }
  const int p = bi;
  const bool sing = p >= n || best == 0 || best >= INFB;
  bv = __shfl_sync(0xffffffffu, bv, p % G, G);  // the value from the lane that holds row p
  const F akk = __shfl_sync(0xffffffffu, a[KQ][KQ], kt, G);
  ip = rcp_rn(sing ? F(1) : bv);
  if (tc == kt && !sing) {
#pragma unroll
    for (int r = KQ; r < T; ++r) {
      if (r >= tn) break;
      const int i = tr + G * r;
      if (i > k && i < n) lb[i] = ((i == p) ? akk : a[r][KQ]) * ip;
    }
  }
  return sing ? -1 : p;
}

// The pivot of step k, published by lane tr = 0 of column k's group.
template <int G, bool PRE, class F>
__device__ __forceinline__ void lu_publish(int k, int p, F ip, int* piv, F* invd, int* sp) {
  const int tid = threadIdx.x;
  if (tid / G == k % G && tid % G == 0) {
    *sp = p;
    if (p >= 0) {
      invd[k] = ip;
      if (PRE) {
        const int t = piv[k];
        piv[k] = piv[p];
        piv[p] = t;
      } else {
        piv[k] = p;
      }
    }
  }
}

// One pivot step at compile-time slot kq (see lu_reg).  Returns false when
// the pivot is zero or not finite.
template <int G, int T, int KQ, bool PRE, bool FULL, class F>
__device__ __forceinline__ bool lu_step(F (&a)[T][T], int n, int kt, int* piv, F* invd, F* scratch) {
  constexpr int GT = G * T;
  const int tid = threadIdx.x, tr = tid % G, tc = tid / G, lane = tid & 31;
  const int k = KQ * G + kt;
  // slots that hold rows / columns below n (warp-uniform); FULL: all T
  const int tn = FULL ? T : (n + G - 1) / G;
  F* lb = scratch + (k & 1) * GT;
  F* ub = scratch + 2 * GT;
  F* xb = scratch + 3 * GT;
  int* sp = reinterpret_cast<int*>(scratch + 4 * GT);
  const unsigned long long INFB = inf_key(F(0));
  // 1. pivot search, reciprocal and multipliers: the warp holding column k.
  // The branch-free form measured faster everywhere but in the full-tile
  // FP64 factorization of the 8 x 8 team, which keeps the owner-group form.
  constexpr bool BF = !(G == 8 && FULL && sizeof(F) == 8);
  const int owner_warp = (kt * G) >> 5;
  if constexpr (BF) {
    if ((tid >> 5) == owner_warp) {
      F ip;
      const int p0 = lu_pivot<G, T, KQ, FULL>(a, n, kt, scratch, ip);
      lu_publish<G, PRE>(k, p0, ip, piv, invd, sp);
    }
  } else if ((tid >> 5) == owner_warp) {
    const int base = (kt * G) & 31;  // first lane of the owner group
    bool sing = false;
    F ip = F(0);
    if (tc == kt) {
      const unsigned gmask = (G >= 32 ? 0xffffffffu : ((1u << G) - 1u)) << base;
      unsigned long long best = 0;
      F bv = F(0);
      int bi = n;
#pragma unroll
      for (int r = KQ; r < T; ++r) {
        if (r >= tn) break;
        const int i = tr + G * r;
        const bool ok = (r > KQ || tr >= kt) && i < n;
        const unsigned long long key = abs_key(a[r][KQ]);
        if (ok && key > best) {
          best = key;
          bv = a[r][KQ];
          bi = i;
        }
      }
#pragma unroll
      for (int off = 1; off < G; off <<= 1) {
        const unsigned long long ok_ = __shfl_xor_sync(gmask, best, off, G);
        const int oi = __shfl_xor_sync(gmask, bi, off, G);
        if (ok_ > best || (ok_ == best && oi < bi)) {
          best = ok_;
          bi = oi;
        }
      }
      const int p = bi;
      sing = p >= n || best == 0 || best >= INFB;
      bv = __shfl_sync(gmask, bv, p % G, G);  // the value from the lane that holds row p
      // column k as it stands after the exchange: row p takes row k's entry
      const F akk = __shfl_sync(gmask, a[KQ][KQ], kt, G);
      if (!sing) {
        ip = rcp_rn(bv);
#pragma unroll
        for (int r = KQ; r < T; ++r) {
          if (r >= tn) break;
          const int i = tr + G * r;
          if (i > k && i < n) lb[i] = (i == p) ? akk : a[r][KQ];
        }
      }
      if (tr == 0) {
        *sp = sing ? -1 : p;
        if (!sing) {
          invd[k] = ip;
          if (PRE) {
            const int t = piv[k];
            piv[k] = piv[p];
            piv[p] = t;
          } else {
            piv[k] = p;
          }
        }
      }
    }
    __syncwarp();
    sing = __shfl_sync(0xffffffffu, (int)sing, base) != 0;
    ip = __shfl_sync(0xffffffffu, ip, base);
    if (!sing)
      for (int i = k + 1 + lane; i < n; i += 32) lb[i] *= ip;
  }
  __syncthreads();
  const int p = *sp;
  if (p < 0) return false;
  // 2. exchange rows k and p; the new row k (the pivot row) lands in ub
  const int pt = p % G, ps = p / G;
  if (tr == kt) {
#pragma unroll
    for (int c = 0; c < T; ++c)
      if (c < tn) (p != k ? xb : ub)[tc + G * c] = a[KQ][c];
  }
  if (p != k && tr == pt) lu_slot_row_out<G, T, KQ>(a, ps, tn, ub);
  __syncthreads();
  if (p != k) {
    if (tr == kt) {
#pragma unroll
      for (int c = 0; c < T; ++c)
        if (c < tn) a[KQ][c] = ub[tc + G * c];
    }
    if (tr == pt) lu_slot_row_in<G, T, KQ>(a, ps, tn, xb);
  }
  // 3. rank-one update of the trailing tile; column k takes the multipliers.
  // Slots at or beyond tn hold only padding and are left alone.
  F u[T];
#pragma unroll
  for (int c = KQ; c < T; ++c) u[c] = c < tn ? ub[tc + G * c] : F(0);
  // slot column KQ needs work only in warps holding a column >= k (the G
  // lanes of a column are consecutive, so the warp's largest tc is its last
  // lane's): a warp-uniform test that lets the other warps skip it.  The
  // FP32 factorization of the precision form measured faster without it.
  const bool wcol = sizeof(F) < 8 || ((tid | 31) / G) >= kt;
#pragma unroll
  for (int r = KQ; r < T; ++r) {
    if (r >= tn) break;
    const bool live = r > KQ || tr > kt;  // row tr + G r lies below row k
    const F li = live ? lb[tr + G * r] : F(0);
#pragma unroll
    for (int c = KQ + 1; c < T; ++c) {
      if (c >= tn) break;
      a[r][c] = fma(-li, u[c], a[r][c]);
    }
    if (wcol) {
      if (tc > kt) a[r][KQ] = fma(-li, u[KQ], a[r][KQ]);
      else if (tc == kt && live) a[r][KQ] = li;
    }
  }
  return true;
}

template <int G, int T, bool PRE, bool FULL, int KQ, class F>
__device__ __forceinline__ int lu_slots(F (&a)[T][T], int n, int* piv, F* invd, F* scratch) {
  if constexpr (KQ < T) {
    for (int kt = 0; kt < G; ++kt) {
      if (KQ * G + kt >= n) return 0;
      if (!lu_step<G, T, KQ, PRE, FULL>(a, n, kt, piv, invd, scratch)) return KQ * G + kt + 1;
    }
    return lu_slots<G, T, PRE, FULL, KQ + 1>(a, n, piv, invd, scratch);
  } else {
    return 0;
  }
}

template <int G, int T, bool PRE = false, class F>
__device__ int lu_reg(F* A, int n, int* piv, F* invd, F* scratch) {
  const int tid = threadIdx.x, tr = tid % G, tc = tid / G;
  for (int e = tid; e < lu_scratch_words<G, T>(); e += blockDim.x) scratch[e] = F(0);
  for (int i = tid; i < n; i += blockDim.x) piv[i] = i;
  F a[T][T];
#pragma unroll
  for (int r = 0; r < T; ++r)
#pragma unroll
    for (int c = 0; c < T; ++c) {
      const int i = tr + G * r, j = tc + G * c;
      a[r][c] = (i < n && j < n) ? A[i * n + j] : F(0);
    }
  __syncthreads();
  // every slot holds real rows and columns (n > G (T - 1)): the steps need no
  // run-time slot bound
  const int info = (n > G * (T - 1)) ? lu_slots<G, T, PRE, true, 0>(a, n, piv, invd, scratch)
                                     : lu_slots<G, T, PRE, false, 0>(a, n, piv, invd, scratch);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < T; ++r) {
    const int i = tr + G * r;
    const F di = (PRE && i < n) ? invd[i] : F(1);
#pragma unroll
    for (int c = 0; c < T; ++c) {
      const int j = tc + G * c;
      // slot (r, c) lies wholly above the diagonal when c > r and wholly
      // below it when c < r (tr, tc < G), so only c == r needs the test
      F v = a[r][c];
      if (PRE && (c > r || (c == r && tc > tr))) v = a[r][c] * di;
      if (i < n && j < n) A[i * n + j] = v;
    }
  }
  __syncthreads();
  return info;
}

// Solve (LU) x = b in place with one warp (b in shared memory).  Must be
// called by all 32 lanes of one warp; the caller orders it against the rest
// of the CTA with a barrier.  Blocked by 32 rows: the dependence of a block on
// earlier blocks is a matrix-vector product (one row per lane, four partial
// sums in a fixed order), the diagonal block a substitution whose solved
// value is broadcast by a shuffle.
// PRE: the factors and permutation come from lu_reg<G, T, true> (gather by
// the composite permutation, U pre-divided by its diagonal).
template <bool PRE = false, class F>
__device__ __forceinline__ void warp_lu_solve(const F* A, int n, const int* piv, const F* invd, F* b) {
  const int lane = threadIdx.x & 31;
  if (PRE) {
    constexpr int MAXR = 5;  // n <= 160 (the team kernels take n <= 144)
    F g[MAXR];
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int i = lane + 32 * q;
      g[q] = i < n ? b[piv[i]] : F(0);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int i = lane + 32 * q;
      if (i < n) b[i] = g[q];
    }
  } else if (lane == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) {
        const F t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
  }
  __syncwarp();
  // forward substitution with the unit lower triangle
  for (int B0 = 0; B0 < n; B0 += 32) {
    const int i = B0 + lane;
    const bool act = i < n;
    F s0 = act ? b[i] : F(0), s1 = F(0), s2 = F(0), s3 = F(0);
    if (act) {
      const F* Li = A + (size_t)i * n;
      int j = 0;
      for (; j + 4 <= B0; j += 4) {
        s0 = fma(-Li[j], b[j], s0);
        s1 = fma(-Li[j + 1], b[j + 1], s1);
        s2 = fma(-Li[j + 2], b[j + 2], s2);
        s3 = fma(-Li[j + 3], b[j + 3], s3);
      }
      for (; j < B0; ++j) s0 = fma(-Li[j], b[j], s0);
    }
    F s = (s0 + s1) + (s2 + s3);
    const int m = min(32, n - B0);
    for (int jj = 0; jj < m; ++jj) {
      const F yj = __shfl_sync(0xffffffffu, s, jj);
      if (act && lane > jj) s = fma(-A[(size_t)i * n + B0 + jj], yj, s);
    }
    if (act) b[i] = s;
    __syncwarp();
  }
  // back substitution with U
  for (int B1 = ((n - 1) / 32) * 32; B1 >= 0; B1 -= 32) {
    const int i = B1 + lane;
    const bool act = i < n;
    const int m = min(32, n - B1);
    F s0 = act ? (PRE ? b[i] * invd[i] : b[i]) : F(0), s1 = F(0), s2 = F(0), s3 = F(0);
    if (act) {
      const F* Ui = A + (size_t)i * n;
      int j = B1 + 32;
      for (; j + 4 <= n; j += 4) {
        s0 = fma(-Ui[j], b[j], s0);
        s1 = fma(-Ui[j + 1], b[j + 1], s1);
        s2 = fma(-Ui[j + 2], b[j + 2], s2);
        s3 = fma(-Ui[j + 3], b[j + 3], s3);
      }
      for (; j < n; ++j) s0 = fma(-Ui[j], b[j], s0);
    }
    F s = (s0 + s1) + (s2 + s3);
    for (int jj = m - 1; jj >= 0; --jj) {
      if (!PRE && lane == jj) s *= invd[i];
      const F xj = __shfl_sync(0xffffffffu, s, jj);
      if (act && lane < jj) s = fma(-A[(size_t)i * n + B1 + jj], xj, s);
    }
    if (act) b[i] = s;
    __syncwarp();
  }
}

}  // namespace ck
