// CPU oracle for the batched constant-pressure reactor path (TEST INFRASTRUCTURE).
//
// A plain, slow FP64 restatement of Stone, Alferman & Niemeyer, "Accelerating
// finite-rate chemical kinetics with coprocessors" (arXiv 1608.05794):
//   * source terms, Sec. 3: Eqs. ydot, tdot, wdot, kfor, krev, kc, tfits, at
//     constant pressure or constant volume (Sec. 3: c_v and u_k), with K_c
//     or explicit reverse Arrhenius coefficients (Sec. 3);
//   * analytic Jacobian of that system (the paper recommends it in Sec. 6;
//     derived here by the chain rule, pinned by complex step), and the
//     forward-difference Jacobian the paper ran ROS4 with (Sec. 5, CVODE's
//     difference quotients);
//   * dense LU with partial pivoting of I/(h gamma) - J (Sec. 2);
//   * RKF45 (Sec. 2, App. B tableau) and ROS4 in transformed form (Sec. 2,
//     App. C coefficients);
//   * the scalar adaptive driver of Algorithm 1.
// Where the paper is silent (error norm, step-size update, initial step) the
// readings are stated at each function.  Nothing here is blocked, fused or
// reordered for speed.  Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline and reference legs may load this library; it shares no code
// with the CUDA path.
#include "oracle_api.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>
#include <complex>
#include <functional>
#include <thread>
#include <vector>

namespace {

const double R_GAS = 8.314462618;  // universal gas constant, J/(mol K)
const double P_STD = 101325.0;     // p0 of Eq. kc: one standard atmosphere, Pa

struct Mech {
  int S = 0, R = 0;
  std::vector<double> mw, nasa, tmid, arrh, arrh0;
  std::vector<int> reac, prod, rtype, rev;
  std::vector<double> eff;       // dense [R][S] third-body efficiencies (1 where unlisted)
  std::vector<double> arrh_rev;  // [R][3] explicit reverse (A, beta, Ea) where rev == 2
  int reactor = 0;               // 0 constant pressure (p given), 1 constant volume (rho given)
};

double re(double x) { return x; }
double re(const std::complex<double>& x) { return x.real(); }

// Eq. tfits, read as the standard NASA seven-term polynomials (the printed
// form is garbled): cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
// H/(RT) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
// S/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
// The low-range set applies when T < T_mid, the high-range set otherwise.
template <class Sc>
void nasa7(const Mech& m, int k, Sc T, Sc& cp_R, Sc& h_RT, Sc& s_R) {
  const double* a = &m.nasa[(size_t)k * 14 + (re(T) < m.tmid[k] ? 0 : 7)];
  Sc T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  cp_R = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
  h_RT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
  s_R = a[0] * std::log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
}

// d(cp/R)/dT of the same polynomial.
double nasa7_dcp(const Mech& m, int k, double T) {
  const double* a = &m.nasa[(size_t)k * 14 + (T < m.tmid[k] ? 0 : 7)];
  return a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T;
}

// Net stoichiometric coefficient nu''_ki - nu'_ki of species k in reaction i.
int net_nu(const Mech& m, int i, int k) {
  int v = 0;
  for (int s = 0; s < 3; ++s) {
    if (m.prod[i * 3 + s] == k) ++v;
    if (m.reac[i * 3 + s] == k) --v;
  }
  return v;
}

// Per-reaction quantities of Sec. 3 at one state.
template <class Sc>
struct Rxn {
  Sc kf, kr, Kc, k0, c, M, Pr, fwd, rev, q;
};

// Eqs. kfor, kc, krev and the c_i factor of Eq. wdot for reaction i.
// c_i = 1 (elementary), [M] = sum_k eff_ik [X_k] (third-body), or the
// Lindemann form P_r/(1 + P_r) with P_r = k0 [M] / k_inf (fall-off; k_f is
// then k_inf).  c_i multiplies both the forward and the reverse term.
template <class Sc>
void reaction(const Mech& m, int i, Sc T, const Sc* X, const Sc* h_RT, const Sc* s_R, Rxn<Sc>& r) {
  const double* ar = &m.arrh[i * 3];
  r.kf = ar[0] * std::pow(T, ar[1]) * std::exp(-ar[2] / (R_GAS * T));
  r.kr = 0.0;
  r.Kc = 0.0;
  if (m.rev[i] == 2) {
    // explicit reverse Arrhenius coefficients (Sec. 3), in place of Eq. krev
    const double* rr = &m.arrh_rev[i * 3];
    r.kr = rr[0] * std::pow(T, rr[1]) * std::exp(-rr[2] / (R_GAS * T));
    r.Kc = r.kf / r.kr;
  } else if (m.rev[i]) {
    Sc sum = 0.0;  // sum_j (nu''_j - nu'_j) (S_j/R - H_j/(R T))
    int dnu = 0;
    for (int s = 0; s < 3; ++s) {
      int j = m.prod[i * 3 + s];
      if (j >= 0) { sum += s_R[j] - h_RT[j]; ++dnu; }
      j = m.reac[i * 3 + s];
      if (j >= 0) { sum -= s_R[j] - h_RT[j]; --dnu; }
    }
    Sc Kp = std::exp(sum);
    r.Kc = std::pow(P_STD / (R_GAS * T), (double)dnu) * Kp;
    r.kr = r.kf / r.Kc;
  }
  r.c = 1.0;
  r.M = 0.0;
  r.k0 = 0.0;
  r.Pr = 0.0;
  if (m.rtype[i] == 1 || m.rtype[i] == 2) {
    for (int k = 0; k < m.S; ++k) r.M += m.eff[(size_t)i * m.S + k] * X[k];
    if (m.rtype[i] == 1) {
      r.c = r.M;
    } else {
      const double* a0 = &m.arrh0[i * 3];
      r.k0 = a0[0] * std::pow(T, a0[1]) * std::exp(-a0[2] / (R_GAS * T));
      r.Pr = r.k0 * r.M / r.kf;
      // P_r/(1+P_r), written as 1/(1 + 1/P_r) above P_r = 1 so that the
      // complex-step twin keeps the derivative 1/(1+P_r)^2 free of cancellation
      if (re(r.Pr) > 1.0) r.c = 1.0 / (1.0 + 1.0 / r.Pr);
      else r.c = r.Pr / (1.0 + r.Pr);
    }
  }
  r.fwd = 1.0;
  r.rev = 1.0;
  for (int s = 0; s < 3; ++s) {
    if (m.reac[i * 3 + s] >= 0) r.fwd *= X[m.reac[i * 3 + s]];
    if (m.prod[i * 3 + s] >= 0) r.rev *= X[m.prod[i * 3 + s]];
  }
  r.q = r.c * (r.kf * r.fwd - r.kr * r.rev);
}

// Mixture state of Sec. 3: mean molar mass, density, and molar
// concentrations [X_k] = rho Y_k / W_k.  Constant pressure: rho from the
// ideal-gas law p = rho (R/W) T with the given p.  Constant volume: the
// second argument is the (fixed) density itself.
template <class Sc>
void mixture(const Mech& m, double p, const Sc* y, Sc& Wbar, Sc& rho, Sc* X) {
  Sc sumYW = 0.0;
  for (int k = 0; k < m.S; ++k) sumYW += y[1 + k] / m.mw[k];
  Wbar = 1.0 / sumYW;
  if (m.reactor == 1) rho = p;
  else rho = p * Wbar / (R_GAS * y[0]);
  for (int k = 0; k < m.S; ++k) X[k] = rho * y[1 + k] / m.mw[k];
}

// Right-hand side of Eqs. ydot and tdot:
//   dY_k/dt = wdot_k W_k / rho,
//   dT/dt   = -(sum_k H_k wdot_k) / (rho cp),
// with H_k the molar enthalpy and cp = sum_k Y_k cp_k / W_k the mass-based
// mixture heat capacity (the printed Eq. tdot omits rho; dimensions need it).
// Constant volume (Sec. 3: c_v for c_p and u_k for h_k): the molar internal
// energy U_k = H_k - R T and c_v = sum_k Y_k (cp_k - R) / W_k in Eq. tdot.
template <class Sc>
void rhs_t(const Mech& m, double p, const Sc* y, Sc* f, Sc* wdot_out, Sc* q_out, double* gross) {
  const int S = m.S;
  std::vector<Sc> X(S), cp_R(S), h_RT(S), s_R(S), wdot(S, Sc(0.0));
  std::vector<double> gw(S, 0.0);
  Sc Wbar, rho;
  mixture(m, p, y, Wbar, rho, X.data());
  Sc T = y[0];
  for (int k = 0; k < S; ++k) nasa7(m, k, T, cp_R[k], h_RT[k], s_R[k]);
  Rxn<Sc> r;
  for (int i = 0; i < m.R; ++i) {
    reaction(m, i, T, X.data(), h_RT.data(), s_R.data(), r);
    if (q_out) q_out[i] = r.q;
    double g = std::abs(r.c) * (std::abs(r.kf * r.fwd) + std::abs(r.kr * r.rev));
    // Eq. wdot: wdot_k = sum_i (nu''_ki - nu'_ki) q_i over distinct species.
    for (int k = 0; k < S; ++k) {
      int v = net_nu(m, i, k);
      if (v != 0) {
        wdot[k] += (double)v * r.q;
        gw[k] += std::abs((double)v) * g;
      }
    }
  }
  const double cv = (m.reactor == 1) ? 1.0 : 0.0;  // subtract R from cp and R T from H
  Sc cp = 0.0, sumHw = 0.0;
  double gT = 0.0;
  for (int k = 0; k < S; ++k) {
    cp += y[1 + k] * (R_GAS * (cp_R[k] - cv)) / m.mw[k];
    sumHw += (R_GAS * T * (h_RT[k] - cv)) * wdot[k];
  }
  for (int k = 0; k < S; ++k) f[1 + k] = wdot[k] * m.mw[k] / rho;
  f[0] = -sumHw / (rho * cp);
  if (wdot_out)
    for (int k = 0; k < S; ++k) wdot_out[k] = wdot[k];
  if (gross) {
    double rr = std::abs(rho), cc = std::abs(cp);
    for (int k = 0; k < S; ++k) {
      gross[1 + k] = gw[k] * m.mw[k] / rr;
      gT += std::abs(R_GAS * T * (h_RT[k] - cv)) * gw[k];
    }
    gross[0] = gT / (rr * cc);
  }
}

// Analytic Jacobian of the same system, d f / d (T, Y_1..Y_S) at constant p.
// Chain rule through rho(T, Y) and [X](rho, Y):
//   d[X_k]/dT = -[X_k]/T,  d[X_k]/dY_j = rho/W_k delta_kj - [X_k] Wbar / W_j;
// at constant volume rho is fixed: d[X_k]/dT = 0, d[X_k]/dY_j = rho/W_k delta_kj,
// and the temperature row uses U_k = H_k - R T, c_v = sum Y_k (cp_k - R)/W_k;
//   d ln k_f/dT = beta/T + Ea/(R T^2);  d ln K_c/dT = sum_j dnu_j (H_j/RT)/T - dnu/T;
//   explicit reverse: d ln k_r/dT = beta_r/T + Ea_r/(R T^2);
//   Lindemann: dc/dP_r = 1/(1+P_r)^2, d ln P_r/dT = d ln k0/dT - d ln k_inf/dT,
//   dP_r/d[X_j] = eff_j k0 / k_inf.
// gross (may be NULL) gets the same sums with every term in absolute value.
void jac_one(const Mech& m, double p, const double* y, double* J, double* G) {
  const int S = m.S, n = S + 1;
  const double cpf = (m.reactor == 1) ? 0.0 : 1.0;  // terms present only at constant pressure
  std::vector<double> X(S), cp_R(S), h_RT(S), s_R(S), dcp_R(S), wdot(S, 0.0);
  std::vector<double> dwdT(S, 0.0), dwdY((size_t)S * S, 0.0);
  std::vector<double> gwdT(S, 0.0), gwdY((size_t)S * S, 0.0), gw(S, 0.0);
  std::vector<double> dqdX(S), gdqdX(S), dqdY(S), gdqdY(S);
  double Wbar, rho;
  mixture(m, p, y, Wbar, rho, X.data());
  const double T = y[0];
  for (int k = 0; k < S; ++k) {
    nasa7(m, k, T, cp_R[k], h_RT[k], s_R[k]);
    dcp_R[k] = nasa7_dcp(m, k, T);
  }
  Rxn<double> r;
  for (int i = 0; i < m.R; ++i) {
    reaction(m, i, T, X.data(), h_RT.data(), s_R.data(), r);
    const double net = r.kf * r.fwd - r.kr * r.rev;
    const double gnet = std::fabs(r.kf * r.fwd) + std::fabs(r.kr * r.rev);
    // d q / d[X_j] at fixed T
    for (int j = 0; j < S; ++j) {
      double dfwd = 0.0, drev = 0.0;
      for (int s = 0; s < 3; ++s) {
        if (m.reac[i * 3 + s] == j) {
          double pr = 1.0;
          for (int t = 0; t < 3; ++t)
            if (t != s && m.reac[i * 3 + t] >= 0) pr *= X[m.reac[i * 3 + t]];
          dfwd += pr;
        }
        if (m.prod[i * 3 + s] == j) {
          double pr = 1.0;
          for (int t = 0; t < 3; ++t)
            if (t != s && m.prod[i * 3 + t] >= 0) pr *= X[m.prod[i * 3 + t]];
          drev += pr;
        }
      }
      double dc = 0.0;
      if (m.rtype[i] == 1) dc = m.eff[(size_t)i * S + j];
      if (m.rtype[i] == 2)
        dc = m.eff[(size_t)i * S + j] * (r.k0 / r.kf) / ((1.0 + r.Pr) * (1.0 + r.Pr));
      dqdX[j] = r.c * (r.kf * dfwd - r.kr * drev) + dc * net;
      gdqdX[j] = std::fabs(r.c) * (std::fabs(r.kf * dfwd) + std::fabs(r.kr * drev)) +
                 std::fabs(dc) * gnet;
    }
    // d q / dT at fixed [X]
    const double* ar = &m.arrh[i * 3];
    double dlnkf = ar[1] / T + ar[2] / (R_GAS * T * T);
    double dlnKc = 0.0;
    if (m.rev[i] == 1) {
      int dnu = 0;
      for (int s = 0; s < 3; ++s) {
        int j = m.prod[i * 3 + s];
        if (j >= 0) { dlnKc += h_RT[j] / T; ++dnu; }
        j = m.reac[i * 3 + s];
        if (j >= 0) { dlnKc -= h_RT[j] / T; --dnu; }
      }
      dlnKc -= (double)dnu / T;
    }
    double dkf = r.kf * dlnkf;
    double dkr = r.kr * (dlnkf - dlnKc);
    if (m.rev[i] == 2) {
      const double* rr = &m.arrh_rev[i * 3];
      dkr = r.kr * (rr[1] / T + rr[2] / (R_GAS * T * T));
    }
    double dc_dT = 0.0;
    if (m.rtype[i] == 2) {
      const double* a0 = &m.arrh0[i * 3];
      double dlnk0 = a0[1] / T + a0[2] / (R_GAS * T * T);
      dc_dT = r.Pr * (dlnk0 - dlnkf) / ((1.0 + r.Pr) * (1.0 + r.Pr));
    }
    double dqdT_X = dc_dT * net + r.c * (dkf * r.fwd - dkr * r.rev);
    double gdqdT_X = std::fabs(dc_dT) * gnet +
                     std::fabs(r.c) * (std::fabs(dkf * r.fwd) + std::fabs(dkr * r.rev));
    // total derivatives at fixed (T, Y) through [X](T, Y)
    double D = 0.0, gD = 0.0;
    for (int j = 0; j < S; ++j) {
      D += dqdX[j] * X[j];
      gD += gdqdX[j] * std::fabs(X[j]);
    }
    double dqdT = dqdT_X - cpf * D / T;
    double gdqdT = gdqdT_X + cpf * gD / T;
    for (int j = 0; j < S; ++j) {
      dqdY[j] = dqdX[j] * rho / m.mw[j] - cpf * (Wbar / m.mw[j]) * D;
      gdqdY[j] = gdqdX[j] * rho / m.mw[j] + cpf * (Wbar / m.mw[j]) * gD;
    }
    double gq = std::fabs(r.c) * gnet;
    for (int k = 0; k < S; ++k) {
      int v = net_nu(m, i, k);
      if (v == 0) continue;
      double av = std::fabs((double)v);
      wdot[k] += (double)v * r.q;
      gw[k] += av * gq;
      dwdT[k] += (double)v * dqdT;
      gwdT[k] += av * gdqdT;
      for (int j = 0; j < S; ++j) {
        dwdY[(size_t)k * S + j] += (double)v * dqdY[j];
        gwdY[(size_t)k * S + j] += av * gdqdY[j];
      }
    }
  }
  // species rows: Y_k' = wdot_k W_k / rho (rho depends on T and Y only at constant p)
  for (int k = 0; k < S; ++k) {
    double wk = m.mw[k];
    J[(size_t)(1 + k) * n + 0] = wk / rho * dwdT[k] + cpf * wdot[k] * wk / (rho * T);
    for (int j = 0; j < S; ++j)
      J[(size_t)(1 + k) * n + 1 + j] =
          wk / rho * dwdY[(size_t)k * S + j] + cpf * wdot[k] * wk * Wbar / (rho * m.mw[j]);
    if (G) {
      G[(size_t)(1 + k) * n + 0] = wk / rho * gwdT[k] + cpf * gw[k] * wk / (rho * T);
      for (int j = 0; j < S; ++j)
        G[(size_t)(1 + k) * n + 1 + j] =
            wk / rho * gwdY[(size_t)k * S + j] + cpf * gw[k] * wk * Wbar / (rho * m.mw[j]);
    }
  }
  // temperature row: T' = -(sum_k E_k wdot_k) / (rho c) with E_k = H_k, c = cp
  // (constant pressure) or E_k = U_k = H_k - R T, c = c_v (constant volume)
  const double cv = 1.0 - cpf;
  double cpm = 0.0, dcpm = 0.0, Q = 0.0, gQ = 0.0;
  for (int k = 0; k < S; ++k) {
    cpm += y[1 + k] * R_GAS * (cp_R[k] - cv) / m.mw[k];
    dcpm += y[1 + k] * R_GAS * dcp_R[k] / m.mw[k];
    Q += R_GAS * T * (h_RT[k] - cv) * wdot[k];
    gQ += std::fabs(R_GAS * T * (h_RT[k] - cv)) * gw[k];
  }
  const double Tdot = -Q / (rho * cpm);
  const double gTdot = gQ / (rho * cpm);
  double dQdT = 0.0, gdQdT = 0.0;
  for (int k = 0; k < S; ++k) {
    dQdT += R_GAS * (cp_R[k] - cv) * wdot[k] + R_GAS * T * (h_RT[k] - cv) * dwdT[k];
    gdQdT += std::fabs(R_GAS * (cp_R[k] - cv)) * gw[k] + std::fabs(R_GAS * T * (h_RT[k] - cv)) * gwdT[k];
  }
  J[0] = -dQdT / (rho * cpm) - Tdot * (-cpf / T + dcpm / cpm);
  if (G) G[0] = gdQdT / (rho * cpm) + gTdot * (cpf / T + std::fabs(dcpm / cpm));
  for (int j = 0; j < S; ++j) {
    double dQdY = 0.0, gdQdY = 0.0;
    for (int k = 0; k < S; ++k) {
      dQdY += R_GAS * T * (h_RT[k] - cv) * dwdY[(size_t)k * S + j];
      gdQdY += std::fabs(R_GAS * T * (h_RT[k] - cv)) * gwdY[(size_t)k * S + j];
    }
    double dlog = R_GAS * (cp_R[j] - cv) / (m.mw[j] * cpm) - cpf * Wbar / m.mw[j];
    J[1 + j] = -dQdY / (rho * cpm) - Tdot * dlog;
    if (G)
      G[1 + j] = gdQdY / (rho * cpm) +
                 gTdot * (std::fabs(R_GAS * (cp_R[j] - cv) / (m.mw[j] * cpm)) + cpf * Wbar / m.mw[j]);
  }
}

// ---------------------------------------------------------------- linear algebra
// LU with partial pivoting (the paper is silent on pivoting; this is the
// reading).  Row-major, in place; unit lower triangle below the diagonal.
int lu_factor(int n, double* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(a[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (!(best > 0.0) || !std::isfinite(best)) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      a[(size_t)i * n + k] /= a[(size_t)k * n + k];
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void lu_solve(int n, const double* a, const int* piv, double* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
    b[i] /= a[(size_t)i * n + i];
  }
}

// ---------------------------------------------------------------- methods
// App. B, Table rkf45: six stages (the text says "five-stage"; the tableau has
// six).  b are the fourth-order weights (propagated), bh the fifth-order ones.
const double RK_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
const double RK_B[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
const double RK_BH[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

// App. C, Table ros4.  gamma = 0.57282 (table value; the text's 0.572816
// breaks the order conditions with the printed a, c, m).  The table's b_i are
// the weights m_i of the transformed scheme; a41 = a31, a42 = a32, a43 = 0.
const double ROS_GAMMA = 0.57282;
const double ROS_A[4][3] = {{0, 0, 0},
                            {2.0, 0, 0},
                            {1.867943637803922, 0.2344449711399156, 0},
                            {1.867943637803922, 0.2344449711399156, 0.0}};
const double ROS_C[4][3] = {{0, 0, 0},
                            {-7.137615036412310, 0, 0},
                            {2.580708087951457, 0.6515950076447975, 0},
                            {-2.137148994382534, -0.3214669691237626, -0.6949742501781779}};
const double ROS_M[4] = {2.255570073418735, 0.2870493262186792, 0.4353179431840180, 1.093502252409163};
const double ROS_E[4] = {-0.2815431932141155, -0.07276199124938920, -0.1082196201495311,
                         -1.093502252409163};

struct System {
  int n;
  std::function<void(const double*, double*)> f;    // f(y)
  std::function<void(const double*, double*)> jac;  // J(y), n x n row-major
  int jac_fd = 0;                                    // 1: forward differences instead of jac
  double rtol = 0.0, atol = 0.0;                     // weights of the difference increments
};

// Number of right-hand-side evaluations made by the reactor systems (all
// threads), so tests can check the evaluations a step costs.
std::atomic<int64_t> g_rhs_evals(0);

// Forward-difference Jacobian, the paper's choice for ROS4 (Sec. 5), built
// as in CVODE's dense difference-quotient routine: with unit roundoff U,
// weights w_i = 1/(atol + rtol |y_i|) and fnorm = WRMS_w(f(y)), the floor
// s0 = 1000 |h| U n fnorm (1 when fnorm = 0); column j is
//   (f(y + s_j e_j) - f(y)) / s_j,  s_j = max(sqrt(U) |y_j|, s0 / w_j).
// f0 = f(y) is given (it is the first stage's right-hand side), so a
// Jacobian costs n further evaluations.
void jac_fd(const System& sys, const double* y, const double* f0, double h, double* J) {
  const int n = sys.n;
  const double U = std::numeric_limits<double>::epsilon();
  double fn = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = f0[i] / (sys.atol + sys.rtol * std::fabs(y[i]));
    fn += v * v;
  }
  fn = std::sqrt(fn / n);
  const double s0 = (fn != 0.0) ? 1000.0 * std::fabs(h) * U * n * fn : 1.0;
  std::vector<double> yj(y, y + n), fj(n);
  for (int j = 0; j < n; ++j) {
    const double sj = std::max(std::sqrt(U) * std::fabs(y[j]), s0 * (sys.atol + sys.rtol * std::fabs(y[j])));
    yj[j] = y[j] + sj;
    sys.f(yj.data(), fj.data());
    for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = (fj[i] - f0[i]) / sj;
    yj[j] = y[j];
  }
}

// RKF45 OneStep (Sec. 2, Eq. rk): k_i = h f(y + sum_j a_ij k_j);
// ynew = y + sum b_j k_j; err = sum (bh_j - b_j) k_j.
void rkf45_step(const System& sys, const double* y, double h, double* ynew, double* err) {
  const int n = sys.n;
  std::vector<double> k((size_t)6 * n), yt(n), ft(n);
  for (int s = 0; s < 6; ++s) {
    for (int i = 0; i < n; ++i) {
      double acc = y[i];
      for (int j = 0; j < s; ++j) acc += RK_A[s][j] * k[(size_t)j * n + i];
      yt[i] = acc;
    }
    sys.f(yt.data(), ft.data());
    for (int i = 0; i < n; ++i) k[(size_t)s * n + i] = h * ft[i];
  }
  for (int i = 0; i < n; ++i) {
    double a = y[i], e = 0.0;
    for (int s = 0; s < 6; ++s) {
      a += RK_B[s] * k[(size_t)s * n + i];
      e += (RK_BH[s] - RK_B[s]) * k[(size_t)s * n + i];
    }
    ynew[i] = a;
    err[i] = e;
  }
}

// ROS4 OneStep in the transformed form of Sec. 2:
//   (I/(h gamma) - J) u_i = f(y + sum_{j<i} a_ij u_j) + sum_{j<i} (c_ij/h) u_j,
//   ynew = y + sum m_i u_i,  err = sum E_i u_i  (App. C).
// J is evaluated at y.  Returns nonzero when the iteration matrix is singular.
int ros4_step(const System& sys, const double* y, double h, double* ynew, double* err) {
  const int n = sys.n;
  std::vector<double> M((size_t)n * n), u((size_t)4 * n), yt(n), ft(n), rhs(n), f0;
  std::vector<int> piv(n);
  if (sys.jac_fd) {
    f0.resize(n);
    sys.f(y, f0.data());
    jac_fd(sys, y, f0.data(), h, M.data());
  } else {
    sys.jac(y, M.data());
  }
  for (size_t i = 0; i < (size_t)n * n; ++i) M[i] = -M[i];
  for (int i = 0; i < n; ++i) M[(size_t)i * n + i] += 1.0 / (h * ROS_GAMMA);
  if (lu_factor(n, M.data(), piv.data()) != 0) return 1;
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < n; ++i) {
      double acc = y[i];
      for (int j = 0; j < s; ++j) acc += ROS_A[s][j] * u[(size_t)j * n + i];
      yt[i] = acc;
    }
    if (s == 0 && sys.jac_fd) ft = f0;  // f(y), already evaluated for the differences
    else sys.f(yt.data(), ft.data());
    for (int i = 0; i < n; ++i) {
      double acc = ft[i];
      for (int j = 0; j < s; ++j) acc += (ROS_C[s][j] / h) * u[(size_t)j * n + i];
      rhs[i] = acc;
    }
    lu_solve(n, M.data(), piv.data(), rhs.data());
    for (int i = 0; i < n; ++i) u[(size_t)s * n + i] = rhs[i];
  }
  for (int i = 0; i < n; ++i) {
    double a = y[i], e = 0.0;
    for (int s = 0; s < 4; ++s) {
      a += ROS_M[s] * u[(size_t)s * n + i];
      e += ROS_E[s] * u[(size_t)s * n + i];
    }
    ynew[i] = a;
    err[i] = e;
  }
  return 0;
}

// Weighted RMS norm (reading): sqrt(mean_i (e_i / (atol + rtol max(|y_i|, |ynew_i|)))^2).
double wrms(int n, const double* e, const double* y, const double* ynew, double rtol, double atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double sc = atol + rtol * std::max(std::fabs(y[i]), std::fabs(ynew[i]));
    double v = e[i] / sc;
    s += v * v;
  }
  return std::sqrt(s / n);
}

// EstimateH0 (reading: the starting-step algorithm of Hairer, Norsett &
// Wanner, Solving ODEs I, Sec. II.4, with order p = 4 for both methods and
// the weights atol + rtol |y0_i|).
double estimate_h0(const System& sys, const double* y0, double tspan, double rtol, double atol) {
  const int n = sys.n;
  std::vector<double> f0(n), y1(n), f1(n), sc(n);
  sys.f(y0, f0.data());
  double d0 = 0.0, d1 = 0.0;
  for (int i = 0; i < n; ++i) {
    sc[i] = atol + rtol * std::fabs(y0[i]);
    d0 += (y0[i] / sc[i]) * (y0[i] / sc[i]);
    d1 += (f0[i] / sc[i]) * (f0[i] / sc[i]);
  }
  d0 = std::sqrt(d0 / n);
  d1 = std::sqrt(d1 / n);
  double ha = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  for (int i = 0; i < n; ++i) y1[i] = y0[i] + ha * f0[i];
  sys.f(y1.data(), f1.data());
  double d2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double v = (f1[i] - f0[i]) / sc[i];
    d2 += v * v;
  }
  d2 = std::sqrt(d2 / n) / ha;
  double dm = std::max(d1, d2);
  double hb = (dm <= 1e-15) ? std::max(1e-6, ha * 1e-3) : std::pow(0.01 / dm, 1.0 / 5.0);
  return std::min(std::min(100.0 * ha, hb), tspan);
}

bool all_finite(int n, const double* v) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Algorithm 1 for one system over [0, tf], with the loop test read as t < t_f
// (the printed "t < t_i" is a misprint).  Step control (reading):
//   accept iff err < 1; h_new = h min(5, max(0.2, 0.9 err^(-1/q))) with
//   q = 4 (ROS4, embedded order 3) or 5 (RKF45, embedded order 4); no growth
//   on the step after a rejection; factor 5 when err == 0; the last step is
//   clamped to end exactly at t_f; a non-finite trial or error is a rejection
//   with factor 0.2; a singular iteration matrix halves h (ORA_SINGULAR after
//   10 in a row); ORA_HMIN when h < 1e-15 t_f; ORA_MAXSTEPS after max_steps
//   attempted steps.
int drive(const System& sys, int method, double* y, double tf, double* h_inout, const ora_opts& o,
          int* acc_out, int* rej_out) {
  const int n = sys.n;
  int acc = 0, rej = 0;
  auto done = [&](int st) {
    if (acc_out) *acc_out = acc;
    if (rej_out) *rej_out = rej;
    return st;
  };
  if (!all_finite(n, y) || !(tf >= 0.0) || !std::isfinite(tf)) return done(ORA_BADINPUT);
  if (tf == 0.0) return done(ORA_OK);
  std::vector<double> ynew(n), err(n);
  const bool fixed = o.fixed_h > 0.0;
  double h;
  if (fixed) h = o.fixed_h;
  else if (h_inout && *h_inout > 0.0) h = *h_inout;
  else if (o.h0 > 0.0) h = o.h0;
  else h = estimate_h0(sys, y, tf, o.rtol, o.atol);
  const double q = (method == ORA_ROS4) ? 4.0 : 5.0;
  const double hmin = 1e-15 * tf;
  double t = 0.0;
  bool last_rejected = false, last_nonfinite = false;
  int singular_run = 0;
  int status = ORA_OK;
  while (t < tf) {
    if (acc + rej >= o.max_steps) { status = ORA_MAXSTEPS; break; }
    bool clamped = h >= tf - t;
    double hh = clamped ? tf - t : h;
    if (hh < hmin) { status = last_nonfinite ? ORA_NONFINITE : ORA_HMIN; break; }
    int sing = 0;
    if (method == ORA_ROS4) sing = ros4_step(sys, y, hh, ynew.data(), err.data());
    else rkf45_step(sys, y, hh, ynew.data(), err.data());
    if (sing) {
      ++rej;
      if (++singular_run >= 10) { status = ORA_SINGULAR; break; }
      h = 0.5 * hh;
      last_rejected = true;
      continue;
    }
    singular_run = 0;
    if (fixed) {
      for (int i = 0; i < n; ++i) y[i] = ynew[i];
      t = clamped ? tf : t + hh;
      ++acc;
      continue;
    }
    double e = wrms(n, err.data(), y, ynew.data(), o.rtol, o.atol);
    if (!std::isfinite(e) || !all_finite(n, ynew.data())) {
      ++rej;
      h = 0.2 * hh;
      last_rejected = true;
      last_nonfinite = true;
      continue;
    }
    last_nonfinite = false;
    if (e < 1.0) {
      for (int i = 0; i < n; ++i) y[i] = ynew[i];
      t = clamped ? tf : t + hh;
      ++acc;
      double fac = (e == 0.0) ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * std::pow(e, -1.0 / q)));
      if (last_rejected) fac = std::min(1.0, fac);
      h = hh * fac;
      last_rejected = false;
    } else {
      ++rej;
      h = hh * std::max(0.2, 0.9 * std::pow(e, -1.0 / q));
      last_rejected = true;
    }
  }
  if (h_inout) *h_inout = h;
  return done(status);
}

System reactor_system(const Mech& m, double p) {
  System s;
  s.n = m.S + 1;
  const Mech* mp = &m;
  s.f = [mp, p](const double* y, double* f) {
    g_rhs_evals.fetch_add(1, std::memory_order_relaxed);
    rhs_t<double>(*mp, p, y, f, nullptr, nullptr, nullptr);
  };
  s.jac = [mp, p](const double* y, double* J) { jac_one(*mp, p, y, J, nullptr); };
  return s;
}

System test_system(int problem, int dim, const double* params) {
  System s;
  s.n = (problem == 1) ? 1 : dim;
  std::vector<double> P;
  if (problem == 0) P.assign(params, params + dim);
  if (problem == 2) P.assign(params, params + (size_t)dim * dim);
  const int n = s.n;
  if (problem == 0) {
    s.f = [P, n](const double* y, double* f) { for (int i = 0; i < n; ++i) f[i] = P[i] * y[i]; };
    s.jac = [P, n](const double*, double* J) {
      for (int i = 0; i < n * n; ++i) J[i] = 0.0;
      for (int i = 0; i < n; ++i) J[i * n + i] = P[i];
    };
  } else if (problem == 1) {
    s.f = [](const double* y, double* f) { f[0] = -y[0] * y[0]; };
    s.jac = [](const double* y, double* J) { J[0] = -2.0 * y[0]; };
  } else if (problem == 3) {
    s.f = [n](const double* y, double* f) { for (int i = 0; i < n; ++i) f[i] = -y[i] * y[i]; };
    s.jac = [n](const double* y, double* J) {
      for (int i = 0; i < n * n; ++i) J[i] = 0.0;
      for (int i = 0; i < n; ++i) J[i * n + i] = -2.0 * y[i];
    };
  } else {
    s.f = [P, n](const double* y, double* f) {
      for (int i = 0; i < n; ++i) {
        double a = 0.0;
        for (int j = 0; j < n; ++j) a += P[(size_t)i * n + j] * y[j];
        f[i] = a;
      }
    };
    s.jac = [P, n](const double*, double* J) { for (int i = 0; i < n * n; ++i) J[i] = P[i]; };
  }
  return s;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (nthreads > n) nthreads = (int)std::max<int64_t>(1, n);
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      fn(i);
    }
  };
  if (nthreads == 1) { work(); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
}

}  // namespace

struct ora_mech {
  Mech m;
};

extern "C" {

ora_mech* ora_mech_create(int32_t S, int32_t R, const double* mw, const double* nasa,
                          const double* tmid, const int32_t* reac, const int32_t* prod,
                          const double* arrh, const int32_t* rtype, const int32_t* rev,
                          const double* arrh0, const int32_t* eff_ptr, const int32_t* eff_sp,
                          const double* eff_val, const double* arrh_rev, int32_t reactor) {
  if (S <= 0 || R < 0 || reactor < 0 || reactor > 1) return nullptr;
  for (int i = 0; i < R; ++i)
    if (rev[i] < 0 || rev[i] > 2 || (rev[i] == 2 && !arrh_rev)) return nullptr;
  ora_mech* h = new ora_mech;
  Mech& m = h->m;
  m.S = S;
  m.R = R;
  m.mw.assign(mw, mw + S);
  m.nasa.assign(nasa, nasa + (size_t)S * 14);
  m.tmid.assign(tmid, tmid + S);
  m.reac.assign(reac, reac + (size_t)R * 3);
  m.prod.assign(prod, prod + (size_t)R * 3);
  m.arrh.assign(arrh, arrh + (size_t)R * 3);
  m.arrh0.assign(arrh0, arrh0 + (size_t)R * 3);
  m.rtype.assign(rtype, rtype + R);
  m.rev.assign(rev, rev + R);
  m.reactor = reactor;
  if (arrh_rev) m.arrh_rev.assign(arrh_rev, arrh_rev + (size_t)R * 3);
  m.eff.assign((size_t)R * S, 1.0);
  for (int i = 0; i < R; ++i)
    for (int e = eff_ptr[i]; e < eff_ptr[i + 1]; ++e) m.eff[(size_t)i * S + eff_sp[e]] = eff_val[e];
  return h;
}

void ora_mech_free(ora_mech* h) { delete h; }

void ora_thermo(const ora_mech* h, double T, double* cp_R, double* h_RT, double* s_R) {
  for (int k = 0; k < h->m.S; ++k) nasa7(h->m, k, T, cp_R[k], h_RT[k], s_R[k]);
}

void ora_rate_coeffs(const ora_mech* h, double T, double* kf, double* kc, double* kr, double* k0) {
  const Mech& m = h->m;
  std::vector<double> cp(m.S), hh(m.S), ss(m.S), X(m.S, 1.0);
  for (int k = 0; k < m.S; ++k) nasa7(m, k, T, cp[k], hh[k], ss[k]);
  Rxn<double> r;
  for (int i = 0; i < m.R; ++i) {
    reaction(m, i, T, X.data(), hh.data(), ss.data(), r);
    kf[i] = r.kf;
    kc[i] = r.Kc;
    kr[i] = r.kr;
    k0[i] = r.k0;
  }
}

void ora_rhs(const ora_mech* h, int64_t n, const double* p, const double* y, double* dydt) {
  const int nn = h->m.S + 1;
  parallel_for(n, 0, [&](int64_t i) {
    rhs_t<double>(h->m, p[i], y + i * nn, dydt + i * nn, nullptr, nullptr, nullptr);
  });
}

void ora_rhs_detail(const ora_mech* h, double p, const double* y, double* wdot, double* q,
                    double* gross) {
  std::vector<double> f(h->m.S + 1);
  rhs_t<double>(h->m, p, y, f.data(), wdot, q, gross);
}

void ora_rhs_complex(const ora_mech* h, double p, const double* y_re, const double* y_im,
                     double* f_re, double* f_im) {
  const int n = h->m.S + 1;
  std::vector<std::complex<double>> y(n), f(n);
  for (int i = 0; i < n; ++i) y[i] = std::complex<double>(y_re[i], y_im[i]);
  rhs_t<std::complex<double>>(h->m, p, y.data(), f.data(), nullptr, nullptr, nullptr);
  for (int i = 0; i < n; ++i) {
    f_re[i] = f[i].real();
    f_im[i] = f[i].imag();
  }
}

void ora_jacobian(const ora_mech* h, int64_t n, const double* p, const double* y, double* jac,
                  double* gross) {
  const int nn = h->m.S + 1;
  parallel_for(n, 0, [&](int64_t i) {
    jac_one(h->m, p[i], y + i * nn, jac + (size_t)i * nn * nn,
            gross ? gross + (size_t)i * nn * nn : nullptr);
  });
}

int32_t ora_lu_factor(int32_t dim, double* a, int32_t* piv) {
  std::vector<int> pv(dim);
  int r = lu_factor(dim, a, pv.data());
  for (int i = 0; i < dim; ++i) piv[i] = pv[i];
  return r;
}

void ora_lu_solve(int32_t dim, const double* lu, const int32_t* piv, double* b) {
  std::vector<int> pv(piv, piv + dim);
  lu_solve(dim, lu, pv.data(), b);
}

void ora_integrate(const ora_mech* h, int32_t method, int64_t n, const double* p, double* y,
                   const double* dt, double* h_inout, const ora_opts* opts, int32_t* steps,
                   int32_t* status, int32_t nthreads) {
  const int nn = h->m.S + 1;
  parallel_for(n, nthreads, [&](int64_t i) {
    int acc = 0, rej = 0;
    int st;
    if (!(p[i] > 0.0) || !std::isfinite(p[i]) || !(y[i * nn] > 0.0)) {
      st = ORA_BADINPUT;
    } else {
      System sys = reactor_system(h->m, p[i]);
      sys.jac_fd = opts->jac == 1;
      sys.rtol = opts->rtol;
      sys.atol = opts->atol;
      st = drive(sys, method, y + i * nn, dt[i], h_inout ? h_inout + i : nullptr, *opts, &acc, &rej);
    }
    status[i] = st;
    if (steps) {
      steps[2 * i] = acc;
      steps[2 * i + 1] = rej;
    }
  });
}

void ora_test_integrate(int32_t problem, int32_t method, int32_t dim, const double* params,
                        double* y, double dt, const ora_opts* opts, int32_t* steps,
                        int32_t* status) {
  System sys = test_system(problem, dim, params);
  int acc = 0, rej = 0;
  *status = drive(sys, method, y, dt, nullptr, *opts, &acc, &rej);
  if (steps) {
    steps[0] = acc;
    steps[1] = rej;
  }
}

void ora_test_onestep(int32_t problem, int32_t method, int32_t dim, const double* params,
                      const double* y, double h, double* ynew, double* err) {
  System sys = test_system(problem, dim, params);
  if (method == ORA_ROS4) ros4_step(sys, y, h, ynew, err);
  else rkf45_step(sys, y, h, ynew, err);
}

void ora_jacobian_fd(const ora_mech* h, int64_t n, const double* p, const double* y, const double* hstep,
                     double rtol, double atol, double* jac) {
  const int nn = h->m.S + 1;
  parallel_for(n, 0, [&](int64_t i) {
    System sys = reactor_system(h->m, p[i]);
    sys.rtol = rtol;
    sys.atol = atol;
    std::vector<double> f0(nn);
    sys.f(y + i * nn, f0.data());
    jac_fd(sys, y + i * nn, f0.data(), hstep[i], jac + (size_t)i * nn * nn);
  });
}

void ora_test_jacobian_fd(int32_t problem, int32_t dim, const double* params, const double* y, double h,
                          double rtol, double atol, double* jac) {
  System sys = test_system(problem, dim, params);
  sys.rtol = rtol;
  sys.atol = atol;
  std::vector<double> f0(sys.n);
  sys.f(y, f0.data());
  jac_fd(sys, y, f0.data(), h, jac);
}

int64_t ora_rhs_evals(int32_t reset) {
  return reset ? g_rhs_evals.exchange(0) : g_rhs_evals.load();
}

int32_t ora_hardware_threads(void) { return (int32_t)std::max(1u, std::thread::hardware_concurrency()); }

}  // extern "C"
