// Device-side data layout and arithmetic shared by the CUDA kernels of the
// batched constant-pressure reactor library (Stone, Alferman & Niemeyer,
// arXiv 1608.05794, Sec. 3 source terms; Sec. 2 integrators).
//
// FP64 is the scarce resource on this GPU (about 1.2 TFLOP/s against
// 70 TFLOP/s FP32), so the tables are pre-scaled at load time to save FP64
// instructions at run time: rate constants are kept as base-2 logarithms
// and evaluated with a table-driven 2^x (8 FP64 instructions), and the
// Gibbs polynomials are pre-divided by ln 2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ck {

constexpr double R_GAS = 8.314462618;       // J/(mol K)
constexpr double P_STD = 101325.0;          // p0 of Eq. kc, Pa
constexpr double LN2 = 0.6931471805599453094;
constexpr double INV_LN2 = 1.4426950408889634074;
constexpr double R_OVER_P0 = R_GAS / P_STD;               // R T / p0 is the molar volume at p0, m^3/mol
constexpr double P0_OVER_R = P_STD / R_GAS;

// One reaction, 96 bytes, read uniformly by all lanes (thread-per-reactor
// kernels) or by one lane per reaction (team kernels).  The loader sorts the
// reactions by (type, reversible, reactant count, product count) so that
// neighbouring lanes of a team kernel take the same branches.
struct __align__(16) RxnRec {
  double lA2;    // log2 A (SI)
  double beta;   // temperature exponent
  double EoR2;   // Ea / (R ln 2), K
  double lA02;   // Lindemann low-pressure limit: log2 A0
  double beta0;
  double E0oR2;
  double dnu_d;    // sum of product minus reactant coefficients, as FP64
  double nreac_d;  // reactant count, as FP64
  double nprod_d;  // product count, as FP64
  int16_t sp[6];    // reactant slots 0..2, product slots 3..5, -1 padded
  int8_t type;      // 0 elementary, 1 third-body, 2 Lindemann
  int8_t rev;       // 1 reversible through K_c, 2 explicit reverse Arrhenius
  int8_t dnu;
  int8_t nreac, nprod, pad0;
  int16_t eff_beg, eff_cnt;  // slice of the efficiency table (eff - 1 != 0)
  int16_t rev_ix;            // rev == 2: row of the explicit reverse table
};
static_assert(sizeof(RxnRec) == 96, "RxnRec layout");

// Jacobian partials stored per reaction: reactant slots 0..2, product slots
// 3..5, and slot 6 = dc/d[M] * (k_f prod' - k_r prod'').
constexpr int JP = 7;

// Per species and temperature range: 18 doubles
//   cp/R  : c0 + c1 T + c2 T^2 + c3 T^3 + c4 T^4               [0..4]
//   H/RT  : h0 + h1 T + h2 T^2 + h3 T^3 + h4 T^4 + h5 / T       [5..10]
//   g/ln2 : (S/R - H/RT)/ln 2 = G0 ln T + G1 + G2 T + G3 T^2 + G4 T^3 + G5 T^4 + G6 / T   [11..17]
constexpr int TH_STRIDE = 18;
constexpr int TH_PER_SPECIES = 2 * TH_STRIDE;

// Packed team-kernel table records (one 16-byte load each).
struct __align__(16) CsrTerm {  // species -> reaction list: net coefficient and reaction
  double nu;
  int32_t rx, pad;
};
struct __align__(16) JcEntry {  // one species-block entry of the Jacobian assembly
  int32_t idx;                  // flat shared-memory index of the entry
  int32_t beg, end;             // its contribution terms
  int32_t pad;
};
struct __align__(16) JcTerm {   // coef * P[pidx]
  double coef;
  int32_t pidx, pad;
};
static_assert(sizeof(CsrTerm) == 16 && sizeof(JcEntry) == 16 && sizeof(JcTerm) == 16, "packed records");

// Device view of a loaded mechanism.  All pointers are device memory (one
// allocation, 16-byte aligned sections).
struct DevMech {
  int S, R, n;            // species, reactions, n = S + 1
  int n_eff;              // entries of the efficiency table
  int csr_nnz;            // entries of the species -> reaction table
  int all_same_tmid;      // every species shares one T_mid
  int cv;                 // 1: constant volume (the parameter is rho), 0: constant pressure
  double tmid0;
  const RxnRec* rxn;      // [R]
  const double* thermo;   // [S][2][TH_STRIDE]
  const double* tmid;     // [S]
  const double* W;        // [S] kg/mol
  const double* invW;     // [S]
  const int16_t* eff_sp;  // [n_eff]
  const double* eff_m1;   // [n_eff] efficiency - 1
  const int32_t* csr_ptr; // [S+1] species -> (reaction, net nu) lists
  const CsrTerm* csr;     // [csr_nnz]
  const double* tab;      // [256] 2^(j/256)
  const double* revp;     // [n_rev][3] explicit reverse: log2 A_r, beta_r, Ea_r / (R ln 2)
  // Team kernels walk the reactions in chunks of `chunk` (= CTA size).
  // csr_cptr[k (n_chunks + 1) + c] = first CSR entry of species k whose
  // reaction lies in chunk c or later.  Jacobian assembly, chunk c: the
  // targets jc[e], e in [jc_ptr[c], jc_ptr[c+1]) (flat index idx: the
  // species-block entry J[idx] below n^2, else the per-species sums wd, aT,
  // E, u at idx - n^2), each add the sum over t in [jc[e].beg, jc[e].end)
  // of jt[t].coef * src[jt[t].pidx] (src: the chunk's q, dq/dT, D and
  // partials P, JP per reaction, contiguous).
  int chunk, n_chunks;
  const int32_t* csr_cptr;
  const int32_t* jc_ptr;
  const JcEntry* jc;
  const JcTerm* jt;
  const int16_t* rsp;     // [S] species order of the one-pass RHS gather, longest row first
};

// ---------------------------------------------------------------- 2^x
// Table-driven 2^x after Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic" (ACM TOMS 15,
// 1989), in base 2: x = e + j/256 + r with |r| <= 1/512, 2^x = 2^e T_j 2^r,
// T_j = 2^(j/256) from a 256-entry table, 2^r - 1 by its degree-4 Taylor
// polynomial in r ln 2 (truncation < 4e-17 relative).  The reduction is
// exact (x - round_{1/256}(x) is representable), so the result is within
// about one ulp.  |x| > 1000 (and NaN) falls back to the library exp2, out of
// line so that the rarely taken branch adds no instructions to the inlined
// fast path.  The range test compares the bits of |x| as an integer (they
// order like |x|, NaN above +inf), which keeps it off the FP64 pipe.
static __device__ __noinline__ double ck_exp2_wide(double x) { return exp2(x); }

__device__ __forceinline__ bool ck_exp2_in_range(double x) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
  return ax <= 0x408F400000000000ULL;  // the bits of 1000.0
}

// 2^r - 1 for |r| <= 1/512 (Taylor, degree 4 in r ln 2), and the step that
// assembles 2^(e + j/256 + r) from it.
__device__ __forceinline__ double ck_exp2_poly(double r) {
  const double c1 = 0.69314718055994530942;
  const double c2 = 0.24022650695910071233;   // ln2^2/2
  const double c3 = 0.055504108664821579953;  // ln2^3/6
  const double c4 = 0.0096181291076284771620; // ln2^4/24
  return fma(fma(fma(c4, r, c3), r, c2), r, c1) * r;
}
__device__ __forceinline__ double ck_exp2_assemble(int i, double q, const double* __restrict__ tab) {
  const int j = i & 255;
  const int e = i >> 8;  // floor division by 256
  const double tj = tab[j];
  const double res = fma(tj, q, tj);
  return __longlong_as_double(__double_as_longlong(res) + ((long long)e << 52));
}

__device__ __forceinline__ double ck_exp2(double x, const double* __restrict__ tab) {
  if (!ck_exp2_in_range(x)) return ck_exp2_wide(x);
  const double SHIFT = 26388279066624.0;  // 1.5 * 2^44: ulp 2^-8
  const double t = x + SHIFT;
  const double r = x - (t - SHIFT);
  const int i = (int)__double2loint(t);  // round(x * 256), low bits of t
  return ck_exp2_assemble(i, ck_exp2_poly(r), tab);
}

// 2^x and 2^-x from one reduction.  Rounding x to a multiple of 1/256 is
// symmetric (ties to even), so -x reduces to -i and -r exactly, and both
// results are bitwise those of ck_exp2(x) and ck_exp2(-x).
__device__ __forceinline__ void ck_exp2_pm(double x, const double* __restrict__ tab, double& ep, double& em) {
  if (!ck_exp2_in_range(x)) {
    ep = ck_exp2_wide(x);
    em = ck_exp2_wide(-x);
    return;
  }
  const double SHIFT = 26388279066624.0;
  const double t = x + SHIFT;
  const double r = x - (t - SHIFT);
  const int i = (int)__double2loint(t);
  ep = ck_exp2_assemble(i, ck_exp2_poly(r), tab);
  em = ck_exp2_assemble(-i, ck_exp2_poly(-r), tab);
}

// 1 / x rounded to nearest: the value IEEE division 1 / x returns, without
// the general-division path.
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }

// (R T / p0)^dnu for dnu = nprod - nreac in [-2, 2]: the concentration
// factor of 1/K_c (Eq. kc), by multiplication instead of an exponential.
__device__ __forceinline__ double rt_over_p0_pow(int dnu, double T, double invT) {
  const double q = dnu >= 0 ? T * R_OVER_P0 : invT * P0_OVER_R;
  const int a = dnu >= 0 ? dnu : -dnu;
  return a == 0 ? 1.0 : (a == 1 ? q : q * q);
}

// ---------------------------------------------------------------- statuses
enum : int32_t { ST_OK = 0, ST_MAXSTEPS = 1, ST_HMIN = 2, ST_NONFINITE = 3, ST_SINGULAR = 4,
                 ST_BADINPUT = 5 };

// Step-control constants (the paper leaves the controller unspecified; these
// are the readings shared with the CPU oracle's documentation).
constexpr double FAC_MAX = 5.0, FAC_MIN = 0.2, SAFETY = 0.9;
constexpr int SINGULAR_LIMIT = 10;

// ROS4 coefficients, App. C Table ros4 (gamma is the table value 0.57282;
// the table's b_i are the transformed-scheme weights m_i; a4j = a3j, a43 = 0
// so the fourth stage reuses the third stage's f).
constexpr double ROS_GAMMA = 0.57282;
constexpr double ROS_A21 = 2.0;
constexpr double ROS_A31 = 1.867943637803922, ROS_A32 = 0.2344449711399156;
constexpr double ROS_C21 = -7.137615036412310;
constexpr double ROS_C31 = 2.580708087951457, ROS_C32 = 0.6515950076447975;
constexpr double ROS_C41 = -2.137148994382534, ROS_C42 = -0.3214669691237626,
                 ROS_C43 = -0.6949742501781779;
constexpr double ROS_M1 = 2.255570073418735, ROS_M2 = 0.2870493262186792,
                 ROS_M3 = 0.4353179431840180, ROS_M4 = 1.093502252409163;
constexpr double ROS_E1 = -0.2815431932141155, ROS_E2 = -0.07276199124938920,
                 ROS_E3 = -0.1082196201495311, ROS_E4 = -1.093502252409163;

// RKF45 tableau, App. B Table rkf45 (b: fourth-order weights, propagated;
// bh: fifth-order weights; the error is sum (bh - b) k).
constexpr double RK_A21 = 1.0 / 4.0;
constexpr double RK_A31 = 3.0 / 32.0, RK_A32 = 9.0 / 32.0;
constexpr double RK_A41 = 1932.0 / 2197.0, RK_A42 = -7200.0 / 2197.0, RK_A43 = 7296.0 / 2197.0;
constexpr double RK_A51 = 439.0 / 216.0, RK_A52 = -8.0, RK_A53 = 3680.0 / 513.0,
                 RK_A54 = -845.0 / 4104.0;
constexpr double RK_A61 = -8.0 / 27.0, RK_A62 = 2.0, RK_A63 = -3544.0 / 2565.0,
                 RK_A64 = 1859.0 / 4104.0, RK_A65 = -11.0 / 40.0;
constexpr double RK_B1 = 25.0 / 216.0, RK_B3 = 1408.0 / 2565.0, RK_B4 = 2197.0 / 4104.0,
                 RK_B5 = -1.0 / 5.0;
constexpr double RK_D1 = 16.0 / 135.0 - 25.0 / 216.0, RK_D3 = 6656.0 / 12825.0 - 1408.0 / 2565.0,
                 RK_D4 = 28561.0 / 56430.0 - 2197.0 / 4104.0, RK_D5 = -9.0 / 50.0 + 1.0 / 5.0,
                 RK_D6 = 2.0 / 55.0;

// Per-CTA global scratch of the ROS4 kernel, in doubles: -J of the current
// state (n x n) and its diagonal (n).
__host__ __device__ constexpr size_t ros4_scratch_doubles(int n) { return (size_t)n * n + (size_t)n; }

struct SolverParams {
  double rtol, atol, h0, fixed_h;
  int max_steps;
  int jac;  // ROS4 Jacobian: 0 analytic, 1 forward differences
};

}  // namespace ck
