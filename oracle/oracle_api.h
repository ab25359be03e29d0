/* CPU oracle for the batched constant-pressure reactor path (TEST INFRASTRUCTURE).
 *
 * Plain, slow, FP64 restatement of Stone, Alferman & Niemeyer (arXiv
 * 1608.05794): the source terms of Sec. 3 (Eqs. ydot, tdot, wdot, kfor, krev,
 * kc, tfits), the RKF45 tableau of App. B, the ROS4 scheme of Sec. 2 with the
 * coefficients of App. C, and the scalar adaptive driver of Algorithm 1.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library.
 *
 * Arrays are host memory owned by the caller, row-major.  A state vector is
 * y = (T [K], Y_1 .. Y_S) of length n = S + 1; p is in Pa.
 */
#ifndef CK_ORACLE_API_H
#define CK_ORACLE_API_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_mech ora_mech;

/* Build a mechanism from plain arrays (copied).  reac/prod are [R][3] species
 * slots padded with -1; arrh/arrh0 are [R][3] (A in SI units, beta, Ea in
 * J/mol); rtype 0 elementary, 1 third-body, 2 Lindemann; rev 1 reversible via
 * K_c, 0 irreversible, 2 reversible with the explicit reverse Arrhenius
 * coefficients arrh_rev[R][3] (Sec. 3; may be NULL when no rev is 2); eff_*
 * is CSR over reactions (default efficiency 1); nasa is [S][2][7] (low range
 * first).  reactor 0: constant pressure, the per-reactor parameter p of the
 * calls below is the pressure in Pa; reactor 1: constant volume (Sec. 3), the
 * parameter is the fixed density in kg/m^3.  Returns NULL on bad input. */
ora_mech* ora_mech_create(int32_t S, int32_t R, const double* mw, const double* nasa,
                          const double* tmid, const int32_t* reac, const int32_t* prod,
                          const double* arrh, const int32_t* rtype, const int32_t* rev,
                          const double* arrh0, const int32_t* eff_ptr, const int32_t* eff_sp,
                          const double* eff_val, const double* arrh_rev, int32_t reactor);
void ora_mech_free(ora_mech* m);

/* NASA-7 properties of every species at T (Eq. tfits, read as the standard
 * seven-term form). */
void ora_thermo(const ora_mech* m, double T, double* cp_R, double* h_RT, double* s_R);
/* Rate coefficients of every reaction at T (Eqs. kfor, kc, krev): k_f, K_c
 * (0 when irreversible) and k_r; k0 is the Lindemann low-pressure limit (0
 * for other types). */
void ora_rate_coeffs(const ora_mech* m, double T, double* kf, double* kc, double* kr, double* k0);

/* Right-hand side f(y) for n reactors: dydt[i] = (dT/dt, dY_k/dt). */
void ora_rhs(const ora_mech* m, int64_t n, const double* p, const double* y, double* dydt);
/* Details for one reactor: net molar production rates wdot[S], rates of
 * progress q[R], and the gross magnitude of every component of f (the same
 * sums with every term taken in absolute value) gross[S+1]. */
void ora_rhs_detail(const ora_mech* m, double p, const double* y, double* wdot, double* q,
                    double* gross);
/* Complex-valued twin of the right-hand side (for complex-step derivatives). */
void ora_rhs_complex(const ora_mech* m, double p, const double* y_re, const double* y_im,
                     double* f_re, double* f_im);
/* Analytic Jacobian J[i][j] = d f_i / d y_j, [n][S+1][S+1]; gross (optional,
 * may be NULL) receives the same sums with every term in absolute value. */
void ora_jacobian(const ora_mech* m, int64_t n, const double* p, const double* y, double* jac,
                  double* gross);

/* Dense LU with partial pivoting of a dim x dim row-major matrix, in place.
 * piv[k] is the row swapped with row k.  Returns 0, or k+1 if pivot k is zero
 * or not finite. */
int32_t ora_lu_factor(int32_t dim, double* a, int32_t* piv);
void ora_lu_solve(int32_t dim, const double* lu, const int32_t* piv, double* b);

/* Solver options (readings of the paper's unspecified step control). */
typedef struct {
  double rtol, atol;
  double h0;       /* > 0: initial step; 0: EstimateH0 */
  double fixed_h;  /* > 0: constant step, every step accepted (order tests) */
  int32_t max_steps;
  int32_t jac;     /* ROS4 Jacobian: 0 analytic (Sec. 6), 1 forward differences (Sec. 5) */
} ora_opts;

enum { ORA_OK = 0, ORA_MAXSTEPS = 1, ORA_HMIN = 2, ORA_NONFINITE = 3, ORA_SINGULAR = 4,
       ORA_BADINPUT = 5 };
enum { ORA_ROS4 = 0, ORA_RKF45 = 1 };

/* Integrate n reactors over [0, dt[i]] (Algorithm 1).  y is in/out;
 * h_inout (may be NULL) supplies the first step when > 0 and receives the
 * step proposed after the last accepted step; steps (may be NULL) receives
 * [accepted, rejected]; status receives ORA_*.  nthreads <= 0 uses all host
 * cores; reactors are handed out one at a time from an atomic counter. */
void ora_integrate(const ora_mech* m, int32_t method, int64_t n, const double* p, double* y,
                   const double* dt, double* h_inout, const ora_opts* opts, int32_t* steps,
                   int32_t* status, int32_t nthreads);

/* Test problems with closed-form solutions, run through the same steppers
 * and driver.  problem 0: y' = diag(lam) y (dim = len(lam)); problem 1:
 * scalar y' = -y^2; problem 2: dense linear y' = A y with A = params
 * (dim x dim); problem 3: dim uncoupled copies y_i' = -y_i^2. */
void ora_test_integrate(int32_t problem, int32_t method, int32_t dim, const double* params,
                        double* y, double dt, const ora_opts* opts, int32_t* steps,
                        int32_t* status);
/* One step of size h from y (no control): ynew and the error vector. */
void ora_test_onestep(int32_t problem, int32_t method, int32_t dim, const double* params,
                      const double* y, double h, double* ynew, double* err);

/* Forward-difference Jacobians (Sec. 5, CVODE's difference quotients), one
 * per reactor at step size hstep[i] with the weights 1/(atol + rtol |y|):
 * the matrix ROS4 uses when ora_opts.jac = 1. */
void ora_jacobian_fd(const ora_mech* m, int64_t n, const double* p, const double* y, const double* hstep,
                     double rtol, double atol, double* jac);

/* The same forward-difference Jacobian for a test problem (see
 * ora_test_integrate) at y with step size h. */
void ora_test_jacobian_fd(int32_t problem, int32_t dim, const double* params, const double* y, double h,
                          double rtol, double atol, double* jac);

/* Right-hand-side evaluations made by ora_integrate's reactor systems since
 * the last reset (all threads); reset != 0 returns the count and zeroes it. */
int64_t ora_rhs_evals(int32_t reset);

int32_t ora_hardware_threads(void);

#ifdef __cplusplus
}
#endif
#endif
