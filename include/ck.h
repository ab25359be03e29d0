/* ck.h — batched constant-pressure chemical kinetics on one GPU (sm_103a).
 *
 * C ABI of the library built from paper_1608_05794_gb300/csrc.  It evaluates
 * and integrates many independent homogeneous constant-pressure reactors —
 * one per CFD cell after operator splitting — as described by Stone, Alferman
 * & Niemeyer, "Accelerating finite-rate chemical kinetics with coprocessors"
 * (arXiv 1608.05794):
 *   Sec. 3  source terms: Eqs. ydot, tdot (state y = (T, Y_1..Y_S)), wdot,
 *           kfor (Arrhenius), krev and kc (reverse rates through K_c from the
 *           NASA-7 fits of Eq. tfits), third-body and Lindemann c_i;
 *   Sec. 2  RKF45 (tableau of App. B) and ROS4 in transformed form
 *           (coefficients of App. C), each driven by Algorithm 1;
 *   Sec. 6  the analytic Jacobian that the paper recommends over finite
 *           differences.
 *
 * Conventions for every call below.
 *   - Units are SI: T in K, p in Pa, concentrations in mol/m^3, molar masses
 *     in kg/mol, activation energies in J/mol, time in s.
 *   - A reactor state is n = S + 1 doubles: y[0] = T, y[1+k] = Y_k (mass
 *     fraction of species k).  Batches are row-major: reactor i occupies
 *     y[i*n .. i*n+n-1].
 *   - Array arguments may be device pointers (cudaMalloc, torch CUDA
 *     tensors) or host pointers.  With device pointers the call only enqueues
 *     work on `stream` (a cudaStream_t, NULL for the legacy default stream)
 *     and returns; the caller keeps the buffers alive until the stream has
 *     reached that point.  If any array argument of a call is host memory,
 *     the library stages every array through device memory on `stream`,
 *     waits for the stream, and returns with the host arrays updated.
 *   - Arrays are owned by the caller; the library never frees them.  Objects
 *     (ck_mech) are owned by the library and freed by their _free call.
 *   - Every call returns CK_OK (0) or a positive call status (CK_E*);
 *     ck_last_error() describes the most recent failure of this thread.
 *     Per-reactor outcomes go to status[] (CK_R_*).  The library never traps
 *     or aborts the process.
 */
#ifndef CK_H
#define CK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Call status. */
enum {
  CK_OK = 0,
  CK_EINVAL = 1,   /* bad argument or mechanism */
  CK_ECUDA = 2,    /* a CUDA call failed (see ck_last_error) */
  CK_ENOMEM = 3,   /* device allocation failed */
  CK_AGAIN = 4,    /* resource temporarily insufficient */
  CK_TIMEOUT = 5,  /* a bounded device wait gave up */
  CK_ERANGE = 6    /* size beyond a documented limit */
};

/* Per-reactor status of the integrators (status[i]).  A reactor that does
 * not finish keeps its last accepted state. */
enum {
  CK_R_OK = 0,
  CK_R_MAXSTEPS = 1,  /* opts.max_steps attempted steps without reaching dt */
  CK_R_HMIN = 2,      /* step size fell below 1e-15 * dt */
  CK_R_NONFINITE = 3, /* trial states stayed NaN/Inf until the step size collapsed */
  CK_R_SINGULAR = 4,  /* ROS4: 10 consecutive singular iteration matrices */
  CK_R_BADINPUT = 5   /* non-finite state, T <= 0, p <= 0 or dt < 0 */
};

/* Limits of this build.  CK_MAX_REACTORS bounds n of every integrating call
 * (ck_integrate_*, a group of ck_integrate_groups, ck_submit): reactors are
 * handed out by a 32-bit device work-queue counter that every CTA or thread
 * advances once past the end, so n + the launch's resident threads must stay
 * below 2^31.  Larger batches are rejected with CK_ERANGE before anything is
 * launched; split them into several calls. */
#define CK_MAX_SPECIES 128
#define CK_MAX_REACTIONS 32767
#define CK_MAX_REACTORS (1LL << 30)

typedef struct ck_mech ck_mech;

/* Mechanism description (host arrays, copied by ck_load_mechanism).
 * Reaction i has reactant slots reac[3i..3i+2] and product slots
 * prod[3i..3i+2] holding species indices, padded with -1; a species listed
 * twice has stoichiometric coefficient 2 (at most 3 slots per side, Eq. wdot).
 * arrh[3i..3i+2] = (A, beta, Ea) of Eq. kfor with A in SI units for the
 * reaction's order (one order higher for third-body reactions).  rtype: 0
 * elementary (c_i = 1), 1 third-body (c_i = [M]), 2 Lindemann fall-off
 * (c_i = P_r/(1+P_r), P_r = k0 [M]/k_inf with k0 from arrh0 and k_inf from
 * arrh).  [M] = sum_k eff_ik [X_k] with eff_ik from the CSR arrays
 * eff_ptr[R+1] / eff_sp / eff_val and 1 for unlisted species.  reversible:
 * 1 = k_r from K_c (Eqs. krev, kc), 0 = irreversible, 2 = k_r from the
 * explicit reverse Arrhenius coefficients arrh_rev[3i..3i+2] = (A_r, beta_r,
 * Ea_r) (Sec. 3; arrh_rev may be NULL when no reaction uses it).  reactor
 * selects the system the handle integrates (Sec. 3): 0 constant pressure,
 * where the per-reactor parameter p of every call is the pressure in Pa; 1
 * constant volume, where p is the reactor's fixed density in kg/m^3 and the
 * temperature equation uses the internal energies u_k and c_v.  nasa[S][2][7] holds
 * the NASA-7 coefficients a1..a7 of the low (index 0, T < t_mid) and high
 * ranges (Eq. tfits).  elem_count[S][n_elements] (optional, may be NULL)
 * enables the atom-balance check; elem_mass[n_elements] (optional) enables
 * the check of mw against the compositions. */
typedef struct {
  int32_t n_species, n_reactions;
  const double* mw;
  const double* nasa;
  const double* t_mid;
  const int32_t* reac;
  const int32_t* prod;
  const double* arrh;
  const int32_t* rtype;
  const int32_t* reversible;
  const double* arrh0;
  const int32_t* eff_ptr;
  const int32_t* eff_sp;
  const double* eff_val;
  int32_t n_elements;
  const int32_t* elem_count;
  const double* elem_mass;
  const double* arrh_rev;
  int32_t reactor;
} ck_mech_desc;

/* Solver options.  The paper leaves the step-size controller unspecified
 * (Sec. 5.2: both solvers share h0 estimation and h adaptation); this
 * library's reading: weighted RMS error norm with weights atol + rtol
 * max(|y|, |y*|); accept iff err < 1; h <- h min(5, max(0.2, 0.9 err^(-1/q)))
 * with q = 4 (ROS4) or 5 (RKF45), no growth right after a rejection; h0 from
 * the Hairer-Norsett-Wanner starting-step algorithm; last step clamped to
 * end exactly at dt. */
typedef struct {
  double rtol;      /* relative tolerance (> 0) */
  double atol;      /* absolute tolerance (> 0) */
  double h0;        /* > 0: first step size; 0: estimate */
  double fixed_h;   /* > 0: constant step, no error control (order tests) */
  int32_t max_steps;/* attempted steps per reactor (accepted + rejected) */
  int32_t precision;/* 0: FP64 throughout; 1 or 2 (ROS4): the LU factor and stage solves in FP32,
                       each solve refined once or twice against the FP64 iteration matrix; the
                       rates, K_c, the temperature equation, the error norm and step control
                       stay FP64 */
  int32_t variant;  /* 0: as many resident CTAs / blocks per SM as fit; > 0: cap per SM */
  int32_t form;     /* RKF45 mapping: 0 automatic, 1 one thread per reactor (shallow),
                       2 one CTA per reactor (deep); ROS4 always uses one CTA per reactor */
  int32_t team;     /* ROS4 thread grid of a reactor team: 0 automatic, 8 (8x8 threads, n <= 56)
                       or 16 (16x16 threads, n <= 112) */
  int32_t jac;      /* ROS4 Jacobian: 0 analytic (Sec. 6), 1 forward differences as the paper
                       ran it (Sec. 5; see ck_jacobian_fd), n further RHS evaluations a step */
} ck_solver_opts;

/* Fills *opts with rtol 1e-9, atol 1e-12, h0 0, fixed_h 0, max_steps 100000. */
void ck_default_opts(ck_solver_opts* opts);

/* Validate a mechanism, pack it into device tables on the current device
 * and return a handle.  Packing (the paper's "binary database", Sec. 5):
 * log2 A, Ea/(R ln 2) and beta per reaction; the Gibbs, enthalpy and heat
 * capacity polynomials pre-divided for FP64-lean evaluation; a
 * species -> reaction table for the team kernels.  Checks: sizes within
 * CK_MAX_*, indices in range, A > 0, finite coefficients, mw > 0, and atom
 * balance of every reaction when elem_count is given.  Returns CK_EINVAL
 * with a message on failure (nothing allocated), CK_ENOMEM/CK_ECUDA on
 * device failures. */
int ck_load_mechanism(const ck_mech_desc* desc, ck_mech** out);
/* Free a handle (device tables included).  NULL is allowed. */
int ck_free_mechanism(ck_mech* mech);
/* Sizes of a loaded mechanism. */
int ck_mech_info(const ck_mech* mech, int32_t* n_species, int32_t* n_reactions);

/* Right-hand side of Eqs. ydot/tdot for n reactors: dydt[i*(S+1)+0] = dT/dt,
 * dydt[i*(S+1)+1+k] = dY_k/dt.  p[n] Pa, y[n][S+1].  One thread per reactor. */
int ck_rhs(const ck_mech* mech, int64_t n, const double* p, const double* y, double* dydt,
           void* stream);

/* Analytic Jacobian jac[i][r][c] = d f_r / d y_c ([n][S+1][S+1], row-major per
 * reactor) of the constant-pressure system at (p[i], y[i]).  One CTA per
 * reactor. */
int ck_jacobian(const ck_mech* mech, int64_t n, const double* p, const double* y, double* jac,
                void* stream);

/* Forward-difference Jacobian, the paper's choice for ROS4 (Sec. 5: first-order
 * forward differences following CVODE, S+1 right-hand-side evaluations per
 * Jacobian), with CVODE's dense difference-quotient increments: unit roundoff
 * U = 2^-52, weights w_c = 1/(atol + rtol |y_c|), fnorm = the weighted RMS
 * norm of f(y), floor s0 = 1000 |h| U (S+1) fnorm (1 when fnorm = 0), and
 * column c = (f(y + s_c e_c) - f(y)) / s_c with s_c = max(2^-26 |y_c|,
 * s0 / w_c).  h[n] is the step size each matrix is for; jac as in
 * ck_jacobian.  One CTA per reactor; host or device pointers (host arrays
 * are staged through device memory and the call synchronises). */
int ck_jacobian_fd(const ck_mech* mech, int64_t n, const double* p, const double* y, const double* h,
                   double rtol, double atol, double* jac, void* stream);

/* Batched dense LU with partial pivoting (the linear algebra of the ROS4
 * stages, Sec. 2).  a[batch][dim][dim] row-major, factored in place into the
 * unit lower and upper triangles; piv[batch][dim] = row exchanged with row k;
 * info[batch] = 0 or k+1 when pivot k is zero or not finite.  dim <= 128. */
int ck_lu_factor(int64_t batch, int32_t dim, double* a, int32_t* piv, int32_t* info, void* stream);
/* Solve A x = b in place for every matrix factored by ck_lu_factor. */
int ck_lu_solve(int64_t batch, int32_t dim, const double* lu, const int32_t* piv, double* b,
                void* stream);

/* Integrate reactor i from t = 0 to dt[i] with ROS4 (Sec. 2, App. C:
 * four-stage L-stable Rosenbrock, transformed form, analytic Jacobian,
 * one LU per step, error = sum E_i u_i) under Algorithm 1.  y[n][S+1] is
 * overwritten with the final states.  h_inout[n] (may be NULL): on entry a
 * positive value is the first step size; on exit the step size proposed
 * after the last accepted step.  steps[n][2] (may be NULL): accepted and
 * rejected steps.  status[n]: CK_R_*.  opts may be NULL for the defaults.
 * One CTA per reactor; reactors are handed out by a device work queue. */
int ck_integrate_ros4(const ck_mech* mech, int64_t n, const double* p, double* y, const double* dt,
                      double* h_inout, const ck_solver_opts* opts, int32_t* steps, int32_t* status,
                      void* stream);
/* Same with RKF45 (Sec. 2, App. B: six stages, fourth-order solution
 * propagated, error = sum (bh - b) k).  One thread per reactor; each thread
 * takes the next reactor from the work queue when its reactor finishes. */
int ck_integrate_rkf45(const ck_mech* mech, int64_t n, const double* p, double* y, const double* dt,
                       double* h_inout, const ck_solver_opts* opts, int32_t* steps, int32_t* status,
                       void* stream);

/* ---------------------------------------------------------------- mixed batches
 * Several groups of reactors, each on its own mechanism, integrated in one
 * call (no counterpart in the paper, which runs one mechanism at a time).
 * Every group runs as a persistent work-queue kernel on a branch forked from
 * `stream`, launched in decreasing order of work_weight (or, when 0, of
 * reactors x the cost of one step of the method from ck_count_work) at full
 * occupancy, so the next group's CTAs take over SMs as the previous group's
 * drain; opts.variant > 0 caps a group's resident CTAs per SM instead.
 * flags: CK_GROUPS_SEQUENTIAL launches the groups one after another on
 * `stream` instead (same order; each then has the whole GPU until its tail);
 * with CK_GROUPS_GRAPH the fork / kernels / join sequence is captured into a
 * CUDA graph on the first call and replayed on later calls with
 * byte-identical arguments and flags (the cache holds 8 graphs; the input
 * arrays may change contents, not addresses).  Every form gives bitwise the
 * same results as one ck_integrate_* call per group.  Device pointers only. */
#define CK_GROUPS_GRAPH 1
#define CK_GROUPS_SEQUENTIAL 2
typedef struct {
  const ck_mech* mech;
  int64_t n;
  const double* p;
  double* y;
  const double* dt;
  double* h_inout;   /* may be NULL */
  int32_t* steps;    /* may be NULL */
  int32_t* status;
  ck_solver_opts opts;
  double work_weight;
} ck_group;
int ck_integrate_groups(int32_t method, int32_t n_groups, const ck_group* groups, int32_t flags,
                        void* stream);
/* Free every cached graph (synchronizes the device). */
int ck_graph_cache_clear(void);

/* ---------------------------------------------------------------- serving
 * A request server for reactor batches that arrive over time (continuous
 * batching; no counterpart in the paper, which integrates one fixed batch).
 * The server's device memory stays within hbm_budget_bytes: at creation each
 * stream reserves the ROS4 solver scratch of its launches (per-CTA copies of
 * the Jacobian and the precision form's FP64 iteration matrices; the SM
 * count x the shared memory of an SM, the most any mechanism can need,
 * about 35 MB on GB300), and a request is admitted, in arrival order, once
 * its device footprint (n * ((S+1)*8 + 28) bytes: state, p, dt, status,
 * step counts) fits in what the reservation leaves; admitted requests are split into chunks of chunk_reactors
 * reactors that a dispatcher thread launches on `streams` CUDA streams, each
 * free stream taking the next chunk of the request with the least estimated
 * remaining work (reactors left x the FP64 cost of one step of its method;
 * a request admitted more than 30 s earlier goes first).  Work that arrives
 * while other requests run therefore starts at once, overlaps them on the
 * device, and short requests are not held behind long ones.  A request's arrays are all host memory
 * (staged by the server; pin them for asynchronous copies) or all device
 * memory (used in place), and must stay valid until the request is done.
 * Each reactor is integrated independently, so results do not depend on the
 * other requests in flight. */
typedef struct ck_server ck_server;
typedef struct {
  int64_t queued, active, completed;
  uint64_t bytes_in_use;  /* reserved scratch + admitted requests */
  uint64_t budget;
  uint64_t reserved;      /* solver scratch held by the streams */
} ck_server_info;
/* Create a server on the current device.  streams in [1, 64];
 * chunk_reactors <= 0 selects 8192.  CK_ERANGE if the budget does not
 * exceed the streams' reserved scratch. */
int ck_server_create(size_t hbm_budget_bytes, int32_t streams, int64_t chunk_reactors, ck_server** out);
/* Queue a request: method 0 ROS4, 1 RKF45; the same arrays and options as
 * ck_integrate_*; steps may be NULL; n in [1, CK_MAX_REACTORS].  *ticket
 * identifies it.  CK_AGAIN if the request alone exceeds what the budget
 * leaves beside the reserved scratch. */
int ck_submit(ck_server* srv, const ck_mech* mech, int32_t method, int64_t n, const double* p, double* y,
              const double* dt, const ck_solver_opts* opts, int32_t* status, int32_t* steps,
              uint64_t* ticket);
/* Non-blocking state: *state = 0 in flight, 1 done, 2 failed (the call
 * returns the failure code), 3 cancelled. */
int ck_poll(ck_server* srv, uint64_t ticket, int32_t* state);
/* Block until the request is done, failed or cancelled, or timeout_s
 * elapses (CK_TIMEOUT). */
int ck_wait(ck_server* srv, uint64_t ticket, double timeout_s);
/* Cancel a request that has not been admitted yet (CK_AGAIN otherwise). */
int ck_cancel(ck_server* srv, uint64_t ticket);
/* Forget a finished request (CK_AGAIN while in flight). */
int ck_release(ck_server* srv, uint64_t ticket);
int ck_server_stats(ck_server* srv, ck_server_info* out);
/* Stop the dispatcher, wait for the device, free everything. */
int ck_server_destroy(ck_server* srv);

/* Allocation-free variant of ck_integrate_ros4 (no counterpart in the paper).
 * Same arguments, arithmetic and results as ck_integrate_ros4 in its FP64
 * form, for callers that cannot let a library allocate device memory: a CFD
 * code that hands all device memory to its own pool at start-up and runs
 * with no headroom, or a process under a fixed device-memory budget where an
 * allocation in the middle of a time step could fail.  ck_integrate_ros4
 * takes its work-queue counter and its per-CTA copies of the Jacobian from a
 * per-call stream-ordered allocation; this entry point uses a statically
 * allocated 256-byte device array for the counter (held on every GPU that
 * loads the library until the process exits), keeps no Jacobian copy (a
 * rejected step recomputes the Jacobian at the unchanged state, which gives
 * the same values), and calls no cudaMalloc, cudaMallocAsync or cudaFree.
 *   - Only the FP64 form is available: opts.precision 1 and 2 need per-CTA
 *     FP64 matrices in device memory and are refused with CK_EINVAL.
 *   - Every array must be a device pointer; host arrays are rejected with
 *     CK_EINVAL because staging them would need device buffers.
 *   - n must not exceed CK_NOALLOC_MAX_REACTORS (CK_ERANGE otherwise).
 *   - The array's device address is looked up once per device, with that
 *     device current: ck_load_mechanism does it for the device it loads on
 *     (so the driver loads the library's device code there, not inside this
 *     call); a call on a device with no mechanism loaded cannot happen, since
 *     the handle must belong to the current device.
 *   - All calls on a device share the array: the counter is zeroed on
 *     `stream` before each launch, so calls that overlap on the GPU (on
 *     different streams, or from several host threads) race and must be
 *     serialized by the caller. */
#define CK_NOALLOC_MAX_REACTORS CK_MAX_REACTORS
int ck_integrate_ros4_noalloc(const ck_mech* mech, int64_t n, const double* p, double* y,
                              const double* dt, double* h_inout, const ck_solver_opts* opts,
                              int32_t* steps, int32_t* status, void* stream);

/* Algorithmic FP64 work, counted from the loaded tables, in FP64 pipe
 * instructions (an FMA, a multiply, an add and a divide count one each; a
 * 2^x counts 8, the cost of the table-driven evaluation this library uses):
 * one RHS, the Jacobian beyond the RHS it also returns, one LU, one pair of
 * triangular solves, one ROS4 step (Jacobian, 3 RHS, LU, 4 solves, vector
 * work) and one RKF45 step (6 RHS, vector work); exps per RHS (one per
 * forward rate, explicit reverse rate and Lindemann k0, and two per species
 * for the Gibbs factors 2^(+-g_k) that give 1/K_c as a product); and the
 * algorithmic bytes per reactor (state in and out, p, dt, status). */
typedef struct {
  double rhs_fp64, rhs_exps, jac_fp64, lu_fp64, solve_fp64;
  double ros4_step_fp64, rkf45_step_fp64;
  double rhs_bytes, integrate_bytes;
  double ros4_fd_step_fp64;  /* one ROS4 step with the forward-difference Jacobian: S+2 RHS
                                (f(y) and one per column) + 2 stage RHS, LU, 4 solves, vector work */
  /* The same work in the flop model of a roofline: an FMA counts 2 flops,
   * any other FP64 add, multiply, divide or comparison 1; exponentials and
   * logarithms are not flops and are counted apart as transcendentals (one
   * ln T and rhs_exps 2^x per RHS).  A ROS4 step that follows a rejected
   * attempt reuses J and f(y) (the state is unchanged): it costs
   * ros4_attempt_flops, and a step at a new state ros4_jeval_flops more (the
   * analytic Jacobian and the RHS it returns; 1 + rhs_exps transcendentals).
   * Each attempt also evaluates 2 stage RHS (2 (1 + rhs_exps)
   * transcendentals).  ros4_fd_jeval_flops replaces ros4_jeval_flops with the
   * forward-difference Jacobian (S+2 RHS). */
  double rhs_flops, rhs_transc, jac_flops, lu_flops, solve_flops;
  double ros4_jeval_flops, ros4_attempt_flops, ros4_step_flops, rkf45_step_flops, ros4_fd_jeval_flops;
} ck_work_counts;
int ck_count_work(const ck_mech* mech, ck_work_counts* out);

/* Throughput probes of the FP64 pipe, the roofline denominators of the
 * integrators (no counterpart in the paper).  kind 0: FMA throughput, 8
 * independent chains a thread over 64 warps an SM; *ops = flops executed (2
 * per FMA).  kind 1: throughput of this library's table-driven 2^x (the
 * mechanism's table), 4 independent chains a thread; *ops = exponentials
 * evaluated (each iteration also takes 2 FP64 adds).  iters in [1, 2^24]
 * loop iterations a thread; the probe is launched four times on a private
 * stream, each timed with CUDA events, and *seconds is the fastest of the
 * last three (the first warms the GPU up).  Synchronizes;
 * allocates one double a thread of the grid for the probe's results. */
int ck_probe_fp64(const ck_mech* mech, int32_t kind, int64_t iters, double* seconds, double* ops);

/* Device error word of a mechanism (bit 1: a bounded shared-memory staging
 * wait gave up).  Synchronizes the device; clears the word when reset != 0. */
int ck_device_errors(const ck_mech* mech, int32_t* bits, int32_t reset);

const char* ck_status_str(int code);
const char* ck_last_error(void);
const char* ck_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CK_H */
