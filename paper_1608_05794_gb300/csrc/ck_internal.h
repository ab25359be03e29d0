// Host-side internal interface between the C ABI (ck_api.cu) and the kernel
// translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ck_common.cuh"

namespace ck {

// Byte offsets of the sections of the staged table block (all 16-byte
// aligned).  The block is [rxn | thermo | tmid | W | invW | eff_sp | eff_m1 | exp2].
struct StageLayout {
  uint32_t rx, th, tmid, W, invW, eff_sp, eff_m1, revp, tab, bytes;
};

struct HostMech {
  int device = -1;
  DevMech d{};
  StageLayout L{};
  void* blob = nullptr;     // device allocation holding every table
  size_t blob_bytes = 0;
  int32_t* dev_err = nullptr;  // device error word (bounded waits that gave up)
  // host copies used for work counting
  std::vector<RxnRec> rx;
  int S = 0, R = 0;
  int n_contrib = 0, csr_nnz = 0;
};

// Device-side error bits reported through HostMech::dev_err.
enum : int32_t { DEVERR_STAGE_TIMEOUT = 1 };

// Launch configuration knobs chosen by the host (variant / autotuner).
struct LaunchCfg {
  int team_warps = 0;   // warps per reactor for team kernels (0: heuristic)
  int ctas_per_sm = 0;  // 0: as many as fit
  int precision = 0;    // ROS4 linear algebra: 0 FP64, 1 FP32 + FP64 refinement
  int grid_side = 0;    // ROS4 team: 0 automatic, 8 or 16 threads per side
};

cudaError_t launch_rhs(const HostMech& hm, int64_t n, const double* p, const double* y, double* f,
                       cudaStream_t st);
cudaError_t launch_jacobian(const HostMech& hm, int64_t n, const double* p, const double* y,
                            double* jac, cudaStream_t st, const LaunchCfg& cfg);
cudaError_t launch_jacobian_fd(const HostMech& hm, int64_t n, const double* p, const double* y, const double* h,
                               double rtol, double atol, double* jac, cudaStream_t st, const LaunchCfg& cfg);
cudaError_t launch_lu_factor(int64_t batch, int dim, double* a, int32_t* piv, int32_t* info,
                             cudaStream_t st);
cudaError_t launch_lu_solve(int64_t batch, int dim, const double* lu, const int32_t* piv,
                            double* b, cudaStream_t st);
// ROS4 over n reactors.  scratch / scratch_bytes: caller-held per-CTA FP64
// matrices (ros4_scratch_doubles(S+1) doubles a CTA; at most
// ros4_scratch_bytes_max() bytes for any mechanism); when absent or too
// small the launch allocates them stream-ordered if may_alloc, and otherwise
// runs the FP64 form without Jacobian copies (the precision form then fails
// with cudaErrorNotSupported).
cudaError_t launch_ros4(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                        double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                        int32_t* queue, cudaStream_t st, const LaunchCfg& cfg, double* scratch,
                        size_t scratch_bytes, bool may_alloc);
size_t ros4_scratch_bytes_max();
// launch_ros4 for one team grid (G x G threads, T x T tiles, n <= G T), each
// in its own translation unit (ck_ros4_GxT.cu).
#define CK_ROS4_TILE_LAUNCHER(NAME)                                                                          \
  cudaError_t NAME(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt, double* h_io, \
                   const SolverParams& sp, int32_t* steps, int32_t* status, int32_t* queue, cudaStream_t st,   \
                   const LaunchCfg& cfg, double* scratch, size_t scratch_bytes, bool may_alloc);
CK_ROS4_TILE_LAUNCHER(launch_ros4_8x7)
CK_ROS4_TILE_LAUNCHER(launch_ros4_16x7)
CK_ROS4_TILE_LAUNCHER(launch_ros4_16x9)
#undef CK_ROS4_TILE_LAUNCHER
cudaError_t launch_rkf45(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                         double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                         int32_t* queue, cudaStream_t st, const LaunchCfg& cfg);

cudaError_t launch_rkf45_team(const HostMech& hm, int64_t n, const double* p, double* y,
                              const double* dt, double* h_io, const SolverParams& sp, int32_t* steps,
                              int32_t* status, int32_t* queue, cudaStream_t st, const LaunchCfg& cfg);

int sm_count();

// Record a failure message for ck_last_error() and return code.
int set_error(int code, const char* msg);
inline int set_error(int code, const std::string& msg) { return set_error(code, msg.c_str()); }

// Allocation-free ROS4 (ck_integrate_ros4_noalloc): the work-queue counter
// lives in a static device array of NOALLOC_SCRATCH_INTS ints.
constexpr int NOALLOC_SCRATCH_INTS = 64;
constexpr int NOALLOC_MAX_DEVICES = 64;
cudaError_t noalloc_scratch(int32_t** out);
cudaError_t launch_ros4_noalloc(const HostMech& hm, int64_t n, const double* p, double* y,
                                const double* dt, double* h_io, const SolverParams& sp,
                                int32_t* steps, int32_t* status, cudaStream_t st,
                                const LaunchCfg& cfg);

}  // namespace ck

// Library-owned handle of a loaded mechanism (opaque in the C ABI).
struct ck_mech {
  ck::HostMech hm;
};
