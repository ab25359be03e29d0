// ROS4 kernels of the 16x16-thread team with 7x7 register tiles
// (n <= 112), in their own translation unit so that the grids compile in
// parallel.
#include "ck_ros4.cuh"

namespace ck {

cudaError_t launch_ros4_16x7(const HostMech& hm, int64_t n, const double* p, double* y, const double* dt,
                          double* h_io, const SolverParams& sp, int32_t* steps, int32_t* status,
                          int32_t* queue, cudaStream_t st, const LaunchCfg& cfg, double* scratch,
                          size_t scratch_bytes, bool may_alloc) {
  return launch_ros4_tile<16, 7>(hm, n, p, y, dt, h_io, sp, steps, status, queue, st, cfg, scratch,
                                 scratch_bytes, may_alloc);
}

}  // namespace ck
