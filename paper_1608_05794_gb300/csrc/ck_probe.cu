// Throughput probes of the FP64 pipe, the roofline denominators of the
// integrators (no counterpart in the paper, which reports speedups only).
//
// Each kind is launched four times; the first warms the GPU up and the
// fastest of the other three is reported.
// kind 0: dependent-chain-free DFMA throughput.  Every thread advances 8
// independent chains a <- a b + c; the grid fills every SM with 64 warps, so
// the pipe, not latency, bounds it.  ops = flops (2 per FMA).
// kind 1: the library's table-driven 2^x (ck_exp2) throughput, 4 independent
// chains a thread, each iteration s += 2^x, x += dx.  ops = exponentials;
// each also costs the loop 2 FP64 adds.
#include <cuda_runtime.h>

#include "../../include/ck.h"
#include "ck_internal.h"

namespace ck {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int64_t iters, double* out, double b, double c) {
  double a0 = 1e-3 * threadIdx.x, a1 = a0 + 1.0, a2 = a0 + 2.0, a3 = a0 + 3.0;
  double a4 = a0 + 4.0, a5 = a0 + 5.0, a6 = a0 + 6.0, a7 = a0 + 7.0;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0 = fma(a0, b, c);
      a1 = fma(a1, b, c);
      a2 = fma(a2, b, c);
      a3 = fma(a3, b, c);
      a4 = fma(a4, b, c);
      a5 = fma(a5, b, c);
      a6 = fma(a6, b, c);
      a7 = fma(a7, b, c);
    }
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_exp2(int64_t iters, const double* __restrict__ tab,
                                                              double* out) {
  const double dx = 1.0 / 1024.0;
  double x0 = -40.0 + 0.25 * (threadIdx.x & 63), x1 = x0 + 10.0, x2 = x0 + 20.0, x3 = x0 + 30.0;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s0 += ck_exp2(x0, tab);
      s1 += ck_exp2(x1, tab);
      s2 += ck_exp2(x2, tab);
      s3 += ck_exp2(x3, tab);
      x0 += dx;
      x1 += dx;
      x2 += dx;
      x3 += dx;
    }
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = (s0 + s1) + (s2 + s3);
}

}  // namespace ck

extern "C" int ck_probe_fp64(const ck_mech* mech, int32_t kind, int64_t iters, double* seconds, double* ops) {
  if (!mech || !seconds || !ops) return ck::set_error(CK_EINVAL, "mech, seconds and ops are required");
  if (kind != 0 && kind != 1) return ck::set_error(CK_EINVAL, "kind must be 0 (DFMA) or 1 (2^x)");
  if (iters < 1 || iters > (1LL << 24)) return ck::set_error(CK_ERANGE, "iters must be in [1, 2^24]");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != mech->hm.device) return ck::set_error(CK_EINVAL, "mechanism was loaded on another device");
  const int blocks = ck::sm_count() * ck::PROBE_BLOCKS_PER_SM;
  const int64_t threads = (int64_t)blocks * ck::PROBE_THREADS;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * threads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    float ms = 0.0f;
    e = cudaEventRecord(a, st);
    if (kind == 0) ck::k_probe_dfma<<<blocks, ck::PROBE_THREADS, 0, st>>>(iters, out, 0.99999999, 1e-9);
    else ck::k_probe_exp2<<<blocks, ck::PROBE_THREADS, 0, st>>>(iters, mech->hm.d.tab, out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (rep == 1 || (rep > 1 && ms < best)) best = ms;
  }
  const float ms = best;
  if (out) cudaFree(out);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return ck::set_error(CK_ECUDA, std::string("ck_probe_fp64: ") + cudaGetErrorString(e));
  *seconds = 1e-3 * ms;
  *ops = (kind == 0 ? 2.0 * 8 * 4 : 4.0 * 4) * (double)iters * (double)threads;
  return CK_OK;
}
