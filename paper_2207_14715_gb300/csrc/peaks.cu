// ALU throughput probes: the denominators of the walker kernels' rooflines (the walker path
// is bound by FP32 FMA, FP64 FMA and the special-function unit, not by HBM).  Each probe runs
// eight independent dependency chains per thread over a grid of 8 blocks x 256 threads per SM
// (full occupancy), so the pipe, not latency, sets the pace; results feed a conditional store
// so the compiler keeps every operation.  Timed with CUDA events, best of three launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/vbqmc.h"

namespace vbq {
int set_error(int code, const std::string& msg);
int set_cuda_error(int cuda_error, const char* what);
}  // namespace vbq

namespace {

__device__ float g_sink_f;
__device__ double g_sink_d;

constexpr int kChains = 8, kUnroll = 16;

__global__ void __launch_bounds__(256) probe_ffma(int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345e-30f) g_sink_f = s;
}

__global__ void __launch_bounds__(256) probe_dfma(int iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345e-300) g_sink_d = s;
}

// x <- exp(-x) stays in (0, 1]: one special-function exponential per step and chain
__global__ void __launch_bounds__(256) probe_exp(int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __expf(-a[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345e-30f) g_sink_f = s;
}

}  // namespace

extern "C" int vbqmc_measure_alu_peaks(int device, double* out, int max, int* n) {
  if (!out || max < 1) return vbq::set_error(VBQMC_ERR_ARG, "measure_alu_peaks: null or empty output");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return vbq::set_cuda_error(e, "cudaSetDevice");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  double res[4] = {0.0, 0.0, 0.0, (double)sms};
  const int blocks = 8 * std::max(sms, 1), threads = 256;
  const double lanes = (double)blocks * threads * kChains * kUnroll;
  // iterations per kind: about 5-20 ms per launch at the nominal rates
  const int iters[3] = {4096, 128, 512};
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // launch 0 warms up
      e = cudaEventRecord(ev0, st);
      if (e != cudaSuccess) break;
      if (kind == 0) probe_ffma<<<blocks, threads, 0, st>>>(iters[0], 0.999999f, 1e-7f);
      else if (kind == 1) probe_dfma<<<blocks, threads, 0, st>>>(iters[1], 0.999999999, 1e-12);
      else probe_exp<<<blocks, threads, 0, st>>>(iters[2]);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
      if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess && best > 0.f) {
      const double ops = lanes * iters[kind] * (kind < 2 ? 2.0 : 1.0);  // FMA = 2 flops
      res[kind] = ops / (best * 1e-3) / 1e12;
    }
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (st) cudaStreamDestroy(st);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return vbq::set_cuda_error(e, "ALU probe");
  for (int i = 0; i < std::min(max, 4); ++i) out[i] = res[i];
  if (n) *n = 4;
  return VBQMC_OK;
}
