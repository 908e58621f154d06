// Context internals shared by the C-ABI translation units (api.cu, batch_api.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"
#include "vbqmc_internal.h"

namespace vbq {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct LoadedSystem {
  bool loaded = false;
  vbq::SysHost host;
  vbq::SysDev dev{};
  void* blob = nullptr;
  size_t blob_bytes = 0;
  vbq::EvalLayout lay_eval[2];
  vbq::SweepLayout lay_sweep[2];
  vbq::ForceLayout lay_force[2];
  int lay_rc_eval[2] = {0, 0};
  int lay_rc_sweep[2] = {0, 0};
  int lay_rc_force[2] = {0, 0};
};

}  // namespace vbq

struct vbqmc_ctx {
  int device = 0;
  int max_smem = 0;
  int last_launches = 0;
  vbq::LoadedSystem sys[VBQMC_MAX_SYSTEMS];
  void* work = nullptr;      // grow-only device workspace of the linear-method accumulation
  size_t work_bytes = 0;
  void* dmc_work = nullptr;  // grow-only device workspace of the DMC steps
  size_t dmc_bytes = 0;
  void* eval_work = nullptr;  // grow-only device workspace of the evaluation kernels
  size_t eval_bytes = 0;
  void* force_work = nullptr;  // grow-only device workspace of the nucleus derivatives
  size_t force_bytes = 0;
  void* red_work = nullptr;    // grow-only device workspace of the weighted column sums
  size_t red_bytes = 0;
  int timing = 0;                               // record events around the evaluation kernels
  cudaEvent_t tev[vbq::kEvalKernels + 1] = {};  // created on first use
  bool tev_valid = false;                       // events of the last timed evaluation are recorded
};

