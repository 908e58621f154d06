// Launch-side view of the VB-QMC kernels: per-warp shared-memory layouts and launchers.
#pragma once

#include <cuda_runtime.h>

#include "vbqmc_internal.h"

namespace vbq {

// One warp evaluates one walker; all per-walker state lives in shared memory.  Offsets are
// bytes from the start of the warp's region.
struct EvalLayout {
  int wpb = 0, warp_bytes = 0;
  int R, vg, G, LJ, Phi, PhiD, Lphi, Gphi, Binv0, Binv1, ldet, dsg, tdet, Wdet, Tdet, rk, scratch, part, partd,
      kacc, red, geo;
  int G0, G1;          // lane-group size per spin for the LU
  int jas_P, jas_S;    // Jastrow lanes: electron = lane % jas_P, group = lane / jas_P (jas_S groups)
};

struct SweepLayout {
  int wpb = 0, warp_bytes = 0;
  int R, Binv0, Binv1, ldet, dsg, wk, PhiO, bas, vrow, part, rho, cvec, scratch, geo;
  int nocc_max;
  int G0, G1;
};

int make_eval_layout(const SysDev& s, int bulk_bytes, int max_smem, EvalLayout& L);
int make_sweep_layout(const SysDev& s, int bulk_bytes, int max_smem, SweepLayout& L);

cudaError_t launch_eval(int precision, const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                        double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out,
                        cudaStream_t st);
cudaError_t launch_sweep(int precision, const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps,
                         int refresh, const double* state_in, double step, uint64_t seed, uint32_t step0, uint32_t tag,
                         uint32_t woff, int* nacc, cudaStream_t st);

}  // namespace vbq
