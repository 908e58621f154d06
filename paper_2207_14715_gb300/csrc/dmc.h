// Launch-side view of the DMC step kernels (dmc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vbq {

// Per-step totals written by the scan kernel and read back by the host.
struct DmcTotals {
  long long total;  // population after branching
  double sum_w;     // sum of the pre-branching weights
  double sum_wE;    // sum of weight x E_L
  double sum_wEb;   // sum of weight x the limited branching energy (feeds E_T)
  int accepted;     // accepted moves in the step
  int pad;
};

// Arrays are walker-major: R, grad [W][N][3]; lp, sg, el, wt, wE [W]; copies, offsets, acc [W].
cudaError_t launch_dmc_propose(int W, int N, const double* R, const double* grad, double tau, uint64_t seed,
                               uint32_t step, uint32_t tag, uint32_t woff, double* Rp, cudaStream_t st);
cudaError_t launch_dmc_accept(int W, int N, double* R, double* lp, double* sg, double* el, double* grad,
                              const double* Rp, const double* lp1, const double* sg1, const double* el1,
                              const double* grad1, double tau, double E_T, uint64_t seed, uint32_t step, uint32_t tag,
                              uint32_t woff, double* wt, double* wE, double* wEb, int* copies, int* acc,
                              cudaStream_t st);
cudaError_t launch_dmc_scan(int W, const int* copies, const double* wt, const double* wE, const double* wEb,
                            const int* acc, int* offsets, DmcTotals* out, cudaStream_t st);
cudaError_t launch_dmc_branch(int W, int N, int cap, const int* copies, const int* offsets, const DmcTotals* tot,
                              const double* R, const double* lp, const double* sg, const double* el,
                              const double* grad, double* Rb, double* lpb, double* sgb, double* elb, double* gradb,
                              cudaStream_t st);

}  // namespace vbq
