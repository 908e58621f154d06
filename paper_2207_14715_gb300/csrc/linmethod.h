// Launch-side view of the linear-method accumulation (linmethod.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace vbq {

// SM count of the current device (1 if it cannot be read).
int lin_sms();
// Split of the M samples into chunks for the tensor-core pass on nsm SMs.
struct LinGrid {
  long long chunk;  // samples per chunk (a multiple of 32)
  int nchunk;
};
LinGrid lin_grid(int P, long long M, int nsm);
// Bytes of device workspace the accumulation needs for P parameters and M samples on nsm SMs.
size_t lin_workspace_bytes(int P, long long M, int nsm);
// O, dEL: [M][P] (float if in_float, else double); E, w: [M] double (w may be null); ws holds
// ws_bytes (cudaErrorInvalidValue if that is less than lin_workspace_bytes(P, M, nsm)).  ev:
// null, or 5 events recorded around the column sums, the centring, the tensor-core pass and
// the final reduction.
cudaError_t launch_lin(int in_float, int P, long long M, const void* O, const void* dEL, const double* E,
                       const double* w, void* ws, size_t ws_bytes, int nsm, double* E0, double* gL, double* gR,
                       double* S, double* H, cudaStream_t st, int* nlaunch, cudaEvent_t* ev = nullptr);

}  // namespace vbq
