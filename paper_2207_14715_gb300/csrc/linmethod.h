// Launch-side view of the linear-method accumulation (linmethod.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace vbq {

// Bytes of device workspace the accumulation needs for P parameters and M samples.
size_t lin_workspace_bytes(int P, long long M);
// Samples per split-K chunk.
long long lin_chunk(long long M);
// O, dEL: [M][P] (float if in_float, else double); E, w: [M] double (w may be null).
cudaError_t launch_lin(int in_float, int P, long long M, const void* O, const void* dEL, const double* E,
                       const double* w, void* ws, double* E0, double* gL, double* gR, double* S, double* H,
                       cudaStream_t st, int* nlaunch);

}  // namespace vbq
