// Allocation-free form of the linear-method accumulation (declared in include/vbqmc.h as
// vbqmc_accumulate_lin_matrices_noalloc).
//
// Some callers cannot let the library allocate device memory: an application that hands the
// whole device to its own caching allocator or to a fixed memory budget, a serving process
// whose memory map must not change after start-up, or code on a latency-critical path where
// cudaMalloc's implicit device synchronization, or its failure under memory pressure, is not
// acceptable.  For them this entry point runs the same kernels as the context's accumulation
// but takes its workspace from one file-scope device array of fixed size, so that no call
// performs any allocation: no cudaMalloc or cudaFree, and no library routine that allocates.
//
// The array is created with the module's other device variables when the module is loaded; its
// address on a device is looked up once, by the first call made with that device current
// (cudaGetSymbolAddress), and cached.  That first call therefore does the set-up and should be
// made before any stream capture begins.
//
// The array is one per device and keeps whatever the previous call left in it.  Each call
// clears, on its own stream and before its kernels run, the accumulators that must start at
// zero (column sums and the centred energy moments); every other byte it reads was written by
// the same call.  Calls on one device whose executions overlap in time (different streams,
// or different host threads without ordering) race on the array: order them on one stream.
#include <mutex>
#include <string>

#include "../../include/vbqmc.h"
#include "linmethod.h"
#include "vbqmc_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// Workspace of vbqmc_accumulate_lin_matrices_noalloc on each device.
static __device__ __align__(256) unsigned char g_lin_scratch[VBQMC_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Address of g_lin_scratch on the current device (looked up on the first use per device).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_lin_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int vbqmc_accumulate_lin_matrices_noalloc(int precision, int P, int64_t M, const void* O,
                                                     const void* dEL, const double* eloc, const double* weights,
                                                     double* E0, double* gL, double* gR, double* S, double* H,
                                                     void* stream) {
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return vbq::set_error(VBQMC_ERR_ARG, "bad precision mode");
  if (P < 1 || M < 1) return vbq::set_error(VBQMC_ERR_ARG, "need P >= 1 and M >= 1");
  if (!O || !dEL || !eloc || !E0 || !gL || !gR || !S || !H)
    return vbq::set_error(VBQMC_ERR_ARG, "null required pointer");
  // Every sample takes at least 8 bytes and the P x P partial tiles at least 16 P^2, so these
  // bounds only keep the size arithmetic below far from overflow.
  const size_t cap = (size_t)VBQMC_NOALLOC_SCRATCH_BYTES;
  const int nsm = vbq::lin_sms();
  const size_t need =
      (P <= 2048 && (uint64_t)M <= cap / 8) ? vbq::lin_workspace_bytes(P, (long long)M, nsm) : cap + 1;
  if (need > cap)
    return vbq::set_error(VBQMC_ERR_CAPACITY,
                          "allocation-free linear-method accumulation: P=" + std::to_string(P) + ", M=" +
                              std::to_string((long long)M) + " needs " +
                              (need == cap + 1 ? "more than " + std::to_string(cap) : std::to_string(need)) +
                              " bytes of scratch; the fixed maximum is " + std::to_string(cap) +
                              " bytes (use vbqmc_accumulate_lin_matrices, or fewer samples per call)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vbq::set_cuda_error((int)e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return vbq::set_error(VBQMC_ERR_ARG, "device index out of range");
  void* ws = nullptr;
  e = scratch_address(dev, &ws);
  if (e != cudaSuccess) return vbq::set_cuda_error((int)e, "cudaGetSymbolAddress(linear-method scratch)");
  int nl = 0;
  e = vbq::launch_lin(precision == VBQMC_MIXED, P, (long long)M, O, dEL, eloc, weights, ws, cap, nsm, E0, gL, gR, S,
                      H, (cudaStream_t)stream, &nl);
  if (e != cudaSuccess) return vbq::set_cuda_error((int)e, "linear-method kernels");
  return VBQMC_OK;
}
