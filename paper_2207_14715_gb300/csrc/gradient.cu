// Weighted sums over walkers of per-walker derivative rows (arXiv:2207.14715, Sec. 2.3.1,
// Eq. H0j: the energy gradient is a sample average of O_j E_L and E_L,j):
//   out[k] = sum_w (ga[w] Ja[w][k] + gb[w] Jb[w][k]),
// the vector-Jacobian product of (ln|Psi|, E_L) over the walkers.  Two passes with a fixed
// summation order (the result does not depend on the launch): blocks of 32 columns x a slice
// of rows write partial sums, then one thread per column adds the slices in order.
#include <algorithm>

#include "ctx_internal.h"

namespace vbq {

namespace {

constexpr int kColTile = 32, kRowWarps = 8;

template <class TJ>
__global__ void __launch_bounds__(32 * kRowWarps) colsum_partial(int W, int K, int rows, const double* __restrict__ ga,
                                                                const TJ* __restrict__ Ja, const double* __restrict__ gb,
                                                                const TJ* __restrict__ Jb, double* __restrict__ part) {
  __shared__ double red[kRowWarps][kColTile];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int k = blockIdx.x * kColTile + lane;
  const int w0 = blockIdx.y * rows, w1 = min(W, w0 + rows);
  double acc = 0.0;
  if (k < K)
    for (int w = w0 + wy; w < w1; w += kRowWarps) {
      acc = fma(__ldg(ga + w), (double)__ldg(Ja + (size_t)w * K + k), acc);
      if (Jb) acc = fma(__ldg(gb + w), (double)__ldg(Jb + (size_t)w * K + k), acc);
    }
  red[wy][lane] = acc;
  __syncthreads();
  if (wy == 0 && k < K) {
    double s = red[0][lane];
    for (int r = 1; r < kRowWarps; ++r) s += red[r][lane];
    part[(size_t)blockIdx.y * K + k] = s;
  }
}

__global__ void colsum_final(int K, int nslice, const double* __restrict__ part, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int j = 0; j < nslice; ++j) s += part[(size_t)j * K + k];
  out[k] = s;
}

}  // namespace

int colsum_slices(int W) { return std::max(1, std::min(128, (W + 511) / 512)); }

cudaError_t launch_weighted_colsum(int W, int K, int jtype, const double* ga, const void* Ja, const double* gb,
                                   const void* Jb, double* out, double* part, cudaStream_t st) {
  const int ns = colsum_slices(W), rows = (W + ns - 1) / ns;
  const dim3 grid((K + kColTile - 1) / kColTile, ns);
  if (jtype == 1)
    colsum_partial<float><<<grid, 32 * kRowWarps, 0, st>>>(W, K, rows, ga, static_cast<const float*>(Ja), gb,
                                                          static_cast<const float*>(Jb), part);
  else
    colsum_partial<double><<<grid, 32 * kRowWarps, 0, st>>>(W, K, rows, ga, static_cast<const double*>(Ja), gb,
                                                           static_cast<const double*>(Jb), part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  colsum_final<<<(K + 255) / 256, 256, 0, st>>>(K, ns, part, out);
  return cudaGetLastError();
}

}  // namespace vbq
