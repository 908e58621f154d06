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

// Structure overlap (Sec. 2.4): per sample the full row R_I = Psi_I/Psi_0 of the Nvb structures
// (columns of O for the structures in cparam; a structure left out of the parameters from the
// sum rule sum_I c_I R_I = 1, which holds at every sample), then the weighted sums of
// R_I R_J (I <= J), R_I and the weights, in double, per slice of samples; a second kernel adds
// the slices in order.  Pair index t < npair(n) over the columns 0..n where column n is 1.
constexpr int kOvTile = 64;

__host__ __device__ inline int ov_npair(int n) { return (n + 1) * (n + 2) / 2; }

template <class TO>
__global__ void __launch_bounds__(256) overlap_partial(int M, int ldo, int rows, const TO* __restrict__ O,
                                                       const double* __restrict__ wts, const OverlapMap map,
                                                       double* __restrict__ part) {
  __shared__ double tile[kOvTile][kOvMaxStruct + 1];
  const int n = map.nvb, np = ov_npair(n);
  const int w0 = blockIdx.x * rows, w1 = min(M, w0 + rows);
  // each thread owns up to 3 pairs (np <= 561 with 32 structures)
  int pi[3], pj[3];
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = threadIdx.x + 256 * r;
    pi[r] = pj[r] = -1;
    if (t < np) {  // t -> (i, j), i <= j <= n, row-major upper triangle
      int i = 0;
      while (t >= n + 1 - i) {
        t -= n + 1 - i;
        ++i;
      }
      pi[r] = i;
      pj[r] = i + t;
    }
  }
  for (int b = w0; b < w1; b += kOvTile) {
    const int nb = min(kOvTile, w1 - b);
    __syncthreads();
    for (int q = threadIdx.x; q < nb * (n + 1); q += 256) {
      const int rr = q / (n + 1), I = q - rr * (n + 1);
      double v;
      if (I == n) v = 1.0;
      else if (map.col[I] >= 0) v = (double)__ldg(O + (size_t)(b + rr) * ldo + map.col[I]);
      else {  // the structure left out of cparam: R_I0 = (1 - sum_I c_I R_I) / c_I0
        double s = 1.0;
        for (int J = 0; J < n; ++J)
          if (map.col[J] >= 0) s -= map.c[J] * (double)__ldg(O + (size_t)(b + rr) * ldo + map.col[J]);
        v = s / map.c[I];
      }
      tile[rr][I] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (pi[r] < 0) continue;
      const int i = pi[r], j = pj[r];
      double a = acc[r];
      for (int rr = 0; rr < nb; ++rr) {
        const double w = wts ? __ldg(wts + b + rr) : 1.0;
        a = fma(w * tile[rr][i], tile[rr][j], a);
      }
      acc[r] = a;
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
    if (pi[r] >= 0) part[(size_t)blockIdx.x * np + threadIdx.x + 256 * r] = acc[r];
}

}  // namespace

int overlap_slices(int M) { return std::max(1, std::min(256, (M + 1023) / 1024)); }
size_t overlap_part_doubles(int M, int nvb) { return (size_t)overlap_slices(M) * ov_npair(nvb); }

cudaError_t launch_structure_overlap(int M, int ldo, int otype, const void* O, const double* wts, const OverlapMap& map,
                                     double* part, double* out, cudaStream_t st) {
  const int ns = overlap_slices(M), rows = (M + ns - 1) / ns, np = ov_npair(map.nvb);
  if (otype == 1)
    overlap_partial<float><<<ns, 256, 0, st>>>(M, ldo, rows, static_cast<const float*>(O), wts, map, part);
  else
    overlap_partial<double><<<ns, 256, 0, st>>>(M, ldo, rows, static_cast<const double*>(O), wts, map, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  colsum_final<<<(np + 255) / 256, 256, 0, st>>>(np, ns, part, out);
  return cudaGetLastError();
}

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
