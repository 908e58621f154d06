// Linear-method estimators (arXiv:2207.14715, Sec. 2.3.1, Eqs. Hi0, H0j, Hij, Sij).
//
// With sample weights w_s (1 for VMC), averages <x> = sum_s w_s x_s / sum_s w_s and centred
// derivatives Ot_si = O_si - <O_i>, the paper's estimators are exactly
//   S_ij = <Ot_i Ot_j>
//   H_ij = <Ot_i (E Ot_j + E_j)>            (E = E_L, E_j = dE_L/dp_j)
//   gL_i = 2 <Ot_i E>,   gR_j = 2 (<Ot_j E> + <E_j>),   E0 = <E>
// (expanding the products recovers the printed sums of averages term by term).
//
// Passes: (1) column sums in double; (2) centring and conversion to float, X = Ot and
// Y = E Ot + dE; (3) split-K products over sample chunks on the FP32 pipe, 128x128 output
// tiles per block, each thread an 8x8 block of S and of H, partial tiles written per chunk;
// (4) deterministic reduction of the chunk partials in double and scaling.
#include <algorithm>

#include "linmethod.h"

namespace vbq {

namespace {

constexpr int kTile = 128;     // output tile edge
constexpr int kKStep = 16;     // samples staged in shared memory per step
constexpr int kThreads = 256;  // 16 x 16 threads, 8 x 8 outputs each

// Column sums: acc = [sum w, sum w E, sum w O_c (P), sum w dE_c (P)]; also float copies of w
// and E per sample.  Each block covers 256 samples; per-thread partial sums in the input type.
template <class Tin>
__global__ void lin_colsum_kernel(int P, long long M, const Tin* __restrict__ O, const Tin* __restrict__ dEL,
                                  const double* __restrict__ E, const double* __restrict__ w,
                                  double* __restrict__ acc, float* __restrict__ wf, float* __restrict__ Ef) {
  const long long s0 = (long long)blockIdx.x * 256, s1 = min(M, s0 + 256);
  __shared__ double red[2][8];
  {
    const long long s = s0 + threadIdx.x;
    double ws = 0.0, we = 0.0;
    if (s < s1) {
      ws = w ? w[s] : 1.0;
      we = ws * E[s];
      wf[s] = (float)ws;
      Ef[s] = (float)E[s];
    }
    for (int o = 16; o > 0; o >>= 1) {
      ws += __shfl_xor_sync(0xffffffffu, ws, o);
      we += __shfl_xor_sync(0xffffffffu, we, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = ws;
      red[1][threadIdx.x >> 5] = we;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sw = 0.0, se = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sw += red[0][q]; se += red[1][q]; }
    atomicAdd(acc, sw);
    atomicAdd(acc + 1, se);
  }
  for (int c = threadIdx.x; c < P; c += blockDim.x) {
    Tin so = 0, sd = 0;
    for (long long s = s0; s < s1; ++s) {
      const Tin ws = (Tin)wf[s];
      so += ws * O[s * P + c];
      sd += ws * dEL[s * P + c];
    }
    atomicAdd(acc + 2 + c, (double)so);
    atomicAdd(acc + 2 + P + c, (double)sd);
  }
}

// X = O - <O>, Y = E X + dE (floats, rows padded to Pp columns with zeros); sxe += sum w X E.
template <class Tin>
__global__ void lin_center_kernel(int P, int Pp, long long M, const Tin* __restrict__ O,
                                  const Tin* __restrict__ dEL, const double* __restrict__ acc,
                                  const float* __restrict__ wf, const float* __restrict__ Ef, float* __restrict__ X,
                                  float* __restrict__ Y, double* __restrict__ sxe /* [P] */) {
  const long long s0 = (long long)blockIdx.x * 256, s1 = min(M, s0 + 256);
  const double isw = 1.0 / acc[0];
  for (int c = threadIdx.x; c < Pp; c += blockDim.x) {
    const Tin mo = c < P ? (Tin)(acc[2 + c] * isw) : (Tin)0;
    float sx = 0.0f;
    for (long long s = s0; s < s1; ++s) {
      const float x = c < P ? (float)(O[s * P + c] - mo) : 0.0f;
      const float y = c < P ? fmaf(Ef[s], x, (float)dEL[s * P + c]) : 0.0f;
      X[s * Pp + c] = x;
      Y[s * Pp + c] = y;
      sx = fmaf(wf[s] * x, Ef[s], sx);
    }
    if (c < P) atomicAdd(sxe + c, (double)sx);
  }
}

// Partial tiles: part[chunk][0][i][j] = sum_{s in chunk} w_s X_si X_sj,
//                part[chunk][1][i][j] = sum_{s in chunk} w_s X_si Y_sj.
__global__ void __launch_bounds__(kThreads, 1)
    lin_tile_kernel(int Pp, long long M, long long chunk, const float* __restrict__ X, const float* __restrict__ Y,
                    const float* __restrict__ wf, double* __restrict__ part) {
  __shared__ __align__(16) float As[kKStep][kTile];
  __shared__ __align__(16) float Bx[kKStep][kTile];
  __shared__ __align__(16) float By[kKStep][kTile];
  const int ntj = Pp / kTile;
  const int ti = blockIdx.x / ntj, tj = blockIdx.x % ntj;
  const int i0 = ti * kTile, j0 = tj * kTile;
  const long long s0 = (long long)blockIdx.y * chunk, s1 = min(M, s0 + chunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float cs[8][8], ch[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) cs[a][b] = ch[a][b] = 0.0f;
  for (long long sb = s0; sb < s1; sb += kKStep) {
    // stage kKStep samples: 16 x 128 floats per operand, 8 per thread
    for (int q = threadIdx.x; q < kKStep * kTile; q += kThreads) {
      const int k = q / kTile, c = q % kTile;
      const long long s = sb + k;
      float a = 0.0f, bx = 0.0f, by = 0.0f;
      if (s < s1) {
        const float ws = wf[s];
        a = X[s * (long long)Pp + i0 + c];
        bx = ws * X[s * (long long)Pp + j0 + c];
        by = ws * Y[s * (long long)Pp + j0 + c];
      }
      As[k][c] = a;
      Bx[k][c] = bx;
      By[k][c] = by;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kKStep; ++k) {
      float a[8], bx[8], by[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Bx[k][tx * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Bx[k][tx * 8 + 4]);
      const float4 y0 = *reinterpret_cast<const float4*>(&By[k][tx * 8]);
      const float4 y1 = *reinterpret_cast<const float4*>(&By[k][tx * 8 + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      bx[0] = x0.x; bx[1] = x0.y; bx[2] = x0.z; bx[3] = x0.w; bx[4] = x1.x; bx[5] = x1.y; bx[6] = x1.z; bx[7] = x1.w;
      by[0] = y0.x; by[1] = y0.y; by[2] = y0.z; by[3] = y0.w; by[4] = y1.x; by[5] = y1.y; by[6] = y1.z; by[7] = y1.w;
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          cs[r][c] = fmaf(a[r], bx[c], cs[r][c]);
          ch[r][c] = fmaf(a[r], by[c], ch[r][c]);
        }
    }
    __syncthreads();
  }
  double* ps = part + (size_t)blockIdx.y * 2 * Pp * Pp;
  double* ph = ps + (size_t)Pp * Pp;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t o = (size_t)(i0 + ty * 8 + r) * Pp + j0 + tx * 8 + c;
      ps[o] = (double)cs[r][c];
      ph[o] = (double)ch[r][c];
    }
}

__global__ void lin_reduce_kernel(int P, int Pp, int nchunk, const double* __restrict__ part,
                                  const double* __restrict__ acc, const double* __restrict__ sxe, double* E0,
                                  double* gL, double* gR, double* S, double* H) {
  const double isw = 1.0 / acc[0];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (long long)P * P) {
    const int i = (int)(q / P), j = (int)(q % P);
    const size_t o = (size_t)i * Pp + j;
    double s = 0.0, h = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      s += part[(size_t)c * 2 * Pp * Pp + o];
      h += part[(size_t)c * 2 * Pp * Pp + (size_t)Pp * Pp + o];
    }
    S[q] = s * isw;
    H[q] = h * isw;
  }
  if (q < P) {
    const double oe = sxe[q] * isw;
    gL[q] = 2.0 * oe;
    gR[q] = 2.0 * (oe + acc[2 + P + q] * isw);
  }
  if (q == 0) *E0 = acc[1] * isw;
}

}  // namespace

size_t lin_workspace_bytes(int P, long long M) {
  const int Pp = ((P + kTile - 1) / kTile) * kTile;
  const long long chunk = lin_chunk(M);
  const long long nchunk = (M + chunk - 1) / chunk;
  size_t b = 0;
  b += sizeof(double) * (2 + 2 * (size_t)P) + 256;        // acc
  b += sizeof(double) * (size_t)P + 256;                  // sxe
  b += sizeof(float) * (size_t)M * Pp * 2 + 256;          // X, Y
  b += 2 * (sizeof(float) * (size_t)M + 256);             // wf, Ef
  b += sizeof(double) * (size_t)nchunk * 2 * Pp * Pp + 256;  // partial tiles
  return b;
}

long long lin_chunk(long long M) {
  // enough chunks to fill the machine with the tile grid, at least 2048 samples per chunk
  long long c = 16384;
  while (c > 2048 && (M + c - 1) / c < 32) c /= 2;
  return c;
}

template <class Tin>
static cudaError_t launch_lin_t(int P, long long M, const Tin* O, const Tin* dEL, const double* E, const double* w,
                                void* ws, double* E0, double* gL, double* gR, double* S, double* H, cudaStream_t st,
                                int* nlaunch) {
  const int Pp = ((P + kTile - 1) / kTile) * kTile;
  const long long chunk = lin_chunk(M);
  const int nchunk = (int)((M + chunk - 1) / chunk);
  unsigned char* p = static_cast<unsigned char*>(ws);
  auto take = [&](size_t bytes) {
    unsigned char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  double* acc = reinterpret_cast<double*>(take(sizeof(double) * (2 + 2 * (size_t)P)));
  double* sxe = reinterpret_cast<double*>(take(sizeof(double) * (size_t)P));
  float* X = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M * Pp));
  float* Y = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M * Pp));
  float* wf = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  float* Ef = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  double* part = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nchunk * 2 * Pp * Pp));
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * (2 + 2 * (size_t)P), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sxe, 0, sizeof(double) * (size_t)P, st);
  if (e != cudaSuccess) return e;
  const int nb = (int)((M + 255) / 256);
  lin_colsum_kernel<Tin><<<nb, 256, 0, st>>>(P, M, O, dEL, E, w, acc, wf, Ef);
  lin_center_kernel<Tin><<<nb, 256, 0, st>>>(P, Pp, M, O, dEL, acc, wf, Ef, X, Y, sxe);
  const int ntile = (Pp / kTile) * (Pp / kTile);
  lin_tile_kernel<<<dim3(ntile, nchunk), kThreads, 0, st>>>(Pp, M, chunk, X, Y, wf, part);
  const long long nq = std::max<long long>((long long)P * P, 1);
  lin_reduce_kernel<<<(int)((nq + 255) / 256), 256, 0, st>>>(P, Pp, nchunk, part, acc, sxe, E0, gL, gR, S, H);
  *nlaunch = 4;
  return cudaGetLastError();
}

cudaError_t launch_lin(int in_float, int P, long long M, const void* O, const void* dEL, const double* E,
                       const double* w, void* ws, double* E0, double* gL, double* gR, double* S, double* H,
                       cudaStream_t st, int* nlaunch) {
  if (in_float)
    return launch_lin_t<float>(P, M, static_cast<const float*>(O), static_cast<const float*>(dEL), E, w, ws, E0, gL,
                               gR, S, H, st, nlaunch);
  return launch_lin_t<double>(P, M, static_cast<const double*>(O), static_cast<const double*>(dEL), E, w, ws, E0, gL,
                              gR, S, H, st, nlaunch);
}

}  // namespace vbq
