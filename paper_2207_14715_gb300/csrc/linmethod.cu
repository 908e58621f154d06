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
// Y = E Ot + dE; (3) the products X^T W X and X^T W Y on the tensor cores (tcgen05, TF32
// operands split into high and low parts so that the products keep float accuracy, FP32
// accumulators in tensor memory) per 128 x 128 output tile and chunk of samples, the chunk
// partials written in double; (4) deterministic reduction of the chunk partials in double
// and scaling.
#include <algorithm>

#include "linmethod.h"
#include "tc_ptx.cuh"

namespace vbq {

namespace {

constexpr int kTile = 128;     // output tile edge

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

// Centred values, transposed (parameter-major, Mp samples per row) and scaled by sqrt(w_s) so
// that the products need no weights: Xt[c][s] = sqrt(w_s) X_sc, Yt[c][s] = sqrt(w_s) Y_sc with
// X = O - <O>, Y = E X + dE (floats; rows c >= P are zero).  sxe[c] += sum_s w_s X_sc E_s.
// A block transposes a 64-sample x 64-parameter tile through shared memory so that both the
// reads (along parameters) and the writes (along samples) are coalesced.
template <class Tin>
__global__ void lin_center_kernel(int P, long long M, long long Mp, const Tin* __restrict__ O,
                                  const Tin* __restrict__ dEL, const double* __restrict__ acc,
                                  const float* __restrict__ wf, const float* __restrict__ Ef, float* __restrict__ Xt,
                                  float* __restrict__ Yt, double* __restrict__ sxe) {
  __shared__ float tx[64][65], ty[64][65];
  __shared__ float red[4][64];
  const long long s0 = (long long)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  const double isw = 1.0 / acc[0];
  {
    const int cl = threadIdx.x & 63, sq = threadIdx.x >> 6;
    const int c = c0 + cl;
    const Tin mo = c < P ? (Tin)(acc[2 + c] * isw) : (Tin)0;
    float sx = 0.0f;
    for (int k = 0; k < 16; ++k) {
      const int sl = sq + 4 * k;
      const long long sm = s0 + sl;
      float xs = 0.0f, ys = 0.0f;
      if (sm < M && c < P) {
        const float x = (float)(O[sm * P + c] - mo);
        const float y = fmaf(Ef[sm], x, (float)dEL[sm * P + c]);
        const float sw = sqrtf(wf[sm]);
        xs = sw * x;
        ys = sw * y;
        sx = fmaf(wf[sm] * x, Ef[sm], sx);
      }
      tx[cl][sl] = xs;
      ty[cl][sl] = ys;
    }
    red[sq][cl] = sx;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int c = c0 + threadIdx.x;
    if (c < P) atomicAdd(sxe + c, (double)(red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] +
                                           red[3][threadIdx.x]));
  }
  const int sl = threadIdx.x & 63, cq = threadIdx.x >> 6;
  const long long sm = s0 + sl;
  if (sm < M)
    for (int k = 0; k < 16; ++k) {
      const int cc = cq + 4 * k;
      Xt[(size_t)(c0 + cc) * Mp + sm] = tx[cc][sl];
      Yt[(size_t)(c0 + cc) * Mp + sm] = ty[cc][sl];
    }
}

// Partial tiles: part[chunk][0][i][j] = sum_{s in chunk} w_s X_si X_sj,
//                part[chunk][1][i][j] = sum_{s in chunk} w_s X_si Y_sj,
// one CTA per (128 x 128 output tile, chunk).  Per step of 16 samples, TMA brings the tiles
// A = Xt[i0..i0+127][s..s+15], Bx = Xt[j0..][s..], By = Yt[j0..][s..] into shared memory,
// K-major with the 64-byte swizzle (the layout the MMA reads), four steps in flight.  Each
// value is x = hi + lo with hi = x with its low 13 mantissa bits cleared, which is what the
// tensor core reads of the raw tile as TF32; the threads write lo = x - hi to a second tile
// at the same offsets.  One thread issues the 8-sample MMAs A_hi B_lo and A_lo B_hi (first,
// while the accumulator is small) and A_hi B_hi, B = [w X_j; w Y_j] (256 rows), into one
// 128 x 256 FP32 accumulator in tensor memory (S and H side by side), starting from zero every
// second step.  The tensor core's accumulation rounds at the accumulator's magnitude, so every
// 32 samples the result is moved to registers and summed there in FP32 (round to nearest)
// instead of accumulating the whole chunk in tensor memory.  Two tensor-memory sets alternate
// so that draining overlaps the MMAs.  Barrier waits are bounded (about a second); on a
// timeout the CTA raises *err and stops.
constexpr int kTcThreads = 256;
constexpr int kTcK = 16;                               // samples per step (64 bytes of TF32)
constexpr int kStages = 4;                             // steps in flight
constexpr int kTileBytes = kTile * kTcK * 4;           // one 128 x 16 TF32 tile: 8 KB
constexpr int kStageBytes = 6 * kTileBytes;            // A hi/lo, Bx hi/lo, By hi/lo
constexpr int kTcSmem = kStages * kStageBytes + 1024 + 128;  // stages, alignment, barriers
constexpr uint64_t kWaitNs = 1000000000ull;

// adds this thread's 128 accumulator columns of TMEM set 'set' to acc (warp w: lanes
// 32 (w % 4) + lane; warps 0-3 the S tile, warps 4-7 the H tile)
__device__ __forceinline__ void drain(uint32_t tmem, int set, int warp, float acc[kTile]) {
  const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * set) + (warp < 4 ? 0u : 128u);
#pragma unroll
  for (int c = 0; c < kTile; c += 16) {
    float v[16];
    tmem_ld16(base + c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[c + q] += v[q];
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    lin_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int Pp,
                  long long M, long long chunk, double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned stage buffers (the swizzle needs 512), barriers after them
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStageBytes);  // [kStages] TMA arrivals
  uint64_t* done = full + kStages;                                            // [kStages] MMA completions
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + kStages);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntj = Pp / kTile;
  const int ti = blockIdx.x / ntj, tj = blockIdx.x % ntj;
  const int i0 = ti * kTile, j0 = tj * kTile;
  const long long s0 = (long long)blockIdx.y * chunk, s1 = min(M, s0 + chunk);
  const int nsteps = (int)((s1 - s0 + kTcK - 1) / kTcK);
  // tiles of a stage: 0 A_hi, 1 A_lo, 2 Bx_hi, 3 By_hi, 4 Bx_lo, 5 By_lo; Bx and By of one part
  // are adjacent, so that they form one 256-row B operand [w X_j; w Y_j]
  auto tile = [&](int st, int t) { return sm + st * kStageBytes + t * kTileBytes; };
  int loaded = 0;  // (thread 0) steps whose TMA was issued
  auto load = [&](int ks) {  // thread 0: TMA of step ks into stage ks % kStages
    const int st = ks % kStages, x = (int)(s0 + (long long)ks * kTcK);
    loaded = ks + 1;
    mbar_arrive_expect_tx(&full[st], 3 * kTileBytes);
    tma_load_2d(tile(st, 0), &tmX, x, i0, &full[st]);
    tma_load_2d(tile(st, 2), &tmX, x, j0, &full[st]);
    tma_load_2d(tile(st, 3), &tmY, x, j0, &full[st]);
  };

  if (tid == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&done[b], 1);
    }
    fence_async_smem();
  }
  if (warp == 0) tmem_alloc(tmem_holder, 512);  // set b at columns 256 b: S tile (+0), H tile (+128)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  if (tid == 0)
    for (int ks = 0; ks < kStages && ks < nsteps; ++ks) load(ks);
  constexpr uint32_t idesc = idesc_tf32(128, 256);
  float acc[kTile];
#pragma unroll
  for (int c = 0; c < kTile; ++c) acc[c] = 0.0f;
  bool ok = true;
  int issued = 0;   // steps whose MMAs were issued
  int drained = 0;  // steps whose results were added to acc

  for (int ks = 0; ks < nsteps; ++ks) {
    // steps 2p and 2p + 1 accumulate into tensor-memory set p & 1
    const int st = ks % kStages, set = (ks >> 1) & 1;
    ok = __syncthreads_and(mbar_wait(&full[st], (uint32_t)((ks / kStages) & 1), kWaitNs)) != 0;
    if (!ok) break;
    // low TF32 parts lo = x - hi (hi: x with its low 13 mantissa bits cleared, which is what
    // the tensor core reads of x) in a second tile at the same (swizzled) offsets
    for (int t = 0; t < 3; ++t) {
      const int th = t == 0 ? 0 : 1 + t, tl = t == 0 ? 1 : 3 + t;  // (0, 1), (2, 4), (3, 5)
      const float4* hi = reinterpret_cast<const float4*>(tile(st, th));
      float4* lo = reinterpret_cast<float4*>(tile(st, tl));
      for (int q = tid; q < kTileBytes / 16; q += kTcThreads) {
        const float4 x = hi[q];
        lo[q] = make_float4(x.x - __uint_as_float(__float_as_uint(x.x) & 0xffffe000u),
                            x.y - __uint_as_float(__float_as_uint(x.y) & 0xffffe000u),
                            x.z - __uint_as_float(__float_as_uint(x.z) & 0xffffe000u),
                            x.w - __uint_as_float(__float_as_uint(x.w) & 0xffffe000u));
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_addr(tile(st, 0)), a_lo = a_hi + kTileBytes;
      const uint32_t b_hi = a_hi + 2 * kTileBytes, b_lo = a_hi + 4 * kTileBytes;
      const uint32_t d = tmem + 256 * set;  // S in columns 0..127, H in 128..255
      const bool fresh = (ks & 1) == 0;
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t ko = kk * 32;  // 8 TF32 = 32 bytes along the swizzled row
        mma_tf32(d, smem_desc_k64(a_hi + ko), smem_desc_k64(b_lo + ko), idesc, (fresh && kk == 0) ? 0u : 1u);
        mma_tf32(d, smem_desc_k64(a_lo + ko), smem_desc_k64(b_hi + ko), idesc, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk)
        mma_tf32(d, smem_desc_k64(a_hi + kk * 32), smem_desc_k64(b_hi + kk * 32), idesc, 1u);
      mma_commit(&done[st]);
    }
    issued = ks + 1;
    if (ks >= 1) {
      // MMAs of step ks-1 done: refill its stage with step ks+3; after the second step of a
      // pair, drain the pair's accumulators
      const int pk = ks - 1, pst = pk % kStages;
      ok = __syncthreads_and(mbar_wait(&done[pst], (uint32_t)((pk / kStages) & 1), kWaitNs)) != 0;
      if (!ok) break;
      if (tid == 0 && pk + kStages < nsteps) load(pk + kStages);
      if (pk & 1) {
        tc_fence_after();
        drain(tmem, (pk >> 1) & 1, warp, acc);
        drained = pk + 1;
        tc_fence_before();
      }
    }
  }
  // the steps not yet drained (the last pair): wait for the last MMAs and drain; on a
  // timeout, still give the copies and MMAs in flight a bounded wait before the shared and
  // tensor memory are released
  if (issued > 0 && drained < issued) {
    const int ks = issued - 1;
    const bool d = mbar_wait(&done[ks % kStages], (uint32_t)((ks / kStages) & 1), kWaitNs);
    ok = __syncthreads_and(ok && d) != 0;
    if (ok) {
      tc_fence_after();
      drain(tmem, (ks >> 1) & 1, warp, acc);
      drained = issued;
    }
  }
  if (!ok && tid == 0)
    for (int ks = issued; ks < loaded; ++ks) mbar_wait(&full[ks % kStages], (uint32_t)((ks / kStages) & 1), kWaitNs);
  if (ok && drained == nsteps) {
    const int row = i0 + 32 * (warp & 3) + (tid & 31);
    double* out = part + (size_t)blockIdx.y * 2 * Pp * Pp + (warp < 4 ? 0 : (size_t)Pp * Pp) + (size_t)row * Pp + j0;
#pragma unroll
    for (int c = 0; c < kTile; ++c) out[c] = (double)acc[c];
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

__global__ void lin_reduce_kernel(int P, int Pp, int nchunk, const double* __restrict__ part,
                                  const double* __restrict__ acc, const double* __restrict__ sxe, double* E0,
                                  double* gL, double* gR, double* S, double* H, const int* __restrict__ err) {
  // a timed-out tensor-core stage leaves NaN outputs
  const double isw = *err ? __longlong_as_double(0x7ff8000000000000ll) : 1.0 / acc[0];
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
  const long long Mp = (M + 31) / 32 * 32;
  b += 2 * (sizeof(float) * (size_t)Mp * Pp + 256);       // Xt, Yt
  b += 2 * (sizeof(float) * (size_t)M + 256);             // wf, Ef
  b += sizeof(double) * (size_t)nchunk * 2 * Pp * Pp + 256;  // partial tiles
  b += 256;                                                  // error flag
  return b;
}

long long lin_chunk(long long M) {
  // enough chunks to fill the machine with the tile grid, at least 2048 samples per chunk
  long long c = 16384;
  while (c > 2048 && (M + c - 1) / c < 32) c /= 2;
  return c;
}

// Tensor map of a [rows][Mp] float array read as M samples per row in 16-sample x 128-row
// boxes with the 64-byte swizzle (samples past M read as zero).  The encoder comes from the
// driver through the runtime, so the library does not link the driver library itself.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_tile_map(CUtensorMap* map, const float* base, int rows, long long M, long long Mp) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Mp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTile};
  const cuuint32_t estr[2] = {1, 1};
  static_assert(kTcK * 4 == 64, "the tile rows are 64 bytes (64-byte swizzle)");
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
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
  const long long Mp = (M + 31) / 32 * 32;
  float* Xt = reinterpret_cast<float*>(take(sizeof(float) * (size_t)Mp * Pp));
  float* Yt = reinterpret_cast<float*>(take(sizeof(float) * (size_t)Mp * Pp));
  float* wf = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  float* Ef = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  double* part = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nchunk * 2 * Pp * Pp));
  int* err = reinterpret_cast<int*>(take(sizeof(int)));
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * (2 + 2 * (size_t)P), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sxe, 0, sizeof(double) * (size_t)P, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int nb = (int)((M + 255) / 256);
  lin_colsum_kernel<Tin><<<nb, 256, 0, st>>>(P, M, O, dEL, E, w, acc, wf, Ef);
  lin_center_kernel<Tin><<<dim3((unsigned)((M + 63) / 64), Pp / 64), 256, 0, st>>>(P, M, Mp, O, dEL, acc, wf, Ef, Xt,
                                                                                    Yt, sxe);
  CUtensorMap tmX, tmY;
  e = encode_tile_map(&tmX, Xt, Pp, M, Mp);
  if (e == cudaSuccess) e = encode_tile_map(&tmY, Yt, Pp, M, Mp);
  if (e != cudaSuccess) return e;
  const int ntile = (Pp / kTile) * (Pp / kTile);
  e = cudaFuncSetAttribute(lin_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  lin_tc_kernel<<<dim3(ntile, nchunk), kTcThreads, kTcSmem, st>>>(tmX, tmY, Pp, M, chunk, part, err);
  const long long nq = std::max<long long>((long long)P * P, 1);
  lin_reduce_kernel<<<(int)((nq + 255) / 256), 256, 0, st>>>(P, Pp, nchunk, part, acc, sxe, E0, gL, gR, S, H, err);
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
