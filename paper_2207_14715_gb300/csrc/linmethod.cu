// Linear-method estimators (arXiv:2207.14715, Sec. 2.3.1, Eqs. Hi0, H0j, Hij, Sij).
//
// With sample weights w_s (1 for VMC), averages <x> = sum_s w_s x_s / sum_s w_s and centred
// derivatives Ot_si = O_si - <O_i>, the paper's estimators are exactly
//   S_ij = <Ot_i Ot_j>
//   H_ij = <Ot_i (E Ot_j + E_j)>            (E = E_L, E_j = dE_L/dp_j)
//   gL_i = 2 <Ot_i E>,   gR_j = 2 (<Ot_j E> + <E_j>),   E0 = <E>
// (expanding the products recovers the printed sums of averages term by term).
//
// Passes:
//  (1) column sums per block of 256 samples (sum w, sum w E in double; sum w O, sum w dE in the
//      input type per thread, then double), written as block partials and added in a fixed
//      order (results do not depend on scheduling), and the column maxima of |O|, |dE| and the
//      maxima of w and |E|;
//  (2) per parameter a power-of-two scale for X = sqrt(w) Ot and Y = sqrt(w) (E Ot + dE) that
//      bounds the scaled values by 2^14, then X and Y scaled, split into high and low half
//      precision parts (v = hi + lo with hi = half(v), lo = half(v - hi): 22 significant bits,
//      the accuracy of a float to 2^-22) and transposed to parameter-major rows; the same pass
//      forms sum w Ot E from the centred values (block partials, fixed-order sum);
//  (3) the products on the tensor cores (tcgen05, kind::f16, FP32 accumulators in tensor
//      memory): per output tile of 128 parameters j x 112 parameters i and chunk of samples,
//      D_S[j][i] = sum_s X_sj X_si and D_H[j][i] = sum_s Y_sj X_si, each product formed as
//      hi*lo + lo*hi + hi*hi (the lo*lo term is below the float accuracy);
//  (4) the chunk partials added in double in a fixed order, unscaled and divided by sum w.
// The half-precision split runs the tensor cores at twice the rate of the TF32 split with the
// same accuracy, because the per-parameter scales keep every value in the normal half range;
// 112-wide i tiles cover 400 parameters with 448 columns instead of 512.
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "linmethod.h"
#include "tc_ptx.cuh"

namespace vbq {

namespace {

constexpr int kTj = 128;          // output tile rows j (MMA M, tensor-memory lanes)
constexpr int kTi = 112;          // output tile columns i (MMA N, a multiple of 16)
constexpr int kColBlock = 256;    // threads of a column-sum block (and samples per sub-tile)
constexpr int kColTiles = 1;      // sub-tiles per column-sum block
constexpr int kCenTiles = 8;      // 64-sample tiles per centring block: 512 samples
constexpr float kScaleTop = 16384.0f;  // scaled values stay below 2^14 (half precision max 65504)

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ inline int rows_j(int P) { return round_up(P, kTj); }
__host__ __device__ inline int rows_i(int P) { return round_up(P, kTi); }
// rows of the transposed arrays: both tile kinds, rounded to the centring kernel's 64-row blocks
__host__ __device__ inline int rows_t(int P) { return round_up(rows_j(P) > rows_i(P) ? rows_j(P) : rows_i(P), 64); }

// (1) Block partials: row b = [sum w, sum w E, sum w O (P), sum w dE (P)] over the block's 2048
// samples (the O and dE sums in the input type per thread, stored in double); maxima as float
// bits (non-negative floats order like unsigned): mx[0] = max w, mx[1] = max |E|,
// mx[2 + c] = max |O_c|, mx[2 + P + c] = max |dE_c|.
template <class Tin>
__global__ void __launch_bounds__(kColBlock) lin_colsum_kernel(int P, long long M, const Tin* __restrict__ O,
                                                               const Tin* __restrict__ dEL,
                                                               const double* __restrict__ E,
                                                               const double* __restrict__ w,
                                                               double* __restrict__ part1, unsigned* __restrict__ mx) {
  __shared__ double sw[kColBlock], se[kColBlock];
  const int L1 = 2 * P + 2;
  double* row = part1 + (size_t)blockIdx.x * L1;
  // each thread keeps its columns' sums over the block's sub-tiles (at most ceil(P / 256)
  // columns per thread; the loop below handles the rest in passes)
  double tot_w = 0.0, tot_we = 0.0;
  for (int c0 = 0; c0 < max(P, 1); c0 += kColBlock) {
    const int c = c0 + threadIdx.x;
    Tin so = 0, sd = 0;
    float mo = 0.0f, md = 0.0f;
    for (int t = 0; t < kColTiles; ++t) {
      const long long s0 = ((long long)blockIdx.x * kColTiles + t) * kColBlock, s1 = min(M, s0 + kColBlock);
      if (s0 >= M) break;
      __syncthreads();
      {
        const long long s = s0 + threadIdx.x;
        double ws = 0.0, e = 0.0;
        if (s < s1) {
          ws = w ? w[s] : 1.0;
          e = E[s];
        }
        sw[threadIdx.x] = ws;
        se[threadIdx.x] = e;
        if (c0 == 0) {
          float mw = (float)ws, me = fabsf((float)e);
          for (int o = 16; o > 0; o >>= 1) {
            mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
            me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
          }
          if ((threadIdx.x & 31) == 0) {
            atomicMax(mx, __float_as_uint(mw));
            atomicMax(mx + 1, __float_as_uint(me));
          }
        }
      }
      __syncthreads();
      const int n = (int)(s1 - s0);
      if (c0 == 0 && threadIdx.x == 0)
        for (int k = 0; k < n; ++k) {
          tot_w += sw[k];
          tot_we = fma(sw[k], se[k], tot_we);
        }
      if (c < P)
        for (int k = 0; k < n; ++k) {
          const Tin o = O[(s0 + k) * P + c], d = dEL[(s0 + k) * P + c];
          const Tin ws = (Tin)sw[k];
          so += ws * o;
          sd += ws * d;
          mo = fmaxf(mo, fabsf((float)o));
          md = fmaxf(md, fabsf((float)d));
        }
    }
    if (c < P) {
      row[2 + c] = (double)so;
      row[2 + P + c] = (double)sd;
      atomicMax(mx + 2 + c, __float_as_uint(mo));
      atomicMax(mx + 2 + P + c, __float_as_uint(md));
    }
  }
  if (threadIdx.x == 0) {
    row[0] = tot_w;
    row[1] = tot_we;
  }
}

// Block partials added in a fixed order: acc[q] = sum over k of (sum of part1[b][q] for the
// blocks b = k mod 8, in block order), eight independent chains for memory-level parallelism.
__global__ void lin_colsum_reduce(int L1, int nb, const double* __restrict__ part1, double* __restrict__ acc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L1) return;
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int b = 0;
  for (; b + 8 <= nb; b += 8)
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += part1[(size_t)(b + k) * L1 + q];
  for (int k = 0; b + k < nb; ++k) s[k] += part1[(size_t)(b + k) * L1 + q];
  acc[q] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// Per-sample float copies for the centring pass: sqrt(w_s) and E_s.
__global__ void lin_sample_kernel(long long M, const double* __restrict__ E, const double* __restrict__ w,
                                  float* __restrict__ rw, float* __restrict__ Ef) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  rw[s] = w ? sqrtf((float)w[s]) : 1.0f;
  Ef[s] = (float)E[s];
}

// (2a) Power-of-two scales: scl[c] for X (bound sqrt(max w)(max|O_c| + |<O_c>|)) and scl[Pr + c]
// for Y (bound sqrt(max w)(max|E| (max|O_c| + |<O_c>|) + max|dE_c|)), 1 for padding rows.
__global__ void lin_scale_kernel(int P, int Pr, const double* __restrict__ acc, const unsigned* __restrict__ mx,
                                 float* __restrict__ scl) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Pr) return;
  float sx = 1.0f, sy = 1.0f;
  if (c < P) {
    const double mu = acc[2 + c] / acc[0];
    const double rw = sqrt((double)__uint_as_float(mx[0]));
    const double ox = (double)__uint_as_float(mx[2 + c]) + fabs(mu);
    const double bx = rw * ox;
    const double by = rw * ((double)__uint_as_float(mx[1]) * ox + (double)__uint_as_float(mx[2 + P + c]));
    int e;
    if (bx > 0.0) {
      frexp(bx, &e);  // bx <= 2^e
      sx = ldexpf(kScaleTop, -max(e, -100));
    }
    if (by > 0.0) {
      frexp(by, &e);
      sy = ldexpf(kScaleTop, -max(e, -100));
    }
  }
  scl[c] = sx;
  scl[Pr + c] = sy;
}

__device__ __forceinline__ void split_half(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// (2b) Scaled, split and transposed values: rows c < Pr of Xh/Xl/Yh/Yl [Pr][Mp] hold the samples
// of parameter c (zero rows c >= P).  A block transposes 64 samples x 64 parameters through
// shared memory: reads along parameters and writes along samples are both coalesced.
template <class Tin>
__global__ void __launch_bounds__(256) lin_center_kernel(int P, long long M, long long Mp, const Tin* __restrict__ O,
                                                         const Tin* __restrict__ dEL, const double* __restrict__ E,
                                                         const double* __restrict__ w, const float* __restrict__ rwf,
                                                         const float* __restrict__ Ef, const double* __restrict__ acc,
                                                         const float* __restrict__ scl, int Pr, __half* __restrict__ Xh,
                                                         __half* __restrict__ Xl, __half* __restrict__ Yh,
                                                         __half* __restrict__ Yl, double* __restrict__ part2) {
  // [array][parameter][sample]: rows of 72 halves (144 bytes) keep the 16-byte chunks aligned
  __shared__ __align__(16) __half t[4][64][72];
  __shared__ double red[4][64];
  const int c0 = blockIdx.y * 64;
  const double isw = 1.0 / acc[0];
  const int cl = threadIdx.x & 63, sq = threadIdx.x >> 6;
  const int c = c0 + cl;
  const Tin mo = c < P ? (Tin)(acc[2 + c] * isw) : (Tin)0;
  const float sx = scl[c], sy = scl[Pr + c];
  double sxe = 0.0;  // sum over this thread's samples of w Ot E (16-sample partials in Tin)
  __half* const dst[4] = {Xh, Xl, Yh, Yl};
  for (int tt = 0; tt < kCenTiles; ++tt) {
    const long long s0 = ((long long)blockIdx.x * kCenTiles + tt) * 64;
    if (s0 >= M) break;
    __syncthreads();
    Tin part = 0;
    for (int k = 0; k < 16; ++k) {
      const int sl = sq + 4 * k;
      const long long sm = s0 + sl;
      float xv = 0.0f, yv = 0.0f;
      if (sm < M && c < P) {
        const Tin x = O[sm * P + c] - mo;
        const Tin e = std::is_same<Tin, double>::value ? (Tin)E[sm] : (Tin)Ef[sm];
        const Tin ex = e * x;
        const Tin y = ex + dEL[sm * P + c];
        const float rw = rwf[sm];
        xv = (float)x * rw * sx;
        yv = (float)y * rw * sy;
        part += (w ? (Tin)w[sm] : (Tin)1) * ex;
      }
      split_half(xv, t[0][cl][sl], t[1][cl][sl]);
      split_half(yv, t[2][cl][sl], t[3][cl][sl]);
    }
    sxe += (double)part;
    __syncthreads();
    // 16-byte stores: per array 64 rows x 8 chunks of 8 samples
    for (int q = threadIdx.x; q < 4 * 64 * 8; q += 256) {
      const int a = q >> 9, rr = (q >> 3) & 63, ch = q & 7;
      const long long sm = s0 + 8 * ch;
      if (sm >= M) continue;
      const uint4 v = *reinterpret_cast<const uint4*>(&t[a][rr][8 * ch]);
      if (sm + 8 <= M) {
        *reinterpret_cast<uint4*>(dst[a] + (size_t)(c0 + rr) * Mp + sm) = v;
      } else {  // the ragged end of the samples
        const __half* hv = reinterpret_cast<const __half*>(&v);
        for (int u = 0; u < (int)(M - sm); ++u) dst[a][(size_t)(c0 + rr) * Mp + sm + u] = hv[u];
      }
    }
  }
  red[sq][cl] = sxe;
  __syncthreads();
  if (threadIdx.x < 64)  // block partial of sum w Ot E, in sample-quarter order
    part2[(size_t)blockIdx.x * Pr + c0 + threadIdx.x] = red[0][threadIdx.x] + red[1][threadIdx.x] +
                                                       red[2][threadIdx.x] + red[3][threadIdx.x];
}

// (3) Partial tiles, one CTA per (128 x 112 output tile, chunk of samples):
//   part[chunk][0][j][i] = sum_{s in chunk} X_sj X_si,   part[chunk][1][j][i] = sum Y_sj X_si
// (scaled values).  Per stage of 32 samples, TMA brings the tiles Xj hi/lo, Yj hi/lo (128 rows)
// and Xi hi/lo (112 rows), 64-byte rows K-major with the 64-byte swizzle (the layout the MMA
// reads), four stages in flight.  One thread issues per 16-sample slice the MMAs
// Xj_hi Xi_lo, Xj_lo Xi_hi, Xj_hi Xi_hi into D_S and the same with Yj into D_H (correction
// products first, while the accumulator is small).  The tensor core's accumulation rounds at
// the accumulator's magnitude, so an accumulator covers 64 samples (two stages) and is then
// moved to registers and summed there in FP32 (round to nearest); two tensor-memory sets
// alternate so that draining overlaps the next MMAs.  Barrier waits are bounded (about a
// second); on a timeout the CTA raises *err and stops.
constexpr int kTcThreads = 256;
constexpr int kK = 32;                                     // samples per stage (64 bytes of f16)
constexpr int kStages = 4;
constexpr int kJBytes = kTj * kK * 2;                      // 8 KB
constexpr int kIBytes = kTi * kK * 2;                      // 7 KB
constexpr int kStageBytes = 4 * kJBytes + 2 * kIBytes;     // Xj hi, Xj lo, Yj hi, Yj lo, Xi hi, Xi lo
constexpr int kTcSmem = kStages * kStageBytes + 1024 + 128;
constexpr int kSetCols = 256;                              // tensor-memory columns per accumulator set
constexpr uint64_t kWaitNs = 1000000000ull;
static_assert(kIBytes % 512 == 0 && kJBytes % 512 == 0, "swizzled tiles stay 512-byte aligned");

// adds this thread's 112 accumulator columns of set 'set' (warp w: lanes 32 (w % 4) + lane;
// warps 0-3 the S tile, warps 4-7 the H tile)
// (the loads go out four and three at a time, each group behind one wait)
__device__ __forceinline__ void drain(uint32_t tmem, int set, int warp, float acc[kTi]) {
  const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kSetCols * set) +
                        (warp < 4 ? 0u : (uint32_t)kTi);
  uint32_t v[4][16];
#pragma unroll
  for (int g = 0; g < 4; ++g) tmem_ld16_async(base + 16 * g, v[g]);
  tmem_wait_ld();
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[16 * g + q] += __uint_as_float(v[g][q]);
#pragma unroll
  for (int g = 0; g < 3; ++g) tmem_ld16_async(base + 64 + 16 * g, v[g]);
  tmem_wait_ld();
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[64 + 16 * g + q] += __uint_as_float(v[g][q]);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    lin_tc_kernel(const __grid_constant__ CUtensorMap tXh, const __grid_constant__ CUtensorMap tXl,
                  const __grid_constant__ CUtensorMap tYh, const __grid_constant__ CUtensorMap tYl,
                  const __grid_constant__ CUtensorMap tXhi, const __grid_constant__ CUtensorMap tXli, int Pj, int Pi,
                  long long M, long long chunk, double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStageBytes);  // [kStages] TMA arrivals
  uint64_t* done = full + kStages;                                            // [kStages] MMA completions
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + kStages);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nti = Pi / kTi;
  const int tj = blockIdx.x / nti, ti = blockIdx.x % nti;
  const int j0 = tj * kTj, i0 = ti * kTi;
  const long long s0 = (long long)blockIdx.y * chunk, s1 = min(M, s0 + chunk);
  const int nsteps = (int)((s1 - s0 + kK - 1) / kK);
  // tiles of a stage: 0 Xj_hi, 1 Xj_lo, 2 Yj_hi, 3 Yj_lo, 4 Xi_hi, 5 Xi_lo
  auto tile = [&](int st, int t) {
    return sm + st * kStageBytes + (t < 4 ? t * kJBytes : 4 * kJBytes + (t - 4) * kIBytes);
  };
  int loaded = 0;  // (thread 0) steps whose TMA was issued
  auto load = [&](int ks) {
    const int st = ks % kStages, x = (int)(s0 + (long long)ks * kK);
    loaded = ks + 1;
    mbar_arrive_expect_tx(&full[st], kStageBytes);
    tma_load_2d(tile(st, 0), &tXh, x, j0, &full[st]);
    tma_load_2d(tile(st, 1), &tXl, x, j0, &full[st]);
    tma_load_2d(tile(st, 2), &tYh, x, j0, &full[st]);
    tma_load_2d(tile(st, 3), &tYl, x, j0, &full[st]);
    tma_load_2d(tile(st, 4), &tXhi, x, i0, &full[st]);  // 112-row boxes
    tma_load_2d(tile(st, 5), &tXli, x, i0, &full[st]);
  };

  if (tid == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&done[b], 1);
    }
    fence_async_smem();
  }
  if (warp == 0) tmem_alloc(tmem_holder, 512);  // set b at columns 256 b: S (+0), H (+112)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  if (tid == 0)
    for (int ks = 0; ks < kStages && ks < nsteps; ++ks) load(ks);
  constexpr uint32_t idesc = idesc_f16(kTj, kTi);
  float acc[kTi];
#pragma unroll
  for (int c = 0; c < kTi; ++c) acc[c] = 0.0f;
  bool ok = true;
  int issued = 0, drained = 0;

  for (int ks = 0; ks < nsteps; ++ks) {
    // steps 2p and 2p + 1 accumulate into tensor-memory set p & 1
    const int st = ks % kStages, set = (ks >> 1) & 1;
    if (tid == 0) {
      const bool arrived = mbar_wait(&full[st], (uint32_t)((ks / kStages) & 1), kWaitNs);
      if (arrived) {
        tc_fence_after();
        const uint32_t xjh = smem_addr(tile(st, 0)), xjl = smem_addr(tile(st, 1));
        const uint32_t yjh = smem_addr(tile(st, 2)), yjl = smem_addr(tile(st, 3));
        const uint32_t xih = smem_addr(tile(st, 4)), xil = smem_addr(tile(st, 5));
        const uint32_t dS = tmem + kSetCols * set, dH = dS + kTi;
        const bool fresh = (ks & 1) == 0;
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint32_t ko = kk * 32;  // 16 halves = 32 bytes along the swizzled row
          const uint32_t a0 = (fresh && kk == 0) ? 0u : 1u;
          mma_f16(dS, smem_desc_k64(xjh + ko), smem_desc_k64(xil + ko), idesc, a0);
          mma_f16(dS, smem_desc_k64(xjl + ko), smem_desc_k64(xih + ko), idesc, 1u);
          mma_f16(dH, smem_desc_k64(yjh + ko), smem_desc_k64(xil + ko), idesc, a0);
          mma_f16(dH, smem_desc_k64(yjl + ko), smem_desc_k64(xih + ko), idesc, 1u);
        }
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint32_t ko = kk * 32;
          mma_f16(dS, smem_desc_k64(xjh + ko), smem_desc_k64(xih + ko), idesc, 1u);
          mma_f16(dH, smem_desc_k64(yjh + ko), smem_desc_k64(xih + ko), idesc, 1u);
        }
        mma_commit(&done[st]);
      }
      ok = arrived;
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
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
    const int row = j0 + 32 * (warp & 3) + (tid & 31);
    double* out = part + ((size_t)blockIdx.y * 2 + (warp < 4 ? 0 : 1)) * Pj * Pi + (size_t)row * Pi + i0;
#pragma unroll
    for (int c = 0; c < kTi; ++c) out[c] = (double)acc[c];
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// (4) thread (j, i): S[i][j] and H[i][j] from the chunk partials [chunk][2][Pj][Pi] (stored as
// [j][i]), unscaled; gL, gR, E0 from the column sums.
__global__ void lin_reduce_kernel(int P, int Pj, int Pi, int Pr, int nchunk, const double* __restrict__ part,
                                  const double* __restrict__ acc, const double* __restrict__ sxe,
                                  const float* __restrict__ scl, double* E0,
                                  double* gL, double* gR, double* S, double* H, const int* __restrict__ err) {
  // a timed-out tensor-core stage leaves NaN outputs
  const double isw = *err ? __longlong_as_double(0x7ff8000000000000ll) : 1.0 / acc[0];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (long long)P * P) {
    const int j = (int)(q / P), i = (int)(q % P);
    const size_t o = (size_t)j * Pi + i;
    double s = 0.0, h = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      s += part[(size_t)c * 2 * Pj * Pi + o];
      h += part[(size_t)c * 2 * Pj * Pi + (size_t)Pj * Pi + o];
    }
    const double sxi = scl[i], sxj = scl[j], syj = scl[Pr + j];
    S[(size_t)i * P + j] = s / (sxi * sxj) * isw;
    H[(size_t)i * P + j] = h / (sxi * syj) * isw;
  }
  if (q < P) {
    const double oe = sxe[q] * isw;  // <Ot E>
    gL[q] = 2.0 * oe;
    gR[q] = 2.0 * (oe + acc[2 + P + q] * isw);
  }
  if (q == 0) *E0 = acc[1] * isw;
}

}  // namespace

long long lin_chunk(long long M) {
  // enough chunks to fill the machine with the tile grid, at least 2048 samples per chunk
  long long c = 32768;
  while (c > 2048 && (M + c - 1) / c < 32) c /= 2;
  return c;
}

namespace {
struct LinWs {
  double *part1, *acc, *part2, *sxe, *part;
  unsigned* mx;
  float *scl, *rw, *Ef;
  __half *Xh, *Xl, *Yh, *Yl;
  int* err;
  size_t bytes;
};
LinWs carve(void* ws, int P, long long M) {
  const int L1 = 2 * P + 2, Pj = rows_j(P), Pi = rows_i(P), Pr = rows_t(P);
  const long long nb1 = (M + kColBlock * kColTiles - 1) / (kColBlock * kColTiles),
                  nb2 = (M + 64 * kCenTiles - 1) / (64 * kCenTiles);
  const long long Mp = (M + 31) / 32 * 32;
  const long long chunk = lin_chunk(M), nchunk = (M + chunk - 1) / chunk;
  unsigned char* p = static_cast<unsigned char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* r = p ? p + off : nullptr;
    off += (bytes + 255) & ~size_t(255);
    return r;
  };
  LinWs w{};
  w.part1 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nb1 * L1));
  w.acc = reinterpret_cast<double*>(take(sizeof(double) * (size_t)L1));
  w.part2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nb2 * Pr));
  w.sxe = reinterpret_cast<double*>(take(sizeof(double) * (size_t)Pr));
  w.mx = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (2 + 2 * (size_t)P)));
  w.scl = reinterpret_cast<float*>(take(sizeof(float) * 2 * (size_t)Pr));
  w.rw = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  w.Ef = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  w.Xh = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * Mp));
  w.Xl = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * Mp));
  w.Yh = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * Mp));
  w.Yl = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * Mp));
  w.part = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nchunk * 2 * Pj * Pi));
  w.err = reinterpret_cast<int*>(take(sizeof(int)));
  w.bytes = off;
  return w;
}
}  // namespace

size_t lin_workspace_bytes(int P, long long M) { return carve(nullptr, P, M).bytes; }

// Tensor map of a [rows][Mp] half array read as M samples per row in 32-sample x box_rows
// boxes with the 64-byte swizzle (samples past M read as zero).  The encoder comes from the
// driver through the runtime, so the library does not link the driver library itself.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_tile_map(CUtensorMap* map, const __half* base, int rows, long long M, long long Mp,
                                   int box_rows) {
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
  const cuuint64_t strides[1] = {(cuuint64_t)Mp * sizeof(__half)};
  const cuuint32_t box[2] = {(cuuint32_t)kK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  static_assert(kK * 2 == 64, "the tile rows are 64 bytes (64-byte swizzle)");
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class Tin>
static cudaError_t launch_lin_t(int P, long long M, const Tin* O, const Tin* dEL, const double* E, const double* w,
                                void* ws, double* E0, double* gL, double* gR, double* S, double* H, cudaStream_t st,
                                int* nlaunch) {
  const int L1 = 2 * P + 2, Pj = rows_j(P), Pi = rows_i(P), Pr = rows_t(P);
  const long long Mp = (M + 31) / 32 * 32;
  const int nb2 = (int)((M + 64 * kCenTiles - 1) / (64 * kCenTiles));
  const long long chunk = lin_chunk(M);
  const int nchunk = (int)((M + chunk - 1) / chunk);
  const int nb1 = (int)((M + kColBlock * kColTiles - 1) / (kColBlock * kColTiles));
  const LinWs L = carve(ws, P, M);
  cudaError_t e = cudaMemsetAsync(L.mx, 0, sizeof(unsigned) * (2 + 2 * (size_t)P), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  lin_colsum_kernel<Tin><<<nb1, kColBlock, 0, st>>>(P, M, O, dEL, E, w, L.part1, L.mx);
  lin_colsum_reduce<<<(L1 + 255) / 256, 256, 0, st>>>(L1, nb1, L.part1, L.acc);
  lin_scale_kernel<<<(Pr + 255) / 256, 256, 0, st>>>(P, Pr, L.acc, L.mx, L.scl);
  lin_sample_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, E, w, L.rw, L.Ef);
  lin_center_kernel<Tin><<<dim3((unsigned)nb2, Pr / 64), 256, 0, st>>>(
      P, M, Mp, O, dEL, E, w, L.rw, L.Ef, L.acc, L.scl, Pr, L.Xh, L.Xl, L.Yh, L.Yl, L.part2);
  lin_colsum_reduce<<<(Pr + 255) / 256, 256, 0, st>>>(Pr, nb2, L.part2, L.sxe);
  CUtensorMap mXh, mXl, mYh, mYl;
  e = encode_tile_map(&mXh, L.Xh, Pr, M, Mp, kTj);
  if (e == cudaSuccess) e = encode_tile_map(&mXl, L.Xl, Pr, M, Mp, kTj);
  if (e == cudaSuccess) e = encode_tile_map(&mYh, L.Yh, Pr, M, Mp, kTj);
  if (e == cudaSuccess) e = encode_tile_map(&mYl, L.Yl, Pr, M, Mp, kTj);
  if (e != cudaSuccess) return e;
  // the i tiles are 112 rows: maps of the same arrays with 112-row boxes
  CUtensorMap mXhi, mXli;
  e = encode_tile_map(&mXhi, L.Xh, Pr, M, Mp, kTi);
  if (e == cudaSuccess) e = encode_tile_map(&mXli, L.Xl, Pr, M, Mp, kTi);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lin_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  const int ntile = (Pj / kTj) * (Pi / kTi);
  lin_tc_kernel<<<dim3(ntile, nchunk), kTcThreads, kTcSmem, st>>>(mXh, mXl, mYh, mYl, mXhi, mXli, Pj, Pi, M, chunk,
                                                                   L.part, L.err);
  const long long nq = std::max<long long>((long long)P * P, 1);
  lin_reduce_kernel<<<(int)((nq + 255) / 256), 256, 0, st>>>(P, Pj, Pi, Pr, nchunk, L.part, L.acc, L.sxe, L.scl, E0,
                                                              gL, gR, S, H, L.err);
  *nlaunch = 8;
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
