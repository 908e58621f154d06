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
//      the accuracy of a float to 2^-22) and transposed into 32-sample groups of parameter
//      rows (each row 32 high halves then 32 low halves); the same pass forms sum w Ot E from
//      the centred values (block partials, fixed-order sum);
//  (3) the products on the tensor cores (tcgen05, kind::f16, FP32 accumulators in tensor
//      memory): per output tile of 128 parameters i x 112 parameters j and chunk of samples,
//      D_S[i][j] = sum_s X_si X_sj and D_H[i][j] = sum_s X_si Y_sj in one MMA of N = 224 whose B
//      operand stacks the j rows of X and of Y, each product formed as hi*lo + lo*hi + hi*hi
//      (the lo*lo term is below the float accuracy);
//  (4) the chunk partials added in double in a fixed order, unscaled and divided by sum w.
// The half-precision split runs the tensor cores at twice the rate of the TF32 split with the
// same accuracy, because the per-parameter scales keep every value in the normal half range;
// 112-wide j tiles cover 400 parameters with 448 columns instead of 512.
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "linmethod.h"
#include "tc_ptx.cuh"

namespace vbq {

namespace {

constexpr int kTa = 128;          // output tile rows i (MMA M, tensor-memory lanes): A = X_i
constexpr int kTb = 112;          // output tile columns j of S and of H: B = [X_j; Y_j], N = 224
constexpr int kColBlock = 256;    // threads of a column-sum block (and samples per sub-tile)
constexpr int kCenTiles = 8;      // 64-sample tiles per centring block: 512 samples
constexpr float kScaleTop = 16384.0f;  // scaled values stay below 2^14 (half precision max 65504)

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ inline int rows_a(int P) { return round_up(P, kTa); }
__host__ __device__ inline int rows_b(int P) { return round_up(P, kTb); }
// stored rows of the transposed arrays: P rounded to the centring kernel's 64-row blocks, at
// least one 128-row tile (the tensor-core pass reads the rows from max(P, 128) up to its tile
// edges as zeros, filled by the copy engine, not from memory)
__host__ __device__ inline int rows_t(int P) { return round_up(P > kTa ? P : kTa, 64); }
// rows the tensor maps cover (never fewer than a box)
__host__ __device__ inline int rows_m(int P) { return P > kTa ? P : kTa; }

// Four consecutive columns c .. c + 3 of one sample row (zero past P): 16-byte loads when VEC
// (P a multiple of 4 and 16-byte aligned arrays), else one element at a time.
template <class Tin, bool VEC>
__device__ __forceinline__ void load4(const Tin* __restrict__ row, int c, int P, Tin v[4]) {
  if (VEC) {
    if (std::is_same<Tin, float>::value) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(row + c));
      v[0] = (Tin)t.x; v[1] = (Tin)t.y; v[2] = (Tin)t.z; v[3] = (Tin)t.w;
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(row + c));
      const double2 b = __ldg(reinterpret_cast<const double2*>(row + c + 2));
      v[0] = (Tin)a.x; v[1] = (Tin)a.y; v[2] = (Tin)b.x; v[3] = (Tin)b.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = c + u < P ? row[c + u] : (Tin)0;
  }
}

// (1) Block partials: row b = [sum w, sum w E, sum w O (P), sum w dE (P)] over samples
// [256 b, 256 b + 256) (the O and dE sums in the input type per thread, added in a fixed order,
// stored in double); maxima as float bits (non-negative floats order like unsigned):
// mx[0] = max w, mx[1] = max |E|, mx[2 + c] = max |O_c|, mx[2 + P + c] = max |dE_c|.
// Block (g, b) (column group fastest, so that the blocks sharing a sample range run together
// and a 128-byte line that straddles two column groups comes from DRAM once) takes columns
// [64 g, 64 g + 64): thread (r, q) = (tid / 16, tid % 16) columns 64 g + 4 q .. + 3 of samples
// 256 b + r, + 16, ...; the 16 row partials are added in row order.
template <class Tin, bool VEC>
__global__ void __launch_bounds__(kColBlock) lin_colsum_kernel(int P, long long M, const Tin* __restrict__ O,
                                                               const Tin* __restrict__ dEL,
                                                               const double* __restrict__ E,
                                                               const double* __restrict__ w,
                                                               double* __restrict__ part1, unsigned* __restrict__ mx,
                                                               long long nb) {
  __shared__ Tin sw[kColBlock];  // the block's weights in the input type (converted once per sample)
  __shared__ Tin red_o[16][64], red_d[16][64];
  __shared__ float red_mo[16][64], red_md[16][64];
  __shared__ double red_w[8][2];
  const int L1 = 2 * P + 2;
  const int tid = threadIdx.x, r = tid >> 4, q = tid & 15;
  // sample blocks blockIdx.y, + gridDim.y, ... (the grid's y extent is limited)
  for (long long sb = blockIdx.y; sb < nb; sb += gridDim.y) {
    __syncthreads();  // the previous sample block is done with the shared arrays
    double* row = part1 + (size_t)sb * L1;
    const long long s0 = sb * kColBlock;
    {
      const long long s = s0 + tid;
      double ws = 0.0, e = 0.0;
      if (s < M) {
        ws = w ? w[s] : 1.0;
        e = E[s];
      }
      sw[tid] = (Tin)ws;
      if (blockIdx.x == 0) {  // sum w, sum w E in a fixed order, and the maxima of w and |E|
        double a = ws, b = ws * e;
        float mw = (float)ws, me = fabsf((float)e);
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
          me = fmaxf(me, __shfl_xor_sync(0xffffffffu, me, o));
        }
        if ((tid & 31) == 0) {
          red_w[tid >> 5][0] = a;
          red_w[tid >> 5][1] = b;
          atomicMax(mx, __float_as_uint(mw));
          atomicMax(mx + 1, __float_as_uint(me));
        }
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && tid == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < 8; ++k) {
        a += red_w[k][0];
        b += red_w[k][1];
      }
      row[0] = a;
      row[1] = b;
    }
    const int c = blockIdx.x * 64 + 4 * q;
    Tin so[4] = {0, 0, 0, 0}, sd[4] = {0, 0, 0, 0};
    float mo[4] = {0.0f, 0.0f, 0.0f, 0.0f}, md[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    auto take = [&](int sl) {
      Tin o[4], d[4];
      load4<Tin, VEC>(O + (s0 + sl) * P, c, P, o);
      load4<Tin, VEC>(dEL + (s0 + sl) * P, c, P, d);
      const Tin ws = sw[sl];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        so[u] += ws * o[u];
        sd[u] += ws * d[u];
        mo[u] = fmaxf(mo[u], fabsf((float)o[u]));
        md[u] = fmaxf(md[u], fabsf((float)d[u]));
      }
    };
    if (c < P) {
      if (s0 + kColBlock <= M) {  // a full block: no per-sample test, so the loads batch
#pragma unroll 4
        for (int k = 0; k < kColBlock / 16; ++k) take(r + 16 * k);
      } else {
        for (int k = 0; k < kColBlock / 16; ++k)
          if (s0 + r + 16 * k < M) take(r + 16 * k);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      red_o[r][4 * q + u] = so[u];
      red_d[r][4 * q + u] = sd[u];
      red_mo[r][4 * q + u] = mo[u];
      red_md[r][4 * q + u] = md[u];
    }
    __syncthreads();
    if (tid < 64) {
      const int cc = blockIdx.x * 64 + tid;
      if (cc < P) {
        Tin a = red_o[0][tid], b = red_d[0][tid];
        float ma = red_mo[0][tid], mb = red_md[0][tid];
        for (int k = 1; k < 16; ++k) {
          a += red_o[k][tid];
          b += red_d[k][tid];
          ma = fmaxf(ma, red_mo[k][tid]);
          mb = fmaxf(mb, red_md[k][tid]);
        }
        row[2 + cc] = (double)a;
        row[2 + P + cc] = (double)b;
        atomicMax(mx + 2 + cc, __float_as_uint(ma));
        atomicMax(mx + 2 + P + cc, __float_as_uint(mb));
      }
    }
  }
}

// Block partials added in a fixed order, in two levels so that the whole machine takes part:
// (a) grid (columns / 32, kSeg): block (x, g) sums for its 32 columns the partial rows of
//     segment g (rows [g nb / kSeg, (g + 1) nb / kSeg)), warp w the rows w, w + 8, ... of the
//     segment, the 8 warp sums added in warp order: seg[g][q];
// (b) acc[q] = sum over g of seg[g][q] in segment order.
constexpr int kSeg = 64;
__global__ void __launch_bounds__(256) lin_seg_reduce(int L, int nb, const double* __restrict__ part,
                                                      double* __restrict__ seg) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int q = blockIdx.x * 32 + lane, g = blockIdx.y;
  const int b0 = (int)((long long)g * nb / kSeg), b1 = (int)((long long)(g + 1) * nb / kSeg);
  double s = 0.0;
  if (q < L)
#pragma unroll 4
    for (int b = b0 + wp; b < b1; b += 8) s += part[(size_t)b * L + q];
  red[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && q < L) {
    double t = red[0][lane];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += red[k][lane];
    seg[(size_t)g * L + q] = t;
  }
}
__global__ void lin_final_reduce(int L, const double* __restrict__ seg, double* __restrict__ acc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L) return;
  double s = 0.0;
  for (int g = 0; g < kSeg; ++g) s += seg[(size_t)g * L + q];
  acc[q] = s;
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

// x and y split into high and low halves (v = hi + lo, hi = half(v), lo = half(v - hi)), the
// two values converted together (one packed conversion each way)
__device__ __forceinline__ void split_half2(float x, float y, __half& xh, __half& xl, __half& yh, __half& yl) {
  const __half2 h = __floats2half2_rn(x, y);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
  xh = __low2half(h);
  yh = __high2half(h);
  xl = __low2half(l);
  yl = __high2half(l);
}

// (2b) Scaled, split and transposed values in sample groups: group g (samples 32 g .. 32 g + 31)
// of XI and YI is a [Pr][64] block of halves whose row c holds parameter c's 32 high halves
// followed by its 32 low halves (one 128-byte row); zero rows c >= P and zero samples
// M <= s < Mp.  A tile of the tensor-core pass (rows r0 .. r0 + 127 of one group) is then one
// contiguous 16 KB block.  A block of this kernel transposes 64 samples x 64 parameters through
// shared memory: reads along parameters and writes along samples are both coalesced.
template <class Tin, bool VEC>
__global__ void __launch_bounds__(256, 4) lin_center_kernel(int P, long long M, long long Mp, const Tin* __restrict__ O,
                                                         const Tin* __restrict__ dEL, const double* __restrict__ E,
                                                         const double* __restrict__ w, const float* __restrict__ rwf,
                                                         const float* __restrict__ Ef, const double* __restrict__ acc,
                                                         const float* __restrict__ scl, int Pr,
                                                         __half* __restrict__ XI, __half* __restrict__ YI,
                                                         double* __restrict__ part2, long long nb) {
  // [array][parameter][sample]: rows of 72 halves (144 bytes) keep the 16-byte chunks aligned
  __shared__ __align__(16) __half t[4][64][72];
  __shared__ double red[16][64];
  const int c0 = blockIdx.x * 64;
  const double isw = 1.0 / acc[0];
  // thread (r, q) = (tid % 16, tid / 16): parameters c0 + 4 q .. + 3 of samples s0 + r + 16 k
  const int r = threadIdx.x & 15, q = threadIdx.x >> 4;
  const int c = c0 + 4 * q;
  Tin mo[4];
  float sx[4], sy[4];
  // sample blocks blockIdx.y, + gridDim.y, ... (the grid's y extent is limited)
  for (long long sb = blockIdx.y; sb < nb; sb += gridDim.y) {
    double sxe[4] = {0.0, 0.0, 0.0, 0.0};  // sums of w Ot E over this thread's samples (16-sample partials in Tin)
    Tin part[4] = {0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      mo[u] = c + u < P ? (Tin)(acc[2 + c + u] * isw) : (Tin)0;
      sx[u] = scl[c + u];
      sy[u] = scl[Pr + c + u];
    }
    for (int tt = 0; tt < kCenTiles; ++tt) {
      const long long s0 = (sb * kCenTiles + tt) * 64;
      if (s0 >= M) break;
      __syncthreads();  // the previous tile's stores have read t
      // the tile's 8 loads of 4 values first (memory-level parallelism), then the arithmetic
      Tin ov[4][4], dv[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long sm = s0 + r + 16 * k;
        if (sm < M && c < P) {
          load4<Tin, VEC>(O + sm * P, c, P, ov[k]);
          load4<Tin, VEC>(dEL + sm * P, c, P, dv[k]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) ov[k][u] = dv[k][u] = (Tin)0;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int sl = r + 16 * k;
        const long long sm = s0 + sl;
        const bool in = sm < M;
        const Tin e = in ? (std::is_same<Tin, double>::value ? (Tin)E[sm] : (Tin)Ef[sm]) : (Tin)0;
        const float rw = in ? rwf[sm] : 0.0f;
        const Tin ws = in ? (w ? (Tin)w[sm] : (Tin)1) : (Tin)0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float xv = 0.0f, yv = 0.0f;
          if (in && c + u < P) {
            const Tin x = ov[k][u] - mo[u];
            const Tin ex = e * x;
            const Tin y = ex + dv[k][u];
            xv = (float)x * rw * sx[u];
            yv = (float)y * rw * sy[u];
            part[u] += ws * ex;
          }
          split_half2(xv, yv, t[0][4 * q + u][sl], t[1][4 * q + u][sl], t[2][4 * q + u][sl], t[3][4 * q + u][sl]);
        }
      }
      if ((tt & 3) == 3) {  // every 4 tiles (16 samples of this thread) into double
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sxe[u] += (double)part[u];
          part[u] = (Tin)0;
        }
      }
      __syncthreads();
      // 16-byte stores: per array (X, Y), group g of the tile's two and row, the 128-byte row
      // [hi 0-31 | lo 0-31] in 8 chunks of 8 halves; groups that start at or past Mp, and rows
      // past the tensor maps' extent (read as zeros by the copy engine), are not stored
      for (int qq = threadIdx.x; qq < 2 * 64 * 16; qq += 256) {
        const int a = qq >> 10, rr = (qq >> 4) & 63, ch = qq & 15;
        const int g = ch >> 3, half = (ch >> 2) & 1, sub = ch & 3;
        if (s0 + 32 * g >= Mp || c0 + rr >= rows_m(P)) continue;
        const uint4 v = *reinterpret_cast<const uint4*>(&t[2 * a + half][rr][32 * g + 8 * sub]);
        __half* const dst = a == 0 ? XI : YI;
        const size_t grp = (size_t)(s0 / 32 + g);
        *reinterpret_cast<uint4*>(dst + (grp * Pr + c0 + rr) * 64 + 32 * half + 8 * sub) = v;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) red[r][4 * q + u] = sxe[u] + (double)part[u];
    __syncthreads();
    if (threadIdx.x < 64) {  // block partial of sum w Ot E, the 16 sample offsets in order
      double v = red[0][threadIdx.x];
      for (int k = 1; k < 16; ++k) v += red[k][threadIdx.x];
      part2[(size_t)sb * Pr + c0 + threadIdx.x] = v;
    }
    __syncthreads();  // red is read before the next sample block writes it
  }
}

// (3) Partial tiles, one CTA per (128 x 112 output tile, chunk of samples):
//   part[chunk][0][i][j] = sum_{s in chunk} X_si X_sj,   part[chunk][1][i][j] = sum X_si Y_sj
// (scaled values).  Per stage of 32 samples (one group), TMA brings the A tile X_i (128 rows) and
// the B tile [X_j; Y_j] (2 x 112 rows), each row 128 bytes [32 high halves | 32 low halves],
// K-major with the 128-byte swizzle (the layout the MMA reads: the high and low operands of a
// 16-sample slice start 32 bytes apart within the swizzled rows, at +32 kk and +64 + 32 kk).  Warp roles: warp 8 issues the copies into a ring of stages;
// warp 9 owns the tensor memory and issues per 16-sample slice the MMAs A_hi B_lo, A_lo B_hi,
// A_hi B_hi (M = 128, N = 224: columns 0-111 accumulate S, 112-223 H; the correction
// products first, while the accumulator is small); warps 0-7 drain the accumulators.  The
// tensor core's accumulation rounds at the accumulator's magnitude, so an accumulator covers 64
// samples (two stages) and is then moved to registers and summed there in FP32 (round to
// nearest); two tensor-memory sets alternate so that draining overlaps the next MMAs.  The
// roles meet only on shared-memory barriers: stage full (copies landed), stage empty (its MMAs
// done), set full (a pair's MMAs done), set empty (all eight drain warps read it).  Every wait
// is bounded (about a second); a timeout sets a shared abort flag that the other roles check
// before each wait, copies and MMAs in flight still get a bounded wait before the shared and
// tensor memory are released, and the CTA raises *err instead of writing its partials.
constexpr int kTcWarps = 10;                               // 8 drain warps, copy warp, MMA warp
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kCopyWarp = 8, kMmaWarp = 9;
constexpr int kK = 32;                                     // samples per stage
constexpr int kRow = 2 * kK * 2;                           // 128-byte rows: high and low halves
constexpr int kStages = 5;
constexpr int kN = 2 * kTb;                                // MMA N: the j rows of X and of Y
constexpr int kABytes = kTa * kRow;                        // 16 KB
constexpr int kHBytes = kTb * kRow;                        // 14 KB: the X_j (or Y_j) half of B
constexpr int kBBytes = 2 * kHBytes;                       // 28 KB
constexpr int kStageBytes = kABytes + kBBytes;             // A, B
constexpr int kNumBars = 2 * kStages + 5;                  // full, empty, set full x2, set empty x2, done
constexpr int kTcSmem = kStages * kStageBytes + 1024 + 8 * kNumBars + 64;
constexpr int kSetCols = 256;                              // tensor-memory columns per accumulator set
constexpr uint64_t kWaitNs = 1000000000ull;
static_assert(kHBytes % 1024 == 0 && kABytes % 1024 == 0, "128-byte swizzled tiles stay 1024-byte aligned");
static_assert(kN % 16 == 0 && kN <= 256 && kN <= kSetCols, "MMA shape M = 128 needs N a multiple of 16, <= 256");
static_assert(kTcSmem <= 232448, "shared memory of one CTA");

// adds this warp's 112 accumulator columns (lanes 32 (warp % 4) + lane; warps 0-3 the S half
// of the set, warps 4-7 the H half) starting at tensor-memory address 'base'; the loads go out
// two at a time behind one wait
__device__ __forceinline__ void drain(uint32_t base, float acc[kTb]) {
  uint32_t v[2][16];
#pragma unroll
  for (int g = 0; g < kTb / 16; g += 2) {
    tmem_ld16_async(base + 16 * g, v[0]);
    if (g + 1 < kTb / 16) tmem_ld16_async(base + 16 * (g + 1), v[1]);
    tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[16 * g + q] += __uint_as_float(v[0][q]);
    if (g + 1 < kTb / 16)
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[16 * (g + 1) + q] += __uint_as_float(v[1][q]);
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    lin_tc_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tBX,
                  const __grid_constant__ CUtensorMap tBY, int Pa, int Pb, long long M, long long chunk,
                  double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStageBytes);  // [kStages] copies landed
  uint64_t* empty = full + kStages;                                           // [kStages] MMAs of the stage done
  uint64_t* sfull = empty + kStages;                                          // [2] a pair's MMAs done
  uint64_t* sempty = sfull + 2;                                               // [2] drained by 8 warps
  uint64_t* mdone = sempty + 2;                                               // every MMA issued done
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntb = Pb / kTb;
  const int ta = blockIdx.x / ntb, tb = blockIdx.x % ntb;
  const int i0 = ta * kTa, j0 = tb * kTb;
  const long long s0 = (long long)blockIdx.y * chunk, s1 = min(M, s0 + chunk);
  const int nsteps = s1 > s0 ? (int)((s1 - s0 + kK - 1) / kK) : 0;
  const int npairs = (nsteps + 1) / 2;
  // stage layout: A = X_i rows, B = [X_j rows; Y_j rows]
  auto a_tile = [&](int st) { return sm + st * kStageBytes; };
  auto b_tile = [&](int st) { return sm + st * kStageBytes + kABytes; };

  if (threadIdx.x == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 8);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_async_smem();
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_holder, 512);  // set b at columns 256 b: S (+0), H (+112)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  float acc[kTb];

  if (warp == kCopyWarp) {
    if (lane == 0) {
      int loaded = 0;
      for (int ks = 0; ks < nsteps; ++ks) {
        const int st = ks % kStages;
        if (ks >= kStages) {  // the stage's previous MMAs must be done
          if (*abort_flag) break;
          if (!mbar_wait(&empty[st], (uint32_t)((ks / kStages - 1) & 1), kWaitNs)) {
            *abort_flag = 1;
            break;
          }
        }
        const int g = (int)(s0 / kK) + ks;  // sample group
        mbar_arrive_expect_tx(&full[st], kStageBytes);
        tma_load_3d(a_tile(st), &tA, 0, i0, g, &full[st]);
        tma_load_3d(b_tile(st), &tBX, 0, j0, g, &full[st]);
        tma_load_3d(b_tile(st) + kHBytes, &tBY, 0, j0, g, &full[st]);
        loaded = ks + 1;
      }
      // after an abort, the copies that may still be in flight land before the CTA ends
      if (*abort_flag)
        for (int ks = max(0, loaded - kStages); ks < loaded; ++ks)
          mbar_wait(&full[ks % kStages], (uint32_t)((ks / kStages) & 1), kWaitNs);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(kTa, kN);
      int issued = 0;
      for (int ks = 0; ks < nsteps; ++ks) {
        const int st = ks % kStages, p = ks >> 1, set = p & 1;
        if (*abort_flag) break;
        if ((ks & 1) == 0 && p >= 2 &&
            !mbar_wait(&sempty[set], (uint32_t)(((p >> 1) - 1) & 1), kWaitNs)) {  // set drained
          *abort_flag = 1;
          break;
        }
        if (!mbar_wait(&full[st], (uint32_t)((ks / kStages) & 1), kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_addr(a_tile(st)), b = smem_addr(b_tile(st));
        const uint32_t d = tmem + kSetCols * set;
        const bool fresh = (ks & 1) == 0;
        // slice kk (16 samples = 32 bytes): high halves at +32 kk, low halves at +64 + 32 kk
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint32_t hi = 32 * kk, lo = 64 + 32 * kk;
          mma_f16(d, smem_desc_k128(a + hi), smem_desc_k128(b + lo), idesc, (fresh && kk == 0) ? 0u : 1u);
          mma_f16(d, smem_desc_k128(a + lo), smem_desc_k128(b + hi), idesc, 1u);
        }
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint32_t hi = 32 * kk;
          mma_f16(d, smem_desc_k128(a + hi), smem_desc_k128(b + hi), idesc, 1u);
        }
        mma_commit(&empty[st]);
        if ((ks & 1) || ks == nsteps - 1) mma_commit(&sfull[set]);
        issued = ks + 1;
      }
      // every MMA issued has completed before the tensor memory is released
      if (issued > 0) {
        mma_commit(mdone);
        if (!mbar_wait(mdone, 0u, kWaitNs)) *abort_flag = 1;
      }
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int c = 0; c < kTb; ++c) acc[c] = 0.0f;
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (warp < 4 ? 0u : (uint32_t)kTb);
    for (int p = 0; p < npairs; ++p) {
      const int set = p & 1;
      int ok = 0;
      if (lane == 0) ok = !*abort_flag && mbar_wait(&sfull[set], (uint32_t)((p >> 1) & 1), kWaitNs);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *abort_flag = 1;
        break;
      }
      tc_fence_after();
      drain(base + kSetCols * set, acc);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sempty[set]);
    }
  }
  __syncthreads();
  const bool good = *abort_flag == 0;  // every role has finished: the flag is final
  if (warp < 8 && good) {
    const int row = i0 + 32 * (warp & 3) + lane;
    double* out = part + ((size_t)blockIdx.y * 2 + (warp < 4 ? 0 : 1)) * Pa * Pb + (size_t)row * Pb + j0;
#pragma unroll
    for (int c = 0; c < kTb; ++c) out[c] = (double)acc[c];
  }
  if (threadIdx.x == 0 && !good) atomicExch(err, 1);
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, 512);
}

// (4) thread (i, j): S[i][j] and H[i][j] from the chunk partials [chunk][2][Pa][Pb], unscaled;
// gL, gR, E0 from the column sums.
__global__ void lin_reduce_kernel(int P, int Pa, int Pb, int Pr, int nchunk, const double* __restrict__ part,
                                  const double* __restrict__ acc, const double* __restrict__ sxe,
                                  const float* __restrict__ scl, double* E0,
                                  double* gL, double* gR, double* S, double* H, const int* __restrict__ err) {
  // a timed-out tensor-core stage leaves NaN outputs
  const double isw = *err ? __longlong_as_double(0x7ff8000000000000ll) : 1.0 / acc[0];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (long long)P * P) {
    const int i = (int)(q / P), j = (int)(q % P);
    const size_t o = (size_t)i * Pb + j, plane = (size_t)Pa * Pb;
    double s = 0.0, h = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      s += part[(size_t)c * 2 * plane + o];
      h += part[(size_t)c * 2 * plane + plane + o];
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

int lin_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n < 1)
    return 1;
  return n;
}

LinGrid lin_grid(int P, long long M, int nsm) {
  // one CTA per SM (the stages take most of the shared memory) and one wave: as many chunks as
  // the SMs hold for every tile at once (the CTAs of a chunk then run side by side and share
  // its tiles through L2), at least kMinChunk samples per chunk
  constexpr long long kMinChunk = 2048;
  const int ntile = (rows_a(P) / kTa) * (rows_b(P) / kTb);
  const long long maxc = std::max<long long>(1, (M + kMinChunk - 1) / kMinChunk);
  const long long n = std::min(maxc, std::max<long long>(1, (long long)std::max(nsm, 1) / ntile));
  LinGrid g;
  g.chunk = std::max<long long>(kK, ((M + n - 1) / n + kK - 1) / kK * kK);
  g.nchunk = (int)((M + g.chunk - 1) / g.chunk);
  return g;
}

namespace {
struct LinWs {
  double *part1, *acc, *part2, *sxe, *seg, *part;
  unsigned* mx;
  float *scl, *rw, *Ef;
  __half *XI, *YI;
  int* err;
  size_t bytes;
};
LinWs carve(void* ws, int P, long long M, int nchunk) {
  const int L1 = 2 * P + 2, Pa = rows_a(P), Pb = rows_b(P), Pr = rows_t(P);
  const long long nb1 = (M + kColBlock - 1) / kColBlock,
                  nb2 = (M + 64 * kCenTiles - 1) / (64 * kCenTiles);
  const long long Mp = (M + 31) / 32 * 32;
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
  w.seg = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kSeg * std::max(L1, Pr)));
  w.mx = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (2 + 2 * (size_t)P)));
  w.scl = reinterpret_cast<float*>(take(sizeof(float) * 2 * (size_t)Pr));
  w.rw = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  w.Ef = reinterpret_cast<float*>(take(sizeof(float) * (size_t)M));
  w.XI = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * 2 * Mp));
  w.YI = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)Pr * 2 * Mp));
  w.part = reinterpret_cast<double*>(take(sizeof(double) * (size_t)nchunk * 2 * Pa * Pb));
  w.err = reinterpret_cast<int*>(take(sizeof(int)));
  w.bytes = off;
  return w;
}
}  // namespace

size_t lin_workspace_bytes(int P, long long M, int nsm) { return carve(nullptr, P, M, lin_grid(P, M, nsm).nchunk).bytes; }

// Tensor map of a grouped [Mp / 32][Pr][64] half array read in boxes of box_rows rows of one
// group (box_rows x 128 contiguous bytes) with the 128-byte swizzle; rows max(P, 128) and above
// lie outside the map and read as zeros.  The encoder comes from the driver through the runtime,
// so the library does not link the driver library itself.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_tile_map(CUtensorMap* map, const __half* base, int P, int Pr, long long Mp, int box_rows) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * kK), (cuuint64_t)rows_m(P), (cuuint64_t)(Mp / kK)};
  const cuuint64_t strides[2] = {(cuuint64_t)kRow, (cuuint64_t)kRow * Pr};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * kK), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  static_assert(kRow == 128, "the tile rows are 128 bytes (128-byte swizzle)");
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class Tin>
static cudaError_t launch_lin_t(int P, long long M, const Tin* O, const Tin* dEL, const double* E, const double* w,
                                void* ws, size_t ws_bytes, int nsm, double* E0, double* gL, double* gR, double* S,
                                double* H, cudaStream_t st, int* nlaunch, cudaEvent_t* ev) {
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], st);
  };
  const int L1 = 2 * P + 2, Pa = rows_a(P), Pb = rows_b(P), Pr = rows_t(P);
  const long long Mp = (M + 31) / 32 * 32;
  const int nb2 = (int)((M + 64 * kCenTiles - 1) / (64 * kCenTiles));
  const LinGrid G = lin_grid(P, M, nsm);
  const int nb1 = (int)((M + kColBlock - 1) / kColBlock);
  const LinWs L = carve(ws, P, M, G.nchunk);
  if (L.bytes > ws_bytes) return cudaErrorInvalidValue;  // workspace sized for another grid
  cudaError_t e = cudaMemsetAsync(L.mx, 0, sizeof(unsigned) * (2 + 2 * (size_t)P), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  mark(0);
  // 16-byte loads of the [M][P] inputs when every row starts on a 16-byte boundary
  const bool vec = P % 4 == 0 && reinterpret_cast<uintptr_t>(O) % 16 == 0 && reinterpret_cast<uintptr_t>(dEL) % 16 == 0;
  const dim3 gcol((unsigned)((P + 63) / 64), (unsigned)std::min(nb1, 65535));
  if (vec)
    lin_colsum_kernel<Tin, true><<<gcol, kColBlock, 0, st>>>(P, M, O, dEL, E, w, L.part1, L.mx, nb1);
  else
    lin_colsum_kernel<Tin, false><<<gcol, kColBlock, 0, st>>>(P, M, O, dEL, E, w, L.part1, L.mx, nb1);
  lin_seg_reduce<<<dim3((L1 + 31) / 32, kSeg), 256, 0, st>>>(L1, nb1, L.part1, L.seg);
  lin_final_reduce<<<(L1 + 255) / 256, 256, 0, st>>>(L1, L.seg, L.acc);
  lin_scale_kernel<<<(Pr + 255) / 256, 256, 0, st>>>(P, Pr, L.acc, L.mx, L.scl);
  lin_sample_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, E, w, L.rw, L.Ef);
  mark(1);
  if (vec)
    lin_center_kernel<Tin, true><<<dim3(Pr / 64, (unsigned)std::min(nb2, 65535)), 256, 0, st>>>(
        P, M, Mp, O, dEL, E, w, L.rw, L.Ef, L.acc, L.scl, Pr, L.XI, L.YI, L.part2, nb2);
  else
    lin_center_kernel<Tin, false><<<dim3(Pr / 64, (unsigned)std::min(nb2, 65535)), 256, 0, st>>>(
        P, M, Mp, O, dEL, E, w, L.rw, L.Ef, L.acc, L.scl, Pr, L.XI, L.YI, L.part2, nb2);
  lin_seg_reduce<<<dim3((Pr + 31) / 32, kSeg), 256, 0, st>>>(Pr, nb2, L.part2, L.seg);
  lin_final_reduce<<<(Pr + 255) / 256, 256, 0, st>>>(Pr, L.seg, L.sxe);
  mark(2);
  // A tiles: 128 rows of X; B tiles: 112 rows of X and of Y
  CUtensorMap mA, mBX, mBY;
  e = encode_tile_map(&mA, L.XI, P, Pr, Mp, kTa);
  if (e == cudaSuccess) e = encode_tile_map(&mBX, L.XI, P, Pr, Mp, kTb);
  if (e == cudaSuccess) e = encode_tile_map(&mBY, L.YI, P, Pr, Mp, kTb);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lin_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  const int ntile = (Pa / kTa) * (Pb / kTb);
  lin_tc_kernel<<<dim3(ntile, G.nchunk), kTcThreads, kTcSmem, st>>>(mA, mBX, mBY, Pa, Pb, M, G.chunk, L.part,
                                                                     L.err);
  mark(3);
  const long long nq = std::max<long long>((long long)P * P, 1);
  lin_reduce_kernel<<<(int)((nq + 255) / 256), 256, 0, st>>>(P, Pa, Pb, Pr, G.nchunk, L.part, L.acc, L.sxe, L.scl,
                                                              E0, gL, gR, S, H, L.err);
  mark(4);
  *nlaunch = 11;
  return cudaGetLastError();
}

cudaError_t launch_lin(int in_float, int P, long long M, const void* O, const void* dEL, const double* E,
                       const double* w, void* ws, size_t ws_bytes, int nsm, double* E0, double* gL, double* gR,
                       double* S, double* H, cudaStream_t st, int* nlaunch, cudaEvent_t* ev) {
  if (in_float)
    return launch_lin_t<float>(P, M, static_cast<const float*>(O), static_cast<const float*>(dEL), E, w, ws, ws_bytes,
                               nsm, E0, gL, gR, S, H, st, nlaunch, ev);
  return launch_lin_t<double>(P, M, static_cast<const double*>(O), static_cast<const double*>(dEL), E, w, ws,
                              ws_bytes, nsm, E0, gL, gR, S, H, st, nlaunch, ev);
}

}  // namespace vbq
