// Device building blocks of the VB-QMC kernels: counter-based random numbers, warp and
// lane-group reductions, the lane-group Slater LU/inverse, Gaussian basis functions and
// the Jastrow pieces (arXiv:2207.14715, Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "dsfloat.cuh"
#include "vbqmc_internal.h"

namespace vbq {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return (int)(threadIdx.x & 31); }

// (q / d, q % d) along q = q0, q0 + 32, q0 + 64, ... without integer division (which this
// part executes through conversions on its slow double-precision pipe): divide once by
// subtraction (q0 < 32), then step.
struct DivStep {
  int hi, lo;
  __device__ __forceinline__ DivStep(int q0, int d) : hi(0), lo(q0) {
    while (lo >= d) { lo -= d; ++hi; }
  }
  __device__ __forceinline__ void next(int d, int stride = 32) {
    lo += stride;
    while (lo >= d) { lo -= d; ++hi; }
  }
};
// dst[i] = (TD)src[i] for i = lane, lane + 32, ... < n by one warp: eight loads issued before
// the first store (the compiler may not move a global load above a store through another
// pointer, so a plain loop waits one memory latency per element).  src is not declared
// __restrict__: in the one-launch batched step it can hold data written earlier in the same
// launch, which the read-only data path may not return.
template <class TD, class TS>
__device__ __forceinline__ void warp_copy(TD* dst, const TS* src, int n, int lane) {
  for (int i0 = lane; i0 < n; i0 += 256) {
    TS v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i0 + 32 * k < n) v[k] = src[i0 + 32 * k];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i0 + 32 * k < n) dst[i0 + 32 * k] = (TD)v[k];
  }
}
// lane-group coordinates for a power-of-two group size G
struct LaneGroup {
  int ng, g, gl;
  __device__ __forceinline__ LaneGroup(int lane, int G) {
    const int lg = __ffs(G) - 1;
    ng = 32 >> lg;
    g = lane >> lg;
    gl = lane & (G - 1);
  }
};

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from the published round function.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Two uniforms in [0, 1): counter (walker, step, slot, (tag << 8) | purpose), key = seed.
__device__ __forceinline__ void uniforms2(uint64_t seed, uint32_t walker, uint32_t step, uint32_t slot, uint32_t tag,
                                          uint32_t purpose, double& u0, double& u1) {
  uint32_t o[4];
  philox4x32_10(walker, step, slot, (tag << 8) | (purpose & 0xffu), (uint32_t)seed, (uint32_t)(seed >> 32), o);
  const uint64_t x0 = ((uint64_t)o[1] << 32) | o[0];
  const uint64_t x1 = ((uint64_t)o[3] << 32) | o[2];
  u0 = (double)(x0 >> 11) * 0x1.0p-53;
  u1 = (double)(x1 >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------------------------------------
// reductions
// ------------------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
template <class T> __device__ __forceinline__ T group_sum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o, G);
  return v;
}

// 1/x in double, four FP64 instructions instead of a division: x = m 2^k with |m| in [1, 2)
// (read from the bit pattern); the float reciprocal of m truncated to 24 bits (a float
// built from the bits, no conversion instruction: conversions to and from double run at the
// double rate) refined by two Newton steps (each doubles the correct bits: 2^-22 -> 2^-44 ->
// below double rounding), then 2^-k added to the exponent field.  Zero, subnormal, huge and
// non-finite x take the division.
__device__ __forceinline__ double recip_dd(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e <= 1 || e >= 2045) return 1.0 / x;
  const double m = __longlong_as_double((b & (long long)0x800fffffffffffffull) | 0x3ff0000000000000ll);
  const unsigned sgn = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  const float mf = __uint_as_float(sgn | 0x3f800000u | (unsigned)((b >> 29) & 0x7fffff));
  const unsigned yb = __float_as_uint(__frcp_rn(mf));  // |1/mf| in (0.5, 1]: a normal float
  // the same value as a double: exponent rebased from 127 to 1023, mantissa moved up 29 bits
  double y = __longlong_as_double(
      (long long)((((unsigned long long)(yb & 0x7fffffffu) << 29) + (896ull << 52)) | ((unsigned long long)sgn << 32)));
  y = y * fma(-m, y, 2.0);
  y = y * fma(-m, y, 2.0);
  // |y| in [0.5, 1]: the result's exponent field stays in 1..2044 over the fast branch's range
  return __longlong_as_double(__double_as_longlong(y) + (long long)(1023 - e) * (1LL << 52));
}

// float -> double by moving the bits (exact, as the conversion): a conversion to or from
// double runs at the double rate, integer operations at the full rate.  Zero, subnormal and
// non-finite values take the conversion (a branch no lane takes costs nothing).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f), ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)f;
  return __longlong_as_double((long long)((((unsigned long long)(u & 0x7fffffffu) << 29) + (896ull << 52)) |
                                          ((unsigned long long)(u & 0x80000000u) << 32)));
}

// a < b for a >= 0 and b >= 0 or NaN (false for NaN), on the bit patterns: for non-negative
// doubles their order is the order of the patterns as integers
__device__ __forceinline__ bool less_nonneg(double a, double b) {
  const long long ib = __double_as_longlong(b);
  return __double_as_longlong(a) < ib && ib <= 0x7ff0000000000000ll;
}

// ------------------------------------------------------------------------------------
// Lane-group LU with partial pivoting and explicit inverse.
// A (n x n, row-major, rows = electrons, columns = orbital slots) is overwritten with its
// LU factors; Binv receives A^{-1} row-major ([slot][electron]).  A group of G lanes
// (G = power of two >= n) handles one matrix; every lane of the warp must call this with
// the same n and G (inactive groups pass active = false).  Pivot ties go to the lowest row.
// Returns ln|det A| and sign(det A) in every lane of the group; a zero pivot gives
// sign 0, ln|det| = -inf and a zero inverse.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void group_lu_inverse(double* A, double* Binv, int* perm, int n, int glane, int G,
                                                 bool active, double& logdet, double& sgn) {
  double s = 1.0;
  bool singular = false;
  if (active && glane < n) perm[glane] = glane;
  __syncwarp();
  for (int c = 0; c < n; ++c) {
    double v = (active && glane >= c && glane < n) ? fabs(A[glane * n + c]) : -1.0;
    int idx = glane;
    for (int o = G >> 1; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(kFull, v, o, G);
      const int oi = __shfl_xor_sync(kFull, idx, o, G);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (v <= 0.0) singular = true;
    if (idx != c) {
      if (active && !singular)
        for (int j = glane; j < n; j += G) {
          const double t = A[c * n + j];
          A[c * n + j] = A[idx * n + j];
          A[idx * n + j] = t;
        }
      if (active && glane == 0) {
        const int t = perm[c];
        perm[c] = perm[idx];
        perm[idx] = t;
      }
      s = -s;
    }
    __syncwarp();
    // pivot reciprocal: computed by the pivot lane and broadcast (one reciprocal per column)
    double ip = 0.0;
    if (active && !singular && glane == c) ip = recip_dd(A[c * n + c]);
    ip = __shfl_sync(kFull, ip, (lane_id() & ~(G - 1)) + c);
    if (active && !singular && glane > c && glane < n) {
      const double l = A[glane * n + c] * ip;
      A[glane * n + c] = l;
      for (int j = c + 1; j < n; ++j) A[glane * n + j] = fma(-l, A[c * n + j], A[glane * n + j]);
    }
    __syncwarp();
  }
  // reciprocal of the U diagonal: lane i of the group holds 1/U_ii; the back substitution
  // multiplies by it (broadcast by shuffle) instead of dividing in every lane
  const double dinv = (active && glane < n && !singular) ? recip_dd(A[glane * n + glane]) : 0.0;
  if (active && glane < n) {
    const int j = glane;
    if (!singular) {
      for (int i = 0; i < n; ++i) {
        double y = (perm[i] == j) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) y = fma(-A[i * n + k], Binv[k * n + j], y);
        Binv[i * n + j] = y;
      }
    } else {
      for (int i = 0; i < n; ++i) Binv[i * n + j] = 0.0;
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    const double di = __shfl_sync(kFull, dinv, (lane_id() & ~(G - 1)) + i);
    if (active && glane < n && !singular) {
      const int j = glane;
      double x = Binv[i * n + j];
      for (int k = i + 1; k < n; ++k) x = fma(-A[i * n + k], Binv[k * n + j], x);
      Binv[i * n + j] = x * di;
    }
  }

  // ln|det| = ln prod |U_ii|: the product of the mantissas (each in [1, 2)) and the sum of the
  // binary exponents over the group, then one logarithm (no overflow for n <= 32)
  double mant = 1.0;
  int ex = 0, neg = 0;
  if (active && glane < n && !singular) {
    const double d = A[glane * n + glane];
    const long long bits = __double_as_longlong(fabs(d));
    ex = (int)((bits >> 52) & 0x7ff) - 1023;
    mant = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
    neg = d < 0.0 ? 1 : 0;
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    mant *= __shfl_xor_sync(kFull, mant, o, G);
    ex += __shfl_xor_sync(kFull, ex, o, G);
    neg += __shfl_xor_sync(kFull, neg, o, G);
  }
  if (singular) {
    logdet = -INFINITY;
    sgn = 0.0;
  } else {
    logdet = log(mant) + (double)ex * 0.6931471805599453;
    sgn = (neg & 1) ? -s : s;
  }
  __syncwarp();
}

// ------------------------------------------------------------------------------------
// math helpers overloaded on the bulk type
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double vexp(double x) { return exp(x); }
__device__ __forceinline__ float vexp(float x) { return expf(x); }
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float vsqrt(float x) { return sqrtf(x); }

template <class T> __device__ __forceinline__ T tload(const double* p) { return (T)__ldg(p); }

// ------------------------------------------------------------------------------------
// Cartesian shell at displacement d = r - center: for every component, with P the cartesian
// monomial (s; x y z; xx yy zz xy xz yz) of degree l,
//   Gaussian (z >= 0):   chi = N P e^{-z r^2},  grad chi = N e (grad P - 2 z d P),
//                        lap chi = N e (lap P + P (4 z^2 r^2 - 6 z - 4 z l));
//   Slater (z = -zeta < 0): chi = N P e^{-zeta r},  grad chi = N e (grad P - (zeta / r) d P),
//                        lap chi = N e (lap P + P (zeta^2 - 2 zeta (l + 1) / r))
// (grad P . d = l P).  Both have the form N e (grad P - t d P) and N e (lap P + P base), so only
// e, t and base depend on the kind.  Writes value (and if out_d is non-null gradient and
// Laplacian) for component c at out[c * stride].
// ------------------------------------------------------------------------------------
template <class T, bool DERIV, class NT, class Emit>
__device__ __forceinline__ void gto_shell_emit(int l, T z, const NT* nrm, T dx, T dy, T dz, Emit&& emit) {
  const T r2 = dx * dx + dy * dy + dz * dz;
  T e, tz, base;
  if (z < (T)0) {
    const T zeta = -z, r = vsqrt(r2);
    const T ir = r > (T)0 ? (T)1 / r : (T)0;
    e = vexp(-zeta * r);
    tz = zeta * ir;
    base = zeta * zeta - (T)2 * zeta * (T)(l + 1) * ir;
  } else {
    e = (z == (T)0) ? (T)1 : vexp(-z * r2);
    tz = (T)2 * z;
    base = (T)4 * z * z * r2 - (T)6 * z - (T)4 * z * (T)l;
  }
  if (l == 0) {
    const T ne = (T)nrm[0] * e;
    if (DERIV) emit(0, ne, -tz * dx * ne, -tz * dy * ne, -tz * dz * ne, base * ne);
    else emit(0, ne, (T)0, (T)0, (T)0, (T)0);
  } else if (l == 1) {
    const T d[3] = {dx, dy, dz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T ne = (T)nrm[c] * e;
      const T P = d[c];
      if (DERIV)
        emit(c, ne * P, ne * ((c == 0 ? (T)1 : (T)0) - tz * dx * P), ne * ((c == 1 ? (T)1 : (T)0) - tz * dy * P),
             ne * ((c == 2 ? (T)1 : (T)0) - tz * dz * P), ne * P * base);
      else
        emit(c, ne * P, (T)0, (T)0, (T)0, (T)0);
    }
  } else {
    // xx yy zz xy xz yz
    const int ia[6] = {0, 1, 2, 0, 0, 1};
    const int ib[6] = {0, 1, 2, 1, 2, 2};
    const T d[3] = {dx, dy, dz};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T ne = (T)nrm[c] * e;
      const T P = d[ia[c]] * d[ib[c]];
      if (DERIV) {
        T g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          T dP = (T)0;
          if (ia[c] == q) dP += d[ib[c]];
          if (ib[c] == q) dP += d[ia[c]];
          g[q] = ne * (dP - tz * d[q] * P);
        }
        const T lapP = (c < 3) ? (T)2 : (T)0;
        emit(c, ne * P, g[0], g[1], g[2], ne * (lapP + P * base));
      } else {
        emit(c, ne * P, (T)0, (T)0, (T)0, (T)0);
      }
    }
  }
}

template <class T, bool DERIV, class NT>
__device__ __forceinline__ void gto_shell(int l, T z, const NT* nrm, T dx, T dy, T dz, T* val, T* gx, T* gy, T* gz,
                                          T* lap, int cs = 1) {
  gto_shell_emit<T, DERIV>(l, z, nrm, dx, dy, dz, [&](int c, T v, T x, T y, T w, T lp) {
    val[c * cs] = v;
    if (DERIV) {
      gx[c * cs] = x;
      gy[c * cs] = y;
      gz[c * cs] = w;
      lap[c] = lp;
    }
  });
}

// ------------------------------------------------------------------------------------
// Jastrow radial pieces.  R(r) = r/(1 + kappa r); f(R) = a1 R/(1 + a2 R) + sum_{p=2..5} q_p R^p
// with q_p = coef[p-2].  Returns f and, with DERIV, df/dr and d2f/dr2.
// ------------------------------------------------------------------------------------
template <class T, bool DERIV>
__device__ __forceinline__ void pade_poly(T r, T kap, T a1, T a2, const T* q, T& f, T& df, T& d2f) {
  const T den = (T)1 / ((T)1 + kap * r);
  const T R = r * den;
  const T pd = (T)1 / ((T)1 + a2 * R);
  const T R2 = R * R, R3 = R2 * R, R4 = R3 * R, R5 = R4 * R;
  f = a1 * R * pd + q[0] * R2 + q[1] * R3 + q[2] * R4 + q[3] * R5;
  if (DERIV) {
    const T dR = den * den;
    const T d2R = (T)-2 * kap * dR * den;
    const T fR = a1 * pd * pd + (T)2 * q[0] * R + (T)3 * q[1] * R2 + (T)4 * q[2] * R3 + (T)5 * q[3] * R4;
    const T fRR = (T)-2 * a1 * a2 * pd * pd * pd + (T)2 * q[0] + (T)6 * q[1] * R + (T)12 * q[2] * R2 +
                  (T)20 * q[3] * R3;
    df = fR * dR;
    d2f = fRR * dR * dR + fR * d2R;
  }
}

// e-e-n terms in the order of the sum of Sec. 2.1: p = 2..5, k = 0..p-1, l = 0..lmax with
// lmax = p-k (k != 0) or p-k-2 (k = 0), kept when p-k-l is even (m = (p-k-l)/2).
struct EenKLM { int k, l, m; };
__host__ __device__ constexpr EenKLM een_klm(int t) {
  int q = 0;
  for (int p = 2; p <= 5; ++p)
    for (int k = 0; k < p; ++k)
      for (int l = 0; l <= (k ? p - k : p - k - 2); ++l)
        if ((p - k - l) % 2 == 0) {
          if (q == t) return EenKLM{k, l, (p - k - l) / 2};
          ++q;
        }
  return EenKLM{-1, -1, -1};
}
static_assert(een_klm(kNeen - 1).k == 4 && een_klm(kNeen).k == -1, "23 e-e-n terms");

template <class F, int... T>
__device__ __forceinline__ void een_for_each_impl(F& f, std::integer_sequence<int, T...>) {
  (f(std::integral_constant<int, T>{}), ...);
}
// Calls f(std::integral_constant<int, t>) for t = 0..22; inside, een_klm(t) is a constant
// expression, so register arrays indexed by the term's powers stay in registers.
template <class F> __device__ __forceinline__ void een_for_each(F&& f) {
  een_for_each_impl(f, std::make_integer_sequence<int, kNeen>{});
}

template <class T> struct Pow6 {
  T v[6];
  __device__ __forceinline__ void set(T x) {
    v[0] = (T)1; v[1] = x; v[2] = x * x; v[3] = v[2] * x; v[4] = v[3] * x; v[5] = v[4] * x;
  }
  __device__ __forceinline__ T p(int n) const { return v[n]; }
  __device__ __forceinline__ T d(int n) const { return n >= 1 ? (T)n * v[n - 1] : (T)0; }
  __device__ __forceinline__ T dd(int n) const { return n >= 2 ? (T)(n * (n - 1)) * v[n - 2] : (T)0; }
};

// Term t of the e-e-n expansion, T = u^k (s^l + t^l)(s t)^m = u^k (s^(l+m) t^m + s^m t^(l+m)).
template <class T>
__device__ __forceinline__ T een_term(const Pow6<T>& U, const Pow6<T>& S, const Pow6<T>& Tt, int k, int l, int m) {
  return U.p(k) * (S.p(l + m) * Tt.p(m) + S.p(m) * Tt.p(l + m));
}

// Value of F = sum_t c_t T_t(u, s, t).
template <class T> __device__ __forceinline__ T een_value(const T* c, T u, T s, T t) {
  Pow6<T> U, S, Tt;
  U.set(u); S.set(s); Tt.set(t);
  T F = (T)0;
  een_for_each([&](auto tc) {
    constexpr int q = decltype(tc)::value;
    constexpr EenKLM x = een_klm(q);
    F += c[q] * een_term(U, S, Tt, x.k, x.l, x.m);
  });
  return F;
}

// F and its partial derivatives with respect to u and s (the electron-i side).
template <class T>
__device__ __forceinline__ void een_partials_us(const T* c, T u, T s, T t, T& F, T& Fu, T& Fs, T& Fuu, T& Fss,
                                                T& Fus) {
  Pow6<T> U, S, Tt;
  U.set(u); S.set(s); Tt.set(t);
  F = Fu = Fs = Fuu = Fss = Fus = (T)0;
  een_for_each([&](auto tc) {
    constexpr int q = decltype(tc)::value;
    constexpr int k = een_klm(q).k, l = een_klm(q).l, m = een_klm(q).m;
    const T f = S.p(l + m) * Tt.p(m) + S.p(m) * Tt.p(l + m);
    const T fs = S.d(l + m) * Tt.p(m) + S.d(m) * Tt.p(l + m);
    const T fss = S.dd(l + m) * Tt.p(m) + S.dd(m) * Tt.p(l + m);
    const T cq = c[q];
    F += cq * U.p(k) * f;
    Fu += cq * U.d(k) * f;
    Fuu += cq * U.dd(k) * f;
    Fs += cq * U.p(k) * fs;
    Fss += cq * U.p(k) * fss;
    Fus += cq * U.d(k) * fs;
  });
}

}  // namespace vbq

namespace vbq {

// ------------------------------------------------------------------------------------
// e-e-n Jastrow through pair sums.  For one nucleus with s_i = Rbar(r_ia) and u_ij = Rbar(r_ij),
// every term c u^k (s_i^l + s_j^l)(s_i s_j)^m summed over pairs i < j equals
//   c sum_{i != j} u_ij^k s_i^A s_j^B  with A = l + m, B = m,
// so f_een = sum_t c_t sum_i S_i^A Y_i^{k,B} with Y_i^{k,q} = sum_{j != i} u_ij^k s_j^q.
// Gradient and Laplacian with respect to r_i follow from the product rule with
//   Z_i^{k,q} = sum_{j != i} grad_i(u_ij^k) s_j^q,  Q_i^{k,q} = sum_{j != i} lap_i(u_ij^k) s_j^q:
//   grad_i = S^A Z^{k,B} + S^B Z^{k,A} + D^A Y^{k,B} + D^B Y^{k,A}
//   lap_i  = S^A Q^{k,B} + S^B Q^{k,A} + 2 D^A.Z^{k,B} + 2 D^B.Z^{k,A} + L^A Y^{k,B} + L^B Y^{k,A}
// with D^q = grad_i s_i^q and L^q = lap_i s_i^q.  For k = 0, Y^{0,q}_i = sum_j s_j^q - s_i^q and
// Z = Q = 0.  Accumulators exist for k in [K0, K1] and q <= 5 - k (the powers the terms use).
// ------------------------------------------------------------------------------------
template <int K0, int K1> struct EenK {
  __host__ __device__ static constexpr int count() {
    int c = 0;
    for (int k = K0; k <= K1; ++k) c += 6 - k;
    return c;
  }
  __host__ __device__ static constexpr int idx(int k, int q) {
    int c = 0;
    for (int kk = K0; kk < k; ++kk) c += 6 - kk;
    return c + q;
  }
};

template <class T, int K0, int K1> struct EenAcc {
  static constexpr int C = EenK<K0, K1>::count();
  T Y[C], Zx[C], Zy[C], Zz[C], Q[C];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < C; ++c) Y[c] = Zx[c] = Zy[c] = Zz[c] = Q[c] = (T)0;
  }
  // adds partner j: u = Rbar(r_ij), ir = 1/r_ij, (ex, ey, ez) = (r_i - r_j)/r_ij, S = s_j^0..5
  __device__ __forceinline__ void add(T u, T ir, T kap, T ex, T ey, T ez, const T* S) {
    const T du = -kap * u * u, d2u = (T)2 * kap * kap * u * u * u;
    T up[5];
    up[0] = (T)1; up[1] = u; up[2] = u * u; up[3] = up[2] * u; up[4] = up[3] * u;
#pragma unroll
    for (int k = K0; k <= K1; ++k) {
      const T Uk = up[k];
      const T dUk = (T)k * up[k - 1] * du;
      const T d2Uk = (k >= 2 ? (T)(k * (k - 1)) * up[k >= 2 ? k - 2 : 0] * du * du : (T)0) + (T)k * up[k - 1] * d2u;
      const T Hk = d2Uk + (T)2 * dUk * ir;
#pragma unroll
      for (int q = 0; q <= 5 - k; ++q) {
        const int c = EenK<K0, K1>::idx(k, q);
        const T sq = S[q];
        Y[c] += Uk * sq;
        const T g = dUk * sq;
        Zx[c] += g * ex; Zy[c] += g * ey; Zz[c] += g * ez;
        Q[c] += Hk * sq;
      }
    }
  }
};

// Per electron-nucleus data: S^q, dS^q/dr and the radial Laplacian of s^q for q = 0..5.
template <class T> struct EenSide {
  T S[6], dS[6], L[6];
  __device__ __forceinline__ void set(T s, T r, T kap) {
    const T ds = -kap * s * s, d2s = (T)2 * kap * kap * s * s * s, ir = (T)1 / r;
    S[0] = (T)1; dS[0] = (T)0; L[0] = (T)0;
#pragma unroll
    for (int q = 1; q <= 5; ++q) {
      S[q] = S[q - 1] * s;
      dS[q] = (T)q * S[q - 1] * ds;
      const T d2 = (q >= 2 ? (T)(q * (q - 1)) * S[q >= 2 ? q - 2 : 0] * ds * ds : (T)0) + (T)q * S[q - 1] * d2s;
      L[q] = d2 + (T)2 * dS[q] * ir;
    }
  }
};

// Calls f(t, val, gx, gy, gz, lap) for every term t with k in [K0, K1] (k = 0 terms when
// K0 == 1): val = s_i^A Y^{k,B}, (gx, gy, gz) = grad_i and lap = lap_i of the term's part
// that involves electron i, as written above.  (ex, ey, ez) = (r_i - r_a)/r_ia; Ssum[q] = sum_j s_j^q (SsumLo[q]: its low float part in the float form, 0 otherwise).
template <class T, int K0, int K1, class F>
__device__ __forceinline__ void een_terms(const EenAcc<T, K0, K1>& acc, const EenSide<T>& si, T ex, T ey, T ez,
                                          const T* Ssum, const T* SsumLo, F&& f) {
  een_for_each([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    constexpr int k = een_klm(t).k, A = een_klm(t).l + een_klm(t).m, B = een_klm(t).m;
    constexpr bool mine = (k >= K0 && k <= K1) || (k == 0 && K0 == 1);
    if (!mine) return;
    T Ya, Yb, Zax = 0, Zay = 0, Zaz = 0, Zbx = 0, Zby = 0, Zbz = 0, Qa = 0, Qb = 0;
    if (k == 0) {
      if constexpr (sizeof(T) == 4) {  // float: the float-float sum minus own term, rounded once
        Ya = ds_diff_f(dsf{Ssum[A], SsumLo[A]}, dsf{si.S[A], 0.0f});
        Yb = ds_diff_f(dsf{Ssum[B], SsumLo[B]}, dsf{si.S[B], 0.0f});
      } else {
        Ya = Ssum[A] - si.S[A];
        Yb = Ssum[B] - si.S[B];
      }
    } else {
      constexpr int ca = EenK<K0, K1>::idx(k >= K0 ? k : K0, A <= 5 - k ? A : 0);
      constexpr int cb = EenK<K0, K1>::idx(k >= K0 ? k : K0, B <= 5 - k ? B : 0);
      Ya = acc.Y[ca]; Yb = acc.Y[cb];
      Zax = acc.Zx[ca]; Zay = acc.Zy[ca]; Zaz = acc.Zz[ca];
      Zbx = acc.Zx[cb]; Zby = acc.Zy[cb]; Zbz = acc.Zz[cb];
      Qa = acc.Q[ca]; Qb = acc.Q[cb];
    }
    const T SA = si.S[A], SB = si.S[B], dA = si.dS[A], dB = si.dS[B];
    const T val = SA * Yb;
    const T gx = SA * Zbx + SB * Zax + (dA * Yb + dB * Ya) * ex;
    const T gy = SA * Zby + SB * Zay + (dA * Yb + dB * Ya) * ey;
    const T gz = SA * Zbz + SB * Zaz + (dA * Yb + dB * Ya) * ez;
    const T lap = SA * Qb + SB * Qa + (T)2 * (dA * (ex * Zbx + ey * Zby + ez * Zbz) + dB * (ex * Zax + ey * Zay + ez * Zaz)) +
                  si.L[A] * Yb + si.L[B] * Ya;
    f(t, val, gx, gy, gz, lap);
  });
}

}  // namespace vbq
