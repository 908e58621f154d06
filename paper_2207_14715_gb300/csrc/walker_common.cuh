// Device helpers shared by the walker kernels (evaluation kernels and the sweep kernel):
// basis functions in the bulk type and in float-float, Jastrow radial coefficients, the
// Slater LU of every unique determinant and the structure sum in the log domain
// (arXiv:2207.14715, Sec. 2.1).
#pragma once

#include <algorithm>
#include <cfloat>

#include "dsfloat.cuh"
#include "kernels.h"
#include "wf_device.cuh"

namespace vbq {

namespace {


__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }
// Threads per block the evaluation kernel is compiled for: the double instantiation keeps
// more live values and runs few walkers per block, so it gets the larger register budget.
template <class Tb> struct EvalBounds { static constexpr int threads = 512; };
template <> struct EvalBounds<double> { static constexpr int threads = 256; };
template <class A, class B> constexpr bool kSameType = false;
template <class A> constexpr bool kSameType<A, A> = true;
inline int group_size(int n) {
  int g = 1;
  while (g < n) g <<= 1;
  return g;
}

template <class Tb> __device__ __forceinline__ const Tb* orb_coefs(const SysDev& s);
template <> __device__ __forceinline__ const double* orb_coefs<double>(const SysDev& s) { return s.orb_coef; }
template <> __device__ __forceinline__ const float* orb_coefs<float>(const SysDev& s) { return s.orb_coef_f; }
template <class Tb> __device__ __forceinline__ const Tb* een_basis_t(const SysDev& s);
template <> __device__ __forceinline__ const double* een_basis_t<double>(const SysDev& s) { return s.een_B; }
template <> __device__ __forceinline__ const float* een_basis_t<float>(const SysDev& s) { return s.een_Bf; }
template <class Tb> __device__ __forceinline__ const Tb* een_coefs(const SysDev& s);
template <> __device__ __forceinline__ const double* een_coefs<double>(const SysDev& s) { return s.een_c; }
template <> __device__ __forceinline__ const float* een_coefs<float>(const SysDev& s) { return s.een_cf; }

// Basis functions (values, or values + gradient + Laplacian) of all shells at point r.
// Lanes take shells round-robin.  Output arrays are indexed by basis function.
template <class Tb, bool DERIV>
__device__ __forceinline__ void basis_at(const SysDev& s, int lane, double x, double y, double z, Tb* bv, Tb* bx,
                                         Tb* by, Tb* bz, Tb* bl) {
  for (int t = lane; t < s.S; t += 32) {
    const int sh = __ldg(s.sh_by_l + t);
    const double* nu = s.nuc4 + 4 * __ldg(s.sh_center + sh);
    const int f = __ldg(s.sh_first + sh);
    gto_shell<Tb, DERIV>(__ldg(s.sh_l + sh), (Tb)__ldg(s.sh_zeta + sh), s.sh_norm + 6 * sh, (Tb)(x - __ldg(nu)),
                         (Tb)(y - __ldg(nu + 1)), (Tb)(z - __ldg(nu + 2)), bv + f, DERIV ? bx + f : nullptr,
                         DERIV ? by + f : nullptr, DERIV ? bz + f : nullptr, DERIV ? bl + f : nullptr);
  }
}

// The same in the mixed form from a point given in float-float (r3[0..2]): the displacement
// from each center is rounded to float from its float-float value, and shell exponents and
// normalisations are float, so no double-precision instruction is issued per shell.
__device__ __forceinline__ dsf nuc_coord_ds(const SysDev& s, int a, int d) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(s.nuc_ds) + 3 * a + d);
  return dsf{v.x, v.y};
}
// PACK4 (with DERIV): value and gradient of function mu as the float4 bv[4 mu .. 4 mu + 3],
// Laplacian at bl[mu] (bx, by, bz and cs unused).
template <bool DERIV, bool PACK4 = false>
__device__ __forceinline__ void basis_at_f(const SysDev& s, int lane, const dsf* r3, float* bv, float* bx, float* by,
                                           float* bz, float* bl, int cs = 1) {
  // the displacement from each nucleus once (lane a: nucleus a), shared by shuffles with the
  // lanes of that nucleus's shells (more than 32 nuclei: each shell forms its own)
  const bool shuf = s.Nn <= 32;
  float cx = 0.0f, cy = 0.0f, cz = 0.0f;
  if (shuf && lane < s.Nn) {
    cx = ds_diff_f(r3[0], nuc_coord_ds(s, lane, 0));
    cy = ds_diff_f(r3[1], nuc_coord_ds(s, lane, 1));
    cz = ds_diff_f(r3[2], nuc_coord_ds(s, lane, 2));
  }
  for (int t0 = 0; t0 < s.S; t0 += 32) {  // every lane takes part in each round (the shuffles)
    const int t = t0 + lane;
    const bool act = t < s.S;
    // one 16-byte record per shell, in the order of l
    const int4 p = act ? __ldg(reinterpret_cast<const int4*>(s.sh_pack_f) + t) : make_int4(0, 0, 0, 0);
    const int c = p.x & 0xffff, l = p.x >> 16, f = p.y, sh = p.z;
    float dx, dy, dz;
    if (shuf) {
      dx = __shfl_sync(kFull, cx, c);
      dy = __shfl_sync(kFull, cy, c);
      dz = __shfl_sync(kFull, cz, c);
    } else {
      dx = ds_diff_f(r3[0], nuc_coord_ds(s, c, 0));
      dy = ds_diff_f(r3[1], nuc_coord_ds(s, c, 1));
      dz = ds_diff_f(r3[2], nuc_coord_ds(s, c, 2));
    }
    if (act) {
      if constexpr (PACK4)  // value and gradient of function f + c as one 16-byte store
        gto_shell_emit<float, true>(l, __int_as_float(p.w), s.sh_norm_f + 6 * sh, dx, dy, dz,
                                    [&](int c, float v, float x, float y, float w, float lp) {
                                      reinterpret_cast<float4*>(bv)[f + c] = make_float4(v, x, y, w);
                                      bl[f + c] = lp;
                                    });
      else
        gto_shell<float, DERIV>(l, __int_as_float(p.w), s.sh_norm_f + 6 * sh, dx, dy, dz,
                                bv + f * cs, DERIV ? bx + f * cs : nullptr, DERIV ? by + f * cs : nullptr,
                                DERIV ? bz + f * cs : nullptr, DERIV ? bl + f : nullptr, cs);
    }
  }
}

// Values of all basis functions at the point r3 (float-float) in float-float (mixed form).
// Per center the displacement and r^2 are float-float; per shell exp(-zeta r^2) and the
// cartesian factors are float-float.  ctab: [Nn][4] scratch (dx, dy, dz, r^2).
__device__ __forceinline__ void basis_values_ds(const SysDev& s, int lane, const dsf* r3, dsf* ctab, dsf* out) {
  for (int c = lane; c < s.Nn; c += 32) {
    const dsf dx = ds_add(r3[0], ds_neg(nuc_coord_ds(s, c, 0)));
    const dsf dy = ds_add(r3[1], ds_neg(nuc_coord_ds(s, c, 1)));
    const dsf dz = ds_add(r3[2], ds_neg(nuc_coord_ds(s, c, 2)));
    ctab[4 * c] = dx;
    ctab[4 * c + 1] = dy;
    ctab[4 * c + 2] = dz;
    ctab[4 * c + 3] = ds_add_nc(ds_add_nc(ds_mul(dx, dx), ds_mul(dy, dy)), ds_mul(dz, dz));
  }
  __syncwarp();
  for (int t = lane; t < s.S; t += 32) {
    const int sh = __ldg(s.sh_by_l + t);
    const int c = __ldg(s.sh_center + sh), l = __ldg(s.sh_l + sh), f = __ldg(s.sh_first + sh);
    const float2 zt = __ldg(reinterpret_cast<const float2*>(s.sh_zeta_ds) + sh);
    dsf e = {1.0f, 0.0f};
    if (zt.x < 0.0f)  // Slater shell: exp(-zeta r), zeta = -z
      e = ds_exp_neg(ds_mul(ds_sqrt(ctab[4 * c + 3]), dsf{-zt.x, -zt.y}));
    else if (zt.x != 0.0f)
      e = ds_exp_neg(ds_mul(ctab[4 * c + 3], dsf{zt.x, zt.y}));
    const float2* nr = reinterpret_cast<const float2*>(s.sh_norm_ds) + 6 * sh;
    if (l == 0) {
      const float2 n0 = __ldg(nr);
      out[f] = ds_mul(dsf{n0.x, n0.y}, e);
    } else if (l == 1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float2 nq = __ldg(nr + q);
        out[f + q] = ds_mul(ds_mul(dsf{nq.x, nq.y}, ctab[4 * c + q]), e);
      }
    } else {
      const int ia[6] = {0, 1, 2, 0, 0, 1};
      const int ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float2 nq = __ldg(nr + q);
        out[f + q] = ds_mul(ds_mul(dsf{nq.x, nq.y}, ds_mul(ctab[4 * c + ia[q]], ctab[4 * c + ib[q]])), e);
      }
    }
  }
}

// e-n Jastrow/e-e Jastrow coefficient blocks as Tb
struct PadeCoef {
  double a1, a2, q[4];
};
// the same in the bulk type, loaded from the bulk-type tables (no conversion per use)
template <class Tb> struct PadeT {
  Tb a1, a2, q[4];
};
template <class Tb> __device__ __forceinline__ PadeT<Tb> en_coef_t(const SysDev& s, int a);
template <class Tb> __device__ __forceinline__ PadeT<Tb> ee_coef_t(const SysDev& s, bool same);
template <class Tb> __device__ __forceinline__ PadeT<Tb> load_pade(const Tb* p, Tb a1) {
  PadeT<Tb> c;
  c.a1 = a1; c.a2 = __ldg(p + 1);
  for (int q = 0; q < 4; ++q) c.q[q] = __ldg(p + 2 + q);
  return c;
}
template <> __device__ __forceinline__ PadeT<double> en_coef_t<double>(const SysDev& s, int a) {
  const double* p = s.jas_a + 6 * __ldg(s.nuc_elem + a);
  return load_pade<double>(p, __ldg(p));
}
template <> __device__ __forceinline__ PadeT<float> en_coef_t<float>(const SysDev& s, int a) {
  const float* p = s.jas_af + 6 * __ldg(s.nuc_elem + a);
  return load_pade<float>(p, __ldg(p));
}
template <> __device__ __forceinline__ PadeT<double> ee_coef_t<double>(const SysDev& s, bool same) {
  return load_pade<double>(s.jas_b, same ? s.b1_par : s.b1_anti);
}
template <> __device__ __forceinline__ PadeT<float> ee_coef_t<float>(const SysDev& s, bool same) {
  return load_pade<float>(s.jas_bf, same ? s.b1_par_f : s.b1_anti_f);
}
// Value of the Pade + polynomial form f(r) = a1 R/(1 + a2 R) + sum_p q_p R^p, R = r/(1 + kappa r),
// in float-float: the e-n and e-e terms of ln J, whose sum over all pairs sets ln|Psi| (the
// mixed form's derivatives keep the float form).  p: [a1 a2 q0 q1 q2 q3] as (hi, lo) pairs
// (a1 replaced by a1r when a1r is given).
__device__ __forceinline__ dsf pade_value_ds(dsf r, const float* p, const float* a1r, const float* kap) {
  const dsf k = {kap[0], kap[1]};
  const dsf R = ds_div(r, ds_add_f(ds_mul(k, r), 1.0f));
  const dsf a1 = a1r ? dsf{a1r[0], a1r[1]} : dsf{__ldg(p), __ldg(p + 1)};
  const dsf a2 = {__ldg(p + 2), __ldg(p + 3)};
  dsf poly = {__ldg(p + 10), __ldg(p + 11)};
  poly = ds_add(ds_mul(poly, R), dsf{__ldg(p + 8), __ldg(p + 9)});
  poly = ds_add(ds_mul(poly, R), dsf{__ldg(p + 6), __ldg(p + 7)});
  poly = ds_add(ds_mul(poly, R), dsf{__ldg(p + 4), __ldg(p + 5)});
  const dsf R2 = ds_mul(R, R);
  return ds_add(ds_div(ds_mul(a1, R), ds_add_f(ds_mul(a2, R), 1.0f)), ds_mul(poly, R2));
}
// |a - b| for float-float 3-vectors
__device__ __forceinline__ dsf ds_dist(const dsf* a, const dsf* b) {
  const dsf dx = ds_sub(a[0], b[0]), dy = ds_sub(a[1], b[1]), dz = ds_sub(a[2], b[2]);
  return ds_sqrt(ds_add(ds_add(ds_mul(dx, dx), ds_mul(dy, dy)), ds_mul(dz, dz)));
}

// 1/x in double (the determinant-ratio updates); see recip_dd.
__device__ __forceinline__ double recip(double x) { return recip_dd(x); }

__device__ __forceinline__ PadeCoef en_coef(const SysDev& s, int a) {
  const double* p = s.jas_a + 6 * __ldg(s.nuc_elem + a);
  PadeCoef c;
  c.a1 = __ldg(p); c.a2 = __ldg(p + 1);
  for (int q = 0; q < 4; ++q) c.q[q] = __ldg(p + 2 + q);
  return c;
}
__device__ __forceinline__ PadeCoef ee_coef(const SysDev& s, bool same) {
  PadeCoef c;
  c.a1 = same ? s.b1_par : s.b1_anti;
  c.a2 = __ldg(s.jas_b + 1);
  for (int q = 0; q < 4; ++q) c.q[q] = __ldg(s.jas_b + 2 + q);
  return c;
}
template <class Tb, bool DERIV>
__device__ __forceinline__ void pade_eval(const PadeT<Tb>& c, Tb r, Tb kap, Tb& f, Tb& df, Tb& d2f) {
  pade_poly<Tb, DERIV>(r, kap, c.a1, c.a2, c.q, f, df, d2f);
}
template <class Tb, bool DERIV>
__device__ __forceinline__ void pade_eval(const PadeCoef& c, Tb r, Tb kap, Tb& f, Tb& df, Tb& d2f) {
  const Tb q[4] = {(Tb)c.q[0], (Tb)c.q[1], (Tb)c.q[2], (Tb)c.q[3]};
  pade_poly<Tb, DERIV>(r, kap, (Tb)c.a1, (Tb)c.a2, q, f, df, d2f);
}

// Lane-group LU + inverse of every unique determinant of spin sp, from orbital values
// Phi[(e0 + e) * ld + idx[u][o]].  Writes Binv[u], ldet[u], dsg[u] (and, if Lphi is given,
// t[u] = tr(Binv L_occ) with L read at Lphi[(e0 + e) * ldL + idx[u][o]]).
template <class TP, class TL>
__device__ __forceinline__ void lu_all(const SysDev& s, int sp, int lane, const TP* Phi, int ld, const TL* Lphi,
                                       int ldL, const int* idx, int G, double* Binv, double* scr, double* ldet,
                                       double* dsg, double* tdet) {
  const int n = s.n[sp], U = s.U[sp], e0 = sp ? s.Nup : 0;
  if (n == 0) {
    for (int u = lane; u < U; u += 32) {
      ldet[u] = 0.0;
      dsg[u] = 1.0;
      if (tdet) tdet[u] = 0.0;
    }
    __syncwarp();
    return;
  }
  const LaneGroup lgp(lane, G);
  const int ng = lgp.ng, g = lgp.g, gl = lgp.gl;
  double* A = scr + g * n * n;
  int* perm = reinterpret_cast<int*>(scr + ng * n * n) + g * n;
  for (int u0 = 0; u0 < U; u0 += ng) {
    const int u = u0 + g;
    const bool act = u < U;
    if (act && gl < n) {  // lane gl fills column (orbital slot) gl
      const int col = __ldg(idx + u * n + gl);
      for (int e = 0; e < n; ++e) A[e * n + gl] = (double)Phi[(e0 + e) * ld + col];
    }
    __syncwarp();
    double lg, sg;
    double* B = Binv + (act ? u : 0) * n * n;
    group_lu_inverse(A, B, perm, n, gl, G, act, lg, sg);
    double t = 0.0;
    if (tdet && act && gl < n) {
      const int o = gl, col = __ldg(idx + u * n + o);
      for (int e = 0; e < n; ++e) t = fma(B[o * n + e], (double)Lphi[(e0 + e) * ldL + col], t);
    }
    t = group_sum(t, G);
    if (act && gl == 0) {
      ldet[u] = lg;
      dsg[u] = sg;
      if (tdet) tdet[u] = t;
    }
    __syncwarp();
  }
}

// r_k = D_k/Phi for every determinant term and ln|Phi|, sign(Phi) (structure sum in the log
// domain relative to the largest term, Sec. 2.1).
__device__ __forceinline__ void term_ratios(const SysDev& s, int lane, const double* ldet, const double* dsg,
                                            double* rk, double& lnPhi, double& sgnPhi) {
  const int U0 = s.U[0];
  double mx = -INFINITY;
  for (int k = lane; k < s.nterm; k += 32) {
    const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
    if (dsg[a] * dsg[U0 + b] != 0.0) mx = fmax(mx, ldet[a] + ldet[U0 + b]);
  }
  mx = warp_max(mx);
  double ph = 0.0;
  for (int k = lane; k < s.nterm; k += 32) {
    const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
    const double sg = dsg[a] * dsg[U0 + b];
    const double r = (sg != 0.0 && mx > -INFINITY) ? sg * exp(ldet[a] + ldet[U0 + b] - mx) : 0.0;
    rk[k] = r;
    ph = fma(__ldg(s.term_coef + k), r, ph);
  }
  ph = warp_sum(ph);
  __syncwarp();
  const double inv = (ph != 0.0) ? 1.0 / ph : 0.0;
  for (int k = lane; k < s.nterm; k += 32) rk[k] *= inv;
  __syncwarp();
  lnPhi = (ph != 0.0) ? mx + log(fabs(ph)) : -INFINITY;
  sgnPhi = ph > 0.0 ? 1.0 : (ph < 0.0 ? -1.0 : 0.0);
}


// Per-walker geometry tables for the Jastrow factor (coordinate differences in double, the
// rest in the bulk type).  Layout of geo (bulk type):
//   rEE [N][N] r_ij, uEE [N][N] Rbar(r_ij), iEE [N][N] 1/r_ij, eEE [N][N][3] (r_i - r_j)/r_ij,
//   rEN [N][Nn] r_ia, eEN [N][Nn][3] (r_i - r_a)/r_ia, Stab [Nn][N][6] Rbar(r_ia)^q,
//   Ssum [Nn][6] sum_i Rbar(r_ia)^q.
// Returns this lane's share of the Coulomb potential V_ee + V_en.
// The electron-pair tables have rows of an odd length ld (N or N + 1), so that lanes on
// consecutive electrons i reading entry (i, j) fall in different shared-memory banks; entry
// (i, j) is at ee(i, j) (eEE: 3 ee(i, j) + component).
template <class Tb> struct GeoTables {
  Tb *rEE, *uEE, *iEE, *eEE, *rEN, *eEN, *Stab, *Ssum, *SsumLo;
  int ld;
  __device__ __forceinline__ GeoTables(Tb* geo, int N, int Nn) {
    ld = N | 1;
    rEE = geo;
    uEE = rEE + N * ld;
    iEE = uEE + N * ld;
    eEE = iEE + N * ld;
    rEN = eEE + 3 * N * ld;
    eEN = rEN + N * Nn;
    Stab = eEN + 3 * N * Nn;
    Ssum = Stab + 6 * N * Nn;
    SsumLo = Ssum + 6 * Nn;
  }
  __device__ __forceinline__ int ee(int i, int j) const { return i * ld + j; }
};
template <class Tb> __host__ __device__ constexpr int geo_elems(int N, int Nn) {
  return 6 * N * (N | 1) + 4 * N * Nn + 6 * N * Nn + 12 * Nn;
}

// Electron coordinates of one walker as the kernels read them: double in the FP64 form;
// float-float in the mixed form, so that differences come out rounded to float without a
// double-precision instruction per pair.
template <class Tb> struct Coords {
  const double* R;  // [N][3]
  __device__ __forceinline__ Tb ee(int i, int j, int d) const { return (Tb)(R[3 * i + d] - R[3 * j + d]); }
  __device__ __forceinline__ Tb en(const SysDev& s, int i, int a, int d) const {
    return (Tb)(R[3 * i + d] - __ldg(s.nuc4 + 4 * a + d));
  }
  __device__ __forceinline__ Tb charge(const SysDev& s, int a) const { return (Tb)__ldg(s.nuc4 + 4 * a + 3); }
};
template <> struct Coords<float> {
  const dsf* R;  // [N][3]
  __device__ __forceinline__ float ee(int i, int j, int d) const { return ds_diff_f(R[3 * i + d], R[3 * j + d]); }
  __device__ __forceinline__ float en(const SysDev& s, int i, int a, int d) const {
    return ds_diff_f(R[3 * i + d], nuc_coord_ds(s, a, d));
  }
  __device__ __forceinline__ float charge(const SysDev& s, int a) const { return __ldg(s.nuc_zf + a); }
};
// Loads a walker's coordinates from global memory (double [N][3]) into the form of Coords<Tb>
// at dst (shared memory, 3N doubles or 3N float pairs).
// (t, stride): this thread's index and the number of threads that share the walker (one warp,
// or the whole block when WIDE).
template <class Tb, bool WIDE = false>
__device__ __forceinline__ Coords<Tb> load_coords(const double* Rg, int N, int t, void* dst, int stride = 32) {
  Coords<Tb> c;
  if constexpr (kSameType<Tb, double>) {
    double* R = static_cast<double*>(dst);
    for (int i = t; i < 3 * N; i += stride) R[i] = Rg[i];
    c.R = R;
  } else {
    dsf* R = static_cast<dsf*>(dst);
    for (int i = t; i < 3 * N; i += stride) R[i] = ds_from_double(Rg[i]);
    c.R = R;
  }
  if constexpr (WIDE) __syncthreads(); else __syncwarp();
  return c;
}

// Rbar(r) = 1/(1 + kappa r).  The float form takes kappa as a float-float pair and rounds only
// the result: kappa = 0.8 is not a float, and its rounding would shift every e-e-n term of
// ln J the same way (a systematic error that grows with the number of terms).
__device__ __forceinline__ double rbar(const SysDev& s, double r) { return 1.0 / (1.0 + s.kappa * r); }
__device__ __forceinline__ float rbar(const SysDev& s, float r) {
  const dsf d = ds_add_f(ds_mul(dsf{s.kappa_ds[0], s.kappa_ds[1]}, dsf{r, 0.0f}), 1.0f);
  const float q = 1.0f / d.hi;
  return fmaf(-q * q, d.lo, q);
}

template <class Tb, bool WIDE = false>
__device__ __forceinline__ double build_geometry(const SysDev& s, int lane, const Coords<Tb>& C, const GeoTables<Tb>& g,
                                                 int stride = 32) {
  const int N = s.N, Nn = s.Nn;
  Tb V_loc = 0;
  for (DivStep ij(lane, N); ij.hi < N; ij.next(N, stride)) {
    const int i = ij.hi, j = ij.lo, p = g.ee(i, j);
    if (i == j) {
      g.rEE[p] = (Tb)0; g.uEE[p] = (Tb)1; g.iEE[p] = (Tb)0;
      g.eEE[3 * p] = g.eEE[3 * p + 1] = g.eEE[3 * p + 2] = (Tb)0;
      continue;
    }
    const Tb dx = C.ee(i, j, 0), dy = C.ee(i, j, 1), dz = C.ee(i, j, 2);
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz), ir = (Tb)1 / r;
    g.rEE[p] = r; g.uEE[p] = rbar(s, r); g.iEE[p] = ir;
    g.eEE[3 * p] = dx * ir; g.eEE[3 * p + 1] = dy * ir; g.eEE[3 * p + 2] = dz * ir;
    if (i < j) V_loc += ir;
  }
  for (DivStep ia(lane, Nn); ia.hi < N; ia.next(Nn, stride)) {
    const int i = ia.hi, a = ia.lo, p = i * Nn + a;
    const Tb dx = C.en(s, i, a, 0), dy = C.en(s, i, a, 1), dz = C.en(s, i, a, 2);
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz), ir = (Tb)1 / r;
    g.rEN[p] = r;
    g.eEN[3 * p] = dx * ir; g.eEN[3 * p + 1] = dy * ir; g.eEN[3 * p + 2] = dz * ir;
    V_loc -= C.charge(s, a) * ir;
    const Tb sv = rbar(s, r);
    Tb* St = g.Stab + (a * N + i) * 6;
    Tb pw = (Tb)1;
#pragma unroll
    for (int q = 0; q < 6; ++q) { St[q] = pw; pw *= sv; }
  }
  if constexpr (WIDE) __syncthreads(); else __syncwarp();
  for (int p = lane; p < Nn * 6; p += stride) {
    const int a = p / 6, q = p - 6 * a;
    // sum over all electrons of s^q, shared by every electron's k = 0 e-e-n terms (which take
    // their own s^q off it): float-float in the float form, so that its rounding does not repeat
    // coherently through every electron
    if constexpr (kSameType<Tb, double>) {
      Tb t = 0;
      for (int i = 0; i < N; ++i) t += g.Stab[(a * N + i) * 6 + q];
      g.Ssum[p] = t;
      g.SsumLo[p] = 0;
    } else {
      dsf t = {0.0f, 0.0f};
      for (int i = 0; i < N; ++i) t = ds_add_f(t, g.Stab[(a * N + i) * 6 + q]);
      g.Ssum[p] = t.hi;
      g.SsumLo[p] = t.lo;
    }
  }
  if constexpr (WIDE) __syncthreads(); else __syncwarp();
  return (double)V_loc;
}

}  // namespace

}  // namespace vbq
