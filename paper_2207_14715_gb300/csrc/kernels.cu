// VB-QMC walker kernels for sm_103a: one warp per walker, per-walker state in shared memory.
//
//   eval_kernel   : ln|Psi|, sign, E_L, grad ln|Psi| and the parameter derivatives
//                   O_j = Psi_j/Psi and E_L,j = dE_L/dp_j            (arXiv:2207.14715, Sec. 2.1-2.3.1)
//   sweep_kernel  : VMC sweeps of single-electron Metropolis moves   (Sec. 2.3.1)
//
// Precision: template parameter Tb is the bulk type (basis functions, orbitals, Jastrow and
// the excitation derivatives); the Slater LU, inverses, determinant ratios, structure sums
// and energy accumulation are always double.
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
template <class Tb> __device__ __forceinline__ const Tb* een_coefs(const SysDev& s);
template <> __device__ __forceinline__ const double* een_coefs<double>(const SysDev& s) { return s.een_c; }
template <> __device__ __forceinline__ const float* een_coefs<float>(const SysDev& s) { return s.een_cf; }

// Basis functions (values, or values + gradient + Laplacian) of all shells at point r.
// Lanes take shells round-robin.  Output arrays are indexed by basis function.
template <class Tb, bool DERIV>
__device__ __forceinline__ void basis_at(const SysDev& s, int lane, double x, double y, double z, Tb* bv, Tb* bx,
                                         Tb* by, Tb* bz, Tb* bl) {
  for (int sh = lane; sh < s.S; sh += 32) {
    const double* nu = s.nuc4 + 4 * __ldg(s.sh_center + sh);
    const int f = __ldg(s.sh_first + sh);
    gto_shell<Tb, DERIV>(__ldg(s.sh_l + sh), (Tb)__ldg(s.sh_zeta + sh), s.sh_norm + 6 * sh, (Tb)(x - __ldg(nu)),
                         (Tb)(y - __ldg(nu + 1)), (Tb)(z - __ldg(nu + 2)), bv + f, DERIV ? bx + f : nullptr,
                         DERIV ? by + f : nullptr, DERIV ? bz + f : nullptr, DERIV ? bl + f : nullptr);
  }
}

// Values of all basis functions at point r in float-float (mixed form).  Per center the
// displacement and r^2 are formed in double and split once; per shell exp(-zeta r^2) and the
// cartesian factors are float-float.  ctab: [Nn][4] scratch (dx, dy, dz, r^2).
__device__ __forceinline__ void basis_values_ds(const SysDev& s, int lane, double x, double y, double z, dsf* ctab,
                                                dsf* out) {
  for (int c = lane; c < s.Nn; c += 32) {
    const double* nu = s.nuc4 + 4 * c;
    const double dx = x - __ldg(nu), dy = y - __ldg(nu + 1), dz = z - __ldg(nu + 2);
    ctab[4 * c] = ds_from_double(dx);
    ctab[4 * c + 1] = ds_from_double(dy);
    ctab[4 * c + 2] = ds_from_double(dz);
    ctab[4 * c + 3] = ds_from_double(fma(dx, dx, fma(dy, dy, dz * dz)));
  }
  __syncwarp();
  for (int sh = lane; sh < s.S; sh += 32) {
    const int c = __ldg(s.sh_center + sh), l = __ldg(s.sh_l + sh), f = __ldg(s.sh_first + sh);
    const float2 zt = __ldg(reinterpret_cast<const float2*>(s.sh_zeta_ds) + sh);
    dsf e = {1.0f, 0.0f};
    if (zt.x != 0.0f) e = ds_exp_neg(ds_mul(ctab[4 * c + 3], dsf{zt.x, zt.y}));
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
// 1/x to about 47 bits: float reciprocal refined by one Newton step in double (one division's
// worth of FP64 work is ~20 instructions on this part; this is 3).
__device__ __forceinline__ double recip(double x) {
  double y = (double)__frcp_rn((float)x);
  return y * fma(-x, y, 2.0);
}

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
  const int ng = 32 / G, g = lane / G, gl = lane % G;
  double* A = scr + g * n * n;
  int* perm = reinterpret_cast<int*>(scr + ng * n * n) + g * n;
  for (int u0 = 0; u0 < U; u0 += ng) {
    const int u = u0 + g;
    const bool act = u < U;
    if (act)
      for (int q = gl; q < n * n; q += G) {
        const int e = q / n, o = q % n;
        A[q] = (double)Phi[(e0 + e) * ld + __ldg(idx + u * n + o)];
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

}  // namespace

// =====================================================================================
// =====================================================================================
// Evaluation kernel
// =====================================================================================
// Phases (one warp per walker):
//   A  Jastrow ln J with grad_i ln J and lap_i ln J (lanes: electron x partner subset), potential
//   B  orbitals at every electron: basis functions, then the contraction in balanced chunks
//   C  Slater LU + inverses of every unique determinant, structure sum in the log domain,
//      E_L and grad ln|Psi|; optionally the walker state (inverses, ln|det|, signs) is stored
//   D  parameter derivatives (structure coefficients, Jastrow, orbital excitations)
template <class Tb>
__global__ void __launch_bounds__(EvalBounds<Tb>::threads, 1) eval_kernel(const SysDev s, const EvalLayout L, int W,
                                                   const double* __restrict__ Rg, double* __restrict__ logpsi,
                                                   double* __restrict__ sgn_out, double* __restrict__ eloc,
                                                   double* __restrict__ grad, Tb* __restrict__ Og,
                                                   Tb* __restrict__ dELg, double* __restrict__ state_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  unsigned char* base = smem + wl * L.warp_bytes;
  double* R = reinterpret_cast<double*>(base + L.R);
  double* vg = reinterpret_cast<double*>(base + L.vg);
  Tb* G = reinterpret_cast<Tb*>(base + L.G);
  Tb* LJ = reinterpret_cast<Tb*>(base + L.LJ);
  Tb* Phi = reinterpret_cast<Tb*>(base + L.Phi);
  double* PhiD = reinterpret_cast<double*>(base + L.PhiD);
  Tb* Lphi = reinterpret_cast<Tb*>(base + L.Lphi);
  Tb* Gphi = reinterpret_cast<Tb*>(base + L.Gphi);
  double* Binv[2] = {reinterpret_cast<double*>(base + L.Binv0), reinterpret_cast<double*>(base + L.Binv1)};
  double* ldet = reinterpret_cast<double*>(base + L.ldet);
  double* dsg = reinterpret_cast<double*>(base + L.dsg);
  double* tdet = reinterpret_cast<double*>(base + L.tdet);
  double* Wdet = reinterpret_cast<double*>(base + L.Wdet);
  double* Tdet = reinterpret_cast<double*>(base + L.Tdet);
  double* rk = reinterpret_cast<double*>(base + L.rk);
  unsigned char* scr = base + L.scratch;
  Tb* part = reinterpret_cast<Tb*>(base + L.part);
  double* partd = reinterpret_cast<double*>(base + L.partd);
  double* kacc = reinterpret_cast<double*>(base + L.kacc);
  double* red = reinterpret_cast<double*>(base + L.red);
  Tb* rEE = reinterpret_cast<Tb*>(base + L.geo);       // [N][N] r_ij
  Tb* uEE = rEE + s.N * s.N;                            // [N][N] Rbar(r_ij)
  Tb* iEE = uEE + s.N * s.N;                            // [N][N] 1/r_ij
  Tb* eEE = iEE + s.N * s.N;                            // [N][N][3] (r_i - r_j)/r_ij
  Tb* rEN = eEE + 3 * s.N * s.N;                        // [N][Nn] r_ia
  Tb* eEN = rEN + s.N * s.Nn;                           // [N][Nn][3] (r_i - r_a)/r_ia
  Tb* Stab = eEN + 3 * s.N * s.Nn;                      // [Nn][N][6] Rbar(r_ia)^q
  Tb* Ssum = Stab + 6 * s.N * s.Nn;                     // [Nn][6] sum_i Rbar(r_ia)^q

  const int N = s.N, Nn = s.Nn, Nup = s.Nup, U0 = s.U[0];
  const Tb kap = (Tb)s.kappa;
  for (int i = lane; i < 3 * N; i += 32) R[i] = Rg[(size_t)w * 3 * N + i];
  __syncwarp();

  // ---- A0. geometry tables: coordinate differences in double, the rest in the bulk type ----
  double lnJ_loc = 0.0, V_loc = 0.0;
  const Tb* cE = een_coefs<Tb>(s);
  for (int p = lane; p < N * N; p += 32) {
    const int i = p / N, j = p % N;
    if (i == j) {
      rEE[p] = (Tb)0; uEE[p] = (Tb)1; iEE[p] = (Tb)0;
      eEE[3 * p] = eEE[3 * p + 1] = eEE[3 * p + 2] = (Tb)0;
      continue;
    }
    const Tb dx = (Tb)(R[3 * i] - R[3 * j]), dy = (Tb)(R[3 * i + 1] - R[3 * j + 1]), dz = (Tb)(R[3 * i + 2] - R[3 * j + 2]);
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz), ir = (Tb)1 / r;
    rEE[p] = r; uEE[p] = (Tb)1 / ((Tb)1 + kap * r); iEE[p] = ir;
    eEE[3 * p] = dx * ir; eEE[3 * p + 1] = dy * ir; eEE[3 * p + 2] = dz * ir;
    if (i < j) V_loc += (double)ir;
  }
  for (int p = lane; p < N * Nn; p += 32) {
    const int i = p / Nn, a = p % Nn;
    const double* nu = s.nuc4 + 4 * a;
    const Tb dx = (Tb)(R[3 * i] - __ldg(nu)), dy = (Tb)(R[3 * i + 1] - __ldg(nu + 1)), dz = (Tb)(R[3 * i + 2] - __ldg(nu + 2));
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz), ir = (Tb)1 / r;
    rEN[p] = r;
    eEN[3 * p] = dx * ir; eEN[3 * p + 1] = dy * ir; eEN[3 * p + 2] = dz * ir;
    V_loc -= __ldg(nu + 3) * (double)ir;
    const Tb sv = (Tb)1 / ((Tb)1 + kap * r);
    Tb* St = Stab + (a * N + i) * 6;
    Tb pw = (Tb)1;
#pragma unroll
    for (int q = 0; q < 6; ++q) { St[q] = pw; pw *= sv; }
  }
  __syncwarp();
  for (int p = lane; p < Nn * 6; p += 32) {
    const int a = p / 6, q = p % 6;
    Tb t = 0;
    for (int i = 0; i < N; ++i) t += Stab[(a * N + i) * 6 + q];
    Ssum[p] = t;
  }
  __syncwarp();

  // ---- A1. Jastrow ln J, grad_i ln J, lap_i ln J: lane -> (electron i, group g); group g takes
  //      nuclei a = g, g + S, ... and partners j = g, g + S, ... ----
  {
    const int Pp = L.jas_P, Sg = L.jas_S;
    for (int b0 = 0; b0 < N; b0 += Pp) {
      const int i = b0 + lane % Pp, g = lane / Pp;
      const bool act = i < N;
      Tb g0 = 0, g1 = 0, g2 = 0, lap = 0;
      double lnj = 0.0;
      if (act) {
        for (int a = g; a < Nn; a += Sg) {
          const int ia = i * Nn + a;
          const Tb r = rEN[ia];
          Tb f, df, d2f;
          pade_eval<Tb, true>(en_coef(s, a), r, kap, f, df, d2f);
          lnj += (double)f;
          g0 += df * eEN[3 * ia]; g1 += df * eEN[3 * ia + 1]; g2 += df * eEN[3 * ia + 2];
          lap += d2f + (Tb)2 * df / r;
        }
        for (int j = g; j < N; j += Sg) {
          if (j == i) continue;
          const int ij = i * N + j;
          Tb f, df, d2f;
          pade_eval<Tb, true>(ee_coef(s, (i < Nup) == (j < Nup)), rEE[ij], kap, f, df, d2f);
          lnj += 0.5 * (double)f;
          g0 += df * eEE[3 * ij]; g1 += df * eEE[3 * ij + 1]; g2 += df * eEE[3 * ij + 2];
          lap += d2f + (Tb)2 * df * iEE[ij];
        }
        if (s.een_on)
          for (int a = g; a < Nn; a += Sg) {
            const int ia = i * Nn + a;
            const Tb* c = cE + kNeen * __ldg(s.nuc_elem + a);
            EenSide<Tb> si;
            si.set(Stab[(a * N + i) * 6 + 1], rEN[ia], kap);
            const Tb ex = eEN[3 * ia], ey = eEN[3 * ia + 1], ez = eEN[3 * ia + 2];
            auto sink = [&](int t, Tb val, Tb gx, Tb gy, Tb gz, Tb lp) {
              const Tb ct = c[t];
              lnj += (double)(ct * val);
              g0 += ct * gx; g1 += ct * gy; g2 += ct * gz;
              lap += ct * lp;
            };
            {
              EenAcc<Tb, 1, 2> acc;
              acc.zero();
              for (int j = 0; j < N; ++j)
                if (j != i) {
                  const int ij = i * N + j;
                  acc.add(uEE[ij], iEE[ij], kap, eEE[3 * ij], eEE[3 * ij + 1], eEE[3 * ij + 2], Stab + (a * N + j) * 6);
                }
              een_terms(acc, si, ex, ey, ez, Ssum + 6 * a, sink);
            }
            {
              EenAcc<Tb, 3, 4> acc;
              acc.zero();
              for (int j = 0; j < N; ++j)
                if (j != i) {
                  const int ij = i * N + j;
                  acc.add(uEE[ij], iEE[ij], kap, eEE[3 * ij], eEE[3 * ij + 1], eEE[3 * ij + 2], Stab + (a * N + j) * 6);
                }
              een_terms(acc, si, ex, ey, ez, Ssum + 6 * a, sink);
            }
          }
        lnJ_loc += lnj;
      }
      for (int o = Pp; o < 32; o <<= 1) {
        g0 += __shfl_xor_sync(kFull, g0, o);
        g1 += __shfl_xor_sync(kFull, g1, o);
        g2 += __shfl_xor_sync(kFull, g2, o);
        lap += __shfl_xor_sync(kFull, lap, o);
      }
      if (act && g == 0) {
        G[3 * i] = g0; G[3 * i + 1] = g1; G[3 * i + 2] = g2;
        LJ[i] = lap;
      }
    }
  }
  const double lnJ = warp_sum(lnJ_loc);
  const double V = warp_sum(V_loc) + s.vnn;
  __syncwarp();

  // ---- B. orbitals: values (double for determinant orbitals), gradients, dressed Laplacian ----
  const int nev = s.n_ev, nevd = s.n_ev_det, M = s.M;
  {
    Tb* bv = reinterpret_cast<Tb*>(scr);
    Tb* bx = bv + M;
    Tb* by = bx + M;
    Tb* bz = by + M;
    Tb* bl = bz + M;
    // mixed form: float-float values of the basis functions for the determinant orbitals
    dsf* bds = reinterpret_cast<dsf*>(scr + align16(5 * M * (int)sizeof(Tb)));
    dsf* ctab = bds + M;
    dsf* partds = reinterpret_cast<dsf*>(partd);
    const Tb* cf = orb_coefs<Tb>(s);
    for (int e = 0; e < N; ++e) {
      basis_at<Tb, true>(s, lane, R[3 * e], R[3 * e + 1], R[3 * e + 2], bv, bx, by, bz, bl);
      if (!kSameType<Tb, double>) basis_values_ds(s, lane, R[3 * e], R[3 * e + 1], R[3 * e + 2], ctab, bds);
      __syncwarp();
      for (int c = lane; c < s.n_ev_chunk; c += 32) {
        const int4 ch = __ldg(reinterpret_cast<const int4*>(s.ev_chunk) + c);
        const Tb* cb = cf + ch.w;
        Tb v = 0, x = 0, y = 0, z = 0, lp = 0;
        for (int mu = ch.y; mu < ch.z; ++mu) {
          const Tb cm = __ldg(cb + mu);
          v += cm * bv[mu]; x += cm * bx[mu]; y += cm * by[mu]; z += cm * bz[mu]; lp += cm * bl[mu];
        }
        Tb* pp = part + 5 * c;
        pp[0] = v; pp[1] = x; pp[2] = y; pp[3] = z; pp[4] = lp;
      }
      if (!kSameType<Tb, double>)
        for (int c = lane; c < s.n_det_chunk; c += 32) {
          const int4 ch = __ldg(reinterpret_cast<const int4*>(s.det_chunk) + c);
          const float2* cb = reinterpret_cast<const float2*>(s.orb_coef_ds) + ch.w;
          dsf acc = {0.0f, 0.0f};
          for (int mu = ch.y; mu < ch.z; ++mu) {
            const float2 lm = __ldg(cb + mu);
            acc = ds_add(acc, ds_mul(dsf{lm.x, lm.y}, bds[mu]));
          }
          partds[c] = acc;
        }
      __syncwarp();
      const Tb G0 = G[3 * e], G1 = G[3 * e + 1], G2 = G[3 * e + 2];
      for (int q = lane; q < nev; q += 32) {
        const int c0 = __ldg(s.ev_chunk_off + q), c1 = __ldg(s.ev_chunk_off + q + 1);
        Tb v = 0, x = 0, y = 0, z = 0, lp = 0;
        for (int c = c0; c < c1; ++c) {
          const Tb* pp = part + 5 * c;
          v += pp[0]; x += pp[1]; y += pp[2]; z += pp[3]; lp += pp[4];
        }
        Lphi[e * nev + q] = lp + (Tb)2 * (G0 * x + G1 * y + G2 * z);
        if (q < nevd) {
          double vd = 0.0;
          if (kSameType<Tb, double>) {
            vd = (double)v;
          } else {
            const int d0 = __ldg(s.det_chunk_off + q), d1 = __ldg(s.det_chunk_off + q + 1);
            dsf acc = {0.0f, 0.0f};
            for (int c = d0; c < d1; ++c) acc = ds_add(acc, partds[c]);
            vd = ds_to_double(acc);
          }
          PhiD[e * nevd + q] = vd;
          v = (Tb)vd;
          Gphi[(e * nevd + q) * 3] = x;
          Gphi[(e * nevd + q) * 3 + 1] = y;
          Gphi[(e * nevd + q) * 3 + 2] = z;
        }
        Phi[e * nev + q] = v;
      }
      __syncwarp();
    }
  }

  // ---- C. Slater matrices: LU, inverses, ln|det|, t_u = tr(A^-1 L) ----
  lu_all(s, 0, lane, PhiD, nevd, Lphi, nev, s.det_ev[0], L.G0, Binv[0], reinterpret_cast<double*>(scr), ldet, dsg,
         tdet);
  lu_all(s, 1, lane, PhiD, nevd, Lphi, nev, s.det_ev[1], L.G1, Binv[1], reinterpret_cast<double*>(scr), ldet + U0,
         dsg + U0, tdet + U0);
  const int Utot = U0 + s.U[1];
  if (state_out) {
    // walker state: [Binv spin 0][Binv spin 1][ln|det| (U0+U1)][sign (U0+U1)]
    double* st = state_out + (size_t)w * s.state_doubles;
    const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1];
    for (int q = lane; q < nb0; q += 32) st[q] = Binv[0][q];
    for (int q = lane; q < nb1; q += 32) st[nb0 + q] = Binv[1][q];
    for (int q = lane; q < Utot; q += 32) {
      st[nb0 + nb1 + q] = ldet[q];
      st[nb0 + nb1 + Utot + q] = dsg[q];
    }
  }
  double lnPhi, sgnPhi;
  term_ratios(s, lane, ldet, dsg, rk, lnPhi, sgnPhi);
  // K[Phi] and the marginal weights W_u = sum_{k contains u} w_k, T_u = sum_{k contains u} w_k t_k
  double kphi = 0.0;
  for (int k = lane; k < s.nterm; k += 32) {
    const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
    kphi += __ldg(s.term_coef + k) * rk[k] * (tdet[a] + tdet[U0 + b]);
  }
  kphi = warp_sum(kphi);
  for (int ud = lane; ud < Utot; ud += 32) {
    const int sp = ud >= U0 ? 1 : 0, u = ud - (sp ? U0 : 0);
    double Wv = 0.0, Tv = 0.0;
    for (int k = 0; k < s.nterm; ++k) {
      const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
      if ((sp ? b : a) != u) continue;
      const double wk = __ldg(s.term_coef + k) * rk[k];
      Wv += wk;
      Tv += wk * (tdet[a] + tdet[U0 + b]);
    }
    Wdet[ud] = Wv;
    Tdet[ud] = Tv;
  }
  __syncwarp();
  // grad_i ln|Psi| = grad_i lnJ + sum_u W_u sum_o Binv_u[o][i] grad phi_o(r_i), in the bulk type
  // (it feeds the Jastrow-parameter derivatives and the drift, not E_L)
  Tb* Bt = reinterpret_cast<Tb*>(scr);
  {
    const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1];
    for (int q = lane; q < nb0; q += 32) Bt[q] = (Tb)Binv[0][q];
    for (int q = lane; q < nb1; q += 32) Bt[nb0 + q] = (Tb)Binv[1][q];
  }
  __syncwarp();
  double kin_loc = 0.0;
  for (int e = lane; e < N; e += 32) {
    const int sp = e >= Nup ? 1 : 0, ie = e - (sp ? Nup : 0), n = s.n[sp], uo = sp ? U0 : 0;
    const Tb* Bs = Bt + (sp ? s.U[0] * s.n[0] * s.n[0] : 0);
    Tb gx = 0, gy = 0, gz = 0;
    for (int u = 0; u < s.U[sp]; ++u) {
      const Tb* B = Bs + u * n * n;
      Tb ax = 0, ay = 0, az = 0;
      for (int o = 0; o < n; ++o) {
        const Tb b = B[o * n + ie];
        const Tb* gp = Gphi + (e * nevd + __ldg(s.det_ev[sp] + u * n + o)) * 3;
        ax += b * gp[0];
        ay += b * gp[1];
        az += b * gp[2];
      }
      const Tb Wu = (Tb)Wdet[uo + u];
      gx += Wu * ax;
      gy += Wu * ay;
      gz += Wu * az;
    }
    const double G0 = (double)G[3 * e], G1 = (double)G[3 * e + 1], G2 = (double)G[3 * e + 2];
    vg[3 * e] = G0 + (double)gx;
    vg[3 * e + 1] = G1 + (double)gy;
    vg[3 * e + 2] = G2 + (double)gz;
    kin_loc += (double)LJ[e] + G0 * G0 + G1 * G1 + G2 * G2;
  }
  const double kin = warp_sum(kin_loc) + kphi;
  const double EL = -0.5 * kin + V;
  __syncwarp();
  if (lane == 0) {
    logpsi[w] = lnJ + lnPhi;
    sgn_out[w] = sgnPhi;
    eloc[w] = EL;
  }
  if (grad)
    for (int q = lane; q < 3 * N; q += 32) grad[(size_t)w * 3 * N + q] = vg[q];
  if (!Og) return;

  // ---- D. parameter derivatives ----
  const int P = s.P;
  Tb* Ow = Og + (size_t)w * P;
  Tb* Ew = dELg ? dELg + (size_t)w * P : nullptr;
  // D1. structure coefficients: O_I = Phi_I/Phi, E_L,I = -1/2 (K[Phi_I] - O_I K[Phi])
  for (int q = lane; q < s.n_cparam; q += 32) {
    const int I = __ldg(s.cparam + q);
    double o = 0.0, kk = 0.0;
    for (int t = 0; t < s.nsterm; ++t) {
      if (__ldg(s.sterm_I + t) != I) continue;
      const int k = __ldg(s.sterm_k + t);
      const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
      const double r = __ldg(s.sterm_d + t) * rk[k];
      o += r;
      kk += r * (tdet[a] + tdet[U0 + b]);
    }
    Ow[q] = (Tb)(o);
    if (Ew) Ew[q] = (Tb)(-0.5 * (kk - o * kphi));
  }
  // D2. Jastrow parameters: O = d lnJ/d alpha, E_L,alpha = -1/2 sum_i (lap_i g + 2 grad_i g . grad_i ln|Psi|)
  if (s.jas_param) {
    // e-n: a_2..a_6 per element (lanes over electron-nucleus pairs).  With h(R) the derivative
    // of f(R) = a1 R/(1 + a2 R) + sum_p a_{p+1} R^p with respect to the parameter:
    //   a_2: h = -a1 R^2/(1+a2 R)^2, h' = -2 a1 R/(1+a2 R)^3, h'' = -2 a1 (1-2 a2 R)/(1+a2 R)^4
    //   a_{p+1}: h = R^p; chain rule to r with R' = 1/(1+kappa r)^2, R'' = -2 kappa/(1+kappa r)^3.
    for (int E = 0; E < s.n_elem; ++E) {
      Tb aO[5] = {0, 0, 0, 0, 0}, aE[5] = {0, 0, 0, 0, 0};
      for (int t = lane; t < N * Nn; t += 32) {
        const int i = t / Nn, a = t % Nn;
        if (__ldg(s.nuc_elem + a) != E) continue;
        const Tb r = rEN[t];
        const PadeCoef c = en_coef(s, a);
        const Tb a1 = (Tb)c.a1, a2 = (Tb)c.a2;
        const Tb den = (Tb)1 / ((Tb)1 + kap * r), Rr = r * den, dR = den * den, d2R = (Tb)-2 * kap * dR * den;
        const Tb cosv = eEN[3 * t] * (Tb)vg[3 * i] + eEN[3 * t + 1] * (Tb)vg[3 * i + 1] + eEN[3 * t + 2] * (Tb)vg[3 * i + 2];
        const Tb pd = (Tb)1 / ((Tb)1 + a2 * Rr);
        Tb h[5], hR[5], hRR[5];
        h[0] = -a1 * Rr * Rr * pd * pd;
        hR[0] = (Tb)-2 * a1 * Rr * pd * pd * pd;
        hRR[0] = (Tb)-2 * a1 * ((Tb)1 - (Tb)2 * a2 * Rr) * pd * pd * pd * pd;
        Tb Rm2 = 1;  // R^(p-2)
#pragma unroll
        for (int p = 2; p <= 5; ++p) {
          h[p - 1] = Rm2 * Rr * Rr;
          hR[p - 1] = (Tb)p * Rm2 * Rr;
          hRR[p - 1] = (Tb)(p * (p - 1)) * Rm2;
          Rm2 *= Rr;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const Tb g1 = hR[q] * dR, g2 = hRR[q] * dR * dR + hR[q] * d2R;
          aO[q] += h[q];
          aE[q] += (Tb)-0.5 * (g2 + (Tb)2 * g1 / r + (Tb)2 * g1 * cosv);
        }
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double o = warp_sum((double)aO[q]), e = warp_sum((double)aE[q]);
        if (lane == 0) {
          Ow[s.p_off_a + 5 * E + q] = (Tb)(o);
          if (Ew) Ew[s.p_off_a + 5 * E + q] = (Tb)(e);
        }
      }
    }
    // e-e: b_2..b_6 (lanes over pairs), same radial forms with b1 (by spins) and b2
    {
      Tb bO[5] = {0, 0, 0, 0, 0}, bE[5] = {0, 0, 0, 0, 0};
      const int npair = N * (N - 1) / 2;
      for (int pp = lane; pp < npair; pp += 32) {
        int i = 0, rem = pp;
        while (rem >= N - 1 - i) { rem -= N - 1 - i; ++i; }
        const int j = i + 1 + rem, ij = i * N + j;
        const Tb r = rEE[ij];
        const PadeCoef c = ee_coef(s, (i < Nup) == (j < Nup));
        const Tb a1 = (Tb)c.a1, a2 = (Tb)c.a2;
        const Tb den = (Tb)1 / ((Tb)1 + kap * r), Rr = r * den, dR = den * den, d2R = (Tb)-2 * kap * dR * den;
        const Tb cosv = eEE[3 * ij] * (Tb)(vg[3 * i] - vg[3 * j]) + eEE[3 * ij + 1] * (Tb)(vg[3 * i + 1] - vg[3 * j + 1]) +
                        eEE[3 * ij + 2] * (Tb)(vg[3 * i + 2] - vg[3 * j + 2]);
        const Tb pd = (Tb)1 / ((Tb)1 + a2 * Rr);
        Tb h[5], hR[5], hRR[5];
        h[0] = -a1 * Rr * Rr * pd * pd;
        hR[0] = (Tb)-2 * a1 * Rr * pd * pd * pd;
        hRR[0] = (Tb)-2 * a1 * ((Tb)1 - (Tb)2 * a2 * Rr) * pd * pd * pd * pd;
        Tb Rm2 = 1;  // R^(p-2)
#pragma unroll
        for (int p = 2; p <= 5; ++p) {
          h[p - 1] = Rm2 * Rr * Rr;
          hR[p - 1] = (Tb)p * Rm2 * Rr;
          hRR[p - 1] = (Tb)(p * (p - 1)) * Rm2;
          Rm2 *= Rr;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const Tb g1 = hR[q] * dR, g2 = hRR[q] * dR * dR + hR[q] * d2R;
          bO[q] += h[q];
          bE[q] += (Tb)-0.5 * ((Tb)2 * (g2 + (Tb)2 * g1 * iEE[ij]) + (Tb)2 * g1 * cosv);
        }
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double o = warp_sum((double)bO[q]), e = warp_sum((double)bE[q]);
        if (lane == 0) {
          Ow[s.p_off_b + q] = (Tb)(o);
          if (Ew) Ew[s.p_off_b + q] = (Tb)(e);
        }
      }
    }
    // e-e-n: per element, the raw-term derivatives from the pair sums (lane -> (electron i,
    // group g), nuclei of the element split among groups), then theta = B^T raw
    if (s.een_on) {
      double* rawO = red;               // [23]
      double* rawE = red + kNeen;       // [23]
      const int Pp = L.jas_P, Sg = L.jas_S;
      for (int E = 0; E < s.n_elem; ++E) {
        Tb accO[kNeen], accE[kNeen];
#pragma unroll
        for (int q = 0; q < kNeen; ++q) accO[q] = accE[q] = (Tb)0;
        for (int b0 = 0; b0 < N; b0 += Pp) {
          const int i = b0 + lane % Pp, g = lane / Pp;
          if (i >= N) continue;
          const Tb vx = (Tb)vg[3 * i], vy = (Tb)vg[3 * i + 1], vz = (Tb)vg[3 * i + 2];
          for (int a = g; a < Nn; a += Sg) {
            if (__ldg(s.nuc_elem + a) != E) continue;
            const int ia = i * Nn + a;
            EenSide<Tb> si;
            si.set(Stab[(a * N + i) * 6 + 1], rEN[ia], kap);
            const Tb ex = eEN[3 * ia], ey = eEN[3 * ia + 1], ez = eEN[3 * ia + 2];
            auto sink = [&](int t, Tb val, Tb gx, Tb gy, Tb gz, Tb lp) {
              accO[t] += val;
              accE[t] += (Tb)-0.5 * (lp + (Tb)2 * (gx * vx + gy * vy + gz * vz));
            };
            {
              EenAcc<Tb, 1, 2> acc;
              acc.zero();
              for (int j = 0; j < N; ++j)
                if (j != i) {
                  const int ij = i * N + j;
                  acc.add(uEE[ij], iEE[ij], kap, eEE[3 * ij], eEE[3 * ij + 1], eEE[3 * ij + 2], Stab + (a * N + j) * 6);
                }
              een_terms(acc, si, ex, ey, ez, Ssum + 6 * a, sink);
            }
            {
              EenAcc<Tb, 3, 4> acc;
              acc.zero();
              for (int j = 0; j < N; ++j)
                if (j != i) {
                  const int ij = i * N + j;
                  acc.add(uEE[ij], iEE[ij], kap, eEE[3 * ij], eEE[3 * ij + 1], eEE[3 * ij + 2], Stab + (a * N + j) * 6);
                }
              een_terms(acc, si, ex, ey, ez, Ssum + 6 * a, sink);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kNeen; ++q) {
          const double o = warp_sum((double)accO[q]), e = warp_sum((double)accE[q]);
          if (lane == 0) {
            rawO[q] = o;
            rawE[q] = e;
          }
        }
        __syncwarp();
        for (int f = lane; f < kNfree; f += 32) {
          double o = 0.0, e = 0.0;
          for (int q = 0; q < kNeen; ++q) {
            const double b = __ldg(s.een_B + q * kNfree + f);
            o = fma(b, rawO[q], o);
            e = fma(b, rawE[q], e);
          }
          Ow[s.p_off_theta + kNfree * E + f] = (Tb)(o);
          if (Ew) Ew[s.p_off_theta + kNfree * E + f] = (Tb)(e);
        }
        __syncwarp();
      }
    }
  }
  // D3. orbital excitations kappa_kl (Sec. 2.2): for determinant u with l at slot o_l and
  //   k unoccupied, x_u = (A^-1 Phi)[o_l][k] = d ln D_u, y_u = (A^-1 L)[o_l][k] -
  //   sum_o' (A^-1 L)[o_l][occ o'] (A^-1 Phi)[o'][k] = d t_u; O = sum_u W_u x_u,
  //   K[Phi_kappa] = sum_u (T_u x_u + W_u y_u), E_L,kappa = -1/2 (K[Phi_kappa] - O K[Phi]).
  if (s.n_kappa > 0) {
    const int nk = s.n_kappa;
    for (int q = lane; q < 2 * nk; q += 32) kacc[q] = 0.0;
    __syncwarp();
    Tb* X = reinterpret_cast<Tb*>(scr);
    for (int sp = 0; sp < 2; ++sp) {
      const int n = s.n[sp], e0 = sp ? Nup : 0, uo = sp ? U0 : 0;
      if (n == 0) continue;
      Tb* Y = X + n * nev;
      Tb* Bt = Y + n * nev;  // bulk-type copy of the inverse
      for (int u = 0; u < s.U[sp]; ++u) {
        const int eb = __ldg(s.kap_off[sp] + u), ee = __ldg(s.kap_off[sp] + u + 1);
        if (eb == ee) continue;
        const double* B = Binv[sp] + u * n * n;
        for (int q = lane; q < n * n; q += 32) Bt[q] = (Tb)B[q];
        __syncwarp();
        for (int q = lane; q < n * nev; q += 32) {
          const int o = q / nev, c = q % nev;
          Tb x = 0, y = 0;
          for (int e = 0; e < n; ++e) {
            const Tb b = Bt[o * n + e];
            x += b * Phi[(e0 + e) * nev + c];
            y += b * Lphi[(e0 + e) * nev + c];
          }
          X[q] = x;
          Y[q] = y;
        }
        __syncwarp();
        const double Wu = Wdet[uo + u], Tu = Tdet[uo + u];
        for (int t = eb + lane; t < ee; t += 32) {
          const int j = __ldg(s.kap_ent[sp] + 4 * t), ol = __ldg(s.kap_ent[sp] + 4 * t + 1),
                    kc = __ldg(s.kap_ent[sp] + 4 * t + 2);
          const Tb x = X[ol * nev + kc];
          Tb y = Y[ol * nev + kc];
          for (int o2 = 0; o2 < n; ++o2) y -= Y[ol * nev + __ldg(s.det_ev[sp] + u * n + o2)] * X[o2 * nev + kc];
          kacc[j] += Wu * (double)x;
          kacc[nk + j] += Tu * (double)x + Wu * (double)y;
        }
        __syncwarp();
      }
    }
    for (int j = lane; j < nk; j += 32) {
      const double o = kacc[j];
      Ow[s.p_off_kappa + j] = (Tb)(o);
      if (Ew) Ew[s.p_off_kappa + j] = (Tb)(-0.5 * (kacc[nk + j] - o * kphi));
    }
  }
}

// =====================================================================================
// VMC sweep kernel
// =====================================================================================
// Each sweep moves every electron once (Sec. 2.3.1).  The determinant inverses come from
// the walker state written by the evaluation at the same positions, or from a fresh LU of
// double-precision orbital values (first sweep without state, and every 'refresh' sweeps).
// The proposed orbital row uses the bulk type; ratios and Sherman-Morrison updates are double.
template <class Tb>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const SysDev s, const SweepLayout L, int W, double* __restrict__ Rg,
                                                    int nsweeps, int refresh, const double* __restrict__ state_in,
                                                    double step, uint64_t seed, uint32_t step0, uint32_t tag,
                                                    uint32_t woff, int* __restrict__ nacc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  unsigned char* base = smem + wl * L.warp_bytes;
  double* R = reinterpret_cast<double*>(base + L.R);
  double* Binv[2] = {reinterpret_cast<double*>(base + L.Binv0), reinterpret_cast<double*>(base + L.Binv1)};
  double* ldet = reinterpret_cast<double*>(base + L.ldet);
  double* dsg = reinterpret_cast<double*>(base + L.dsg);
  double* wk = reinterpret_cast<double*>(base + L.wk);
  double* PhiO = reinterpret_cast<double*>(base + L.PhiO);
  double* basd = reinterpret_cast<double*>(base + L.bas);
  Tb* bas = reinterpret_cast<Tb*>(base + L.bas);
  double* vrowd = reinterpret_cast<double*>(base + L.vrow);
  Tb* part = reinterpret_cast<Tb*>(base + L.part);
  double* partd = reinterpret_cast<double*>(base + L.part);
  double* rho = reinterpret_cast<double*>(base + L.rho);
  double* cvec = reinterpret_cast<double*>(base + L.cvec);
  double* scr = reinterpret_cast<double*>(base + L.scratch);
  Tb* rEE = reinterpret_cast<Tb*>(base + L.geo);       // [N][N] r_ij
  Tb* rEN = rEE + s.N * s.N;                            // [N][Nn] r_ia
  Tb* Stab = rEN + s.N * s.Nn;                          // [Nn][N][6] Rbar(r_ia)^q
  Tb* rnE = Stab + 6 * s.N * s.Nn;                      // [N] r from the proposed position
  Tb* rnN = rnE + s.N;                                  // [Nn]
  Tb* Snew = rnN + s.Nn;                                // [Nn][6]
  Tb* Upo = Snew + 6 * s.Nn;                            // [5][N] Rbar(r_ej)^k, current position of e
  Tb* Upn = Upo + 5 * s.N;                              // [5][N] Rbar(r_ej)^k, proposed position

  const int N = s.N, Nn = s.Nn, Nup = s.Nup, U0 = s.U[0], ldo = L.nocc_max;
  const Tb kap = (Tb)s.kappa;
  const Tb* cf = orb_coefs<Tb>(s);
  const Tb* cE = een_coefs<Tb>(s);
  for (int i = lane; i < 3 * N; i += 32) R[i] = Rg[(size_t)w * 3 * N + i];
  __syncwarp();
  // geometry tables (coordinate differences in double, the rest in the bulk type)
  for (int p = lane; p < N * N; p += 32) {
    const int i = p / N, j = p % N;
    const Tb dx = (Tb)(R[3 * i] - R[3 * j]), dy = (Tb)(R[3 * i + 1] - R[3 * j + 1]), dz = (Tb)(R[3 * i + 2] - R[3 * j + 2]);
    rEE[p] = i == j ? (Tb)0 : vsqrt(dx * dx + dy * dy + dz * dz);
  }
  for (int p = lane; p < N * Nn; p += 32) {
    const int i = p / Nn, a = p % Nn;
    const double* nu = s.nuc4 + 4 * a;
    const Tb dx = (Tb)(R[3 * i] - __ldg(nu)), dy = (Tb)(R[3 * i + 1] - __ldg(nu + 1)), dz = (Tb)(R[3 * i + 2] - __ldg(nu + 2));
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz);
    rEN[p] = r;
    const Tb sv = (Tb)1 / ((Tb)1 + kap * r);
    Tb pw = (Tb)1;
#pragma unroll
    for (int q = 0; q < 6; ++q) { Stab[(a * N + i) * 6 + q] = pw; pw *= sv; }
  }
  if (state_in) {
    const double* st = state_in + (size_t)w * s.state_doubles;
    const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1], Ut = U0 + s.U[1];
    for (int q = lane; q < nb0; q += 32) Binv[0][q] = st[q];
    for (int q = lane; q < nb1; q += 32) Binv[1][q] = st[nb0 + q];
    for (int q = lane; q < Ut; q += 32) {
      ldet[q] = st[nb0 + nb1 + q];
      dsg[q] = st[nb0 + nb1 + Ut + q];
    }
  }
  __syncwarp();
  int accepted = 0;
  const uint32_t wid = woff + (uint32_t)w;

  for (int sw = 0; sw < nsweeps; ++sw) {
    const bool do_refresh = (sw == 0) ? (state_in == nullptr) : (refresh > 0 && sw % refresh == 0);
    if (do_refresh) {
      // double-precision orbital values of every electron, then LU of every unique determinant
      for (int e = 0; e < N; ++e) {
        const int sp = e >= Nup ? 1 : 0;
        basis_at<double, false>(s, lane, R[3 * e], R[3 * e + 1], R[3 * e + 2], basd, nullptr, nullptr, nullptr,
                                nullptr);
        __syncwarp();
        for (int c = lane; c < s.n_occ_chunk[sp]; c += 32) {
          const int4 ch = __ldg(reinterpret_cast<const int4*>(s.occ_chunk[sp]) + c);
          const double* cb = s.orb_coef + ch.w;
          double v = 0.0;
          for (int mu = ch.y; mu < ch.z; ++mu) v = fma(__ldg(cb + mu), basd[mu], v);
          partd[c] = v;
        }
        __syncwarp();
        for (int q = lane; q < s.nocc[sp]; q += 32) {
          const int c0 = __ldg(s.occ_chunk_off[sp] + q), c1 = __ldg(s.occ_chunk_off[sp] + q + 1);
          double v = 0.0;
          for (int c = c0; c < c1; ++c) v += partd[c];
          PhiO[e * ldo + q] = v;
        }
        __syncwarp();
      }
      lu_all(s, 0, lane, PhiO, ldo, (const double*)nullptr, 0, s.det_loc[0], L.G0, Binv[0], scr, ldet, dsg, nullptr);
      lu_all(s, 1, lane, PhiO, ldo, (const double*)nullptr, 0, s.det_loc[1], L.G1, Binv[1], scr, ldet + U0, dsg + U0,
             nullptr);
    }
    if (do_refresh || sw == 0) {
      double lnPhi, sgnPhi;
      term_ratios(s, lane, ldet, dsg, wk, lnPhi, sgnPhi);
      for (int k = lane; k < s.nterm; k += 32) wk[k] *= __ldg(s.term_coef + k);  // w_k = C_k D_k / Phi
      __syncwarp();
    }
    const uint32_t st = step0 + (uint32_t)sw;
    for (int e = 0; e < N; ++e) {
      const int sp = e >= Nup ? 1 : 0, ie = e - (sp ? Nup : 0), n = s.n[sp], G = sp ? L.G1 : L.G0;
      double u0, u1, u2, uacc;
      uniforms2(seed, wid, st, (uint32_t)e, tag, 0, u0, u1);
      uniforms2(seed, wid, st, (uint32_t)e, tag, 1, u2, uacc);
      double rn[3];
      rn[0] = __dadd_rn(R[3 * e], __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u0), 1.0)));
      rn[1] = __dadd_rn(R[3 * e + 1], __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u1), 1.0)));
      rn[2] = __dadd_rn(R[3 * e + 2], __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u2), 1.0)));
      // orbital row at the proposed position (bulk type), contraction in balanced chunks
      basis_at<Tb, false>(s, lane, rn[0], rn[1], rn[2], bas, nullptr, nullptr, nullptr, nullptr);
      __syncwarp();
      for (int c = lane; c < s.n_occ_chunk[sp]; c += 32) {
        const int4 ch = __ldg(reinterpret_cast<const int4*>(s.occ_chunk[sp]) + c);
        const Tb* cb = cf + ch.w;
        Tb v = 0;
        for (int mu = ch.y; mu < ch.z; ++mu) v += __ldg(cb + mu) * bas[mu];
        part[c] = v;
      }
      __syncwarp();
      for (int q = lane; q < s.nocc[sp]; q += 32) {
        const int c0 = __ldg(s.occ_chunk_off[sp] + q), c1 = __ldg(s.occ_chunk_off[sp] + q + 1);
        Tb v = 0;
        for (int c = c0; c < c1; ++c) v += part[c];
        vrowd[q] = (double)v;
      }
      __syncwarp();
      // determinant ratios rho_u = sum_o v_occ(o) Binv_u[o][ie]
      const int U = s.U[sp], ng = 32 / G, g = lane / G, gl = lane % G;
      const int* dl = s.det_loc[sp];
      for (int ub = 0; ub < U; ub += ng) {
        const int u = ub + g;
        double r = 0.0;
        if (u < U && gl < n) r = vrowd[__ldg(dl + u * n + gl)] * Binv[sp][u * n * n + gl * n + ie];
        r = group_sum(r, G);
        if (u < U && gl == 0) rho[u] = r;
      }
      __syncwarp();
      double rphi = 0.0;
      for (int k = lane; k < s.nterm; k += 32) rphi += wk[k] * rho[__ldg(s.term_det + 2 * k + sp)];
      rphi = warp_sum(rphi);
      // Jastrow change of the terms that involve electron e (Sec. 2.1): distances from the
      // proposed position, then items e-n (a), e-e (j) and e-e-n (a, k), the last through the
      // pair sums Y^{k,q} = sum_{j != e} u_ej^k s_j^q (the terms of e are s_e^A Y^{k,B} + s_e^B Y^{k,A}).
      for (int j = lane; j < N; j += 32) {
        const Tb dx = (Tb)(rn[0] - R[3 * j]), dy = (Tb)(rn[1] - R[3 * j + 1]), dz = (Tb)(rn[2] - R[3 * j + 2]);
        const Tb rnew = j == e ? (Tb)0 : vsqrt(dx * dx + dy * dy + dz * dz);
        rnE[j] = rnew;
        const Tb uo = (Tb)1 / ((Tb)1 + kap * rEE[e * N + j]), un = (Tb)1 / ((Tb)1 + kap * rnew);
        Tb po = (Tb)1, pn = (Tb)1;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          Upo[k * N + j] = po;
          Upn[k * N + j] = pn;
          po *= uo;
          pn *= un;
        }
      }
      for (int a = lane; a < Nn; a += 32) {
        const double* nu = s.nuc4 + 4 * a;
        const Tb dx = (Tb)(rn[0] - __ldg(nu)), dy = (Tb)(rn[1] - __ldg(nu + 1)), dz = (Tb)(rn[2] - __ldg(nu + 2));
        const Tb r = vsqrt(dx * dx + dy * dy + dz * dz);
        rnN[a] = r;
        const Tb sv = (Tb)1 / ((Tb)1 + kap * r);
        Tb pw = (Tb)1;
#pragma unroll
        for (int q = 0; q < 6; ++q) { Snew[a * 6 + q] = pw; pw *= sv; }
      }
      __syncwarp();
      Tb dj = 0;
      const int nitem = Nn + N + (s.een_on ? 5 * Nn : 0);
      for (int t = lane; t < nitem; t += 32) {
        if (t < Nn) {
          const PadeCoef c = en_coef(s, t);
          Tb f1, f0, t0, t1;
          pade_eval<Tb, false>(c, rnN[t], kap, f1, t0, t1);
          pade_eval<Tb, false>(c, rEN[e * Nn + t], kap, f0, t0, t1);
          dj += f1 - f0;
        } else if (t < Nn + N) {
          const int j = t - Nn;
          if (j == e) continue;
          const PadeCoef c = ee_coef(s, (e < Nup) == (j < Nup));
          Tb f1, f0, t0, t1;
          pade_eval<Tb, false>(c, rnE[j], kap, f1, t0, t1);
          pade_eval<Tb, false>(c, rEE[e * N + j], kap, f0, t0, t1);
          dj += f1 - f0;
        } else {
          const int tt = t - Nn - N, a = tt / 5, k = tt % 5;
          Tb Yo[6], Yn[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) Yo[q] = Yn[q] = (Tb)0;
          for (int j = 0; j < N; ++j) {
            if (j == e) continue;
            const Tb po = Upo[k * N + j], pn = Upn[k * N + j];
            const Tb* Sj = Stab + (a * N + j) * 6;
#pragma unroll
            for (int q = 0; q < 6; ++q)
              if (q <= 5 - k) {
                Yo[q] += po * Sj[q];
                Yn[q] += pn * Sj[q];
              }
          }
          const Tb* So = Stab + (a * N + e) * 6;
          const Tb* Sn = Snew + a * 6;
          const Tb* c = cE + kNeen * __ldg(s.nuc_elem + a);
          een_for_each([&](auto tc) {
            constexpr int q = decltype(tc)::value;
            constexpr int tk = een_klm(q).k, A = een_klm(q).l + een_klm(q).m, B = een_klm(q).m;
            if (tk != k) return;
            dj += c[q] * ((Sn[A] * Yn[B] + Sn[B] * Yn[A]) - (So[A] * Yo[B] + So[B] * Yo[A]));
          });
        }
      }
      const Tb dJ = warp_sum(dj);
      const double prob = rphi * rphi * (double)vexp((Tb)2 * dJ);
      if (uacc < prob) {
        // Sherman-Morrison: Binv <- Binv - Binv[:, ie] (v^T Binv - e_ie^T) / rho
        for (int ub = 0; ub < U; ub += ng) {
          const int u = ub + g;
          const bool act = u < U;
          double* B = Binv[sp] + (act ? u : 0) * n * n;
          double* cv = cvec + g * n;
          if (act && gl < n) cv[gl] = B[gl * n + ie];
          __syncwarp();
          if (act && gl < n) {
            const int j = gl;
            double wj = (j == ie) ? -1.0 : 0.0;
            for (int o = 0; o < n; ++o) wj = fma(vrowd[__ldg(dl + u * n + o)], B[o * n + j], wj);
            const double f = wj * recip(rho[u]);
            for (int o = 0; o < n; ++o) B[o * n + j] = fma(-cv[o], f, B[o * n + j]);
          }
          __syncwarp();
        }
        const double irphi = recip(rphi);
        for (int k = lane; k < s.nterm; k += 32) wk[k] *= rho[__ldg(s.term_det + 2 * k + sp)] * irphi;
        if (lane < 3) R[3 * e + lane] = rn[lane];
        for (int j = lane; j < N; j += 32) rEE[e * N + j] = rEE[j * N + e] = rnE[j];
        for (int a = lane; a < Nn; a += 32) {
          rEN[e * Nn + a] = rnN[a];
#pragma unroll
          for (int q = 0; q < 6; ++q) Stab[(a * N + e) * 6 + q] = Snew[a * 6 + q];
        }
        ++accepted;
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < 3 * N; i += 32) Rg[(size_t)w * 3 * N + i] = R[i];
  if (nacc && lane == 0) nacc[w] += accepted;
}

// =====================================================================================
// layouts and launchers
// =====================================================================================
int make_eval_layout(const SysDev& s, int tb, int max_smem, EvalLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1];
  L.G0 = group_size(s.n[0]);
  L.G1 = group_size(s.n[1]);
  L.R = take(8 * 3 * N);
  L.vg = take(8 * 3 * N);
  L.G = take(tb * 3 * N);
  L.LJ = take(tb * N);
  L.Phi = take(tb * N * s.n_ev);
  L.PhiD = take(8 * N * std::max(s.n_ev_det, 1));
  L.Lphi = take(tb * N * s.n_ev);
  L.Gphi = take(tb * N * s.n_ev_det * 3);
  L.Binv0 = take(8 * s.U[0] * s.n[0] * s.n[0]);
  L.Binv1 = take(8 * s.U[1] * s.n[1] * s.n[1]);
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.tdet = take(8 * Ut);
  L.Wdet = take(8 * Ut);
  L.Tdet = take(8 * Ut);
  L.rk = take(8 * s.nterm);
  int scr = align16(5 * s.M * tb) + 8 * s.M + 32 * s.Nn;
  scr = std::max(scr, tb * (s.U[0] * s.n[0] * s.n[0] + s.U[1] * s.n[1] * s.n[1]));
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], G = sp ? L.G1 : L.G0, ng = 32 / G;
    scr = std::max(scr, ng * (8 * n * n + 4 * n) + 16);
    scr = std::max(scr, (2 * n * s.n_ev + n * n) * tb);
  }
  L.scratch = take(scr);
  L.part = take(5 * tb * std::max(s.n_ev_chunk, 1));
  L.partd = take(8 * std::max(s.n_det_chunk, 1));
  L.kacc = take(8 * 2 * std::max(s.n_kappa, 1));
  L.red = take(8 * 64);
  L.geo = take(tb * (6 * N * N + 4 * N * s.Nn + 6 * N * s.Nn + 6 * s.Nn));
  {
    int P = 1;
    while (P < N && P < 32) P <<= 1;
    L.jas_P = P;
    L.jas_S = 32 / P;
  }
  L.warp_bytes = off;
  int wpb = max_smem / off;
  const int cap = (tb == 8 ? EvalBounds<double>::threads : EvalBounds<float>::threads) / 32;
  if (wpb > cap) wpb = cap;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

int make_sweep_layout(const SysDev& s, int tb, int max_smem, SweepLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1];
  L.G0 = group_size(s.n[0]);
  L.G1 = group_size(s.n[1]);
  L.nocc_max = std::max(std::max(s.nocc[0], s.nocc[1]), 1);
  L.R = take(8 * 3 * N);
  L.Binv0 = take(8 * s.U[0] * s.n[0] * s.n[0]);
  L.Binv1 = take(8 * s.U[1] * s.n[1] * s.n[1]);
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.wk = take(8 * s.nterm);
  L.PhiO = take(8 * N * L.nocc_max);
  L.bas = take(8 * s.M);
  L.vrow = take(8 * L.nocc_max);
  L.part = take(8 * std::max(std::max(s.n_occ_chunk[0], s.n_occ_chunk[1]), 1));
  L.rho = take(8 * std::max(s.U[0], s.U[1]));
  int cv = 0, scr = 0;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], G = sp ? L.G1 : L.G0, ng = 32 / G;
    cv = std::max(cv, 8 * ng * n);
    scr = std::max(scr, ng * (8 * n * n + 4 * n) + 16);
  }
  L.cvec = take(std::max(cv, 8));
  L.scratch = take(std::max(scr, 16));
  L.geo = take(tb * (N * N + N * s.Nn + 6 * N * s.Nn + N + s.Nn + 6 * s.Nn + 10 * N));
  L.warp_bytes = off;
  int wpb = max_smem / off;
  if (wpb > 16) wpb = 16;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

template <class Tb>
static cudaError_t launch_eval_t(const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                                 double* sign, double* eloc, double* grad, Tb* O, Tb* dEL, double* state_out,
                                 cudaStream_t st) {
  const int smem = L.wpb * L.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(eval_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (W + L.wpb - 1) / L.wpb;
  eval_kernel<Tb><<<blocks, 32 * L.wpb, smem, st>>>(s, L, W, R, logpsi, sign, eloc, grad, O, dEL, state_out);
  return cudaGetLastError();
}

template <class Tb>
static cudaError_t launch_sweep_t(const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps, int refresh,
                                  const double* state_in, double step, uint64_t seed, uint32_t step0, uint32_t tag,
                                  uint32_t woff, int* nacc, cudaStream_t st) {
  const int smem = L.wpb * L.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (W + L.wpb - 1) / L.wpb;
  sweep_kernel<Tb><<<blocks, 32 * L.wpb, smem, st>>>(s, L, W, R, nsweeps, refresh, state_in, step, seed, step0, tag,
                                                     woff, nacc);
  return cudaGetLastError();
}

cudaError_t launch_eval(int precision, const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                        double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out,
                        cudaStream_t st) {
  if (precision == VBQMC_MIXED)
    return launch_eval_t<float>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<float*>(O),
                                static_cast<float*>(dEL), state_out, st);
  return launch_eval_t<double>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<double*>(O),
                               static_cast<double*>(dEL), state_out, st);
}

cudaError_t launch_sweep(int precision, const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps,
                         int refresh, const double* state_in, double step, uint64_t seed, uint32_t step0, uint32_t tag,
                         uint32_t woff, int* nacc, cudaStream_t st) {
  if (precision == VBQMC_MIXED)
    return launch_sweep_t<float>(s, L, W, R, nsweeps, refresh, state_in, step, seed, step0, tag, woff, nacc, st);
  return launch_sweep_t<double>(s, L, W, R, nsweeps, refresh, state_in, step, seed, step0, tag, woff, nacc, st);
}

}  // namespace vbq
