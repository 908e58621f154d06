// Per-walker bodies of the Jastrow kernels (arXiv:2207.14715, Sec. 2.1, Jastrow factor): ln J,
// its electron gradients and Laplacians, the Coulomb potential, and the Jastrow-parameter
// derivatives; shared by the single-system, batched and fused batch kernels.
#pragma once

#include "batch.h"
#include "walker_common.cuh"

namespace vbq {

namespace {

// Blocks per SM the Jastrow kernels are compiled for (the double instantiation keeps more
// live values, so it gets the whole register file of one block).
template <class Tb> struct JasBounds { static constexpr int min_blocks = 2; };
template <> struct JasBounds<double> { static constexpr int min_blocks = 1; };

// Per-lane sum of ln J terms: double in the FP64 form; in the mixed form a compensated float
// sum (the value enters ln|Psi|, so it keeps about double accuracy without double
// instructions): the running sum s and, in c, the rounding error of every addition (TwoSum)
// and of every coefficient product (TwoProduct), added to s once at the end.
template <class Tb> struct LnSum {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(const LnSum& o) { v += o.v; }
  __device__ __forceinline__ double value() const { return v; }
};
template <> struct LnSum<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void acc(float x) {
    const dsf t = ds_two_sum(s, x);
    s = t.hi;
    c += t.lo;
  }
  __device__ __forceinline__ void add(float x) { acc(x); }
  __device__ __forceinline__ void add(dsf x) {
    acc(x.hi);
    c += x.lo;
  }
  // (chi + clo) val, the coefficient a float-float pair
  __device__ __forceinline__ void add_prod(float chi, float clo, float val) {
    const float p = chi * val;
    c += fmaf(clo, val, fmaf(chi, val, -p));
    acc(p);
  }
  __device__ __forceinline__ void add(const LnSum& o) {
    acc(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// lanes -> (electron i, group g); group g takes nuclei a = g, g + S, ... and partners
// j = g, g + S, ...
// WIDE: the whole block works on walker w (warp rank r takes groups r Sg .. r Sg + Sg - 1 of
// nuclei and partners), the per-walker tables are shared, and the per-electron sums of the
// warps meet in shared memory; otherwise one warp per walker.
template <class Tb, bool WIDE = false>
__device__ __forceinline__ void jastrow_body(const SysDev& s, const JasLayout& L, int w, unsigned char* base,
                                             const double* Rg, Tb* __restrict__ JG, Tb* __restrict__ JL,
                                             double* __restrict__ JS) {
  const int lane = threadIdx.x & 31;
  const int rank = WIDE ? (int)(threadIdx.x >> 5) : 0, nw = WIDE ? (int)(blockDim.x >> 5) : 1;
  const int N = s.N, Nn = s.Nn, Nup = s.Nup;
  const GeoTables<Tb> g(reinterpret_cast<Tb*>(base + L.geo), N, Nn);
  const Tb kap = (Tb)s.kappa;
  const Coords<Tb> C = load_coords<Tb, WIDE>(Rg + (size_t)w * 3 * N, N, 32 * rank + lane, base + L.R, 32 * nw);
  const double V_loc = build_geometry<Tb, WIDE>(s, 32 * rank + lane, C, g, 32 * nw);
  LnSum<Tb> lnJ_loc;
  const Tb* cE = een_coefs<Tb>(s);
  const int Pp = L.jas_P, Sg = L.jas_S * nw;
  for (int b0 = 0; b0 < N; b0 += Pp) {
    const int i = b0 + (lane & (Pp - 1)), gr = rank * L.jas_S + (lane >> (__ffs(Pp) - 1));
    const bool act = i < N;
    Tb g0 = 0, g1 = 0, g2 = 0, lap = 0;
    LnSum<Tb> lnj;
    if (act) {
      for (int a = gr; a < Nn; a += Sg) {
        const int ia = i * Nn + a;
        const Tb r = g.rEN[ia];
        Tb f, df, d2f;
        pade_eval<Tb, true>(en_coef_t<Tb>(s, a), r, kap, f, df, d2f);
        if constexpr (kSameType<Tb, double>) {
          lnj.add(f);
        } else {  // the value in float-float from float-float coordinates
          const dsf na[3] = {nuc_coord_ds(s, a, 0), nuc_coord_ds(s, a, 1), nuc_coord_ds(s, a, 2)};
          lnj.add(pade_value_ds(ds_dist(C.R + 3 * i, na), s.jas_a_ds + 12 * __ldg(s.nuc_elem + a), nullptr,
                                s.kappa_ds));
        }
        g0 += df * g.eEN[3 * ia]; g1 += df * g.eEN[3 * ia + 1]; g2 += df * g.eEN[3 * ia + 2];
        lap += d2f + (Tb)2 * df / r;
      }
      for (int j = gr; j < N; j += Sg) {
        if (j == i) continue;
        const int ij = g.ee(i, j);
        Tb f, df, d2f;
        pade_eval<Tb, true>(ee_coef_t<Tb>(s, (i < Nup) == (j < Nup)), g.rEE[ij], kap, f, df, d2f);
        if constexpr (kSameType<Tb, double>) {
          lnj.add((Tb)0.5 * f);
        } else {
          const dsf v = pade_value_ds(ds_dist(C.R + 3 * i, C.R + 3 * j), s.jas_b_ds,
                                      (i < Nup) == (j < Nup) ? s.b1_par_ds : s.b1_anti_ds, s.kappa_ds);
          lnj.add(dsf{0.5f * v.hi, 0.5f * v.lo});
        }
        g0 += df * g.eEE[3 * ij]; g1 += df * g.eEE[3 * ij + 1]; g2 += df * g.eEE[3 * ij + 2];
        lap += d2f + (Tb)2 * df * g.iEE[ij];
      }
      if (s.een_on)
        for (int a = gr; a < Nn; a += Sg) {
          const int ia = i * Nn + a;
          const Tb* c = cE + kNeen * __ldg(s.nuc_elem + a);
          EenSide<Tb> si;
          si.set(g.Stab[(a * N + i) * 6 + 1], g.rEN[ia], kap);
          const Tb ex = g.eEN[3 * ia], ey = g.eEN[3 * ia + 1], ez = g.eEN[3 * ia + 2];
          const float* cds = s.een_c_ds + 2 * kNeen * __ldg(s.nuc_elem + a);
          auto sink = [&](int t, Tb val, Tb gx, Tb gy, Tb gz, Tb lp) {
            const Tb ct = c[t];
            if constexpr (kSameType<Tb, double>)
              lnj.add(ct * val);
            else  // coefficient as a float-float pair: its rounding would shift every triple alike
              lnj.add_prod(__ldg(cds + 2 * t), __ldg(cds + 2 * t + 1), val);
            g0 += ct * gx; g1 += ct * gy; g2 += ct * gz;
            lap += ct * lp;
          };
          {
            EenAcc<Tb, 1, 2> acc;
            acc.zero();
            for (int j = 0; j < N; ++j)
              if (j != i) {
                const int ij = g.ee(i, j);
                acc.add(g.uEE[ij], g.iEE[ij], kap, g.eEE[3 * ij], g.eEE[3 * ij + 1], g.eEE[3 * ij + 2],
                        g.Stab + (a * N + j) * 6);
              }
            een_terms(acc, si, ex, ey, ez, g.Ssum + 6 * a, g.SsumLo + 6 * a, sink);
          }
          {
            EenAcc<Tb, 3, 4> acc;
            acc.zero();
            for (int j = 0; j < N; ++j)
              if (j != i) {
                const int ij = g.ee(i, j);
                acc.add(g.uEE[ij], g.iEE[ij], kap, g.eEE[3 * ij], g.eEE[3 * ij + 1], g.eEE[3 * ij + 2],
                        g.Stab + (a * N + j) * 6);
              }
            een_terms(acc, si, ex, ey, ez, g.Ssum + 6 * a, g.SsumLo + 6 * a, sink);
          }
        }
      lnJ_loc.add(lnj);
    }
    for (int o = Pp; o < 32; o <<= 1) {
      g0 += __shfl_xor_sync(kFull, g0, o);
      g1 += __shfl_xor_sync(kFull, g1, o);
      g2 += __shfl_xor_sync(kFull, g2, o);
      lap += __shfl_xor_sync(kFull, lap, o);
    }
    if constexpr (WIDE) {
      Tb* red = reinterpret_cast<Tb*>(base + L.wred);  // [nw][Pp][4]
      if (act && lane < Pp) {
        Tb* r = red + (rank * Pp + lane) * 4;
        r[0] = g0; r[1] = g1; r[2] = g2; r[3] = lap;
      }
      __syncthreads();
      if (rank == 0 && act && lane < Pp) {
        Tb a[4] = {0, 0, 0, 0};
        for (int q = 0; q < nw; ++q)
#pragma unroll
          for (int c = 0; c < 4; ++c) a[c] += red[(q * Pp + lane) * 4 + c];
        Tb* Gw = JG + (size_t)w * 3 * N;
        Gw[3 * i] = a[0]; Gw[3 * i + 1] = a[1]; Gw[3 * i + 2] = a[2];
        JL[(size_t)w * N + i] = a[3];
      }
      __syncthreads();
    } else if (act && gr == 0) {
      Tb* Gw = JG + (size_t)w * 3 * N;
      Gw[3 * i] = g0; Gw[3 * i + 1] = g1; Gw[3 * i + 2] = g2;
      JL[(size_t)w * N + i] = lap;
    }
  }
  double lnJ = warp_sum(lnJ_loc.value());
  double V = warp_sum(V_loc);
  if constexpr (WIDE) {
    double* dred = reinterpret_cast<double*>(base + L.wred2);  // [nw][2]
    if (lane == 0) {
      dred[2 * rank] = lnJ;
      dred[2 * rank + 1] = V;
    }
    __syncthreads();
    lnJ = 0.0;
    V = 0.0;
    for (int q = 0; q < nw; ++q) {
      lnJ += dred[2 * q];
      V += dred[2 * q + 1];
    }
  }
  if (lane == 0 && rank == 0) {
    JS[2 * (size_t)w] = lnJ;
    JS[2 * (size_t)w + 1] = V + s.vnn;
  }
}

// Radial parameter derivatives of the Pade + polynomial form f(R) = a1 R/(1 + a2 R) +
// sum_p a_{p+1} R^p, R = r/(1 + kappa r): with h the derivative of f with respect to the
// parameter,
//   a_2: h = -a1 R^2/(1+a2 R)^2, h' = -2 a1 R/(1+a2 R)^3, h'' = -2 a1 (1-2 a2 R)/(1+a2 R)^4
//   a_{p+1}: h = R^p; chain rule to r with R' = 1/(1+kappa r)^2, R'' = -2 kappa/(1+kappa r)^3.
template <class Tb>
__device__ __forceinline__ void pade_param_derivs(Tb r, Tb kap, Tb a1, Tb a2, Tb h[5], Tb g1[5], Tb g2[5]) {
  const Tb den = (Tb)1 / ((Tb)1 + kap * r), Rr = r * den, dR = den * den, d2R = (Tb)-2 * kap * dR * den;
  const Tb pd = (Tb)1 / ((Tb)1 + a2 * Rr);
  Tb hR[5], hRR[5];
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
    g1[q] = hR[q] * dR;
    g2[q] = hRR[q] * dR * dR + hR[q] * d2R;
  }
}

template <class Tb>
__device__ __forceinline__ void jastrow_deriv_body(const SysDev& s, const JasLayout& L, int w, unsigned char* base,
                                                   const double* Rg, const double* vgg,
                                                   Tb* __restrict__ Og, Tb* __restrict__ dELg) {
  const int lane = threadIdx.x & 31;
  Tb* vg = reinterpret_cast<Tb*>(base + L.vg);  // grad ln|Psi| in the bulk type
  Tb* red = reinterpret_cast<Tb*>(base + L.red);
  const int N = s.N, Nn = s.Nn, Nup = s.Nup;
  const GeoTables<Tb> g(reinterpret_cast<Tb*>(base + L.geo), N, Nn);
  const Tb kap = (Tb)s.kappa;
  for (int i = lane; i < 3 * N; i += 32) vg[i] = (Tb)vgg[(size_t)w * 3 * N + i];
  const Coords<Tb> C = load_coords<Tb>(Rg + (size_t)w * 3 * N, N, lane, base + L.R);
  build_geometry<Tb>(s, lane, C, g);
  const int P = s.P;
  Tb* Ow = Og + (size_t)w * P;
  Tb* Ew = dELg ? dELg + (size_t)w * P : nullptr;
  // e-n: a_2..a_6 per element (lanes over electron-nucleus pairs)
  for (int E = 0; E < s.n_elem; ++E) {
    Tb aO[5] = {0, 0, 0, 0, 0}, aE[5] = {0, 0, 0, 0, 0};
    for (DivStep ia(lane, Nn); ia.hi < N; ia.next(Nn)) {
      const int i = ia.hi, a = ia.lo, t = i * Nn + a;
      if (__ldg(s.nuc_elem + a) != E) continue;
      const Tb r = g.rEN[t];
      const PadeT<Tb> c = en_coef_t<Tb>(s, a);
      const Tb cosv = g.eEN[3 * t] * vg[3 * i] + g.eEN[3 * t + 1] * vg[3 * i + 1] + g.eEN[3 * t + 2] * vg[3 * i + 2];
      Tb h[5], g1[5], g2[5];
      pade_param_derivs<Tb>(r, kap, c.a1, c.a2, h, g1, g2);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        aO[q] += h[q];
        aE[q] += (Tb)-0.5 * (g2[q] + (Tb)2 * g1[q] / r + (Tb)2 * g1[q] * cosv);
      }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const Tb o = warp_sum(aO[q]), e = warp_sum(aE[q]);
      if (lane == 0) {
        Ow[s.p_off_a + 5 * E + q] = o;
        if (Ew) Ew[s.p_off_a + 5 * E + q] = e;
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
      const int j = i + 1 + rem, ij = g.ee(i, j);
      const Tb r = g.rEE[ij];
      const PadeT<Tb> c = ee_coef_t<Tb>(s, (i < Nup) == (j < Nup));
      const Tb cosv = g.eEE[3 * ij] * (vg[3 * i] - vg[3 * j]) + g.eEE[3 * ij + 1] * (vg[3 * i + 1] - vg[3 * j + 1]) +
                      g.eEE[3 * ij + 2] * (vg[3 * i + 2] - vg[3 * j + 2]);
      Tb h[5], g1[5], g2[5];
      pade_param_derivs<Tb>(r, kap, c.a1, c.a2, h, g1, g2);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        bO[q] += h[q];
        bE[q] += (Tb)-0.5 * ((Tb)2 * (g2[q] + (Tb)2 * g1[q] * g.iEE[ij]) + (Tb)2 * g1[q] * cosv);
      }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const Tb o = warp_sum(bO[q]), e = warp_sum(bE[q]);
      if (lane == 0) {
        Ow[s.p_off_b + q] = o;
        if (Ew) Ew[s.p_off_b + q] = e;
      }
    }
  }
  // e-e-n: per element, the raw-term derivatives from the pair sums (lane -> (electron i,
  // group g), nuclei of the element split among groups), then theta = B^T raw
  if (s.een_on) {
    Tb* rawO = red;          // [23]
    Tb* rawE = red + kNeen;  // [23]
    const int Pp = L.jas_P, Sg = L.jas_S;
    for (int E = 0; E < s.n_elem; ++E) {
      Tb accO[kNeen], accE[kNeen];
#pragma unroll
      for (int q = 0; q < kNeen; ++q) accO[q] = accE[q] = (Tb)0;
      for (int b0 = 0; b0 < N; b0 += Pp) {
        const int i = b0 + (lane & (Pp - 1)), gr = lane >> (__ffs(Pp) - 1);
        if (i >= N) continue;
        const Tb vx = vg[3 * i], vy = vg[3 * i + 1], vz = vg[3 * i + 2];
        for (int a = gr; a < Nn; a += Sg) {
          if (__ldg(s.nuc_elem + a) != E) continue;
          const int ia = i * Nn + a;
          EenSide<Tb> si;
          si.set(g.Stab[(a * N + i) * 6 + 1], g.rEN[ia], kap);
          const Tb ex = g.eEN[3 * ia], ey = g.eEN[3 * ia + 1], ez = g.eEN[3 * ia + 2];
          auto sink = [&](int t, Tb val, Tb gx, Tb gy, Tb gz, Tb lp) {
            accO[t] += val;
            accE[t] += (Tb)-0.5 * (lp + (Tb)2 * (gx * vx + gy * vy + gz * vz));
          };
          {
            EenAcc<Tb, 1, 2> acc;
            acc.zero();
            for (int j = 0; j < N; ++j)
              if (j != i) {
                const int ij = g.ee(i, j);
                acc.add(g.uEE[ij], g.iEE[ij], kap, g.eEE[3 * ij], g.eEE[3 * ij + 1], g.eEE[3 * ij + 2],
                        g.Stab + (a * N + j) * 6);
              }
            een_terms(acc, si, ex, ey, ez, g.Ssum + 6 * a, g.SsumLo + 6 * a, sink);
          }
          {
            EenAcc<Tb, 3, 4> acc;
            acc.zero();
            for (int j = 0; j < N; ++j)
              if (j != i) {
                const int ij = g.ee(i, j);
                acc.add(g.uEE[ij], g.iEE[ij], kap, g.eEE[3 * ij], g.eEE[3 * ij + 1], g.eEE[3 * ij + 2],
                        g.Stab + (a * N + j) * 6);
              }
            een_terms(acc, si, ex, ey, ez, g.Ssum + 6 * a, g.SsumLo + 6 * a, sink);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kNeen; ++q) {
        const Tb o = warp_sum(accO[q]), e = warp_sum(accE[q]);
        if (lane == 0) {
          rawO[q] = o;
          rawE[q] = e;
        }
      }
      __syncwarp();
      const Tb* Bmat = een_basis_t<Tb>(s);
      for (int f = lane; f < kNfree; f += 32) {
        Tb o = 0, e = 0;
        for (int q = 0; q < kNeen; ++q) {
          const Tb b = __ldg(Bmat + q * kNfree + f);
          o += b * rawO[q];
          e += b * rawE[q];
        }
        Ow[s.p_off_theta + kNfree * E + f] = o;
        if (Ew) Ew[s.p_off_theta + kNfree * E + f] = e;
      }
      __syncwarp();
    }
  }
}

}  // namespace

}  // namespace vbq
