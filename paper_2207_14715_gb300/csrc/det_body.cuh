// Per-walker body of the determinant kernel (arXiv:2207.14715, Sec. 2.1 determinant expansion,
// Sec. 2.3.1): Slater LU or carried inverses, structure sum, E_L, grad ln|Psi| and the
// structure and orbital-excitation derivatives; shared by the single-system, batched and
// fused batch kernels.
#pragma once

#include "batch.h"
#include "walker_common.cuh"

namespace vbq {

namespace {

// Lane-group LU + inverse of every unique determinant of spin sp from the double orbital
// values PhiD[(e0 + e) * ld + idx[u][o]]: Bt[u] = A^-1 in the bulk type, ln|det|, sign,
// t_u = tr(A^-1 L) with L read at Lphi[(e0 + e) * ldL + idx[u][o]]; the double inverse is
// also written to st_binv[u] when st_binv is not null.
template <class Tb>
__device__ __forceinline__ void lu_det_all(const SysDev& s, int sp, int lane, const double* PhiD, int ld,
                                           const Tb* Lphi, int ldL, const int* idx, int G, Tb* Bt, double* scr,
                                           double* ldet, double* dsg, double* tdet, double* st_binv) {
  const int n = s.n[sp], U = s.U[sp], e0 = sp ? s.Nup : 0;
  if (n == 0) {
    for (int u = lane; u < U; u += 32) {
      ldet[u] = 0.0;
      dsg[u] = 1.0;
      tdet[u] = 0.0;
    }
    __syncwarp();
    return;
  }
  const LaneGroup lgp(lane, G);
  const int ng = lgp.ng, g = lgp.g, gl = lgp.gl;
  double* A = scr + g * n * n;
  double* B = scr + ng * n * n + g * n * n;
  int* perm = reinterpret_cast<int*>(scr + 2 * ng * n * n) + g * n;
  for (int u0 = 0; u0 < U; u0 += ng) {
    const int u = u0 + g;
    const bool act = u < U;
    if (act && gl < n) {  // lane gl fills column (orbital slot) gl
      const int col = __ldg(idx + u * n + gl);
      for (int e = 0; e < n; ++e) A[e * n + gl] = PhiD[(e0 + e) * ld + col];
    }
    __syncwarp();
    double lg, sg;
    group_lu_inverse(A, B, perm, n, gl, G, act, lg, sg);
    __syncwarp();
    double t = 0.0;
    if (act && gl < n) {
      const int o = gl, col = __ldg(idx + u * n + o);
      for (int e = 0; e < n; ++e) t = fma(B[o * n + e], (double)Lphi[(e0 + e) * ldL + col], t);
    }
    t = group_sum(t, G);
    if (act) {
      for (int q = gl; q < n * n; q += G) {
        Bt[u * n * n + q] = (Tb)B[q];
        if (st_binv) st_binv[u * n * n + q] = B[q];
      }
      if (gl == 0) {
        ldet[u] = lg;
        dsg[u] = sg;
        tdet[u] = t;
      }
    }
    __syncwarp();
  }
}

template <class Tb>
__device__ __forceinline__ void det_body(const SysDev& s, const DetLayout& L, int w, unsigned char* base,
                                         const Tb* JG, const Tb* JL, const double* JS, const Tb* OB,
                                         const double* OD, double* __restrict__ logpsi,
                                         double* __restrict__ sgn_out, double* __restrict__ eloc,
                                         double* __restrict__ vg_ws, double* __restrict__ grad, Tb* __restrict__ Og,
                                         Tb* __restrict__ dELg, double* __restrict__ state_out,
                                         double* __restrict__ aux, const double* carry) {
  const int lane = threadIdx.x & 31;
  double* vg = reinterpret_cast<double*>(base + L.vg);
  Tb* G = reinterpret_cast<Tb*>(base + L.G);
  Tb* LJ = reinterpret_cast<Tb*>(base + L.LJ);
  double* PhiD = reinterpret_cast<double*>(base + L.PhiD);
  Tb* Lphi = reinterpret_cast<Tb*>(base + L.Lphi);
  Tb* Gphi = reinterpret_cast<Tb*>(base + L.Gphi);
  Tb* Bt[2] = {reinterpret_cast<Tb*>(base + L.Bt0), reinterpret_cast<Tb*>(base + L.Bt1)};
  double* ldet = reinterpret_cast<double*>(base + L.ldet);
  double* dsg = reinterpret_cast<double*>(base + L.dsg);
  double* tdet = reinterpret_cast<double*>(base + L.tdet);
  double* Wdet = reinterpret_cast<double*>(base + L.Wdet);
  double* Tdet = reinterpret_cast<double*>(base + L.Tdet);
  double* rk = reinterpret_cast<double*>(base + L.rk);
  unsigned char* scr = base + L.scratch;

  const int N = s.N, Nup = s.Nup, U0 = s.U[0];
  const int nev = s.n_ev, nevd = s.n_ev_det;
  // Jastrow results and orbitals from the workspace; dressed Laplacian L = lap phi + 2 grad lnJ . grad phi
  for (int q = lane; q < 3 * N; q += 32) G[q] = JG[(size_t)w * 3 * N + q];
  for (int q = lane; q < N; q += 32) LJ[q] = JL[(size_t)w * N + q];
  const double lnJ = JS[2 * (size_t)w], V = JS[2 * (size_t)w + 1];
  __syncwarp();
  // four (electron, orbital) entries per lane requested before the first is used (the
  // workspace comes from memory: one latency per four entries)
  for (DivStep eq(lane, nev); eq.hi < N;) {
    int ee[4], qq[4];
    Tb x[4], y[4], z[4], lp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ee[k] = eq.hi;
      qq[k] = eq.lo;
      if (eq.hi < N) {
        const Tb* ob = OB + ((size_t)w * N + eq.hi) * 5 * nev + eq.lo;
        x[k] = ob[nev];
        y[k] = ob[2 * nev];
        z[k] = ob[3 * nev];
        lp[k] = ob[4 * nev];
        eq.next(nev);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = ee[k], q = qq[k];
      if (e >= N) break;
      const Tb lq = lp[k] + (Tb)2 * (G[3 * e] * x[k] + G[3 * e + 1] * y[k] + G[3 * e + 2] * z[k]);
      Lphi[e * nev + q] = lq;
      if (q < nevd) {
        // PhiD: double orbital values for the LU, or with carried inverses (no LU) the dressed
        // Laplacians of the determinant orbitals widened once for the traces t_u
        PhiD[e * nevd + q] = carry ? (double)lq : OD[((size_t)w * N + e) * nevd + q];
        Gphi[(e * nevd + q) * 3] = x[k];
        Gphi[(e * nevd + q) * 3 + 1] = y[k];
        Gphi[(e * nevd + q) * 3 + 2] = z[k];
      }
    }
  }
  __syncwarp();

  // ---- C. Slater matrices: LU, inverses, ln|det|, t_u = tr(A^-1 L) ----
  // walker state: [Binv spin 0][Binv spin 1][ln|det| (Utot)][sign (Utot)][r_k (nterm)][ln|Phi|][sign]
  const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1];
  const int Utot = U0 + s.U[1];
  double lnPhi, sgnPhi;
  if (carry) {
    // inverses, term ratios and ln|Phi| carried by the sweep to these positions: no factorisation
    const double* cs = carry + (size_t)w * s.state_doubles;
    double* part = reinterpret_cast<double*>(scr);
    for (int sp = 0; sp < 2; ++sp) {
      const int n = s.n[sp], U = s.U[sp], e0 = sp ? Nup : 0, uo = sp ? U0 : 0;
      const double* Bc = cs + (sp ? nb0 : 0);
      warp_copy(Bt[sp], Bc, U * n * n, lane);
      // t_u = tr(B_u L_u): partial sums per (u, slot o), then per u
      for (int i = lane; i < U * n; i += 32) {
        const int u = i / n, o = i - u * n, col = __ldg(s.det_ev[sp] + u * n + o);
        const double* B = Bc + u * n * n + o * n;
        double t = 0.0;
        for (int e = 0; e < n; ++e) t = fma(B[e], PhiD[(e0 + e) * nevd + col], t);
        part[i] = t;
      }
      __syncwarp();
      for (int u = lane; u < U; u += 32) {
        double t = 0.0;
        for (int o = 0; o < n; ++o) t += part[u * n + o];
        tdet[uo + u] = t;
      }
      __syncwarp();
    }
    for (int k = lane; k < s.nterm; k += 32) rk[k] = cs[nb0 + nb1 + 2 * Utot + k];
    lnPhi = cs[nb0 + nb1 + 2 * Utot + s.nterm];
    sgnPhi = cs[nb0 + nb1 + 2 * Utot + s.nterm + 1];
    __syncwarp();
  } else {
    double* st = state_out ? state_out + (size_t)w * s.state_doubles : nullptr;
    lu_det_all<Tb>(s, 0, lane, PhiD, nevd, Lphi, nev, s.det_ev[0], L.G0, Bt[0], reinterpret_cast<double*>(scr), ldet,
                   dsg, tdet, st);
    lu_det_all<Tb>(s, 1, lane, PhiD, nevd, Lphi, nev, s.det_ev[1], L.G1, Bt[1], reinterpret_cast<double*>(scr),
                   ldet + U0, dsg + U0, tdet + U0, st ? st + nb0 : nullptr);
    term_ratios(s, lane, ldet, dsg, rk, lnPhi, sgnPhi);
    if (st) {
      for (int q = lane; q < Utot; q += 32) {
        st[nb0 + nb1 + q] = ldet[q];
        st[nb0 + nb1 + Utot + q] = dsg[q];
      }
      for (int k = lane; k < s.nterm; k += 32) st[nb0 + nb1 + 2 * Utot + k] = rk[k];
      if (lane == 0) {
        st[nb0 + nb1 + 2 * Utot + s.nterm] = lnPhi;
        st[nb0 + nb1 + 2 * Utot + s.nterm + 1] = sgnPhi;
      }
    }
  }
  // K[Phi] and the marginal weights W_u = sum_{k contains u} w_k, T_u = sum_{k contains u} w_k t_k
  double kphi = 0.0;
  for (int k = lane; k < s.nterm; k += 32) {
    const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
    kphi += __ldg(s.term_coef + k) * rk[k] * (tdet[a] + tdet[U0 + b]);
  }
  kphi = warp_sum(kphi);
  for (int ud = lane; ud < Utot; ud += 32) {
    double Wv = 0.0, Tv = 0.0;
    for (int t = __ldg(s.det_term_off + ud); t < __ldg(s.det_term_off + ud + 1); ++t) {
      const int k = __ldg(s.det_term + t);
      const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
      const double wk = __ldg(s.term_coef + k) * rk[k];
      Wv += wk;
      Tv += wk * (tdet[a] + tdet[U0 + b]);
    }
    // the rows below read W_u and T_u in the bulk type: converted here once per determinant
    // (a conversion costs a double instruction) instead of once per use by the whole warp
    reinterpret_cast<Tb*>(Wdet)[ud] = (Tb)Wv;
    reinterpret_cast<Tb*>(Tdet)[ud] = (Tb)Tv;
    if (aux) {
      aux[(size_t)w * (2 * Utot + 1) + ud] = Wv;
      aux[(size_t)w * (2 * Utot + 1) + Utot + ud] = Tv;
    }
  }
  if (aux && lane == 0) aux[(size_t)w * (2 * Utot + 1) + 2 * Utot] = kphi;
  __syncwarp();
  // Rows over the evaluation columns c < n_ev_det, one entry per electron of the spin:
  //   Gam_c = sum over determinants u holding column c (at slot o) of W_u B_u[o],
  // and, when orbital-excitation derivatives are wanted (D3 below),
  //   Aux_c = sum over the same u of (T_u B_u - W_u B_u L_u B_u)[o],
  // L_u the dressed Laplacians of u's own columns.
  const bool kap = Og && s.n_kappa > 0;
  Tb* Gam[2];
  Tb* Aux[2];
  Gam[0] = reinterpret_cast<Tb*>(scr);
  Gam[1] = Gam[0] + nevd * s.n[0];
  Aux[0] = Gam[1] + nevd * s.n[1];
  Aux[1] = Aux[0] + nevd * s.n[0];
  Tb* M = Aux[1] + nevd * s.n[1];
  double kin_loc = 0.0;
  if (kap) {
    for (int q = lane; q < 2 * nevd * N; q += 32) Gam[0][q] = (Tb)0;
    __syncwarp();
    for (int sp = 0; sp < 2; ++sp) {
      const int n = s.n[sp], e0 = sp ? Nup : 0, uo = sp ? U0 : 0;
      if (n == 0) continue;
      const int* ev_u = s.det_ev[sp];
      for (int u = 0; u < s.U[sp]; ++u) {
        const Tb* B = Bt[sp] + u * n * n;
        // M = B_u L_u
        for (DivStep oc(lane, n); oc.hi < n; oc.next(n)) {
          const int col = __ldg(ev_u + u * n + oc.lo);
          const Tb* Br = B + oc.hi * n;
          Tb m = 0;
          for (int e = 0; e < n; ++e) m += Br[e] * Lphi[(e0 + e) * nev + col];
          M[oc.hi * n + oc.lo] = m;
        }
        __syncwarp();
        const Tb Wu = reinterpret_cast<const Tb*>(Wdet)[uo + u], Tu = reinterpret_cast<const Tb*>(Tdet)[uo + u];
        for (DivStep oc(lane, n); oc.hi < n; oc.next(n)) {
          const int o = oc.hi, e = oc.lo, r = __ldg(ev_u + u * n + o) * n + e;
          const Tb b = B[o * n + e];
          Tb z = 0;
          for (int o2 = 0; o2 < n; ++o2) z += M[o * n + o2] * B[o2 * n + e];
          Gam[sp][r] += Wu * b;
          Aux[sp][r] += Tu * b - Wu * z;
        }
        __syncwarp();
      }
    }
    // grad_i ln|Psi| = grad_i lnJ + sum_c Gam_c[i] grad phi_c(r_i), in the bulk type
    for (int q = lane; q < 3 * N; q += 32) {
      const int e = q / 3, x = q - 3 * e;
      const int sp = e >= Nup ? 1 : 0, n = s.n[sp];
      const Tb* g = Gam[sp] + (e - (sp ? Nup : 0));
      const Tb* gp = Gphi + e * nevd * 3 + x;
      Tb acc = 0;
      for (int c = 0; c < nevd; ++c) acc += g[c * n] * gp[3 * c];
      vg[q] = (double)G[q] + (double)acc;
    }
  } else {
    // grad_i ln|Psi| = grad_i lnJ + sum_u W_u sum_o B_u[o][i] grad phi_o(r_i), in the bulk type
    for (int e = lane; e < N; e += 32) {
      const int sp = e >= Nup ? 1 : 0, ie = e - (sp ? Nup : 0), n = s.n[sp], uo = sp ? U0 : 0;
      const Tb* Bs = Bt[sp];
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
        const Tb Wu = reinterpret_cast<const Tb*>(Wdet)[uo + u];
        gx += Wu * ax;
        gy += Wu * ay;
        gz += Wu * az;
      }
      vg[3 * e] = (double)G[3 * e] + (double)gx;
      vg[3 * e + 1] = (double)G[3 * e + 1] + (double)gy;
      vg[3 * e + 2] = (double)G[3 * e + 2] + (double)gz;
    }
  }
  for (int e = lane; e < N; e += 32) {
    const double G0 = (double)G[3 * e], G1 = (double)G[3 * e + 1], G2 = (double)G[3 * e + 2];
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
  for (int q = lane; q < 3 * N; q += 32) {
    vg_ws[(size_t)w * 3 * N + q] = vg[q];
    if (grad) grad[(size_t)w * 3 * N + q] = vg[q];
  }
  if (!Og) return;

  // ---- D. parameter derivatives (the Jastrow parameters are done by the Jastrow kernel) ----
  const int P = s.P;
  Tb* Ow = Og + (size_t)w * P;
  Tb* Ew = dELg ? dELg + (size_t)w * P : nullptr;
  // D1. structure coefficients: O_I = Phi_I/Phi, E_L,I = -1/2 (K[Phi_I] - O_I K[Phi])
  for (int q = lane; q < s.n_cparam; q += 32) {
    double o = 0.0, kk = 0.0;
    for (int ts = __ldg(s.cpar_off + q); ts < __ldg(s.cpar_off + q + 1); ++ts) {
      const int t = __ldg(s.cpar_st + ts), k = __ldg(s.sterm_k + t);
      const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
      const double r = __ldg(s.sterm_d + t) * rk[k];
      o += r;
      kk += r * (tdet[a] + tdet[U0 + b]);
    }
    Ow[q] = (Tb)(o);
    if (Ew) Ew[q] = (Tb)(-0.5 * (kk - o * kphi));
  }
  // D3. orbital excitations kappa_kl (Sec. 2.2), phi_l -> phi_l + kappa phi_k.  For determinant u
  //   holding l at slot o (and not k): x_u = (B_u Phi)[o][k] = d ln D_u and
  //   y_u = (B_u L)[o][k] - (B_u L_u B_u Phi)[o][k] = d t_u.  Both vanish identically when u
  //   also holds k (B_u Phi has the unit vector there), so the sums over u factor through the
  //   rows Gam_l and Aux_l built above:
  //   O = sum_spin Gam_l . Phi_k,  K[Phi_kappa] = sum_u (T_u x_u + W_u y_u)
  //     = sum_spin (Aux_l . Phi_k + Gam_l . L_k),  E_L,kappa = -1/2 (K[Phi_kappa] - O K[Phi]).
  if (kap) {
    for (int j = lane; j < s.n_kappa; j += 32) {
      const int4 kx = __ldg(reinterpret_cast<const int4*>(s.kap_x) + j);
      const int kc = kx.z;
      Tb o = 0, kk = 0;
      for (int sp = 0; sp < 2; ++sp) {
        const int l = sp ? kx.y : kx.x;
        if (l < 0) continue;
        const int n = s.n[sp], e0 = sp ? Nup : 0;
        const Tb* g = Gam[sp] + l * n;
        const Tb* a = Aux[sp] + l * n;
        // orbital values from the workspace (not staged in shared memory: the walker region
        // then fits 16 walkers per SM)
        const Tb* pv = OB + ((size_t)w * N + e0) * 5 * nev + kc;
        // eight electrons' values requested before the first is used (the workspace rows are
        // mostly not cached by now: one memory latency per eight loads instead of per load)
        for (int eb = 0; eb < n; eb += 8) {
          Tb ph[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) ph[t] = eb + t < n ? pv[(size_t)(eb + t) * 5 * nev] : (Tb)0;
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (eb + t < n) {
              const int e = eb + t;
              const Tb lph = Lphi[(e0 + e) * nev + kc];
              o += g[e] * ph[t];
              kk += a[e] * ph[t] + g[e] * lph;
            }
        }
      }
      Ow[s.p_off_kappa + j] = o;
      if (Ew) Ew[s.p_off_kappa + j] = (Tb)-0.5 * (kk - o * (Tb)kphi);
    }
  }
}

}  // namespace

}  // namespace vbq
