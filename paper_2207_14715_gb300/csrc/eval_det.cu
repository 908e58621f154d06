// Determinant part of the evaluation and the evaluation driver (arXiv:2207.14715, Sec. 2.1,
// Sec. 2.2, Sec. 2.3.1).  One warp per walker:
//   C  Slater LU + inverses of every unique determinant (double), structure sum in the log
//      domain, E_L and grad ln|Psi|; optionally the walker state (inverses, ln|det|, signs)
//   D1 structure-coefficient derivatives; D3 orbital-excitation derivatives
// from the Jastrow and orbital results in the evaluation workspace.  The inverses are kept in
// shared memory in the bulk type only (the double inverses go straight to the walker state).
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
                                         const Tb* __restrict__ JG, const Tb* __restrict__ JL,
                                         const double* __restrict__ JS, const Tb* __restrict__ OB,
                                         const double* __restrict__ OD, double* __restrict__ logpsi,
                                         double* __restrict__ sgn_out, double* __restrict__ eloc,
                                         double* __restrict__ vg_ws, double* __restrict__ grad, Tb* __restrict__ Og,
                                         Tb* __restrict__ dELg, double* __restrict__ state_out,
                                         double* __restrict__ aux, const double* __restrict__ carry) {
  const int lane = threadIdx.x & 31;
  double* vg = reinterpret_cast<double*>(base + L.vg);
  Tb* G = reinterpret_cast<Tb*>(base + L.G);
  Tb* LJ = reinterpret_cast<Tb*>(base + L.LJ);
  Tb* Phi = reinterpret_cast<Tb*>(base + L.Phi);
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
  for (DivStep eq(lane, nev); eq.hi < N; eq.next(nev)) {
    const int e = eq.hi, q = eq.lo;
    const Tb* ob = OB + ((size_t)w * N + e) * 5 * nev;
    const Tb v = ob[q], x = ob[nev + q], y = ob[2 * nev + q], z = ob[3 * nev + q], lp = ob[4 * nev + q];
    const Tb lq = lp + (Tb)2 * (G[3 * e] * x + G[3 * e + 1] * y + G[3 * e + 2] * z);
    Lphi[e * nev + q] = lq;
    if (q < nevd) {
      // PhiD: double orbital values for the LU, or with carried inverses (no LU) the dressed
      // Laplacians of the determinant orbitals widened once for the traces t_u
      PhiD[e * nevd + q] = carry ? (double)lq : OD[((size_t)w * N + e) * nevd + q];
      Gphi[(e * nevd + q) * 3] = x;
      Gphi[(e * nevd + q) * 3 + 1] = y;
      Gphi[(e * nevd + q) * 3 + 2] = z;
    }
    Phi[e * nev + q] = v;
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
      for (int q = lane; q < U * n * n; q += 32) Bt[sp][q] = (Tb)Bc[q];
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
    Wdet[ud] = Wv;
    Tdet[ud] = Tv;
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
        const Tb Wu = (Tb)Wdet[uo + u], Tu = (Tb)Tdet[uo + u];
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
        const Tb Wu = (Tb)Wdet[uo + u];
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
        for (int e = 0; e < n; ++e) {
          const Tb ph = Phi[(e0 + e) * nev + kc], lph = Lphi[(e0 + e) * nev + kc];
          o += g[e] * ph;
          kk += a[e] * ph + g[e] * lph;
        }
      }
      Ow[s.p_off_kappa + j] = o;
      if (Ew) Ew[s.p_off_kappa + j] = (Tb)-0.5 * (kk - o * (Tb)kphi);
    }
  }
}

template <class Tb>
__global__ void __launch_bounds__(EvalBounds<Tb>::threads, 1)
    det_kernel(const SysDev s, const DetLayout L, int W, const Tb* __restrict__ JG, const Tb* __restrict__ JL,
               const double* __restrict__ JS, const Tb* __restrict__ OB, const double* __restrict__ OD,
               double* __restrict__ logpsi, double* __restrict__ sgn_out, double* __restrict__ eloc,
               double* __restrict__ vg_ws, double* __restrict__ grad, Tb* __restrict__ Og, Tb* __restrict__ dELg,
               double* __restrict__ state_out, double* __restrict__ aux, const double* __restrict__ carry) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  det_body<Tb>(s, L, w, smem + wl * L.warp_bytes, JG, JL, JS, OB, OD, logpsi, sgn_out, eloc, vg_ws, grad, Og, dELg,
               state_out, aux, carry);
}

template <class Tb>
__global__ void __launch_bounds__(EvalBounds<Tb>::threads, 1)
    det_batch_kernel(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items, int nitems,
                     const BatchCall* __restrict__ call) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    const bool d = call->derivs && b.O && b.dev.P > 0;
    det_body<Tb>(b.dev, b.lay.det, item.first + wl, smem + wl * b.lay.det.warp_bytes, static_cast<const Tb*>(b.JG),
                 static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD, b.logpsi, b.sign, b.eloc, b.VG,
                 nullptr, d ? static_cast<Tb*>(b.O) : nullptr, d ? static_cast<Tb*>(b.dEL) : nullptr, b.state,
                 nullptr, nullptr);
  }
}

}  // namespace

int make_det_layout(const SysDev& s, int tb, int max_smem, DetLayout& L, bool carried) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1];
  L.G0 = group_size(s.n[0]);
  L.G1 = group_size(s.n[1]);
  L.vg = take(8 * 3 * N);
  L.G = take(tb * 3 * N);
  L.LJ = take(tb * N);
  L.Phi = take(tb * N * s.n_ev);
  L.PhiD = take(8 * N * std::max(s.n_ev_det, 1));
  L.Lphi = take(tb * N * s.n_ev);
  L.Gphi = take(tb * N * s.n_ev_det * 3);
  L.Bt0 = take(tb * s.U[0] * s.n[0] * s.n[0]);
  L.Bt1 = take(tb * s.U[1] * s.n[1] * s.n[1]);
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.tdet = take(8 * Ut);
  L.Wdet = take(8 * Ut);
  L.Tdet = take(8 * Ut);
  L.rk = take(8 * s.nterm);
  int scr = 16;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], G = sp ? L.G1 : L.G0, ng = 32 / G;
    if (!carried) scr = std::max(scr, ng * (16 * n * n + 4 * n) + 16);  // LU: A, inverse, pivots per group
    scr = std::max(scr, 8 * s.U[sp] * n);                  // carried state: trace partials
  }
  // Gam and Aux rows of both spins, one product B_u L_u
  scr = std::max(scr, tb * (2 * std::max(s.n_ev_det, 1) * N + std::max(s.n[0] * s.n[0], s.n[1] * s.n[1])));
  L.scratch = take(scr);
  L.warp_bytes = off;
  int wpb = max_smem / off;
  const int cap = (tb == 8 ? EvalBounds<double>::threads : EvalBounds<float>::threads) / 32;
  if (wpb > cap) wpb = cap;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

namespace {
inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

EvalWs carve_eval_ws(const SysDev& s, int tb, int W, void* ws) {
  const size_t N = s.N, Wz = W;
  unsigned char* p = static_cast<unsigned char*>(ws);
  EvalWs r;
  auto take = [&](size_t b) {
    unsigned char* q = p;
    p += al256(b);
    return q;
  };
  r.JG = take(Wz * 3 * N * tb);
  r.JL = take(Wz * N * tb);
  r.JS = reinterpret_cast<double*>(take(Wz * 2 * 8));
  r.OB = take(Wz * N * 5 * s.n_ev * tb);
  r.OD = reinterpret_cast<double*>(take(Wz * N * std::max(s.n_ev_det, 1) * 8));
  r.VG = reinterpret_cast<double*>(take(Wz * 3 * N * 8));
  return r;
}

namespace {

template <class Tb>
cudaError_t launch_eval_t(const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi, double* sign,
                          double* eloc, double* grad, Tb* O, Tb* dEL, double* state_out, void* ws, cudaStream_t st,
                          int* nlaunch, cudaEvent_t* ev, double* aux, const double* carry) {
  const EvalWs b = carve_eval_ws(s, (int)sizeof(Tb), W, ws);
  *nlaunch = 0;
  auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], st) : cudaSuccess; };
  cudaError_t e = mark(0);
  if (e != cudaSuccess) return e;
  e = launch_jastrow<Tb>(s, L.jas, W, R, static_cast<Tb*>(b.JG), static_cast<Tb*>(b.JL), b.JS, st);
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(1)) != cudaSuccess) return e;
  e = launch_orbitals<Tb>(s, L.orb, W, R, static_cast<Tb*>(b.OB), carry ? nullptr : b.OD, st);
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(2)) != cudaSuccess) return e;
  if (s.msd) {
    e = launch_dettab<Tb>(s, L.tab, W, static_cast<const Tb*>(b.JG), static_cast<const Tb*>(b.JL), b.JS,
                          static_cast<const Tb*>(b.OB), b.OD, logpsi, sign, eloc, b.VG, grad, O, dEL, st);
  } else {
    const DetLayout& D = carry ? L.detc : L.det;
    const int smem = D.wpb * D.warp_bytes;
    e = cudaFuncSetAttribute(det_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    det_kernel<Tb><<<(W + D.wpb - 1) / D.wpb, 32 * D.wpb, smem, st>>>(
        s, D, W, static_cast<const Tb*>(b.JG), static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD,
        logpsi, sign, eloc, b.VG, grad, O, dEL, carry ? nullptr : state_out, aux, carry);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(3)) != cudaSuccess) return e;
  if (O && s.jas_param) {
    e = launch_jastrow_deriv<Tb>(s, L.jas, W, R, b.VG, O, dEL, st);
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return mark(4);
}

}  // namespace

template <class Tb>
cudaError_t launch_det_batch(const BatchSys* sys, const BatchItem* items, int nitems, const BatchCall* call, int grid,
                             int warps, int smem, cudaStream_t st) {
  det_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems, call);
  return cudaGetLastError();
}
int det_batch_grid(int is_float, int nitems, int warps, int smem, int persist) {
  return batch_grid(is_float ? (const void*)det_batch_kernel<float> : (const void*)det_batch_kernel<double>, nitems,
                    warps, smem, persist);
}
template cudaError_t launch_det_batch<float>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_det_batch<double>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                              cudaStream_t);

int make_eval_layout(const SysDev& s, int tb, int max_smem, EvalLayout& L) {
  int rc = make_jas_layout(s, tb, max_smem, L.jas);
  if (rc == VBQMC_OK) rc = make_orb_layout(s, tb, max_smem, L.orb);
  if (rc == VBQMC_OK)
    rc = s.msd ? make_dettab_layout(s, tb, max_smem, L.tab) : make_det_layout(s, tb, max_smem, L.det);
  if (rc == VBQMC_OK && !s.msd) rc = make_det_layout(s, tb, max_smem, L.detc, true);
  return rc;
}

size_t eval_workspace_bytes(const SysDev& s, int tb, int W) {
  const size_t N = s.N, Wz = std::max(W, 1);
  return al256(Wz * 3 * N * tb) + al256(Wz * N * tb) + al256(Wz * 2 * 8) + al256(Wz * N * 5 * s.n_ev * tb) +
         al256(Wz * N * std::max(s.n_ev_det, 1) * 8) + al256(Wz * 3 * N * 8);
}

cudaError_t launch_eval(int precision, const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                        double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out, void* ws,
                        cudaStream_t st, int* nlaunch, cudaEvent_t* ev, double* aux, const double* carry) {
  if (precision == VBQMC_MIXED)
    return launch_eval_t<float>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<float*>(O),
                                static_cast<float*>(dEL), state_out, ws, st, nlaunch, ev, aux, carry);
  return launch_eval_t<double>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<double*>(O),
                               static_cast<double*>(dEL), state_out, ws, st, nlaunch, ev, aux, carry);
}

}  // namespace vbq
