// Per-walker body of the determinant kernel on reference-determinant tables (arXiv:2207.14715,
// Sec. 2.1 determinant expansion): shared by the single-system and the fused batch kernels.
#pragma once

#include "walker_common.cuh"

namespace vbq {

namespace {

// det and inverse of the k x k leading block of M (k <= 4; the rest is treated as identity) by
// Gauss-Jordan elimination with partial pivoting, fully unrolled so that M stays in registers.
__device__ __forceinline__ double small_inverse(double M[4][4], double Mi[4][4], int k) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i >= k || j >= k) M[i][j] = (i == j) ? 1.0 : 0.0;
      Mi[i][j] = (i == j) ? 1.0 : 0.0;
    }
  double det = 1.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    // pivot: the largest |M[r][c]| for r >= c, swapped into row c (conditional swaps keep
    // every index static)
#pragma unroll
    for (int r = c + 1; r < 4; ++r)
      if (fabs(M[r][c]) > fabs(M[c][c])) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double t = M[c][j];
          M[c][j] = M[r][j];
          M[r][j] = t;
          t = Mi[c][j];
          Mi[c][j] = Mi[r][j];
          Mi[r][j] = t;
        }
        det = -det;
      }
    const double p = M[c][c];
    det *= p;
    if (p == 0.0) return 0.0;
    const double ip = 1.0 / p;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      M[c][j] *= ip;
      Mi[c][j] *= ip;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = M[r][c];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          M[r][j] = fma(-f, M[c][j], M[r][j]);
          Mi[r][j] = fma(-f, Mi[c][j], Mi[r][j]);
        }
      }
  }
  return det;
}

template <class Tb>
__device__ __forceinline__ void dettab_body(const SysDev& s, const DetTabLayout& L, int w, unsigned char* base,
                                            const Tb* JG, const Tb* JL, const double* JS, const Tb* OB,
                                            const double* OD, double* __restrict__ logpsi,
                                            double* __restrict__ sgn_out, double* __restrict__ eloc,
                                            double* __restrict__ vg_ws, double* __restrict__ grad,
                                            Tb* __restrict__ Og, Tb* __restrict__ dELg) {
  const int lane = threadIdx.x & 31;
  const int N = s.N, Nup = s.Nup, U0 = s.U[0], Utot = s.U[0] + s.U[1];
  const int nev = s.n_ev, nevd = s.n_ev_det;
  double* vg = reinterpret_cast<double*>(base + L.vg);
  double* Bd[2] = {reinterpret_cast<double*>(base + L.B0), reinterpret_cast<double*>(base + L.B1)};
  double* TX[2] = {reinterpret_cast<double*>(base + L.T0), reinterpret_cast<double*>(base + L.T1)};
  double* YH[2] = {reinterpret_cast<double*>(base + L.Y0), reinterpret_cast<double*>(base + L.Y1)};
  double* A = reinterpret_cast<double*>(base + L.A);
  double* Bs = reinterpret_cast<double*>(base + L.Bs);
  int* perm = reinterpret_cast<int*>(base + L.perm);
  double* Ls = reinterpret_cast<double*>(base + L.Ls);  // [n][nevd] dressed Laplacian of the spin's electrons
  double* ldet = reinterpret_cast<double*>(base + L.ldet);
  double* dsg = reinterpret_cast<double*>(base + L.dsg);
  double* tdet = reinterpret_cast<double*>(base + L.tdet);
  double* Wdet = reinterpret_cast<double*>(base + L.Wdet);
  double* rk = reinterpret_cast<double*>(base + L.rk);
  double* Minv = reinterpret_cast<double*>(base + L.Minv);  // per determinant its k x k minor inverse, packed
  double* Gam = reinterpret_cast<double*>(base + L.Gam);    // [n_x][n] of one spin: h = Gamma B
  Tb* G = reinterpret_cast<Tb*>(base + L.G);

  for (int q = lane; q < 3 * N; q += 32) G[q] = JG[(size_t)w * 3 * N + q];
  const double lnJ = JS[2 * (size_t)w], V = JS[2 * (size_t)w + 1];
  __syncwarp();

  // ---- per spin: reference LU, tables, every determinant's ratio and trace ----
  int moff_spin = 0;  // start of the spin's packed minor inverses
  int mstart[2] = {0, 0};
  for (int sp = 0; sp < 2; ++sp) {
    mstart[sp] = moff_spin;
    const int n = s.n[sp], e0 = sp ? Nup : 0, nx = s.n_x[sp], uo = sp ? U0 : 0;
    if (n == 0) {
      for (int u = lane; u < s.U[sp]; u += 32) {
        ldet[uo + u] = 0.0;
        dsg[uo + u] = 1.0;
        tdet[uo + u] = 0.0;
      }
      __syncwarp();
      continue;
    }
    const int* ref = s.det_ev[sp];
    const int* xl = s.tab_x[sp];
    int Gs = 1;
    while (Gs < n) Gs <<= 1;
    const LaneGroup lg(lane, Gs);
    const bool act = lg.g == 0;  // one group: n <= 32
    if (act && lg.gl < n) {
      const int col = __ldg(ref + lg.gl);
      for (int e = 0; e < n; ++e) A[e * n + lg.gl] = OD[((size_t)w * N + e0 + e) * nevd + col];
    }
    for (int i = lane; i < n * nevd; i += 32) {
      const int e = i / nevd, q = i - e * nevd;
      const Tb* ob = OB + ((size_t)w * N + e0 + e) * 5 * nev;
      const Tb* g = G + 3 * (e0 + e);
      Ls[i] = (double)ob[4 * nev + q] +
              2.0 * ((double)g[0] * (double)ob[nev + q] + (double)g[1] * (double)ob[2 * nev + q] +
                     (double)g[2] * (double)ob[3 * nev + q]);
    }
    __syncwarp();
    double lg0 = 0.0, sg0 = 1.0;
    double* B = Bd[sp];
    group_lu_inverse(A, B, perm, n, lg.gl, Gs, act, lg0, sg0);
    lg0 = __shfl_sync(kFull, lg0, 0);
    sg0 = __shfl_sync(kFull, sg0, 0);
    __syncwarp();
    // Y0 = B L_0 (into A), t0 = tr Y0
    for (int i = lane; i < n * n; i += 32) {
      const int o = i / n, o2 = i - o * n, col = __ldg(ref + o2);
      double y = 0.0;
      for (int e = 0; e < n; ++e) y = fma(B[o * n + e], Ls[e * nevd + col], y);
      A[i] = y;
    }
    __syncwarp();
    double t0 = 0.0;
    for (int o = lane; o < n; o += 32) t0 += A[o * n + o];
    t0 = warp_sum(t0);
    // T = B Phi_X, then Yhat = B L_X - Y0 T
    double* T = TX[sp];
    double* Yh = YH[sp];
    for (int i = lane; i < n * nx; i += 32) {
      const int o = i / nx, x = i - o * nx, col = __ldg(xl + x);
      double t = 0.0, y = 0.0;
      for (int e = 0; e < n; ++e) {
        const double b = B[o * n + e];
        t = fma(b, OD[((size_t)w * N + e0 + e) * nevd + col], t);
        y = fma(b, Ls[e * nevd + col], y);
      }
      T[i] = t;
      Yh[i] = y;
    }
    __syncwarp();
    for (int i = lane; i < n * nx; i += 32) {
      const int o = i / nx, x = i - o * nx;
      double y = Yh[i];
      for (int o2 = 0; o2 < n; ++o2) y = fma(-A[o * n + o2], T[o2 * nx + x], y);
      Bs[i] = y;
    }
    __syncwarp();
    for (int i = lane; i < n * nx; i += 32) Yh[i] = Bs[i];
    __syncwarp();
    // every determinant of the spin: lanes over determinants; the packed minor inverses start
    // at the running sum of k^2 (a scan over each round of 32 determinants)
    int mbase = moff_spin;
    for (int ub = 0; ub < s.U[sp]; ub += 32) {
      const int u = ub + lane;
      const int* tab = s.tab_det[sp] + (u < s.U[sp] ? u : 0) * kTabStride;
      const int k = u < s.U[sp] ? __ldg(tab) : 0;
      int incl = k * k;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int moff = mbase + incl - k * k;
      mbase += __shfl_sync(kFull, incl, 31);
      if (u >= s.U[sp]) continue;
      const double sgu = (double)__ldg(tab + 1);
      int S[kMaxExc], Q[kMaxExc];
#pragma unroll
      for (int j = 0; j < kMaxExc; ++j) {
        S[j] = j < k ? __ldg(tab + 2 + j) : 0;
        Q[j] = j < k ? __ldg(tab + 2 + kMaxExc + j) : 0;
      }
      double M[4][4], Mi[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) M[j][jp] = (j < k && jp < k) ? T[S[j] * nx + Q[jp]] : 0.0;
      const double dm = small_inverse(M, Mi, k);
      double tr = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp)
          if (j < k && jp < k) tr = fma(Mi[jp][j], Yh[S[j] * nx + Q[jp]], tr);
      const bool ok = dm != 0.0 && sg0 != 0.0;
      ldet[uo + u] = ok ? lg0 + log(fabs(dm)) : -INFINITY;
      dsg[uo + u] = ok ? sg0 * sgu * (dm > 0.0 ? 1.0 : -1.0) : 0.0;
      tdet[uo + u] = ok ? t0 + tr : 0.0;
      double* mo = Minv + moff;
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp)
          if (j < k && jp < k) mo[k * j + jp] = ok ? Mi[j][jp] : 0.0;
    }
    moff_spin = mbase;
    __syncwarp();
  }

  // ---- structure sum, K[Phi]/Phi and the marginal weights (as in the direct kernel) ----
  double lnPhi, sgnPhi;
  term_ratios(s, lane, ldet, dsg, rk, lnPhi, sgnPhi);
  double kphi = 0.0;
  for (int k = lane; k < s.nterm; k += 32) {
    const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
    kphi += __ldg(s.term_coef + k) * rk[k] * (tdet[a] + tdet[U0 + b]);
  }
  kphi = warp_sum(kphi);
  for (int ud = lane; ud < Utot; ud += 32) {
    double Wv = 0.0;
    for (int t = __ldg(s.det_term_off + ud); t < __ldg(s.det_term_off + ud + 1); ++t) {
      const int k = __ldg(s.det_term + t);
      Wv += __ldg(s.term_coef + k) * rk[k];
    }
    Wdet[ud] = Wv;
  }
  __syncwarp();

  // ---- grad_i ln|Phi| per spin through Gamma ----
  double kin_loc = 0.0;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], e0 = sp ? Nup : 0, nx = s.n_x[sp], uo = sp ? U0 : 0;
    if (n == 0) continue;
    const int* ref = s.det_ev[sp];
    const int* xl = s.tab_x[sp];
    double* B = Bd[sp];
    const double* T = TX[sp];
    // Gamma[x][o] = sum over determinants with o in S_u and x in Q_u of W_u (M_u^-1)[x][o]
    for (int i = lane; i < nx * n; i += 32) {
      const int x = i / n, o = i - x * n;
      double gsum = 0.0;
      const int k0 = __ldg(s.tab_det[sp]);
      int mo = mstart[sp] + k0 * k0;  // packed minor inverse of determinant u
      for (int u = 1; u < s.U[sp]; ++u) {
        const int* tab = s.tab_det[sp] + u * kTabStride;
        const int k = __ldg(tab);
        int jo = -1, jx = -1;
        for (int j = 0; j < k; ++j) {
          if (__ldg(tab + 2 + j) == o) jo = j;
          if (__ldg(tab + 2 + kMaxExc + j) == x) jx = j;
        }
        if (jo >= 0 && jx >= 0) gsum = fma(Wdet[uo + u], Minv[mo + k * jx + jo], gsum);
        mo += k * k;
      }
      A[i] = gsum;
    }
    __syncwarp();
    // h[x][i] = sum_o Gamma[x][o] B[o][i]
    for (int i = lane; i < nx * n; i += 32) {
      const int x = i / n, e = i - x * n;
      double h = 0.0;
      for (int o = 0; o < n; ++o) h = fma(A[x * n + o], B[o * n + e], h);
      Gam[i] = h;
    }
    __syncwarp();
    // grad_i ln|Phi| = sum_o B[o][i] grad phi_o + sum_x h[x][i] (grad phi_x - sum_o T[o][x] grad phi_o)
    //               = sum_o C[o][i] grad phi_o + sum_x h[x][i] grad phi_x,  C = B - T h
    // (C in double, in place of B, which is not read again; the sums in the bulk type: the
    // gradient feeds the drift and the Jastrow-parameter derivatives, not E_L)
    for (int i = lane; i < n * n; i += 32) {
      const int o = i / n, e = i - o * n;
      double c = B[i];
      for (int x = 0; x < nx; ++x) c = fma(-T[o * nx + x], Gam[x * n + e], c);
      B[i] = c;
    }
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
      const Tb* ob = OB + ((size_t)w * N + e0 + e) * 5 * nev;
      Tb g[3] = {0, 0, 0};
      for (int o = 0; o < n; ++o) {
        const int col = __ldg(ref + o);
        const Tb c = (Tb)B[o * n + e];
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] += c * ob[(1 + d) * nev + col];
      }
      for (int x = 0; x < nx; ++x) {
        const Tb h = (Tb)Gam[x * n + e];
        const int colx = __ldg(xl + x);
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] += h * ob[(1 + d) * nev + colx];
      }
      const int i = e0 + e;
      const double G0 = (double)G[3 * i], G1 = (double)G[3 * i + 1], G2 = (double)G[3 * i + 2];
      vg[3 * i] = G0 + (double)g[0];
      vg[3 * i + 1] = G1 + (double)g[1];
      vg[3 * i + 2] = G2 + (double)g[2];
      kin_loc += (double)JL[(size_t)w * N + i] + G0 * G0 + G1 * G1 + G2 * G2;
    }
    __syncwarp();
  }
  const double kin = warp_sum(kin_loc) + kphi;
  const double EL = -0.5 * kin + V;
  if (lane == 0) {
    logpsi[w] = lnJ + lnPhi;
    sgn_out[w] = sgnPhi;
    eloc[w] = EL;
  }
  __syncwarp();
  for (int q = lane; q < 3 * N; q += 32) {
    vg_ws[(size_t)w * 3 * N + q] = vg[q];
    if (grad) grad[(size_t)w * 3 * N + q] = vg[q];
  }
  if (!Og) return;
  // structure coefficients: O_I = Phi_I/Phi, E_L,I = -1/2 (K[Phi_I] - O_I K[Phi])
  const int P = s.P;
  Tb* Ow = Og + (size_t)w * P;
  Tb* Ew = dELg ? dELg + (size_t)w * P : nullptr;
  for (int q = lane; q < s.n_cparam; q += 32) {
    double o = 0.0, kk = 0.0;
    for (int ts = __ldg(s.cpar_off + q); ts < __ldg(s.cpar_off + q + 1); ++ts) {
      const int t = __ldg(s.cpar_st + ts), k = __ldg(s.sterm_k + t);
      const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
      const double r = __ldg(s.sterm_d + t) * rk[k];
      o += r;
      kk += r * (tdet[a] + tdet[U0 + b]);
    }
    Ow[q] = (Tb)o;
    if (Ew) Ew[q] = (Tb)(-0.5 * (kk - o * kphi));
  }
}

}  // namespace

}  // namespace vbq
