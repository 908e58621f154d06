// Per-walker body of the VMC sweep (arXiv:2207.14715, Sec. 2.3.1): single-electron Metropolis
// moves with the determinants carried by per-determinant inverses or reference tables;
// shared by the single-system, batched and fused batch kernels.
#pragma once

#include "batch.h"
#include "walker_common.cuh"

namespace vbq {

// q_u = D_u / D_0 of a determinant u given by the reference-determinant tables: sign_u times
// the k x k determinant of T[S_u, Q_u] + b[S_u] c[Q_u]^T (k <= 4; b = null: T alone), by
// elimination with partial pivoting.  T [n][nx] row-major; td = the determinant's table row.
__device__ __forceinline__ double tab_ratio(const double* T, int nx, const int* __restrict__ td, const double* b,
                                            const double* c) {
  const int k = __ldg(td);
  double M[kMaxExc][kMaxExc];
#pragma unroll
  for (int i = 0; i < kMaxExc; ++i)
#pragma unroll
    for (int j = 0; j < kMaxExc; ++j) {
      double v = (i == j) ? 1.0 : 0.0;
      if (i < k && j < k) {
        const int si = __ldg(td + 2 + i), qj = __ldg(td + 2 + kMaxExc + j);
        v = T[si * nx + qj];
        if (b) v = fma(b[si], c[qj], v);
      }
      M[i][j] = v;
    }
  double det = (double)__ldg(td + 1);
#pragma unroll
  for (int col = 0; col < kMaxExc; ++col) {
#pragma unroll
    for (int r = col + 1; r < kMaxExc; ++r)
      if (fabs(M[r][col]) > fabs(M[col][col])) {
#pragma unroll
        for (int j = 0; j < kMaxExc; ++j) {
          const double t = M[col][j];
          M[col][j] = M[r][j];
          M[r][j] = t;
        }
        det = -det;
      }
    const double p = M[col][col];
    det *= p;
    if (p == 0.0) return 0.0;
    const double ip = 1.0 / p;
#pragma unroll
    for (int r = col + 1; r < kMaxExc; ++r) {
      const double f = M[r][col] * ip;
#pragma unroll
      for (int j = col + 1; j < kMaxExc; ++j) M[r][j] = fma(-f, M[col][j], M[r][j]);
    }
  }
  return det;
}

// =====================================================================================
// VMC sweep kernel
// =====================================================================================
// Two ways of carrying the determinants through the moves (template parameter TAB):
//  - per-determinant inverses (TAB = false): every unique determinant's inverse is updated by
//    Sherman-Morrison on an accepted move (Sec. 2.3.1); the ratio of determinant u is
//    rho_u = sum_o v_o Binv_u[o][i].
//  - reference-determinant tables (TAB = true; systems whose per-determinant inverses do not
//    fit in shared memory): each spin carries the inverse B of its reference determinant
//    (u = 0), T = B Phi_X over the orbitals X outside the reference, and q_u = D_u / D_0 =
//    sgn_u det T[S_u, Q_u].  Moving electron i to a point with orbital row v gives
//      rho_0 = sum_o v_o B[o][i],  c_x = v_x - sum_o v_o T[o][x],  b = B[:, i] / rho_0,
//      T' = T + b c^T,  q'_u = sgn_u det T'[S_u, Q_u],
//    and Phi'/Phi = rho_0 Sigma' / Sigma with Sigma = sum_k C_k q_up(k) q_dn(k); an accepted move
//    updates B by Sherman-Morrison, T to T' and q to q'.
// Each sweep moves every electron once (Sec. 2.3.1).  The determinant inverses come from
// the walker state written by the evaluation at the same positions, or from a fresh LU of
// double-precision orbital values (first sweep without state, and every 'refresh' sweeps).
// The proposed orbital row uses the bulk type; ratios and Sherman-Morrison updates are double.
// One warp, walker w, shared-memory region 'base' of L.warp_bytes bytes.
template <class Tb, bool TAB>
__device__ __forceinline__ void sweep_body(const SysDev& s, const SweepLayout& L, int w, unsigned char* base,
                                           double* __restrict__ Rg, int nsweeps, int refresh,
                                           double* __restrict__ state, int state_valid, double step, uint64_t seed,
                                           uint32_t step0, uint32_t tag, uint32_t woff, int* __restrict__ nacc) {
  const int lane = threadIdx.x & 31;
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
  double* rinv = reinterpret_cast<double*>(base + L.rinv);
  double* cvec = reinterpret_cast<double*>(base + L.cvec);
  double* scr = reinterpret_cast<double*>(base + L.scratch);
  // the pair distances r_ij are formed where a move needs them (the distances of the moving
  // electron, from the same coordinate differences the tables would hold)
  Tb* rEN = reinterpret_cast<Tb*>(base + L.geo);       // [N][Nn] r_ia
  // row strides padded by one so that lanes on different nuclei (powers) read different banks
  const int SA = s.N + 1, UP = s.N + 1;
  Tb* Sv = rEN + s.N * s.Nn;                            // [Nn][SA]: Rbar(r_ja) at a*SA + j (its powers formed where used)
  Tb* rnE = reinterpret_cast<Tb*>(base + L.geom);       // [N] r from the proposed position
  Tb* roE = rnE + s.N;                                  // [N] r from the current position
  Tb* rnN = roE + s.N;                                  // [Nn]
  Tb* Snew = rnN + s.Nn;                                // [Nn][6]
  Tb* Upo = Snew + 6 * s.Nn;                            // [5][UP] Rbar(r_ej)^k, current position of e
  Tb* Upn = Upo + 5 * UP;                               // [5][UP] Rbar(r_ej)^k, proposed position

  const int N = s.N, Nn = s.Nn, Nup = s.Nup, U0 = s.U[0], ldo = L.nocc_max;
  const Tb kap = (Tb)s.kappa;
  const Tb* cf = orb_coefs<Tb>(s);
  const Tb* cE = een_coefs<Tb>(s);
  for (int i = lane; i < 3 * N; i += 32) R[i] = Rg[(size_t)w * 3 * N + i];
  // positions as the bulk-type arithmetic reads them (float-float copies in the mixed form)
  dsf* Rds = reinterpret_cast<dsf*>(base + L.Rds);
  Coords<Tb> C;
  if constexpr (kSameType<Tb, double>) {
    C.R = R;
  } else {
    for (int i = lane; i < 3 * N; i += 32) Rds[i] = ds_from_double(Rg[(size_t)w * 3 * N + i]);
    C.R = Rds;
  }
  __syncwarp();
  // geometry tables
  for (DivStep ia(lane, Nn); ia.hi < N; ia.next(Nn)) {
    const int i = ia.hi, a = ia.lo, p = i * Nn + a;
    const Tb dx = C.en(s, i, a, 0), dy = C.en(s, i, a, 1), dz = C.en(s, i, a, 2);
    const Tb r = vsqrt(dx * dx + dy * dy + dz * dz);
    rEN[p] = r;
    Sv[a * SA + i] = (Tb)1 / ((Tb)1 + kap * r);
  }
  // walker state: [Binv spin 0][Binv spin 1][ln|det| (Ut)][sign (Ut)][r_k = D_k/Phi (nterm)]
  // [ln|Phi|][sign Phi]; the sweep starts from the inverses and the term ratios and carries
  // both (and ln|Phi|) through its moves
  const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1], Ut = U0 + s.U[1];
  double lnPhi = 0.0, sgnPhi = 1.0;
  // product of the accepted moves' |Phi'/Phi| since ln|Phi| was last set, as a mantissa in
  // [1, 2) and a binary exponent (bit operations; one logarithm per sweep instead of one per move)
  double pm = 1.0;
  int pe = 0;
  // reference-determinant tables (TAB): T per spin, q_u of both spins in wk, proposed q_u,
  // the move's c_x, and Sigma = sum_k C_k q_up q_dn
  double* Tt[2] = {reinterpret_cast<double*>(base + L.T0), reinterpret_cast<double*>(base + L.T1)};
  double* qn = reinterpret_cast<double*>(base + L.qn);
  double* cxv = reinterpret_cast<double*>(base + L.cx);
  double Sig = 1.0;
  const bool from_state = !TAB && state && state_valid;
  if (from_state) {
    const double* st = state + (size_t)w * s.state_doubles;
    warp_copy(Binv[0], st, nb0, lane);
    warp_copy(Binv[1], st + nb0, nb1, lane);
    warp_copy(wk, st + nb0 + nb1 + 2 * Ut, s.nterm, lane);
    lnPhi = st[nb0 + nb1 + 2 * Ut + s.nterm];
    sgnPhi = st[nb0 + nb1 + 2 * Ut + s.nterm + 1];
  }
  __syncwarp();
  int accepted = 0;
  const uint32_t wid = woff + (uint32_t)w;

  for (int sw = 0; sw < nsweeps; ++sw) {
    const bool do_refresh = (sw == 0) ? !from_state : (refresh > 0 && sw % refresh == 0);
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
      if constexpr (TAB) {
        // per spin: LU of the reference determinant, T = B Phi_X, every q_u
        for (int sp = 0; sp < 2; ++sp) {
          const int n = s.n[sp], e0 = sp ? Nup : 0, nx = s.n_x[sp], U = s.U[sp], uo = sp ? U0 : 0;
          if (n == 0) {
            for (int u = lane; u < U; u += 32) wk[uo + u] = 1.0;
            __syncwarp();
            continue;
          }
          int G = 1;
          while (G < n) G <<= 1;
          const LaneGroup lg(lane, G);
          const bool act = lg.g == 0;
          double* A = scr;
          int* perm = reinterpret_cast<int*>(scr + n * n);
          if (act && lg.gl < n) {
            const int col = __ldg(s.det_loc[sp] + lg.gl);
            for (int e = 0; e < n; ++e) A[e * n + lg.gl] = PhiO[(e0 + e) * ldo + col];
          }
          __syncwarp();
          double lgd, sgd;
          group_lu_inverse(A, Binv[sp], perm, n, lg.gl, G, act, lgd, sgd);
          const double* B = Binv[sp];
          for (int t = lane; t < n * nx; t += 32) {
            const int o = t / nx, x = t - o * nx, col = __ldg(s.tab_xl[sp] + x);
            double v = 0.0;
            for (int e = 0; e < n; ++e) v = fma(B[o * n + e], PhiO[(e0 + e) * ldo + col], v);
            Tt[sp][t] = v;
          }
          __syncwarp();
          for (int u = lane; u < U; u += 32)
            wk[uo + u] = tab_ratio(Tt[sp], nx, s.tab_det[sp] + u * kTabStride, nullptr, nullptr);
          __syncwarp();
        }
        double sg = 0.0;
        for (int k = lane; k < s.nterm; k += 32)
          sg = fma(__ldg(s.term_coef + k), wk[__ldg(s.term_det + 2 * k)] * wk[U0 + __ldg(s.term_det + 2 * k + 1)], sg);
        Sig = warp_sum(sg);
      } else {
        lu_all(s, 0, lane, PhiO, ldo, (const double*)nullptr, 0, s.det_loc[0], L.G0, Binv[0], scr, ldet, dsg,
               nullptr);
        lu_all(s, 1, lane, PhiO, ldo, (const double*)nullptr, 0, s.det_loc[1], L.G1, Binv[1], scr, ldet + U0,
               dsg + U0, nullptr);
      }
    }
    if (!TAB && do_refresh) {
      term_ratios(s, lane, ldet, dsg, wk, lnPhi, sgnPhi);  // wk: r_k = D_k / Phi
      pm = 1.0;
      pe = 0;
      __syncwarp();
    }
    const uint32_t st = step0 + (uint32_t)sw;
    // the sweep's random numbers, one electron per lane: the proposed position R_e + step
    // (2u - 1) per coordinate (electron e has not moved yet in this sweep when its turn comes)
    // and the acceptance uniform; in the mixed form also the float-float copy of the proposal
    double* rtab = reinterpret_cast<double*>(base + L.rtab);
    dsf* rtds = reinterpret_cast<dsf*>(base + L.rtds);
    for (int e = lane; e < N; e += 32) {
      double u[4];
      uniforms2(seed, wid, st, (uint32_t)e, tag, 0, u[0], u[1]);
      uniforms2(seed, wid, st, (uint32_t)e, tag, 1, u[2], u[3]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double x = __dadd_rn(R[3 * e + d], __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u[d]), 1.0)));
        rtab[4 * e + d] = x;
        if constexpr (!kSameType<Tb, double>) rtds[3 * e + d] = ds_from_double(x);
      }
      rtab[4 * e + 3] = u[3];
    }
    __syncwarp();
    for (int e = 0; e < N; ++e) {
      const int sp = e >= Nup ? 1 : 0, ie = e - (sp ? Nup : 0), n = s.n[sp], G = sp ? L.G1 : L.G0;
      const double uacc = rtab[4 * e + 3];
      const double rn[3] = {rtab[4 * e], rtab[4 * e + 1], rtab[4 * e + 2]};
      // the proposed position as the bulk-type arithmetic reads it
      dsf rnd[3];
      if constexpr (!kSameType<Tb, double>) {
        rnd[0] = rtds[3 * e];
        rnd[1] = rtds[3 * e + 1];
        rnd[2] = rtds[3 * e + 2];
      }
      auto dnew_e = [&](int j, int d) -> Tb {  // proposed position minus electron j
        if constexpr (kSameType<Tb, double>) return (Tb)(rn[d] - R[3 * j + d]);
        else return ds_diff_f(rnd[d], Rds[3 * j + d]);
      };
      auto dnew_n = [&](int a, int d) -> Tb {  // proposed position minus nucleus a
        if constexpr (kSameType<Tb, double>) return (Tb)(rn[d] - __ldg(s.nuc4 + 4 * a + d));
        else return ds_diff_f(rnd[d], nuc_coord_ds(s, a, d));
      };
      // orbital row at the proposed position (bulk type), contraction in balanced chunks
      if constexpr (kSameType<Tb, double>)
        basis_at<double, false>(s, lane, rn[0], rn[1], rn[2], bas, nullptr, nullptr, nullptr, nullptr);
      else
        basis_at_f<false>(s, lane, rnd, bas, nullptr, nullptr, nullptr, nullptr);
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
        if constexpr (kSameType<Tb, double>) vrowd[q] = v;
        else vrowd[q] = f2d_bits(v);
      }
      __syncwarp();
      const LaneGroup lgp(lane, G);
      const int U = s.U[sp], ng = lgp.ng, g = lgp.g, gl = lgp.gl;
      const int* dl = s.det_loc[sp];
      double rphi = 0.0, r0 = 0.0, Sig_new = 0.0;
      if constexpr (TAB) {
        // rho_0, c_x, b = B[:, i] / rho_0 (in cvec), the proposed q_u and Sigma'
        const int nx = s.n_x[sp], uo = sp ? U0 : 0;
        const double* B = Binv[sp];
        const double* T = Tt[sp];
        if (lane < n) r0 = vrowd[__ldg(dl + lane)] * B[lane * n + ie];
        r0 = warp_sum(r0);
        for (int x = lane; x < nx; x += 32) {
          double cc = vrowd[__ldg(s.tab_xl[sp] + x)];
          for (int o = 0; o < n; ++o) cc = fma(-vrowd[__ldg(dl + o)], T[o * nx + x], cc);
          cxv[x] = cc;
        }
        const double ir0 = r0 != 0.0 ? 1.0 / r0 : 0.0;
        if (lane < n) cvec[lane] = B[lane * n + ie] * ir0;
        __syncwarp();
        for (int u = lane; u < U; u += 32) qn[u] = tab_ratio(T, nx, s.tab_det[sp] + u * kTabStride, cvec, cxv);
        __syncwarp();
        double sg = 0.0;
        for (int k = lane; k < s.nterm; k += 32) {
          const int a = __ldg(s.term_det + 2 * k), b = __ldg(s.term_det + 2 * k + 1);
          const double qa = sp == 0 ? qn[a] : wk[a], qb = sp == 1 ? qn[b] : wk[U0 + b];
          sg = fma(__ldg(s.term_coef + k), qa * qb, sg);
        }
        Sig_new = warp_sum(sg);
        rphi = (r0 != 0.0 && Sig != 0.0) ? r0 * Sig_new / Sig : 0.0;
        if (!isfinite(rphi)) rphi = 0.0;  // an overflowing ratio is rejected (the tables are refreshed)
        (void)uo;
      }
      // determinant ratios rho_u = sum_o v_occ(o) Binv_u[o][ie], RG lanes per determinant.  With
      // one pass over the determinants (the usual case) the lanes' products are formed here and
      // reduced after the Jastrow distances below, whose float work then covers their latency.
      const int RG = sp ? L.RG1 : L.RG0;
      const LaneGroup lgr(lane, RG);
      const bool one_pass = U <= lgr.ng;
      const int ur = lgr.g;
      double rpart = 0.0;
      if constexpr (!TAB) {
        if (one_pass) {
          if (ur < U) {
            const double* Bu = Binv[sp] + ur * n * n + ie;
            const int* du = dl + ur * n;
            for (int o = lgr.gl; o < n; o += RG) rpart = fma(vrowd[__ldg(du + o)], Bu[o * n], rpart);
          }
        } else {
          for (int ub = 0; ub < U; ub += lgr.ng) {
            const int u = ub + lgr.g;
            double r = 0.0;
            if (u < U) {
              const double* Bu = Binv[sp] + u * n * n + ie;
              const int* du = dl + u * n;
              for (int o = lgr.gl; o < n; o += RG) r = fma(vrowd[__ldg(du + o)], Bu[o * n], r);
            }
            r = group_sum(r, RG);
            if (u < U && lgr.gl == 0) rho[u] = r;
          }
        }
      }
      // Jastrow change of the terms that involve electron e (Sec. 2.1): distances from the
      // proposed position, then items e-n (a), e-e (j) and e-e-n (a, k), the last through the
      // pair sums Y^{k,q} = sum_{j != e} u_ej^k s_j^q (the terms of e are s_e^A Y^{k,B} + s_e^B Y^{k,A}).
      for (int j = lane; j < N; j += 32) {
        const Tb dx = dnew_e(j, 0), dy = dnew_e(j, 1), dz = dnew_e(j, 2);
        const Tb rnew = j == e ? (Tb)0 : vsqrt(dx * dx + dy * dy + dz * dz);
        const Tb ox = C.ee(e, j, 0), oy = C.ee(e, j, 1), oz = C.ee(e, j, 2);
        const Tb rold = j == e ? (Tb)0 : vsqrt(ox * ox + oy * oy + oz * oz);
        rnE[j] = rnew;
        roE[j] = rold;
        const Tb uo = (Tb)1 / ((Tb)1 + kap * rold), un = (Tb)1 / ((Tb)1 + kap * rnew);
        Tb po = (Tb)1, pn = (Tb)1;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          Upo[k * UP + j] = po;
          Upn[k * UP + j] = pn;
          po *= uo;
          pn *= un;
        }
      }
      for (int a = lane; a < Nn; a += 32) {
        const Tb dx = dnew_n(a, 0), dy = dnew_n(a, 1), dz = dnew_n(a, 2);
        const Tb r = vsqrt(dx * dx + dy * dy + dz * dz);
        rnN[a] = r;
        const Tb sv = (Tb)1 / ((Tb)1 + kap * r);
        Tb pw = (Tb)1;
#pragma unroll
        for (int q = 0; q < 6; ++q) { Snew[a * 6 + q] = pw; pw *= sv; }
      }
      if constexpr (!TAB) {
        if (one_pass) {
          rpart = group_sum(rpart, RG);
          if (ur < U && lgr.gl == 0) rho[ur] = rpart;
        }
      }
      __syncwarp();
      if constexpr (!TAB) {
        // the structure sum's per-lane parts; they are reduced after the Jastrow change,
        // together with its sum: the double reduction's latency then overlaps the float work
        for (int k = lane; k < s.nterm; k += 32)
          rphi += __ldg(s.term_coef + k) * wk[k] * rho[__ldg(s.term_det + 2 * k + sp)];
      }
      Tb dj = 0;
      for (int t = lane; t < Nn + N; t += 32) {
        if (t < Nn) {
          const PadeT<Tb> c = en_coef_t<Tb>(s, t);
          Tb f1, f0, t0, t1;
          pade_eval<Tb, false>(c, rnN[t], kap, f1, t0, t1);
          pade_eval<Tb, false>(c, rEN[e * Nn + t], kap, f0, t0, t1);
          dj += f1 - f0;
        } else {
          const int j = t - Nn;
          if (j == e) continue;
          const PadeT<Tb> c = ee_coef_t<Tb>(s, (e < Nup) == (j < Nup));
          Tb f1, f0, t0, t1;
          pade_eval<Tb, false>(c, rnE[j], kap, f1, t0, t1);
          pade_eval<Tb, false>(c, roE[j], kap, f0, t0, t1);
          dj += f1 - f0;
        }
      }
      if (s.een_on) {
        // e-e-n items (nucleus a, part of the partners j), every k in each: the pair sums
        // are linear in the partners, so each part adds its own share of the change, and all
        // lanes run the same code (no divergence over k)
        const int np = max(1, 32 / Nn);
        for (int t = lane; t < np * Nn; t += 32) {
          const int a = t / np, part = t - np * a;
          Tb Yo[5][6], Yn[5][6];
#pragma unroll
          for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int q = 0; q < 6; ++q) Yo[k][q] = Yn[k][q] = (Tb)0;
          for (int j = part * N / np; j < (part + 1) * N / np; ++j) {
            if (j == e) continue;
            const Tb svj = Sv[a * SA + j];
            Tb sj[6];
            sj[0] = (Tb)1;
#pragma unroll
            for (int q = 1; q < 6; ++q) sj[q] = sj[q - 1] * svj;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              const Tb po = Upo[k * UP + j], pn = Upn[k * UP + j];
#pragma unroll
              for (int q = 0; q <= 5 - k; ++q) {
                Yo[k][q] += po * sj[q];
                Yn[k][q] += pn * sj[q];
              }
            }
          }
          Tb So[6];
          So[0] = (Tb)1;
          {
            const Tb sve = Sv[a * SA + e];
#pragma unroll
            for (int q = 1; q < 6; ++q) So[q] = So[q - 1] * sve;
          }
          const Tb* Sn = Snew + a * 6;
          const Tb* c = cE + kNeen * __ldg(s.nuc_elem + a);
          een_for_each([&](auto tc) {
            constexpr int q = decltype(tc)::value;
            constexpr int tk = een_klm(q).k, A = een_klm(q).l + een_klm(q).m, B = een_klm(q).m;
            dj += c[q] * ((Sn[A] * Yn[tk][B] + Sn[B] * Yn[tk][A]) - (So[A] * Yo[tk][B] + So[B] * Yo[tk][A]));
          });
        }
      }
      Tb dJ;
      if constexpr (TAB) {
        dJ = warp_sum(dj);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          rphi += __shfl_xor_sync(kFull, rphi, o);
          dj += __shfl_xor_sync(kFull, dj, o);
        }
        dJ = dj;
      }
      double ej;
      if constexpr (kSameType<Tb, double>) ej = vexp(2.0 * dJ);
      else ej = f2d_bits(vexp(2.0f * dJ));
      const double prob = rphi * rphi * ej;
      const bool acc = less_nonneg(uacc, prob);  // uacc in [0, 1), prob >= 0 or NaN
      if (TAB && acc) {
        // T <- T + b c^T; B <- B - b (v^T B - e_i^T) (b = B[:, i] / rho_0, lane j owns column j:
        // it reads only its own column before writing it); q <- q'
        const int nx = s.n_x[sp], uo = sp ? U0 : 0;
        double* T = Tt[sp];
        double* B = Binv[sp];
        for (int t = lane; t < n * nx; t += 32) {
          const int o = t / nx, x = t - o * nx;
          T[t] = fma(cvec[o], cxv[x], T[t]);
        }
        if (lane < n) {
          const int j = lane;
          double w = (j == ie) ? -1.0 : 0.0;
          for (int o = 0; o < n; ++o) w = fma(vrowd[__ldg(dl + o)], B[o * n + j], w);
          for (int o = 0; o < n; ++o) B[o * n + j] = fma(-cvec[o], w, B[o * n + j]);
        }
        for (int u = lane; u < U; u += 32) wk[uo + u] = qn[u];
        Sig = Sig_new;
        if (lane < 3) {
          R[3 * e + lane] = lane == 0 ? rn[0] : (lane == 1 ? rn[1] : rn[2]);
          if constexpr (!kSameType<Tb, double>) Rds[3 * e + lane] = lane == 0 ? rnd[0] : (lane == 1 ? rnd[1] : rnd[2]);
        }
        for (int a = lane; a < Nn; a += 32) {
          rEN[e * Nn + a] = rnN[a];
          Sv[a * SA + e] = Snew[a * 6 + 1];
        }
        ++accepted;
      } else if (!TAB && acc) {
        // the reciprocals 1/rho_u and 1/(Phi'/Phi), one per lane
        for (int q = lane; q <= U; q += 32) rinv[q] = recip(q < U ? rho[q] : rphi);
        __syncwarp();
        // Sherman-Morrison: Binv <- Binv - Binv[:, ie] (v^T Binv - e_ie^T) / rho, two lane-group
        // passes at a time (determinants u and u + ng): their row products are independent
        // chains, so each hides the other's latency without extra double instructions
        for (int ub = 0; ub < U; ub += 2 * ng) {
          const int ua = ub + g, uc = ub + ng + g;
          const bool aa = ua < U, ac = uc < U, two = ub + ng < U;  // ac implies aa; two: warp-uniform
          double* Ba = Binv[sp] + (aa ? ua : 0) * n * n;
          double* Bc = Binv[sp] + (ac ? uc : 0) * n * n;
          double* cva = cvec + g * n;
          double* cvc = cvec + (ng + g) * n;
          if (aa && gl < n) cva[gl] = Ba[gl * n + ie];
          if (ac && gl < n) cvc[gl] = Bc[gl * n + ie];
          const double ira = aa ? rinv[ua] : 0.0, irc = ac ? rinv[uc] : 0.0;
          __syncwarp();
          if (aa && gl < n) {
            const int j = gl;
            const int* da = dl + ua * n;
            const int* dc = dl + (ac ? uc : ua) * n;
            double wa = (j == ie) ? -1.0 : 0.0, wc = wa;
            if (two) {
              for (int o = 0; o < n; ++o) {
                wa = fma(vrowd[__ldg(da + o)], Ba[o * n + j], wa);
                if (ac) wc = fma(vrowd[__ldg(dc + o)], Bc[o * n + j], wc);
              }
            } else {
              for (int o = 0; o < n; ++o) wa = fma(vrowd[__ldg(da + o)], Ba[o * n + j], wa);
            }
            const double fa = wa * ira, fc = wc * irc;
            for (int o = 0; o < n; ++o) {
              Ba[o * n + j] = fma(-cva[o], fa, Ba[o * n + j]);
              if (ac) Bc[o * n + j] = fma(-cvc[o], fc, Bc[o * n + j]);
            }
          }
          __syncwarp();
        }
        const double irphi = rinv[U];
        {
          const long long b = __double_as_longlong(fabs(rphi) * pm);
          pe += (int)((b >> 52) & 0x7ff) - 1023;
          pm = __longlong_as_double((b & 0x800fffffffffffffLL) | (1023LL << 52));
        }
        // an accepted rphi is nonzero: its sign bit is its sign; flip sgnPhi's sign bit
        if (__double_as_longlong(rphi) < 0)
          sgnPhi = __longlong_as_double(__double_as_longlong(sgnPhi) ^ (long long)0x8000000000000000ull);
        for (int k = lane; k < s.nterm; k += 32) wk[k] *= rho[__ldg(s.term_det + 2 * k + sp)] * irphi;
        if (lane < 3) {
          R[3 * e + lane] = lane == 0 ? rn[0] : (lane == 1 ? rn[1] : rn[2]);
          if constexpr (!kSameType<Tb, double>) Rds[3 * e + lane] = lane == 0 ? rnd[0] : (lane == 1 ? rnd[1] : rnd[2]);
        }
        for (int a = lane; a < Nn; a += 32) {
          rEN[e * Nn + a] = rnN[a];
          Sv[a * SA + e] = Snew[a * 6 + 1];
        }
        ++accepted;
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < 3 * N; i += 32) Rg[(size_t)w * 3 * N + i] = R[i];
  if (nacc && lane == 0) nacc[w] += accepted;
  lnPhi += log(pm) + (double)pe * 0.69314718055994530942;  // ln 2
  if (!TAB && state) {  // the carried inverses, term ratios and ln|Phi| at the final positions
    double* st = state + (size_t)w * s.state_doubles;
    for (int q = lane; q < nb0; q += 32) st[q] = Binv[0][q];
    for (int q = lane; q < nb1; q += 32) st[nb0 + q] = Binv[1][q];
    for (int k = lane; k < s.nterm; k += 32) st[nb0 + nb1 + 2 * Ut + k] = wk[k];
    if (lane == 0) {
      st[nb0 + nb1 + 2 * Ut + s.nterm] = lnPhi;
      st[nb0 + nb1 + 2 * Ut + s.nterm + 1] = sgnPhi;
    }
  }
}

}  // namespace vbq
