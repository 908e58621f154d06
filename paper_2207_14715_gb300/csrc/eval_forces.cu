// Derivatives of ln|Psi| and E_L with respect to the nucleus positions, at fixed electron
// positions (arXiv:2207.14715, Sec. 2.3.1: E_L,j = dE_L/dp_j, here with p_j a nucleus
// coordinate R_{a,c}).  Moving nucleus a moves the basis functions centred on it, its e-n and
// e-e-n Jastrow terms and the potential.  One warp per walker, after an evaluation that left
// grad_i ln J and the orbital gradients/Laplacians in its workspace, the inverses in the walker
// state and the determinant weights W_u, T_u and K = K[Phi]/Phi in 'aux' (eval_det.cu).
//
// For the tangent t = d/dR_{a,c}:
//   t ln|Psi| = t ln J + sum_u W_u x_u,             x_u = tr(A_u^-1 tA_u)
//   t E_L     = -1/2 [ sum_i (t lap_i ln J + 2 grad_i ln J . t grad_i ln J)
//                      + sum_u (T_u x_u + W_u y_u) - K sum_u W_u x_u ] + tV
//   y_u = t tr(A_u^-1 L_u) = tr(A_u^-1 tL_u) - tr(Z_u tA_u),   Z_u = A_u^-1 L_u A_u^-1,
// L the dressed Laplacian lap phi + 2 grad ln J . grad phi, so that
//   tL = t lap phi + 2 t(grad ln J) . grad phi + 2 grad ln J . t(grad phi).
// Orbital tangents: t phi_q(r_i) = -sum_{mu on a} lambda_{q mu} d_c chi_mu(r_i), and the same
// for grad phi (Hessian row c of chi) and lap phi (d_c lap chi); the Gaussian derivatives come
// from the 1-D factors x^n e^{-zeta x^2} up to third order.  Jastrow tangents: the terms of
// nucleus a depend on R_a only through r_ia and r_ja, so
//   t s = -s^_c (s = r_ia, s^ = (r_i - R_a)/s),   t s^ = -(e_c - s^ s^_c)/s,
// and t grad_i ln J, t lap_i ln J follow from the partial derivatives of f_en(s) and of
// f_een(u, s, t) (u = r_ij, t = r_ja) up to third order, written out below.
#include "walker_common.cuh"

namespace vbq {

namespace {

constexpr int kForceMaxWarps = 8;

template <class Tb> __device__ __forceinline__ Tb shell_zeta(const SysDev& s, int sh);
template <> __device__ __forceinline__ double shell_zeta<double>(const SysDev& s, int sh) { return __ldg(s.sh_zeta + sh); }
template <> __device__ __forceinline__ float shell_zeta<float>(const SysDev& s, int sh) { return __ldg(s.sh_zeta_f + sh); }
template <class Tb> __device__ __forceinline__ Tb shell_norm(const SysDev& s, int sh, int q);
template <> __device__ __forceinline__ double shell_norm<double>(const SysDev& s, int sh, int q) {
  return __ldg(s.sh_norm + 6 * sh + q);
}
template <> __device__ __forceinline__ float shell_norm<float>(const SysDev& s, int sh, int q) {
  return __ldg(s.sh_norm_f + 6 * sh + q);
}

// cartesian exponents of component q of a shell of angular momentum l (s; x y z; xx yy zz xy xz yz)
__device__ __forceinline__ void cart_exponents(int l, int q, int e[3]) {
  e[0] = e[1] = e[2] = 0;
  if (l == 1) {
    e[q] = 1;
  } else if (l == 2) {
    if (q < 3) {
      e[q] = 2;
    } else {
      const int a = q == 5 ? 1 : 0, b = q == 3 ? 1 : 2;
      e[a] = 1;
      e[b] = 1;
    }
  }
}

// Polynomial parts p_n of the derivatives of g(x) = x^a e^{-z x^2}: g^(n) = p_n(x) e^{-z x^2},
//   p_0 = x^a,  p_1 = a x^{a-1} - 2 z x^{a+1},
//   p_2 = a(a-1) x^{a-2} - 2 z (2a+1) x^a + 4 z^2 x^{a+2},
//   p_3 = a(a-1)(a-2) x^{a-3} - 6 z a^2 x^{a-1} + 12 z^2 (a+1) x^{a+1} - 8 z^3 x^{a+3}.
// pw[k] = x^k for k = 0..5; a <= 2.
template <class Tb> __device__ __forceinline__ void gauss_1d(int a, Tb z, const Tb pw[6], Tb p[4]) {
  const Tb z2 = z * z;
  const Tb am1 = a >= 1 ? pw[a - 1] : (Tb)0, am2 = a >= 2 ? pw[a - 2] : (Tb)0;
  p[0] = pw[a];
  p[1] = (Tb)a * am1 - (Tb)2 * z * pw[a + 1];
  p[2] = (Tb)(a * (a - 1)) * am2 - (Tb)2 * z * (Tb)(2 * a + 1) * pw[a] + (Tb)4 * z2 * pw[a + 2];
  p[3] = (Tb)(-6 * a * a) * z * am1 + (Tb)12 * z2 * (Tb)(a + 1) * pw[a + 1] - (Tb)8 * z2 * z * pw[a + 3];
}

// Padé + polynomial f(r) = g(R), R = r/(1 + kappa r), g(R) = a1 R/(1 + a2 R) + sum_p q_p R^p:
// first three derivatives with respect to r (chain rule with R' = 1/(1+kappa r)^2,
// R'' = -2 kappa/(1+kappa r)^3, R''' = 6 kappa^2/(1+kappa r)^4).
template <class Tb>
__device__ __forceinline__ void pade_d123(const PadeT<Tb>& c, Tb r, Tb kap, Tb& f1, Tb& f2, Tb& f3) {
  const Tb den = (Tb)1 / ((Tb)1 + kap * r), R = r * den;
  const Tb pd = (Tb)1 / ((Tb)1 + c.a2 * R), pd2 = pd * pd;
  const Tb R2 = R * R, R3 = R2 * R, R4 = R3 * R;
  const Tb g1 = c.a1 * pd2 + (Tb)2 * c.q[0] * R + (Tb)3 * c.q[1] * R2 + (Tb)4 * c.q[2] * R3 + (Tb)5 * c.q[3] * R4;
  const Tb g2 = (Tb)-2 * c.a1 * c.a2 * pd2 * pd + (Tb)2 * c.q[0] + (Tb)6 * c.q[1] * R + (Tb)12 * c.q[2] * R2 +
                (Tb)20 * c.q[3] * R3;
  const Tb g3 = (Tb)6 * c.a1 * c.a2 * c.a2 * pd2 * pd2 + (Tb)6 * c.q[1] + (Tb)24 * c.q[2] * R + (Tb)60 * c.q[3] * R2;
  const Tb R1 = den * den, Rr2 = (Tb)-2 * kap * R1 * den, Rr3 = (Tb)6 * kap * kap * R1 * R1;
  f1 = g1 * R1;
  f2 = g2 * R1 * R1 + g1 * Rr2;
  f3 = g3 * R1 * R1 * R1 + (Tb)3 * g2 * R1 * Rr2 + g1 * Rr3;
}

// Partial derivatives of f_een(u, s, t) = sum_q c_q ub^k (sb^l + tb^l) (sb tb)^m, with
// xb = 1/(1 + kappa x), in the raw distances u = r_ij, s = r_ia, t = r_ja.
template <class Tb> struct EenPartials {
  Tb s, t, us, ut, ss, st, uus, uut, uss, ust, sss, sst;
};
__host__ __device__ constexpr int rising(int n, int a) {
  int r = 1;
  for (int i = 0; i < a; ++i) r *= n + i;
  return r;
}
// Each term is the sum of two separable monomials ub^k sb^A tb^B with (A, B) = (l+m, m) and
// (m, l+m); d^a/dx^a xb^n = (-kappa)^a n (n+1)...(n+a-1) xb^{n+a}.  S[k][j] collects, per
// power k of ub, the s,t derivatives of orders (1,0) (0,1) (2,0) (1,1) (3,0) (2,1) without
// their (-kappa) factors.
template <class Tb>
__device__ __forceinline__ EenPartials<Tb> een_partials(const Tb* c, Tb ub, Tb sb, Tb tb, Tb kap) {
  Tb up[7], sp[9], tp[7];
  up[0] = sp[0] = tp[0] = (Tb)1;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    sp[i] = sp[i - 1] * sb;
    if (i < 7) {
      up[i] = up[i - 1] * ub;
      tp[i] = tp[i - 1] * tb;
    }
  }
  Tb S[5][6];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int j = 0; j < 6; ++j) S[k][j] = (Tb)0;
  een_for_each([&](auto tc) {
    constexpr int q = decltype(tc)::value;
    constexpr int k = een_klm(q).k, A = een_klm(q).l + een_klm(q).m, B = een_klm(q).m;
    const Tb cq = __ldg(c + q);
    // (b, c) -> rising(A,b) rising(B,c) sb^{A+b} tb^{B+c} + rising(B,b) rising(A,c) sb^{B+b} tb^{A+c}
    S[k][0] += cq * ((Tb)rising(A, 1) * sp[A + 1] * tp[B] + (Tb)rising(B, 1) * sp[B + 1] * tp[A]);
    S[k][1] += cq * ((Tb)rising(B, 1) * sp[A] * tp[B + 1] + (Tb)rising(A, 1) * sp[B] * tp[A + 1]);
    S[k][2] += cq * ((Tb)rising(A, 2) * sp[A + 2] * tp[B] + (Tb)rising(B, 2) * sp[B + 2] * tp[A]);
    S[k][3] += cq * ((Tb)(rising(A, 1) * rising(B, 1)) * (sp[A + 1] * tp[B + 1] + sp[B + 1] * tp[A + 1]));
    S[k][4] += cq * ((Tb)rising(A, 3) * sp[A + 3] * tp[B] + (Tb)rising(B, 3) * sp[B + 3] * tp[A]);
    S[k][5] += cq * ((Tb)(rising(A, 2) * rising(B, 1)) * sp[A + 2] * tp[B + 1] +
                     (Tb)(rising(B, 2) * rising(A, 1)) * sp[B + 2] * tp[A + 1]);
  });
  // u factors: U0 = ub^k, U1 = k ub^{k+1}, U2 = k (k+1) ub^{k+2}
  Tb a[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) a[i] = (Tb)0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const Tb U0 = up[k], U1 = (Tb)k * up[k + 1], U2 = (Tb)(k * (k + 1)) * up[k + 2];
    a[0] += U0 * S[k][0];   // s
    a[1] += U0 * S[k][1];   // t
    a[2] += U1 * S[k][0];   // us
    a[3] += U1 * S[k][1];   // ut
    a[4] += U0 * S[k][2];   // ss
    a[5] += U0 * S[k][3];   // st
    a[6] += U2 * S[k][0];   // uus
    a[7] += U2 * S[k][1];   // uut
    a[8] += U1 * S[k][2];   // uss
    a[9] += U1 * S[k][3];   // ust
    a[10] += U0 * S[k][4];  // sss
    a[11] += U0 * S[k][5];  // sst
  }
  const Tb k1 = -kap, k2 = k1 * k1, k3 = k2 * k1;
  EenPartials<Tb> f;
  f.s = k1 * a[0];
  f.t = k1 * a[1];
  f.us = k2 * a[2];
  f.ut = k2 * a[3];
  f.ss = k2 * a[4];
  f.st = k2 * a[5];
  f.uus = k3 * a[6];
  f.uut = k3 * a[7];
  f.uss = k3 * a[8];
  f.ust = k3 * a[9];
  f.sss = k3 * a[10];
  f.sst = k3 * a[11];
  return f;
}

// symmetric 3x3 index -> slot of the Hessian (xx yy zz xy xz yz)
__device__ __forceinline__ int hslot(int d, int c) {
  if (d == c) return d;
  const int s = d + c;  // 1: xy, 2: xz, 3: yz
  return 2 + s;
}

template <class Tb>
__device__ __forceinline__ void force_body(const SysDev& s, const ForceLayout& L, int w, unsigned char* base,
                                           const double* __restrict__ Rg, const Tb* __restrict__ JG,
                                           const Tb* __restrict__ OB, const double* __restrict__ state,
                                           const double* __restrict__ aux, double* __restrict__ dlp,
                                           double* __restrict__ dEL) {
  const int lane = threadIdx.x & 31;
  const int N = s.N, Nn = s.Nn, Nup = s.Nup, nev = s.n_ev, nevd = s.n_ev_det;
  const int U0 = s.U[0], Utot = s.U[0] + s.U[1];
  const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1];
  double* R = reinterpret_cast<double*>(base + L.R);
  double* wt = reinterpret_cast<double*>(base + L.wt);
  Tb* G = reinterpret_cast<Tb*>(base + L.G);
  Tb* Gphi = reinterpret_cast<Tb*>(base + L.Gphi);
  Tb* Bt = reinterpret_cast<Tb*>(base + L.B);
  Tb* Zt = reinterpret_cast<Tb*>(base + L.Z);
  Tb* D = reinterpret_cast<Tb*>(base + L.D);
  Tb* bd = reinterpret_cast<Tb*>(base + L.bd);
  Tb* dG = reinterpret_cast<Tb*>(base + L.dG);
  Tb* dLJ = reinterpret_cast<Tb*>(base + L.dLJ);
  const Tb kap = (Tb)s.kappa;

  // ---- walker inputs ----
  for (int i = lane; i < 3 * N; i += 32) {
    R[i] = Rg[(size_t)w * 3 * N + i];
    G[i] = JG[(size_t)w * 3 * N + i];
  }
  const double* st = state + (size_t)w * s.state_doubles;
  for (int i = lane; i < nb0 + nb1; i += 32) Bt[i] = (Tb)st[i];
  const double* ax = aux + (size_t)w * (2 * Utot + 1);
  for (int i = lane; i < 2 * Utot + 1; i += 32) wt[i] = ax[i];
  __syncwarp();
  // orbital gradients and the dressed Laplacian L (in D, before D is used for the tangents)
  Tb* Ld = D;
  for (int i = lane; i < N * nevd; i += 32) {
    const int e = i / nevd, q = i - e * nevd;
    const Tb* ob = OB + ((size_t)w * N + e) * 5 * nev;
    const Tb gx = ob[nev + q], gy = ob[2 * nev + q], gz = ob[3 * nev + q];
    Gphi[3 * i] = gx;
    Gphi[3 * i + 1] = gy;
    Gphi[3 * i + 2] = gz;
    Ld[i] = ob[4 * nev + q] + (Tb)2 * (G[3 * e] * gx + G[3 * e + 1] * gy + G[3 * e + 2] * gz);
  }
  __syncwarp();
  // Z_u = B_u L_u B_u (B = A^-1 stored [o][e]; L_u[e][o] = L at column det_ev[u][o])
  Tb* Y = D + N * nevd;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], e0 = sp ? Nup : 0;
    const int* dev = s.det_ev[sp];
    for (int u = 0; u < s.U[sp]; ++u) {
      const Tb* B = Bt + (sp ? nb0 : 0) + u * n * n;
      Tb* Z = Zt + (sp ? nb0 : 0) + u * n * n;
      for (int i = lane; i < n * n; i += 32) {
        const int o = i / n, o2 = i - o * n, col = __ldg(dev + u * n + o2);
        Tb y = 0;
        for (int e = 0; e < n; ++e) y += B[o * n + e] * Ld[(e0 + e) * nevd + col];
        Y[i] = y;
      }
      __syncwarp();
      for (int i = lane; i < n * n; i += 32) {
        const int o = i / n, e = i - o * n;
        Tb z = 0;
        for (int o2 = 0; o2 < n; ++o2) z += Y[o * n + o2] * B[o2 * n + e];
        Z[i] = z;
      }
      __syncwarp();
    }
  }

  int Pe = 1;
  while (Pe < N && Pe < 32) Pe <<= 1;
  const int ngr = 32 / Pe;
  const Tb* cE = een_coefs<Tb>(s);
  const double kphi = wt[2 * Utot];

  for (int a = 0; a < Nn; ++a) {
    const double Xa = __ldg(s.nuc4 + 4 * a), Ya = __ldg(s.nuc4 + 4 * a + 1), Za = __ldg(s.nuc4 + 4 * a + 2);
    // ---- Jastrow tangents of nucleus a: t ln J, t grad_i ln J (dG[i][d][c]), t lap_i ln J ----
    double lnj[3] = {0.0, 0.0, 0.0};
    for (int eb = 0; eb < N; eb += Pe) {
      const int e = eb + (lane & (Pe - 1)), gr = lane / Pe;
      const bool act = e < N;
      Tb g[3][3], lj[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lj[d] = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) g[d][c] = 0;
      }
      if (act) {
        const double dx = R[3 * e] - Xa, dy = R[3 * e + 1] - Ya, dz = R[3 * e + 2] - Za;
        const double sd = sqrt(dx * dx + dy * dy + dz * dz);
        const Tb sv = (Tb)sd, is = (Tb)(1.0 / sd);
        const Tb sh[3] = {(Tb)(dx / sd), (Tb)(dy / sd), (Tb)(dz / sd)};
        if (gr == 0) {
          Tb f1, f2, f3;
          pade_d123<Tb>(en_coef_t<Tb>(s, a), sv, kap, f1, f2, f3);
          const Tb rad = f3 + (Tb)2 * f2 * is - (Tb)2 * f1 * is * is;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            lnj[d] -= (double)(f1 * sh[d]);
#pragma unroll
            for (int c = 0; c < 3; ++c)
              g[d][c] -= f2 * sh[d] * sh[c] + f1 * ((d == c ? (Tb)1 : (Tb)0) - sh[c] * sh[d]) * is;
            lj[d] -= rad * sh[d];
          }
        }
        if (s.een_on) {
          const Tb* c = cE + kNeen * __ldg(s.nuc_elem + a);
          const Tb sb = (Tb)1 / ((Tb)1 + kap * sv);
          for (int j = gr; j < N; j += ngr) {
            if (j == e) continue;
            const double ux = R[3 * e] - R[3 * j], uy = R[3 * e + 1] - R[3 * j + 1], uz = R[3 * e + 2] - R[3 * j + 2];
            const double ud = sqrt(ux * ux + uy * uy + uz * uz);
            const double tx = R[3 * j] - Xa, ty = R[3 * j + 1] - Ya, tz = R[3 * j + 2] - Za;
            const double td = sqrt(tx * tx + ty * ty + tz * tz);
            const Tb uv = (Tb)ud, iu = (Tb)(1.0 / ud), tv = (Tb)td;
            const Tb uh[3] = {(Tb)(ux / ud), (Tb)(uy / ud), (Tb)(uz / ud)};
            const Tb sj[3] = {(Tb)(tx / td), (Tb)(ty / td), (Tb)(tz / td)};
            const EenPartials<Tb> f =
                een_partials<Tb>(c, (Tb)1 / ((Tb)1 + kap * uv), sb, (Tb)1 / ((Tb)1 + kap * tv), kap);
            const Tb us = uh[0] * sh[0] + uh[1] * sh[1] + uh[2] * sh[2];
            const Tb Xs = f.uus + (Tb)2 * f.us * iu + f.sss + (Tb)2 * f.ss * is - (Tb)2 * f.s * is * is +
                          (Tb)2 * f.uss * us;
            const Tb Xt = f.uut + (Tb)2 * f.ut * iu + f.sst + (Tb)2 * f.st * is + (Tb)2 * f.ust * us;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              // ordered pairs (e, j) and (j, e) both visit the unordered pair: half each
              lnj[d] -= 0.5 * (double)(f.s * sh[d] + f.t * sj[d]);
              const Tb A = f.us * sh[d] + f.ut * sj[d], Bc = f.ss * sh[d] + f.st * sj[d];
#pragma unroll
              for (int cc = 0; cc < 3; ++cc)
                g[d][cc] -= A * uh[cc] + Bc * sh[cc] + f.s * ((d == cc ? (Tb)1 : (Tb)0) - sh[cc] * sh[d]) * is;
              lj[d] -= Xs * sh[d] + Xt * sj[d] + (Tb)2 * f.us * (uh[d] - us * sh[d]) * is;
            }
          }
        }
      }
      for (int o = Pe; o < 32; o <<= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          lj[d] += __shfl_xor_sync(kFull, lj[d], o);
#pragma unroll
          for (int c = 0; c < 3; ++c) g[d][c] += __shfl_xor_sync(kFull, g[d][c], o);
        }
      }
      if (act && gr == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dLJ[3 * e + d] = lj[d];
#pragma unroll
          for (int c = 0; c < 3; ++c) dG[9 * e + 3 * d + c] = g[d][c];
        }
      }
    }
    __syncwarp();

    // ---- orbital tangents of nucleus a: D[i][q][0..2] t phi, [3..8] t grad phi (Hessian
    //      slots), [9..11] t L (dressed Laplacian) ----
    const int sh0 = __ldg(s.nuc_sh + 4 * a), sh1 = __ldg(s.nuc_sh + 4 * a + 1);
    const int mu0 = __ldg(s.nuc_sh + 4 * a + 2), mu1 = __ldg(s.nuc_sh + 4 * a + 3);
    const int nsh = sh1 - sh0;
    for (int ec = 0; ec < N; ec += L.Ec) {
      const int ne = min(L.Ec, N - ec);
      // basis derivatives of the shells of a at electrons ec .. ec+ne-1
      for (int it = lane; it < ne * nsh; it += 32) {
        const int el = it / nsh, sh = sh0 + (it - el * nsh), e = ec + el;
        const int l = __ldg(s.sh_l + sh);
        const Tb z = shell_zeta<Tb>(s, sh);
        const Tb x[3] = {(Tb)(R[3 * e] - Xa), (Tb)(R[3 * e + 1] - Ya), (Tb)(R[3 * e + 2] - Za)};
        const Tb E = vexp(-z * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
        Tb p[3][3][4];  // [axis][power a][derivative order]
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          Tb pw[6];
          pw[0] = (Tb)1;
#pragma unroll
          for (int k = 1; k < 6; ++k) pw[k] = pw[k - 1] * x[d];
#pragma unroll
          for (int pa = 0; pa < 3; ++pa) gauss_1d<Tb>(pa, z, pw, p[d][pa]);
        }
        const int ncomp = l == 0 ? 1 : (l == 1 ? 3 : 6);
        const int mb = __ldg(s.sh_first + sh) - mu0;
        for (int q = 0; q < ncomp; ++q) {
          int ex[3];
          cart_exponents(l, q, ex);
          const Tb nE = shell_norm<Tb>(s, sh, q) * E;
          const Tb* px = p[0][ex[0]];
          const Tb* py = p[1][ex[1]];
          const Tb* pz = p[2][ex[2]];
          Tb* o = bd + (el * L.max_mu + mb + q) * 12;
          o[0] = nE * px[1] * py[0] * pz[0];
          o[1] = nE * px[0] * py[1] * pz[0];
          o[2] = nE * px[0] * py[0] * pz[1];
          o[3] = nE * px[2] * py[0] * pz[0];
          o[4] = nE * px[0] * py[2] * pz[0];
          o[5] = nE * px[0] * py[0] * pz[2];
          o[6] = nE * px[1] * py[1] * pz[0];
          o[7] = nE * px[1] * py[0] * pz[1];
          o[8] = nE * px[0] * py[1] * pz[1];
          o[9] = nE * (px[3] * py[0] * pz[0] + px[1] * (py[2] * pz[0] + py[0] * pz[2]));
          o[10] = nE * (py[3] * px[0] * pz[0] + py[1] * (px[2] * pz[0] + px[0] * pz[2]));
          o[11] = nE * (pz[3] * px[0] * py[0] + pz[1] * (px[2] * py[0] + px[0] * py[2]));
        }
      }
      __syncwarp();
      // contraction with the coefficients of the orbitals on a's functions, and the dressing
      const Tb* cf = orb_coefs<Tb>(s);
      for (int it = lane; it < ne * nevd; it += 32) {
        const int el = it / nevd, q = it - el * nevd, e = ec + el;
        const int k = __ldg(s.ev_orb + q), lo = __ldg(s.orb_lo + k), hi = __ldg(s.orb_hi + k);
        const int m0 = max(lo, mu0), m1 = min(hi, mu1);
        const Tb* cb = cf + __ldg(s.orb_off + k) - lo;
        Tb acc[12];
#pragma unroll
        for (int v = 0; v < 12; ++v) acc[v] = 0;
        for (int mu = m0; mu < m1; ++mu) {
          const Tb cm = __ldg(cb + mu);
          const Tb* b = bd + (el * L.max_mu + mu - mu0) * 12;
#pragma unroll
          for (int v = 0; v < 12; ++v) acc[v] += cm * b[v];
        }
        Tb* Dq = D + (e * nevd + q) * 12;
        const Tb* gp = Gphi + 3 * (e * nevd + q);
#pragma unroll
        for (int v = 0; v < 9; ++v) Dq[v] = -acc[v];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const Tb* tg = dG + 9 * e + 3 * d;
          Tb t = -acc[9 + d];
#pragma unroll
          for (int c = 0; c < 3; ++c) t += (Tb)2 * (tg[c] * gp[c] - G[3 * e + c] * acc[3 + hslot(d, c)]);
          Dq[9 + d] = t;
        }
      }
      __syncwarp();
    }

    // ---- determinant tangents: x_u, y_u summed with the weights ----
    double accL[3] = {0.0, 0.0, 0.0}, accK[3] = {0.0, 0.0, 0.0};
    for (int sp = 0; sp < 2; ++sp) {
      const int n = s.n[sp], e0 = sp ? Nup : 0, uo = sp ? U0 : 0;
      const int* dev = s.det_ev[sp];
      for (int it = lane; it < s.U[sp] * n; it += 32) {
        const int u = it / n, o = it - u * n, q = __ldg(dev + u * n + o);
        const Tb* B = Bt + (sp ? nb0 : 0) + u * n * n + o * n;
        const Tb* Z = Zt + (sp ? nb0 : 0) + u * n * n + o * n;
        Tb xp[3] = {0, 0, 0}, yp[3] = {0, 0, 0};
        for (int e = 0; e < n; ++e) {
          const Tb b = B[e], zz = Z[e];
          const Tb* Dq = D + ((e0 + e) * nevd + q) * 12;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            xp[d] += b * Dq[d];
            yp[d] += b * Dq[9 + d] - zz * Dq[d];
          }
        }
        const double Wu = wt[uo + u], Tu = wt[Utot + uo + u];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          accL[d] += Wu * (double)xp[d];
          accK[d] += Tu * (double)xp[d] + Wu * (double)yp[d];
        }
      }
    }
    // ---- Jastrow kinetic terms and the potential ----
    double jk[3] = {0.0, 0.0, 0.0}, dV[3] = {0.0, 0.0, 0.0};
    const double Zn = __ldg(s.nuc4 + 4 * a + 3);
    for (int e = lane; e < N; e += 32) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Tb* tg = dG + 9 * e + 3 * d;
        jk[d] += (double)(dLJ[3 * e + d] + (Tb)2 * (G[3 * e] * tg[0] + G[3 * e + 1] * tg[1] + G[3 * e + 2] * tg[2]));
      }
      const double dx = R[3 * e] - Xa, dy = R[3 * e + 1] - Ya, dz = R[3 * e + 2] - Za;
      const double r2 = dx * dx + dy * dy + dz * dz, ir3 = 1.0 / (r2 * sqrt(r2));
      dV[0] -= Zn * dx * ir3;
      dV[1] -= Zn * dy * ir3;
      dV[2] -= Zn * dz * ir3;
    }
    for (int b = lane; b < Nn; b += 32) {
      if (b == a) continue;
      const double dx = Xa - __ldg(s.nuc4 + 4 * b), dy = Ya - __ldg(s.nuc4 + 4 * b + 1),
                   dz = Za - __ldg(s.nuc4 + 4 * b + 2);
      const double r2 = dx * dx + dy * dy + dz * dz, f = Zn * __ldg(s.nuc4 + 4 * b + 3) / (r2 * sqrt(r2));
      dV[0] -= f * dx;
      dV[1] -= f * dy;
      dV[2] -= f * dz;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double tl = warp_sum(accL[d]), tk = warp_sum(accK[d]), tj = warp_sum(jk[d]), tv = warp_sum(dV[d]);
      const double tJ = warp_sum(lnj[d]);
      if (lane == 0) {
        dlp[((size_t)w * Nn + a) * 3 + d] = tJ + tl;
        if (dEL) dEL[((size_t)w * Nn + a) * 3 + d] = -0.5 * (tj + tk - tl * kphi) + tv;
      }
    }
    __syncwarp();
  }
}

template <class Tb>
__global__ void __launch_bounds__(32 * kForceMaxWarps, 1)
    force_kernel(const SysDev s, const ForceLayout L, int W, const double* __restrict__ Rg, const Tb* __restrict__ JG,
                 const Tb* __restrict__ OB, const double* __restrict__ state, const double* __restrict__ aux,
                 double* __restrict__ dlp, double* __restrict__ dEL) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  force_body<Tb>(s, L, w, smem + wl * L.warp_bytes, Rg, JG, OB, state, aux, dlp, dEL);
}

}  // namespace

int make_force_layout(const SysDev& s, int tb, int max_smem, ForceLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, nevd = std::max(s.n_ev_det, 1), Ut = s.U[0] + s.U[1];
  const int nb = s.U[0] * s.n[0] * s.n[0] + s.U[1] * s.n[1] * s.n[1];
  const int nmax = std::max(s.n[0], s.n[1]);
  L.max_mu = std::max(s.max_nuc_mu, 1);
  // electrons per chunk of basis derivatives: about 16 KB of table
  L.Ec = std::max(1, std::min(N, 16384 / (12 * tb * L.max_mu)));
  L.R = take(8 * 3 * N);
  L.wt = take(8 * (2 * Ut + 1));
  L.G = take(tb * 3 * N);
  L.Gphi = take(tb * 3 * N * nevd);
  L.B = take(tb * std::max(nb, 1));
  L.Z = take(tb * std::max(nb, 1));
  L.D = take(tb * std::max(12 * N * nevd, N * nevd + nmax * nmax));
  L.bd = take(tb * 12 * L.Ec * L.max_mu);
  L.dG = take(tb * 9 * N);
  L.dLJ = take(tb * 3 * N);
  L.warp_bytes = off;
  int wpb = max_smem / off;
  if (wpb > kForceMaxWarps) wpb = kForceMaxWarps;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

size_t force_workspace_bytes(const SysDev& s, int W) {
  const size_t Wz = std::max(W, 1), Ut = s.U[0] + s.U[1];
  return ((Wz * s.state_doubles * 8 + 255) & ~size_t(255)) + ((Wz * (2 * Ut + 1) * 8 + 255) & ~size_t(255));
}

cudaError_t launch_nuclear_derivs(int precision, const SysDev& s, const EvalLayout& LE, const ForceLayout& LF, int W,
                                  const double* R, double* logpsi, double* sign, double* eloc, double* dlp,
                                  double* dEL, void* ws, void* fws, cudaStream_t st, int* nlaunch) {
  const int tb = precision == VBQMC_MIXED ? 4 : 8;
  double* state = static_cast<double*>(fws);
  double* aux = reinterpret_cast<double*>(static_cast<unsigned char*>(fws) +
                                          (((size_t)std::max(W, 1) * s.state_doubles * 8 + 255) & ~size_t(255)));
  cudaError_t e = launch_eval(precision, s, LE, W, R, logpsi, sign, eloc, nullptr, nullptr, nullptr, state, ws, st,
                              nlaunch, nullptr, aux);
  if (e != cudaSuccess) return e;
  const EvalWs b = carve_eval_ws(s, tb, W, ws);
  const int smem = LF.wpb * LF.warp_bytes;
  const int grid = (W + LF.wpb - 1) / LF.wpb;
  if (precision == VBQMC_MIXED) {
    e = cudaFuncSetAttribute(force_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    force_kernel<float><<<grid, 32 * LF.wpb, smem, st>>>(s, LF, W, R, static_cast<const float*>(b.JG),
                                                          static_cast<const float*>(b.OB), state, aux, dlp, dEL);
  } else {
    e = cudaFuncSetAttribute(force_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    force_kernel<double><<<grid, 32 * LF.wpb, smem, st>>>(s, LF, W, R, static_cast<const double*>(b.JG),
                                                           static_cast<const double*>(b.OB), state, aux, dlp, dEL);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) ++*nlaunch;
  return e;
}

}  // namespace vbq
