// Derivatives of ln|Psi| and E_L with respect to the nucleus positions, at fixed electron
// positions (arXiv:2207.14715, Sec. 2.3.1: E_L,j = dE_L/dp_j, here with p_j a nucleus
// coordinate R_{a,c}).  Moving nucleus a moves the basis functions centred on it, its e-n and
// e-e-n Jastrow terms and the potential.  Runs after an evaluation that left
// grad_i ln J and the orbital gradients/Laplacians in its workspace, the inverses in the walker
// state and the determinant weights W_u, T_u and K = K[Phi]/Phi in 'aux' (eval_det.cu).
// One block per walker: the walker's tables (positions, pair distances, inverses B_u and
// Z_u, orbital gradients) are shared by the block's warps, and each warp takes one nucleus.
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
// blocks per SM the kernel is compiled for: the float form fits two 6-warp blocks at 128
// registers; the double form keeps its larger working set in registers
template <class Tb> struct ForceBounds { static constexpr int min_blocks = 2; };
template <> struct ForceBounds<double> { static constexpr int min_blocks = 1; };

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

// exponent of axis d in component q of a shell of angular momentum L (s; x y z; xx yy zz xy xz yz)
__host__ __device__ constexpr int cart_e(int L, int q, int d) {
  return L == 0 ? 0
                : (L == 1 ? (q == d ? 1 : 0)
                          : (q < 3 ? (q == d ? 2 : 0)
                                   : (((q == 3 && d != 2) || (q == 4 && d != 1) || (q == 5 && d != 0)) ? 1 : 0)));
}
__host__ __device__ constexpr int ncomp_of(int L) { return L == 0 ? 1 : (L == 1 ? 3 : 6); }

// Polynomial parts p_n of the derivatives of g(x) = x^a e^{-z x^2}: g^(n) = p_n(x) e^{-z x^2},
//   p_0 = x^a,  p_1 = a x^{a-1} - 2 z x^{a+1},
//   p_2 = a(a-1) x^{a-2} - 2 z (2a+1) x^a + 4 z^2 x^{a+2},
//   p_3 = a(a-1)(a-2) x^{a-3} - 6 z a^2 x^{a-1} + 12 z^2 (a+1) x^{a+1} - 8 z^3 x^{a+3}
// (a <= 2 here, so the x^{a-3} term is absent).  pw[k] = x^k, k = 0..5.
template <int A, class Tb> __device__ __forceinline__ void gauss_1d(Tb z, const Tb pw[6], Tb p[4]) {
  const Tb z2 = z * z;
  p[0] = pw[A];
  p[1] = -(Tb)2 * z * pw[A + 1];
  p[2] = -(Tb)2 * z * (Tb)(2 * A + 1) * pw[A] + (Tb)4 * z2 * pw[A + 2];
  p[3] = (Tb)12 * z2 * (Tb)(A + 1) * pw[A + 1] - (Tb)8 * z2 * z * pw[A + 3];
  if constexpr (A >= 1) {
    p[1] += (Tb)A * pw[A - 1];
    p[3] -= (Tb)(6 * A * A) * z * pw[A - 1];
  }
  if constexpr (A >= 2) p[2] += (Tb)(A * (A - 1)) * pw[A - 2];
}

// The twelve derivatives of every component of shell sh (angular momentum L) at x = r - R_a:
// out[q][0..2] d_c chi, [3..8] Hessian (xx yy zz xy xz yz), [9..11] d_c lap chi.
template <int L, class Tb>
__device__ __forceinline__ void shell_d3(const SysDev& s, int sh, const Tb x[3], Tb* out) {
  const Tb z = shell_zeta<Tb>(s, sh);
  const Tb E = vexp(-z * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
  Tb p[3][L + 1][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Tb pw[6];
    pw[0] = (Tb)1;
#pragma unroll
    for (int k = 1; k < 6; ++k) pw[k] = pw[k - 1] * x[d];
    gauss_1d<0, Tb>(z, pw, p[d][0]);
    if constexpr (L >= 1) gauss_1d<1, Tb>(z, pw, p[d][1]);
    if constexpr (L >= 2) gauss_1d<2, Tb>(z, pw, p[d][2]);
  }
#pragma unroll
  for (int q = 0; q < ncomp_of(L); ++q) {
    const Tb nE = shell_norm<Tb>(s, sh, q) * E;
    const Tb* px = p[0][cart_e(L, q, 0)];
    const Tb* py = p[1][cart_e(L, q, 1)];
    const Tb* pz = p[2][cart_e(L, q, 2)];
    Tb* o = out + 12 * q;
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
// (m, l+m); d^a/dx^a xb^n = (-kappa)^a n (n+1)...(n+a-1) xb^{n+a}.  Per term, v[j] are the
// s,t derivatives of orders (1,0) (0,1) (2,0) (1,1) (3,0) (2,1) and U0, U1, U2 the u
// derivatives of orders 0, 1, 2, all without their (-kappa) factors.
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
  Tb a[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) a[i] = (Tb)0;
  een_for_each([&](auto tc) {
    constexpr int q = decltype(tc)::value;
    constexpr int k = een_klm(q).k, A = een_klm(q).l + een_klm(q).m, B = een_klm(q).m;
    const Tb cq = __ldg(c + q);
    const Tb v0 = cq * ((Tb)rising(A, 1) * sp[A + 1] * tp[B] + (Tb)rising(B, 1) * sp[B + 1] * tp[A]);
    const Tb v1 = cq * ((Tb)rising(B, 1) * sp[A] * tp[B + 1] + (Tb)rising(A, 1) * sp[B] * tp[A + 1]);
    const Tb v2 = cq * ((Tb)rising(A, 2) * sp[A + 2] * tp[B] + (Tb)rising(B, 2) * sp[B + 2] * tp[A]);
    const Tb v3 = cq * ((Tb)(rising(A, 1) * rising(B, 1)) * (sp[A + 1] * tp[B + 1] + sp[B + 1] * tp[A + 1]));
    const Tb v4 = cq * ((Tb)rising(A, 3) * sp[A + 3] * tp[B] + (Tb)rising(B, 3) * sp[B + 3] * tp[A]);
    const Tb v5 = cq * ((Tb)(rising(A, 2) * rising(B, 1)) * sp[A + 2] * tp[B + 1] +
                        (Tb)(rising(B, 2) * rising(A, 1)) * sp[B + 2] * tp[A + 1]);
    const Tb U0 = up[k];
    a[0] += U0 * v0;   // s
    a[1] += U0 * v1;   // t
    a[4] += U0 * v2;   // ss
    a[5] += U0 * v3;   // st
    a[10] += U0 * v4;  // sss
    a[11] += U0 * v5;  // sst
    if constexpr (k >= 1) {
      const Tb U1 = (Tb)k * up[k + 1], U2 = (Tb)(k * (k + 1)) * up[k + 2];
      a[2] += U1 * v0;  // us
      a[3] += U1 * v1;  // ut
      a[6] += U2 * v0;  // uus
      a[7] += U2 * v1;  // uut
      a[8] += U1 * v2;  // uss
      a[9] += U1 * v3;  // ust
    }
  });
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
__device__ __forceinline__ int hslot(int d, int c) { return d == c ? d : 2 + d + c; }

// Block = one walker; warp wid takes nuclei a = wid, wid + nwarps, ...
template <class Tb>
__device__ __forceinline__ void force_body(const SysDev& s, const ForceLayout& L, int w, unsigned char* sm,
                                           const double* __restrict__ Rg, const Tb* __restrict__ JG,
                                           const Tb* __restrict__ OB, const double* __restrict__ state,
                                           const double* __restrict__ aux, double* __restrict__ dlp,
                                           double* __restrict__ dEL) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int N = s.N, Nn = s.Nn, Nup = s.Nup, nev = s.n_ev, nevd = s.n_ev_det;
  const int U0 = s.U[0], Utot = s.U[0] + s.U[1];
  const int nb0 = s.U[0] * s.n[0] * s.n[0], nb1 = s.U[1] * s.n[1] * s.n[1];
  // block-shared tables
  double* R = reinterpret_cast<double*>(sm + L.R);
  double* wt = reinterpret_cast<double*>(sm + L.wt);
  Tb* G = reinterpret_cast<Tb*>(sm + L.G);
  Tb* uE = reinterpret_cast<Tb*>(sm + L.uE);   // [N][N] r_ij
  Tb* uH = reinterpret_cast<Tb*>(sm + L.uH);   // [N][N][3] (r_i - r_j)/r_ij
  Tb* Gphi = reinterpret_cast<Tb*>(sm + L.Gphi);
  Tb* Ld = reinterpret_cast<Tb*>(sm + L.Ld);
  Tb* Bt = reinterpret_cast<Tb*>(sm + L.B);
  Tb* Zt = reinterpret_cast<Tb*>(sm + L.Z);
  // this warp's tables
  unsigned char* wb = sm + L.shared_bytes + wid * L.warp_bytes;
  Tb* D = reinterpret_cast<Tb*>(wb + L.D);      // [N][nevd][6]: t phi (3), t L (3)
  Tb* bd = reinterpret_cast<Tb*>(wb + L.bd);    // [Ec][max_mu][12]
  Tb* dG = reinterpret_cast<Tb*>(wb + L.dG);    // [N][3][3]
  Tb* dLJ = reinterpret_cast<Tb*>(wb + L.dLJ);  // [N][3]
  Tb* sN = reinterpret_cast<Tb*>(wb + L.sN);    // [N][4]: r_ia, (r_i - R_a)/r_ia
  Tb* Y = reinterpret_cast<Tb*>(wb + L.Y);      // [n][n] scratch of Z_u
  const Tb kap = (Tb)s.kappa;

  // ---- walker inputs (whole block) ----
  for (int i = tid; i < 3 * N; i += blockDim.x) {
    R[i] = Rg[(size_t)w * 3 * N + i];
    G[i] = JG[(size_t)w * 3 * N + i];
  }
  const double* st = state + (size_t)w * s.state_doubles;
  for (int i = tid; i < nb0 + nb1; i += blockDim.x) Bt[i] = (Tb)st[i];
  const double* ax = aux + (size_t)w * (2 * Utot + 1);
  for (int i = tid; i < 2 * Utot + 1; i += blockDim.x) wt[i] = ax[i];
  __syncthreads();
  for (int i = tid; i < N * N; i += blockDim.x) {
    const int e = i / N, j = i - e * N;
    const double dx = R[3 * e] - R[3 * j], dy = R[3 * e + 1] - R[3 * j + 1], dz = R[3 * e + 2] - R[3 * j + 2];
    const double r = e == j ? 1.0 : sqrt(dx * dx + dy * dy + dz * dz), ir = 1.0 / r;
    uE[i] = (Tb)r;
    uH[3 * i] = (Tb)(dx * ir);
    uH[3 * i + 1] = (Tb)(dy * ir);
    uH[3 * i + 2] = (Tb)(dz * ir);
  }
  // orbital gradients and the dressed Laplacian L = lap phi + 2 grad ln J . grad phi
  for (int i = tid; i < N * nevd; i += blockDim.x) {
    const int e = i / nevd, q = i - e * nevd;
    const Tb* ob = OB + ((size_t)w * N + e) * 5 * nev;
    const Tb gx = ob[nev + q], gy = ob[2 * nev + q], gz = ob[3 * nev + q];
    Gphi[3 * i] = gx;
    Gphi[3 * i + 1] = gy;
    Gphi[3 * i + 2] = gz;
    Ld[i] = ob[4 * nev + q] + (Tb)2 * (G[3 * e] * gx + G[3 * e + 1] * gy + G[3 * e + 2] * gz);
  }
  __syncthreads();
  // Z_u = B_u L_u B_u (B = A^-1 stored [o][e]; L_u[e][o] = L at column det_ev[u][o]), warps over determinants
  for (int ud = wid; ud < Utot; ud += nw) {
    const int sp = ud >= U0 ? 1 : 0, u = ud - (sp ? U0 : 0), n = s.n[sp], e0 = sp ? Nup : 0;
    const int* dev = s.det_ev[sp];
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
  __syncthreads();

  int Pe = 1;
  while (Pe < N && Pe < 32) Pe <<= 1;
  const int ngr = 32 / Pe;
  const Tb* cE = een_coefs<Tb>(s);
  const double kphi = wt[2 * Utot];
  const Tb* cf = orb_coefs<Tb>(s);

  for (int a = wid; a < Nn; a += nw) {
    const double Xa = __ldg(s.nuc4 + 4 * a), Ya = __ldg(s.nuc4 + 4 * a + 1), Za = __ldg(s.nuc4 + 4 * a + 2);
    // distances to nucleus a (double differences, then the bulk type)
    for (int i = lane; i < N; i += 32) {
      const double dx = R[3 * i] - Xa, dy = R[3 * i + 1] - Ya, dz = R[3 * i + 2] - Za;
      const double r = sqrt(dx * dx + dy * dy + dz * dz), ir = 1.0 / r;
      sN[4 * i] = (Tb)r;
      sN[4 * i + 1] = (Tb)(dx * ir);
      sN[4 * i + 2] = (Tb)(dy * ir);
      sN[4 * i + 3] = (Tb)(dz * ir);
    }
    __syncwarp();
    // ---- Jastrow tangents of nucleus a: t ln J, t grad_i ln J (dG[i][d][c]), t lap_i ln J ----
    Tb lnj[3] = {0, 0, 0};
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
        const Tb sv = sN[4 * e], is = (Tb)1 / sv;
        const Tb sh[3] = {sN[4 * e + 1], sN[4 * e + 2], sN[4 * e + 3]};
        if (gr == 0) {
          Tb f1, f2, f3;
          pade_d123<Tb>(en_coef_t<Tb>(s, a), sv, kap, f1, f2, f3);
          const Tb rad = f3 + (Tb)2 * f2 * is - (Tb)2 * f1 * is * is;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            lnj[d] -= f1 * sh[d];
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
            const Tb uv = uE[e * N + j], iu = (Tb)1 / uv, tv = sN[4 * j];
            const Tb uh[3] = {uH[3 * (e * N + j)], uH[3 * (e * N + j) + 1], uH[3 * (e * N + j) + 2]};
            const Tb sj[3] = {sN[4 * j + 1], sN[4 * j + 2], sN[4 * j + 3]};
            const EenPartials<Tb> f =
                een_partials<Tb>(c, (Tb)1 / ((Tb)1 + kap * uv), sb, (Tb)1 / ((Tb)1 + kap * tv), kap);
            const Tb us = uh[0] * sh[0] + uh[1] * sh[1] + uh[2] * sh[2];
            const Tb Xs = f.uus + (Tb)2 * f.us * iu + f.sss + (Tb)2 * f.ss * is - (Tb)2 * f.s * is * is +
                          (Tb)2 * f.uss * us;
            const Tb Xt = f.uut + (Tb)2 * f.ut * iu + f.sst + (Tb)2 * f.st * is + (Tb)2 * f.ust * us;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              // ordered pairs (e, j) and (j, e) both visit the unordered pair: half each
              lnj[d] -= (Tb)0.5 * (f.s * sh[d] + f.t * sj[d]);
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

    // ---- orbital tangents of nucleus a: D[i][q][0..2] t phi, [3..5] t L ----
    const int sh0 = __ldg(s.nuc_sh + 4 * a), sh1 = __ldg(s.nuc_sh + 4 * a + 1);
    const int mu0 = __ldg(s.nuc_sh + 4 * a + 2), mu1 = __ldg(s.nuc_sh + 4 * a + 3);
    const int nsh = sh1 - sh0;
    for (int ec = 0; ec < N; ec += L.Ec) {
      const int ne = min(L.Ec, N - ec);
      // basis derivatives of the shells of a at electrons ec .. ec+ne-1
      for (int it = lane; it < ne * nsh; it += 32) {
        const int el = it / nsh, sh = sh0 + (it - el * nsh), e = ec + el;
        const Tb x[3] = {(Tb)(R[3 * e] - Xa), (Tb)(R[3 * e + 1] - Ya), (Tb)(R[3 * e + 2] - Za)};
        Tb* o = bd + (el * L.max_mu + __ldg(s.sh_first + sh) - mu0) * 12;
        const int l = __ldg(s.sh_l + sh);
        if (l == 0)
          shell_d3<0, Tb>(s, sh, x, o);
        else if (l == 1)
          shell_d3<1, Tb>(s, sh, x, o);
        else
          shell_d3<2, Tb>(s, sh, x, o);
      }
      __syncwarp();
      // contraction with the coefficients of the orbitals on a's functions, and the dressing
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
        Tb* Dq = D + (e * nevd + q) * 6;
        const Tb* gp = Gphi + 3 * (e * nevd + q);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const Tb* tg = dG + 9 * e + 3 * d;
          Tb t = -acc[9 + d];
#pragma unroll
          for (int c = 0; c < 3; ++c) t += (Tb)2 * (tg[c] * gp[c] - G[3 * e + c] * acc[3 + hslot(d, c)]);
          Dq[d] = -acc[d];
          Dq[3 + d] = t;
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
          const Tb* Dq = D + ((e0 + e) * nevd + q) * 6;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            xp[d] += b * Dq[d];
            yp[d] += b * Dq[3 + d] - zz * Dq[d];
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
      const double tJ = warp_sum((double)lnj[d]);
      if (lane == 0) {
        dlp[((size_t)w * Nn + a) * 3 + d] = tJ + tl;
        if (dEL) dEL[((size_t)w * Nn + a) * 3 + d] = -0.5 * (tj + tk - tl * kphi) + tv;
      }
    }
    __syncwarp();
  }
}

template <class Tb>
__global__ void __launch_bounds__(32 * kForceMaxWarps, ForceBounds<Tb>::min_blocks)
    force_kernel(const SysDev s, const ForceLayout L, const double* __restrict__ Rg, const Tb* __restrict__ JG,
                 const Tb* __restrict__ OB, const double* __restrict__ state, const double* __restrict__ aux,
                 double* __restrict__ dlp, double* __restrict__ dEL) {
  extern __shared__ __align__(16) unsigned char smem[];
  force_body<Tb>(s, L, blockIdx.x, smem, Rg, JG, OB, state, aux, dlp, dEL);
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
  L.nwarps = std::max(1, std::min(s.Nn, kForceMaxWarps));
  L.max_mu = std::max(s.max_nuc_mu, 1);
  // electrons per chunk of basis derivatives: about 4 KB of table per warp
  L.Ec = std::max(1, std::min(N, 4096 / (12 * tb * L.max_mu)));
  L.R = take(8 * 3 * N);
  L.wt = take(8 * (2 * Ut + 1));
  L.G = take(tb * 3 * N);
  L.uE = take(tb * N * N);
  L.uH = take(tb * 3 * N * N);
  L.Gphi = take(tb * 3 * N * nevd);
  L.Ld = take(tb * N * nevd);
  L.B = take(tb * std::max(nb, 1));
  L.Z = take(tb * std::max(nb, 1));
  L.shared_bytes = off;
  off = 0;
  L.D = take(tb * 6 * N * nevd);
  L.bd = take(tb * 12 * L.Ec * L.max_mu);
  L.dG = take(tb * 9 * N);
  L.dLJ = take(tb * 3 * N);
  L.sN = take(tb * 4 * N);
  L.Y = take(tb * std::max(nmax * nmax, 1));
  L.warp_bytes = off;
  // fewer warps (each taking more nuclei) when the tables of one warp per nucleus do not fit
  while (L.nwarps > 1 && L.shared_bytes + L.nwarps * L.warp_bytes > max_smem) --L.nwarps;
  L.block_bytes = L.shared_bytes + L.nwarps * L.warp_bytes;
  return L.block_bytes <= max_smem ? VBQMC_OK : VBQMC_ERR_CAPACITY;
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
  const int smem = LF.block_bytes, threads = 32 * LF.nwarps;
  if (precision == VBQMC_MIXED) {
    e = cudaFuncSetAttribute(force_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    force_kernel<float><<<W, threads, smem, st>>>(s, LF, R, static_cast<const float*>(b.JG),
                                                  static_cast<const float*>(b.OB), state, aux, dlp, dEL);
  } else {
    e = cudaFuncSetAttribute(force_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    force_kernel<double><<<W, threads, smem, st>>>(s, LF, R, static_cast<const double*>(b.JG),
                                                   static_cast<const double*>(b.OB), state, aux, dlp, dEL);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) ++*nlaunch;
  return e;
}

}  // namespace vbq
