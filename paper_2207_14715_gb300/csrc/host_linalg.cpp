// Host FP64 linear algebra of the library: the linear-method eigenproblem (Sec. 2.3.1,
// Eq. geneigeqM) and the structure weights (Sec. 2.4).  Both act on small matrices, (P+1)^2
// and Nvb^2, once per optimisation step or analysis, so they run on the host in double.
//
// Method of vbqmc_lin_solve.  The pencil of Eq. geneigeqM is
//     A = [[E0, gR^T/2], [gL/2, H + a I]],   B = [[1, 0], [0, S]],   A v = E B v,
// with S symmetric positive semi-definite.  S = U diag(s) U^T (Householder tridiagonal form,
// then implicit QR with Wilkinson shifts); the directions with s_i <= P eps max(s) carry no
// information (redundant parameters) and are dropped, X = U_k diag(s_k^-1/2).  With
// v = [y_0; X y'] the pencil becomes the standard nonsymmetric problem
//     C y = E y,   C = [[E0, gR^T X / 2], [X^T gL / 2, X^T (H + a I) X]],
// whose eigenvalues come from a Householder reduction to Hessenberg form and Francis
// double-shift QR.  The real eigenvalues are examined in ascending order.  The reduction
// multiplies by s_i^-1/2, which loses accuracy in the eigenvectors when S is ill-conditioned
// (near-redundant parameters), so each candidate's eigenvector is then taken from the pencil
// itself: inverse iteration v <- (A - sigma B)^-1 B v (LU with partial pivoting of the full
// (P+1)^2 matrix, sigma just off the eigenvalue) from the reduced problem's vector, and
// E = (Bv)^T A v / |Bv|^2 (the least-squares fit of A v = E B v).  The first candidate whose
// component v_0 holds at least 1e-3 of |v| is the answer, scaled to v_0 = 1: dp = v[1:] / v_0.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/vbqmc.h"

namespace vbq {
int set_error(int code, const std::string& msg);
}

namespace {

using Mat = std::vector<double>;  // row-major square matrices

constexpr double kEps = 2.220446049250313e-16;

// Symmetric eigendecomposition A = Q diag(d) Q^T of the n x n row-major matrix a (destroyed).
// Householder reduction to tridiagonal form with the reflections accumulated in Q, then
// implicit symmetric QR steps with Wilkinson shifts (each rotation applied to a window of the
// band and to the columns of Q).  Returns false if the QR iteration does not converge.
bool sym_eig(int n, Mat& a, std::vector<double>& d, Mat& q) {
  q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) q[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    // reflector H = I - 2 v v^T (|v| = 1) mapping a[k+1:, k] onto a multiple of e_{k+1}
    double xn = 0.0;
    for (int i = k + 1; i < n; ++i) xn += a[(size_t)i * n + k] * a[(size_t)i * n + k];
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    const double x0 = a[(size_t)(k + 1) * n + k];
    const double alpha = x0 >= 0.0 ? -xn : xn;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = a[(size_t)i * n + k] - (i == k + 1 ? alpha : 0.0);
      vn += v[i] * v[i];
    }
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    // trailing block: A <- A - 2 (v w^T + w v^T), p = A v, w = p - (v^T p) v
    double K = 0.0;
    for (int i = k + 1; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += a[(size_t)i * n + j] * v[j];
      p[i] = s;
      K += v[i] * s;
    }
    for (int i = k + 1; i < n; ++i) w[i] = p[i] - K * v[i];
    for (int i = k + 1; i < n; ++i)
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= 2.0 * (v[i] * w[j] + w[i] * v[j]);
    a[(size_t)(k + 1) * n + k] = a[(size_t)k * n + k + 1] = alpha;
    for (int i = k + 2; i < n; ++i) a[(size_t)i * n + k] = a[(size_t)k * n + i] = 0.0;
    // Q <- Q H on columns k+1..n-1
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += q[(size_t)r * n + j] * v[j];
      s *= 2.0;
      for (int j = k + 1; j < n; ++j) q[(size_t)r * n + j] -= s * v[j];
    }
  }
  d.assign(n, 0.0);
  std::vector<double> e(std::max(n - 1, 1), 0.0);
  for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)i * n + i + 1];

  int iter = 0;
  int m = n - 1;
  while (m > 0) {
    // deflate converged off-diagonal entries at the bottom
    if (std::fabs(e[m - 1]) <= kEps * (std::fabs(d[m - 1]) + std::fabs(d[m]))) {
      e[m - 1] = 0.0;
      --m;
      continue;
    }
    int l = m - 1;
    while (l > 0 && std::fabs(e[l - 1]) > kEps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
    if (l > 0) e[l - 1] = 0.0;
    if (++iter > 60 * n) return false;
    // Wilkinson shift from the trailing 2x2 block of [l, m]
    const double dl = 0.5 * (d[m - 1] - d[m]);
    const double em = e[m - 1];
    const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * std::hypot(dl, em);
    const double mu = d[m] - (den != 0.0 ? em * em / den : 0.0);
    double x = d[l] - mu, z = e[l];
    double bulge = 0.0;  // T[k+1][k-1] during the chase
    for (int k = l; k < m; ++k) {
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
      // window [j0, j1] of the band around rows k, k+1: dense copy, G T G^T, write back
      const int j0 = std::max(k - 1, l), j1 = std::min(k + 2, m);
      double T[4][4] = {};
      const int nw = j1 - j0 + 1;
      for (int i = 0; i < nw; ++i) {
        const int gi = j0 + i;
        T[i][i] = d[gi];
        if (i + 1 < nw) T[i][i + 1] = T[i + 1][i] = e[gi];
      }
      if (k > l) {  // bulge at (k+1, k-1)
        const int bi = k + 1 - j0, bj = k - 1 - j0;
        T[bi][bj] = T[bj][bi] = bulge;
      }
      const int rk = k - j0;
      for (int col = 0; col < nw; ++col) {
        const double t0 = T[rk][col], t1 = T[rk + 1][col];
        T[rk][col] = c * t0 + s * t1;
        T[rk + 1][col] = -s * t0 + c * t1;
      }
      for (int row = 0; row < nw; ++row) {
        const double t0 = T[row][rk], t1 = T[row][rk + 1];
        T[row][rk] = c * t0 + s * t1;
        T[row][rk + 1] = -s * t0 + c * t1;
      }
      for (int i = 0; i < nw; ++i) {
        d[j0 + i] = T[i][i];
        if (i + 1 < nw) e[j0 + i] = T[i][i + 1];
      }
      if (k > l) e[k - 1] = T[rk][rk - 1];  // the bulge has been moved into the band
      bulge = (k + 2 <= m) ? T[rk + 2][rk] : 0.0;
      if (k + 2 <= m) {
        x = e[k];
        z = bulge;
      }
      for (int row = 0; row < n; ++row) {
        const double q0 = q[(size_t)row * n + k], q1 = q[(size_t)row * n + k + 1];
        q[(size_t)row * n + k] = c * q0 + s * q1;
        q[(size_t)row * n + k + 1] = -s * q0 + c * q1;
      }
    }
  }
  return true;
}

// Eigenvalues (wr + i wi) of the n x n row-major matrix h (destroyed): Householder reduction to
// upper Hessenberg form, then Francis double-shift QR steps on the active block with
// deflation of 1x1 and 2x2 blocks.  Returns false if the iteration does not converge.
bool hess_eigvals(int n, Mat& h, std::vector<double>& wr, std::vector<double>& wi) {
  auto H = [&](int i, int j) -> double& { return h[(size_t)i * n + j]; };
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0.0;
    for (int i = k + 1; i < n; ++i) xn += H(i, k) * H(i, k);
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    const double alpha = H(k + 1, k) >= 0.0 ? -xn : xn;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = H(i, k) - (i == k + 1 ? alpha : 0.0);
      vn += v[i] * v[i];
    }
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    for (int j = 0; j < n; ++j) {  // rows: H <- (I - 2vv^T) H
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * H(i, j);
      s *= 2.0;
      for (int i = k + 1; i < n; ++i) H(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {  // columns: H <- H (I - 2vv^T)
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += H(i, j) * v[j];
      s *= 2.0;
      for (int j = k + 1; j < n; ++j) H(i, j) -= s * v[j];
    }
    for (int i = k + 2; i < n; ++i) H(i, k) = 0.0;
  }
  wr.assign(n, 0.0);
  wi.assign(n, 0.0);
  // applies the reflector I - 2 u u^T (u of length len, |u| = 1) to rows r0.. and columns c0..
  auto refl_rows = [&](const double* u, int len, int r0, int c0, int c1) {
    for (int j = c0; j <= c1; ++j) {
      double s = 0.0;
      for (int t = 0; t < len; ++t) s += u[t] * H(r0 + t, j);
      s *= 2.0;
      for (int t = 0; t < len; ++t) H(r0 + t, j) -= s * u[t];
    }
  };
  auto refl_cols = [&](const double* u, int len, int c0, int r0, int r1) {
    for (int i = r0; i <= r1; ++i) {
      double s = 0.0;
      for (int t = 0; t < len; ++t) s += H(i, c0 + t) * u[t];
      s *= 2.0;
      for (int t = 0; t < len; ++t) H(i, c0 + t) -= s * u[t];
    }
  };
  auto make_refl = [](double* x, int len) -> bool {  // x -> unit u with (I - 2uu^T) x = alpha e_0
    double xn = 0.0;
    for (int t = 0; t < len; ++t) xn += x[t] * x[t];
    xn = std::sqrt(xn);
    if (xn == 0.0) return false;
    x[0] -= x[0] >= 0.0 ? -xn : xn;
    double un = 0.0;
    for (int t = 0; t < len; ++t) un += x[t] * x[t];
    un = std::sqrt(un);
    if (un == 0.0) return false;
    for (int t = 0; t < len; ++t) x[t] /= un;
    return true;
  };
  int m = n - 1, its = 0, total = 0;
  while (m >= 0) {
    if (m == 0) {
      wr[0] = H(0, 0);
      --m;
      continue;
    }
    int l = m;
    while (l > 0) {
      const double sc = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
      if (std::fabs(H(l, l - 1)) <= kEps * (sc == 0.0 ? 1.0 : sc)) break;
      --l;
    }
    if (l > 0) H(l, l - 1) = 0.0;
    if (l == m) {  // 1x1 block
      wr[m] = H(m, m);
      --m;
      its = 0;
      continue;
    }
    if (l == m - 1) {  // 2x2 block: roots of its characteristic polynomial
      const double a = H(m - 1, m - 1), b = H(m - 1, m), c = H(m, m - 1), dd = H(m, m);
      const double tr = 0.5 * (a + dd), det = a * dd - b * c;
      const double disc = tr * tr - det;
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        const double r1 = tr + (tr >= 0.0 ? sq : -sq);
        const double r2 = r1 != 0.0 ? det / r1 : tr - (tr >= 0.0 ? sq : -sq);
        wr[m - 1] = r1;
        wr[m] = r2;
      } else {
        const double sq = std::sqrt(-disc);
        wr[m - 1] = wr[m] = tr;
        wi[m - 1] = sq;
        wi[m] = -sq;
      }
      m -= 2;
      its = 0;
      continue;
    }
    if (++total > 100 * n) return false;
    ++its;
    // shifts: eigenvalues of the trailing 2x2 block (trace s, determinant t); exceptional
    // shifts after 10 and 20 steps without deflation
    double s, t;
    if (its % 10 == 0) {
      const double ex = std::fabs(H(m, m - 1)) + std::fabs(H(m - 1, m - 2));
      s = 1.5 * ex + H(m, m);
      t = ex * ex;
    } else {
      s = H(m - 1, m - 1) + H(m, m);
      t = H(m - 1, m - 1) * H(m, m) - H(m - 1, m) * H(m, m - 1);
    }
    double x[3];
    x[0] = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
    x[1] = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
    x[2] = H(l + 1, l) * H(l + 2, l + 1);
    for (int k = l; k <= m - 2; ++k) {
      double u[3] = {x[0], x[1], x[2]};
      if (make_refl(u, 3)) {
        refl_rows(u, 3, k, std::max(l, k - 1), m);
        refl_cols(u, 3, k, l, std::min(k + 3, m));
      }
      x[0] = H(k + 1, k);
      x[1] = H(k + 2, k);
      if (k < m - 2) x[2] = H(k + 3, k);
    }
    double u[2] = {x[0], x[1]};
    if (make_refl(u, 2)) {
      refl_rows(u, 2, m - 1, m - 2, m);
      refl_cols(u, 2, m - 1, l, m);
    }
  }
  return true;
}

// Solves (C - lam I) y = b in place for the n x n matrix c by LU with partial pivoting;
// a zero pivot is replaced by eps |C| (the shifted matrix is singular by construction).
void shifted_solve(int n, const Mat& c, double lam, double cnorm, std::vector<double>& b) {
  Mat a(c);
  for (int i = 0; i < n; ++i) a[(size_t)i * n + i] -= lam;
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + k]) > std::fabs(a[(size_t)p * n + k])) p = i;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    double& pk = a[(size_t)k * n + k];
    if (std::fabs(pk) < kEps * cnorm) pk = (pk >= 0.0 ? 1.0 : -1.0) * kEps * cnorm;
    for (int i = k + 1; i < n; ++i) {
      const double f = a[(size_t)i * n + k] / pk;
      a[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
    }
  }
  for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
    b[i] /= a[(size_t)i * n + i];
  }
}

// LU factorisation with partial pivoting of the n x n row-major matrix a (in place); pivots
// below tiny are replaced by +-tiny (the matrix is singular by construction in inverse iteration).
void lu_factor(int n, Mat& a, std::vector<int>& piv, double tiny) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + k]) > std::fabs(a[(size_t)p * n + k])) p = i;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    double& pk = a[(size_t)k * n + k];
    if (std::fabs(pk) < tiny) pk = (pk >= 0.0 ? 1.0 : -1.0) * tiny;
    for (int i = k + 1; i < n; ++i) {
      const double f = a[(size_t)i * n + k] / pk;
      a[(size_t)i * n + k] = f;
      if (f != 0.0)
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
    }
  }
}

void lu_solve(int n, const Mat& a, const std::vector<int>& piv, std::vector<double>& b) {
  for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
    b[i] /= a[(size_t)i * n + i];
  }
}

bool all_finite(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

}  // namespace

extern "C" {

int vbqmc_lin_solve(int P, double E0, const double* gL, const double* gR, const double* H, const double* S,
                    double shift, double* dp, double* e_lin) {
  if (P < 1 || !gL || !gR || !H || !S || !dp || !e_lin) return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: bad argument");
  const size_t PP = (size_t)P * P;
  if (!std::isfinite(E0) || !std::isfinite(shift) || !all_finite(gL, P) || !all_finite(gR, P) || !all_finite(H, PP) ||
      !all_finite(S, PP))
    return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: non-finite input");
  // S = U diag(s) U^T on its symmetric part
  Mat a(PP);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) a[(size_t)i * P + j] = 0.5 * (S[(size_t)i * P + j] + S[(size_t)j * P + i]);
  std::vector<double> s;
  Mat U;
  if (!sym_eig(P, a, s, U)) return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: eigendecomposition of S did not converge");
  double smax = 0.0;
  for (double x : s) smax = std::max(smax, x);
  if (!(smax > 0.0)) return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: S has no positive eigenvalue");
  std::vector<int> keep;
  for (int i = 0; i < P; ++i)
    if (s[i] > P * kEps * smax) keep.push_back(i);
  const int k = (int)keep.size(), n = k + 1;
  Mat X((size_t)P * k);  // X = U_k diag(s_k^-1/2), P x k
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < k; ++c) X[(size_t)r * k + c] = U[(size_t)r * P + keep[c]] / std::sqrt(s[keep[c]]);
  // C = [[E0, gR^T X / 2], [X^T gL / 2, X^T (H + shift I) X]]
  Mat HX((size_t)P * k, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      const double hij = H[(size_t)i * P + j] + (i == j ? shift : 0.0);
      if (hij == 0.0) continue;
      const double* xr = &X[(size_t)j * k];
      double* o = &HX[(size_t)i * k];
      for (int c = 0; c < k; ++c) o[c] += hij * xr[c];
    }
  Mat C((size_t)n * n, 0.0);
  C[0] = E0;
  for (int c = 0; c < k; ++c) {
    double r = 0.0, l = 0.0;
    for (int i = 0; i < P; ++i) {
      r += gR[i] * X[(size_t)i * k + c];
      l += gL[i] * X[(size_t)i * k + c];
    }
    C[1 + c] = 0.5 * r;
    C[(size_t)(1 + c) * n] = 0.5 * l;
  }
  for (int i = 0; i < P; ++i) {
    const double* xr = &X[(size_t)i * k];
    const double* hr = &HX[(size_t)i * k];
    for (int r = 0; r < k; ++r) {
      const double xi = xr[r];
      if (xi == 0.0) continue;
      double* o = &C[(size_t)(1 + r) * n + 1];
      for (int c = 0; c < k; ++c) o[c] += xi * hr[c];
    }
  }
  double cnorm = 0.0;
  for (double x : C) cnorm = std::max(cnorm, std::fabs(x));
  cnorm = std::max(cnorm, 1e-300);
  Mat hw(C);
  std::vector<double> wr, wi;
  if (!hess_eigvals(n, hw, wr, wi)) return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: QR iteration did not converge");
  std::vector<int> order;
  for (int i = 0; i < n; ++i)
    if (std::isfinite(wr[i]) && std::fabs(wi[i]) <= 1e-8 * std::max(1.0, std::fabs(wr[i]))) order.push_back(i);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return wr[x] < wr[y]; });
  std::vector<double> y(n), v(P + 1);
  for (int idx : order) {
    const double lam = wr[idx];
    double refined = lam;
    // inverse iteration at a shift just off the eigenvalue: beyond its rounding error in C
    // (a few eps |C|), close enough for fast convergence
    const double sh = lam + std::max(1e-10 * std::max(std::fabs(lam), 1.0), 64.0 * kEps * cnorm);
    for (int i = 0; i < n; ++i) y[i] = 1.0 / std::sqrt((double)n) * (1.0 + 0.01 * (i % 7));
    for (int it = 0; it < 3; ++it) {
      shifted_solve(n, C, sh, cnorm, y);
      double yn = 0.0;
      for (double t : y) yn = std::max(yn, std::fabs(t));
      if (!(yn > 0.0) || !std::isfinite(yn)) break;
      for (double& t : y) t /= yn;
    }
    if (!all_finite(y.data(), n)) continue;
    v[0] = y[0];
    for (int i = 0; i < P; ++i) {
      double t = 0.0;
      const double* xr = &X[(size_t)i * k];
      for (int c = 0; c < k; ++c) t += xr[c] * y[1 + c];
      v[1 + i] = t;
    }
    // refinement on the pencil: v <- (A - sigma B)^-1 B v, then E from A v = E B v; a second
    // round shifted just off the refined E
    for (int round = 0; round < 2; ++round) {
      const double sig = round == 0 ? sh : refined + 1e-10 * std::max(std::fabs(refined), 1.0);
      const int m = P + 1;
      Mat K((size_t)m * m);
      double knorm = 0.0;
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          double aij, bij;
          if (i == 0 && j == 0) aij = E0, bij = 1.0;
          else if (i == 0) aij = 0.5 * gR[j - 1], bij = 0.0;
          else if (j == 0) aij = 0.5 * gL[i - 1], bij = 0.0;
          else {
            aij = H[(size_t)(i - 1) * P + (j - 1)] + (i == j ? shift : 0.0);
            bij = S[(size_t)(i - 1) * P + (j - 1)];
          }
          K[(size_t)i * m + j] = aij - sig * bij;
          knorm = std::max(knorm, std::fabs(aij) + std::fabs(sig * bij));
        }
      std::vector<int> piv;
      lu_factor(m, K, piv, kEps * std::max(knorm, 1e-300));
      auto applyB = [&](const std::vector<double>& x, std::vector<double>& out) {
        out.assign(m, 0.0);
        out[0] = x[0];
        for (int i = 0; i < P; ++i) {
          double t = 0.0;
          const double* sr = S + (size_t)i * P;
          for (int j = 0; j < P; ++j) t += sr[j] * x[1 + j];
          out[1 + i] = t;
        }
      };
      std::vector<double> bv, Av(m);
      bool ok = true;
      for (int it = 0; it < 2 && ok; ++it) {
        applyB(v, bv);
        lu_solve(m, K, piv, bv);
        double bn = 0.0;
        for (double t : bv) bn = std::max(bn, std::fabs(t));
        ok = bn > 0.0 && std::isfinite(bn);
        if (ok)
          for (int i = 0; i < m; ++i) v[i] = bv[i] / bn;
      }
      if (!ok || !all_finite(v.data(), v.size())) break;
      applyB(v, bv);
      Av[0] = E0 * v[0];
      for (int j = 0; j < P; ++j) Av[0] += 0.5 * gR[j] * v[1 + j];
      for (int i = 0; i < P; ++i) {
        double t = 0.5 * gL[i] * v[0] + shift * v[1 + i];
        const double* hr = H + (size_t)i * P;
        for (int j = 0; j < P; ++j) t += hr[j] * v[1 + j];
        Av[1 + i] = t;
      }
      double num = 0.0, den = 0.0;
      for (int i = 0; i < m; ++i) {
        num += bv[i] * Av[i];
        den += bv[i] * bv[i];
      }
      if (den > 0.0 && std::isfinite(num / den)) refined = num / den;
    }
    if (!all_finite(v.data(), v.size())) continue;
    double vn = 0.0;
    for (double t : v) vn += t * t;
    vn = std::sqrt(vn);
    if (!(std::fabs(v[0]) >= 1e-3 * vn)) continue;
    for (int i = 0; i < P; ++i) dp[i] = v[1 + i] / v[0];
    *e_lin = refined;
    return VBQMC_OK;
  }
  return vbq::set_error(VBQMC_ERR_ARG, "lin_solve: no real eigenvalue with an admissible eigenvector");
}

int vbqmc_lin_merge(int nparts, int P, const double* wsum, const double* mean, const double* E0, const double* gL,
                    const double* gR, const double* S, const double* H, double* E0_out, double* mean_out,
                    double* gL_out, double* gR_out, double* S_out, double* H_out) {
  if (nparts < 1 || P < 1 || !wsum || !mean || !E0 || !gL || !gR || !S || !H || !E0_out || !gL_out || !gR_out ||
      !S_out || !H_out)
    return vbq::set_error(VBQMC_ERR_ARG, "lin_merge: bad argument");
  const size_t PP = (size_t)P * P;
  double n = 0.0;
  for (int r = 0; r < nparts; ++r) {
    if (!(wsum[r] >= 0.0) || !std::isfinite(wsum[r])) return vbq::set_error(VBQMC_ERR_ARG, "lin_merge: bad weight sum");
    n += wsum[r];
  }
  if (!(n > 0.0)) return vbq::set_error(VBQMC_ERR_ARG, "lin_merge: the weight sums add up to zero");
  // global mean of O and of E_L
  std::vector<double> mu(P, 0.0);
  double e0 = 0.0;
  for (int r = 0; r < nparts; ++r) {
    const double f = wsum[r] / n;
    e0 += f * E0[r];
    for (int i = 0; i < P; ++i) mu[i] += f * mean[(size_t)r * P + i];
  }
  std::vector<double> gl(P, 0.0), del(P, 0.0), s(PP, 0.0), h(PP, 0.0), d(P), ej(P);
  for (int r = 0; r < nparts; ++r) {
    const double f = wsum[r] / n;
    if (f == 0.0) continue;
    const double* gLr = gL + (size_t)r * P;
    const double* gRr = gR + (size_t)r * P;
    const double* Sr = S + (size_t)r * PP;
    const double* Hr = H + (size_t)r * PP;
    // O - mu = (O - mu_r) + d within part r: the part's estimators re-centred on the global mean
    for (int i = 0; i < P; ++i) {
      d[i] = mean[(size_t)r * P + i] - mu[i];
      ej[i] = 0.5 * (gRr[i] - gLr[i]);  // <dE_L/dp_i> of the part
      gl[i] += f * (gLr[i] + 2.0 * d[i] * E0[r]);
      del[i] += f * ej[i];
    }
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) {
        const size_t q = (size_t)i * P + j;
        s[q] += f * (Sr[q] + d[i] * d[j]);
        h[q] += f * (Hr[q] + 0.5 * (d[j] * gLr[i] + d[i] * gLr[j]) + d[i] * d[j] * E0[r] + d[i] * ej[j]);
      }
  }
  *E0_out = e0;
  if (mean_out) std::copy(mu.begin(), mu.end(), mean_out);
  for (int i = 0; i < P; ++i) {
    gL_out[i] = gl[i];
    gR_out[i] = gl[i] + 2.0 * del[i];
  }
  std::copy(s.begin(), s.end(), S_out);
  std::copy(h.begin(), h.end(), H_out);
  return VBQMC_OK;
}

int vbqmc_structure_weights(int nvb, const double* S, const double* c, double* w_cc, double* w_lowdin) {
  if (nvb < 1 || !S || !c || (!w_cc && !w_lowdin)) return vbq::set_error(VBQMC_ERR_ARG, "structure_weights: bad argument");
  if (!all_finite(S, (size_t)nvb * nvb) || !all_finite(c, nvb))
    return vbq::set_error(VBQMC_ERR_ARG, "structure_weights: non-finite input");
  Mat a((size_t)nvb * nvb);
  for (int i = 0; i < nvb; ++i)
    for (int j = 0; j < nvb; ++j) a[(size_t)i * nvb + j] = 0.5 * (S[(size_t)i * nvb + j] + S[(size_t)j * nvb + i]);
  if (w_cc) {  // Chirgwin-Coulson: c_I (S c)_I / c^T S c
    std::vector<double> Sc(nvb, 0.0);
    double norm = 0.0;
    for (int i = 0; i < nvb; ++i) {
      for (int j = 0; j < nvb; ++j) Sc[i] += a[(size_t)i * nvb + j] * c[j];
      norm += c[i] * Sc[i];
    }
    if (!(norm > 0.0)) return vbq::set_error(VBQMC_ERR_ARG, "structure_weights: c^T S c is not positive");
    for (int i = 0; i < nvb; ++i) w_cc[i] = c[i] * Sc[i] / norm;
  }
  if (w_lowdin) {  // Loewdin: (S^1/2 c)_I^2 / |S^1/2 c|^2, negative rounding-size eigenvalues as 0
    std::vector<double> lam;
    Mat U;
    Mat a2(a);
    if (!sym_eig(nvb, a2, lam, U)) return vbq::set_error(VBQMC_ERR_ARG, "structure_weights: eigendecomposition failed");
    std::vector<double> t(nvb, 0.0), cb(nvb, 0.0);
    for (int m = 0; m < nvb; ++m) {
      double s = 0.0;
      for (int i = 0; i < nvb; ++i) s += U[(size_t)i * nvb + m] * c[i];
      t[m] = std::sqrt(std::max(lam[m], 0.0)) * s;
    }
    double norm = 0.0;
    for (int i = 0; i < nvb; ++i) {
      for (int m = 0; m < nvb; ++m) cb[i] += U[(size_t)i * nvb + m] * t[m];
      norm += cb[i] * cb[i];
    }
    if (!(norm > 0.0)) return vbq::set_error(VBQMC_ERR_ARG, "structure_weights: S^1/2 c vanishes");
    for (int i = 0; i < nvb; ++i) w_lowdin[i] = cb[i] * cb[i] / norm;
  }
  return VBQMC_OK;
}

}  // extern "C"
