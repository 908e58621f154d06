// VB-QMC oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of the Jastrow-Valence-Bond (JVB) quantum Monte
// Carlo method of Radenkovic, Domin, Toulouse and Braida, "The Valence-Bond Quantum
// Monte Carlo Method" (arXiv:2207.14715).  Only the tests, the package smoke check and
// the CPU-baseline leg of the benchmark may load it; the CUDA library never does, and
// this file shares no code, header or table with it.
//
// What is computed, and where the paper defines it:
//   * Psi_0 = J * sum_I c_I Phi_I                                   (Sec. 2.1, Eq. PsiJVBSCF)
//   * HLSP structures Phi_I as creation strings, expanded into 2^Npairs signed
//     determinants                                                   (Sec. 2.1, Eq. PhiI and the
//                                                                     determinant expansion after it)
//   * orbitals phi_p = sum_mu lambda_{p,mu} chi_mu                   (Sec. 2.1, orbital expansion)
//   * Jastrow J = exp(f_en + f_ee + f_een) with R(r)=r/(1+kappa r),
//     Rbar(r)=1/(1+kappa r), kappa = 0.8                            (Sec. 2.1, Jastrow equations)
//   * local energy E_L = (H Psi)/Psi                                 (Sec. 2.3.1, definition before Eq. Elav)
//   * parameters p = (alpha, c, kappa_kl); derivatives O_j = Psi_j/Psi_0 and
//     E_L,j = dE_L/dp_j                                              (Sec. 2.2, Eq. PsiJVBp; Sec. 2.3.1 Eq. H0j)
//   * VMC Metropolis sampling of Psi^2                               (Sec. 2.3.1)
//   * fixed-node DMC weighted walk with birth/death                  (Sec. 2.3.2, Eq. E0DMCweights)
//
// Readings where the paper is silent (each is listed in the design notes of the repo):
//   * basis: uncontracted, normalised cartesian Gaussians, d shells with 6 components;
//     zeta = 0 denotes the constant function 1 (normalisation taken as 1).  Shells may instead
//     be Slater-type (the paper's all-electron basis, Sec. 2.1): N x^a y^b z^c exp(-zeta r)
//     with n = l + 1, zeta > 0, normalised to 1.
//   * i = j self-pairs: the factor 2 of Sec. 2.1 is dropped (structures are unnormalised).
//   * determinant columns: orbitals in creation-string order after moving all up-spin
//     operators in front of all down-spin ones; the permutation parity is the sign d_{I,k}.
//   * e-e-n cusp constraints: the coefficients c_{pkl} are c = B theta, with B the
//     reduced-row-echelon null-space basis of the linear conditions that keep
//     d f_een / d r_ij = 0 at r_ij = 0 and d f_een / d r_ia = 0 at r_ia = 0.
//   * orbital-rotation derivative: at kappa = 0 the first-order action of E_kl replaces
//     phi_l by phi_l + eps * phi_k in every determinant (both spins).
//   * V includes the nucleus-nucleus repulsion.
//   * DMC: the paper names the algorithm of Umrigar, Nightingale and Runge (J. Chem. Phys.
//     99, 2865 (1993)) without printing it.  The step here keeps that algorithm's two limits
//     near nodes on an all-electron drift-diffusion move with Metropolis acceptance: each
//     electron's drift v_i = grad_i ln|Psi| is replaced by
//       vbar_i = v_i (-1 + sqrt(1 + 2 a |v_i|^2 tau)) / (a |v_i|^2 tau),  a = 1,
//     and in the branching weight E_L is replaced by E_T + (E_L - E_T) |Vbar| / |V| (V, Vbar the
//     whole-walker drift vectors), the difference E_L - E_T being further cut off at
//     +-0.2 sqrt(N / tau) (the cutoff of Zen, Sorella, Gillan, Michaelides and Alfe, Phys. Rev. B
//     93, 241118(R) (2016), which keeps a walker far from any node but at a huge |E_L| from
//     multiplying without bound); node rejection, weight
//     exp(-tau[(E'_L(R) + E'_L(R_kept))/2 - E_T]) with E'_L the limited energy, branching
//     copies = floor(w + U) capped at 3, children in parent order,
//     E_T = E_b,mean - (0.1/tau) ln(pop/target) with E_b,mean the weighted mean of the limited
//     energies at the kept positions (the energies that set the weights, so that the population
//     settles at the target); the reported estimator stays the weighted mean of the raw E_L.
//     Random numbers are keyed by walker_offset + (the walker's index in the population).
//
// Derivatives:
//   * electron gradients/Laplacians of the Slater part: each determinant is linear in the
//     row of electron i, so d/dx_i D is the determinant with that row replaced by the
//     derivative row (fresh LU each time);
//   * electron gradients/Laplacians of ln J: hyper-dual numbers (exact second derivatives);
//   * parameter derivatives: forward-mode dual numbers, one tangent per parameter, pushed
//     through the whole evaluation above;
//   * nucleus-position derivatives of ln|Psi| and E_L (the ingredients of forces): the same,
//     one tangent per nucleus coordinate (basis centres, Jastrow e-n/e-e-n terms and V move).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) written from its
// published definition; uniforms are (x >> 11) * 2^-53 of a 64-bit word.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -shared -fPIC -pthread.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace orc {

// ----------------------------------------------------------------------------------
// Philox4x32-10 from its published definition.
// ----------------------------------------------------------------------------------
static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c[0], &hi0, &lo0);
    mulhilo32(M1, c[2], &hi1, &lo1);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// Two uniforms in [0,1) from one Philox block keyed by the 64-bit seed.
// Counter words: (walker, step, slot, (system << 8) | purpose).
static void uniforms2(uint64_t seed, uint32_t walker, uint32_t step, uint32_t slot,
                      uint32_t system, uint32_t purpose, double u[2]) {
  uint32_t ctr[4] = {walker, step, slot, (system << 8) | (purpose & 0xffu)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  uint64_t x0 = ((uint64_t)o[1] << 32) | o[0];
  uint64_t x1 = ((uint64_t)o[3] << 32) | o[2];
  u[0] = (double)(x0 >> 11) * 0x1.0p-53;
  u[1] = (double)(x1 >> 11) * 0x1.0p-53;
}

// ----------------------------------------------------------------------------------
// Forward-mode AD types.  Dual<T>: value + one tangent.  HD<T>: hyper-dual number
// f + d1 e1 + d2 e2 + d12 e1 e2 (e1^2 = e2^2 = 0), giving exact second derivatives.
// ----------------------------------------------------------------------------------
template <class T> struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& a, const T& b) : v(a), d(b) {}
};
template <class T> struct HD {
  T f, d1, d2, d12;
  HD() : f(0.0), d1(0.0), d2(0.0), d12(0.0) {}
  template <class U> HD(const U& x) : f(T(x)), d1(0.0), d2(0.0), d12(0.0) {}
  HD(const T& a, const T& b, const T& c, const T& e) : f(a), d1(b), d2(c), d12(e) {}
};

inline double val(double x) { return x; }
template <class T> double val(const Dual<T>& x) { return val(x.v); }
template <class T> double val(const HD<T>& x) { return val(x.f); }

// Dual arithmetic
template <class T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> Dual<T> operator-(const Dual<T>& a) { return Dual<T>(-a.v, -a.d); }
template <class T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return Dual<T>(a.v * b.v, a.v * b.d + a.d * b.v); }
template <class T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> Dual<T> operator+(const Dual<T>& a, double b) { return Dual<T>(a.v + b, a.d); }
template <class T> Dual<T> operator+(double b, const Dual<T>& a) { return Dual<T>(a.v + b, a.d); }
template <class T> Dual<T> operator-(const Dual<T>& a, double b) { return Dual<T>(a.v - b, a.d); }
template <class T> Dual<T> operator-(double b, const Dual<T>& a) { return Dual<T>(b - a.v, -a.d); }
template <class T> Dual<T> operator*(const Dual<T>& a, double b) { return Dual<T>(a.v * b, a.d * b); }
template <class T> Dual<T> operator*(double b, const Dual<T>& a) { return Dual<T>(a.v * b, a.d * b); }
template <class T> Dual<T> operator/(const Dual<T>& a, double b) { return Dual<T>(a.v / b, a.d / b); }
template <class T> Dual<T> operator/(double b, const Dual<T>& a) { return Dual<T>(b) / a; }
template <class T> Dual<T>& operator+=(Dual<T>& a, const Dual<T>& b) { a = a + b; return a; }
template <class T> Dual<T>& operator-=(Dual<T>& a, const Dual<T>& b) { a = a - b; return a; }
template <class T> Dual<T>& operator*=(Dual<T>& a, const Dual<T>& b) { a = a * b; return a; }

// HD arithmetic
template <class T> HD<T> operator+(const HD<T>& a, const HD<T>& b) { return HD<T>(a.f + b.f, a.d1 + b.d1, a.d2 + b.d2, a.d12 + b.d12); }
template <class T> HD<T> operator-(const HD<T>& a, const HD<T>& b) { return HD<T>(a.f - b.f, a.d1 - b.d1, a.d2 - b.d2, a.d12 - b.d12); }
template <class T> HD<T> operator-(const HD<T>& a) { return HD<T>(-a.f, -a.d1, -a.d2, -a.d12); }
template <class T> HD<T> operator*(const HD<T>& a, const HD<T>& b) {
  return HD<T>(a.f * b.f, a.f * b.d1 + a.d1 * b.f, a.f * b.d2 + a.d2 * b.f,
               a.f * b.d12 + a.d1 * b.d2 + a.d2 * b.d1 + a.d12 * b.f);
}
template <class T> HD<T> operator+(const HD<T>& a, double b) { return HD<T>(a.f + b, a.d1, a.d2, a.d12); }
template <class T> HD<T> operator+(double b, const HD<T>& a) { return a + b; }
template <class T> HD<T> operator-(const HD<T>& a, double b) { return HD<T>(a.f - b, a.d1, a.d2, a.d12); }
template <class T> HD<T> operator-(double b, const HD<T>& a) { return HD<T>(b - a.f, -a.d1, -a.d2, -a.d12); }
template <class T> HD<T> operator*(const HD<T>& a, double b) { return HD<T>(a.f * b, a.d1 * b, a.d2 * b, a.d12 * b); }
template <class T> HD<T> operator*(double b, const HD<T>& a) { return a * b; }
template <class T> HD<T>& operator+=(HD<T>& a, const HD<T>& b) { a = a + b; return a; }

// unary functions: value g, first derivative g1, second derivative g2 at a point
inline double vsqrt(double x) { return std::sqrt(x); }
inline double vexp(double x) { return std::exp(x); }
inline double vlog(double x) { return std::log(x); }
template <class T> Dual<T> vsqrt(const Dual<T>& a) { T s = vsqrt(a.v); return Dual<T>(s, a.d / (2.0 * s)); }
template <class T> Dual<T> vexp(const Dual<T>& a) { T e = vexp(a.v); return Dual<T>(e, e * a.d); }
template <class T> Dual<T> vlog(const Dual<T>& a) { return Dual<T>(vlog(a.v), a.d / a.v); }

template <class T> HD<T> hd_apply(const HD<T>& a, const T& g, const T& g1, const T& g2) {
  return HD<T>(g, g1 * a.d1, g1 * a.d2, g1 * a.d12 + g2 * a.d1 * a.d2);
}
template <class T> HD<T> vsqrt(const HD<T>& a) {
  T g = vsqrt(a.f);
  T g1 = 0.5 / g;
  T g2 = -1.0 * g1 / (2.0 * a.f);
  return hd_apply(a, g, g1, g2);
}
template <class T> HD<T> vexp(const HD<T>& a) { T g = vexp(a.f); return hd_apply(a, g, g, g); }
template <class T> HD<T> vlog(const HD<T>& a) {
  T g1 = 1.0 / a.f;
  return hd_apply(a, vlog(a.f), g1, -1.0 * g1 * g1);
}
template <class T> HD<T> vinv(const HD<T>& a) {
  T g = 1.0 / a.f;
  return hd_apply(a, g, -1.0 * g * g, 2.0 * g * g * g);
}
template <class T> HD<T> operator/(const HD<T>& a, const HD<T>& b) { return a * vinv(b); }
template <class T> HD<T> operator/(double a, const HD<T>& b) { return vinv(b) * a; }
template <class T> HD<T> operator/(const HD<T>& a, double b) { return a * (1.0 / b); }

template <class S> S ipow(const S& x, int p) {
  S r(1.0);
  for (int i = 0; i < p; ++i) r = r * x;
  return r;
}

}  // namespace orc

// ----------------------------------------------------------------------------------
// Input description (host arrays, borrowed for the duration of a call).
// ----------------------------------------------------------------------------------
extern "C" {
typedef struct orc_system {
  int Nn, n_elem;
  const double* nuc_xyz;  // [Nn][3]
  const double* nuc_Z;    // [Nn]
  const int* nuc_elem;    // [Nn]
  int S;
  const int* sh_center;   // [S]
  const int* sh_l;        // [S] 0,1,2
  const double* sh_zeta;  // [S]
  int Norb;
  const double* orb_coef; // [Norb][M]
  int Nup, Ndn;
  int Nvb;
  const double* c_vb;     // [Nvb]
  const int* inact_off;   // [Nvb+1]
  const int* inact;
  const int* pair_off;    // [Nvb+1]
  const int* pairs;       // [npairs][2]
  const int* unp_off;     // [Nvb+1]
  const int* unp;
  double kappa;
  const double* jas_a;    // [n_elem][6]  a1..a6
  const double* jas_b;    // [6]          b1 (unused), b2..b6
  double b1_anti, b1_par;
  int een_on;
  const double* een_theta;  // [n_elem][15]
  int n_cparam;
  const int* cparam;      // structure indices whose c_I are parameters
  int jas_param;          // 1: a2..a6 per element, b2..b6, theta per element are parameters
  int n_kappa;
  const int* kappa_kl;    // [n_kappa][2] = (k, l): excitation from l to k
  const int* sh_kind;     // [S] 0 Gaussian, 1 Slater (NULL: all Gaussian)
} orc_system;
}

namespace orc {

// e-e-n expansion terms (p, k, l, m) in the order of the triple sum of Sec. 2.1.
struct EenTerm { int p, k, l, m; };
static std::vector<EenTerm> een_terms() {
  std::vector<EenTerm> t;
  for (int p = 2; p <= 5; ++p)
    for (int k = 0; k <= p - 1; ++k) {
      int lmax = (k != 0) ? (p - k) : (p - k - 2);
      for (int l = 0; l <= lmax; ++l)
        if (((p - k - l) % 2) == 0) t.push_back({p, k, l, (p - k - l) / 2});
    }
  return t;
}

// Cusp conditions on the e-e-n coefficients.  With u = Rbar(r_ij), s = Rbar(r_ia),
// t = Rbar(r_ja) and Rbar'(0) = -kappa:
//   e-e (r_ij -> 0, s = t):   d/dr_ij term = -kappa k s^(l+2m) * 2        -> per power q=p-k: sum k c = 0
//   e-n (r_ia -> 0, s = 1, u = t): d/ds term = (l+m) t^(k+m) + m t^(k+l+m) -> per power q: sum = 0
// Free parameters: null space of that matrix in reduced row echelon form.
static int een_null_basis(std::vector<double>& B, int& nfree) {
  std::vector<EenTerm> T = een_terms();
  const int nt = (int)T.size();
  std::vector<std::vector<double>> C;
  for (int q = 1; q <= 5; ++q) {  // e-e rows
    std::vector<double> row(nt, 0.0);
    bool any = false;
    for (int i = 0; i < nt; ++i)
      if (T[i].k >= 1 && T[i].p - T[i].k == q) { row[i] = (double)T[i].k; any = true; }
    if (any) C.push_back(row);
  }
  for (int q = 0; q <= 6; ++q) {  // e-n rows
    std::vector<double> row(nt, 0.0);
    bool any = false;
    for (int i = 0; i < nt; ++i) {
      double v = 0.0;
      if (T[i].k + T[i].m == q) v += (double)(T[i].l + T[i].m);
      if (T[i].k + T[i].l + T[i].m == q) v += (double)T[i].m;
      if (v != 0.0) { row[i] = v; any = true; }
    }
    if (any) C.push_back(row);
  }
  // reduced row echelon form by Gauss-Jordan elimination, columns in order
  int nr = (int)C.size();
  std::vector<int> pivcol;
  int r = 0;
  for (int col = 0; col < nt && r < nr; ++col) {
    int best = -1;
    double bv = 1e-9;
    for (int i = r; i < nr; ++i)
      if (std::fabs(C[i][col]) > bv) { bv = std::fabs(C[i][col]); best = i; }
    if (best < 0) continue;
    std::swap(C[r], C[best]);
    double pv = C[r][col];
    for (int j = 0; j < nt; ++j) C[r][j] /= pv;
    for (int i = 0; i < nr; ++i)
      if (i != r && C[i][col] != 0.0) {
        double f = C[i][col];
        for (int j = 0; j < nt; ++j) C[i][j] -= f * C[r][j];
      }
    pivcol.push_back(col);
    ++r;
  }
  std::vector<int> is_piv(nt, -1);
  for (int i = 0; i < (int)pivcol.size(); ++i) is_piv[pivcol[i]] = i;
  std::vector<int> freecols;
  for (int j = 0; j < nt; ++j)
    if (is_piv[j] < 0) freecols.push_back(j);
  nfree = (int)freecols.size();
  B.assign((size_t)nt * nfree, 0.0);
  for (int f = 0; f < nfree; ++f) {
    int fc = freecols[f];
    B[(size_t)fc * nfree + f] = 1.0;
    for (int i = 0; i < (int)pivcol.size(); ++i) B[(size_t)pivcol[i] * nfree + f] = -C[i][fc];
  }
  return (int)pivcol.size();
}

struct DetTerm {
  int I;        // structure
  double d;     // sign from the creation-string reordering
  std::vector<int> up, dn;  // ordered occupations
};

static const int NCOMP[3] = {1, 3, 6};
// cartesian exponents (a,b,c) of each component, in the fixed order
// s; x y z; xx yy zz xy xz yz
static const int CART[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
static const int CART_OFF[3] = {0, 1, 4};

struct Sys {
  int Nn, n_elem, S, M, Norb, Nup, Ndn, N, Nvb;
  std::vector<double> nuc_xyz, nuc_Z;
  std::vector<int> nuc_elem;
  std::vector<int> sh_center, sh_l, sh_first;
  std::vector<double> sh_zeta, sh_norm;  // norm per component: [S][6]
  std::vector<int> sh_kind;              // 0 Gaussian, 1 Slater
  std::vector<double> lam;               // [Norb][M]
  std::vector<double> c_vb;
  std::vector<DetTerm> terms;
  double kappa;
  std::vector<double> a, b;  // [n_elem*6], [6]
  double b1_anti, b1_par;
  int een_on;
  std::vector<double> theta;  // [n_elem*nfree]
  std::vector<EenTerm> et;
  std::vector<double> B;      // [23][nfree]
  int nfree;
  std::vector<int> cparam;
  int jas_param;
  std::vector<int> kap_k, kap_l;
  int P;
};

static double dfact(int n) {  // double factorial, (-1)!! = 1
  double r = 1.0;
  for (int i = n; i > 1; i -= 2) r *= i;
  return r;
}

// Expansion of one HLSP structure (Eq. PhiI) into signed determinants.
static void expand_structure(int I, const std::vector<int>& inact,
                             const std::vector<std::pair<int, int>>& pairs,
                             const std::vector<int>& unp, std::vector<DetTerm>& out) {
  int np = (int)pairs.size();
  // choice per pair: 0 -> (i up, j down) weight +1 ; 1 -> (i down, j up) weight -1 ; i==j -> only 0
  std::vector<int> nchoice(np);
  for (int q = 0; q < np; ++q) nchoice[q] = (pairs[q].first == pairs[q].second) ? 1 : 2;
  std::vector<int> ch(np, 0);
  while (true) {
    // build creation string of (orbital, spin) with spin 0 = up, 1 = down
    std::vector<std::pair<int, int>> s;
    double w = 1.0;
    for (int p : inact) { s.push_back({p, 0}); s.push_back({p, 1}); }
    for (int q = 0; q < np; ++q) {
      int i = pairs[q].first, j = pairs[q].second;
      if (ch[q] == 0) { s.push_back({i, 0}); s.push_back({j, 1}); }
      else { s.push_back({i, 1}); s.push_back({j, 0}); w = -w; }
    }
    for (int qq : unp) s.push_back({qq, 0});
    // parity of moving every up operator in front of all down operators (stable)
    int ndown_before = 0, inv = 0;
    for (auto& o : s) {
      if (o.second == 1) ++ndown_before;
      else inv += ndown_before;
    }
    if (inv & 1) w = -w;
    DetTerm t;
    t.I = I;
    t.d = w;
    for (auto& o : s) (o.second == 0 ? t.up : t.dn).push_back(o.first);
    // Pauli: a repeated spin-orbital gives a zero determinant
    bool zero = false;
    for (auto* v : {&t.up, &t.dn}) {
      std::vector<int> c = *v;
      std::sort(c.begin(), c.end());
      for (size_t x = 1; x < c.size(); ++x)
        if (c[x] == c[x - 1]) zero = true;
    }
    if (!zero) out.push_back(t);
    int q = 0;
    while (q < np) {
      if (++ch[q] < nchoice[q]) break;
      ch[q] = 0;
      ++q;
    }
    if (q == np) break;
  }
}

static int build_sys(const orc_system* in, Sys& s) {
  s.Nn = in->Nn; s.n_elem = in->n_elem; s.S = in->S; s.Norb = in->Norb;
  s.Nup = in->Nup; s.Ndn = in->Ndn; s.N = in->Nup + in->Ndn; s.Nvb = in->Nvb;
  s.nuc_xyz.assign(in->nuc_xyz, in->nuc_xyz + 3 * s.Nn);
  s.nuc_Z.assign(in->nuc_Z, in->nuc_Z + s.Nn);
  s.nuc_elem.assign(in->nuc_elem, in->nuc_elem + s.Nn);
  s.sh_center.assign(in->sh_center, in->sh_center + s.S);
  s.sh_l.assign(in->sh_l, in->sh_l + s.S);
  s.sh_zeta.assign(in->sh_zeta, in->sh_zeta + s.S);
  s.sh_kind.assign(s.S, 0);
  if (in->sh_kind) s.sh_kind.assign(in->sh_kind, in->sh_kind + s.S);
  s.sh_first.resize(s.S);
  s.sh_norm.assign((size_t)s.S * 6, 0.0);
  int M = 0;
  for (int i = 0; i < s.S; ++i) {
    int l = s.sh_l[i];
    if (l < 0 || l > 2) return -1;
    s.sh_first[i] = M;
    double z = s.sh_zeta[i];
    for (int c = 0; c < NCOMP[l]; ++c) {
      const int* e = CART[CART_OFF[l] + c];
      double nrm;
      if (s.sh_kind[i] == 1) {
        // Slater: int x^2a y^2b z^2c e^{-2 z r} d^3r = [4 pi (2a-1)!!(2b-1)!!(2c-1)!! / (2l+1)!!]
        //         x (2l+2)! / (2z)^(2l+3)
        if (!(z > 0.0)) return -1;
        double fact = 1.0;
        for (int k = 2; k <= 2 * l + 2; ++k) fact *= k;
        const double integral = 4.0 * M_PI * dfact(2 * e[0] - 1) * dfact(2 * e[1] - 1) * dfact(2 * e[2] - 1) /
                                dfact(2 * l + 1) * fact / std::pow(2.0 * z, 2 * l + 3);
        nrm = 1.0 / std::sqrt(integral);
      } else if (z == 0.0) nrm = 1.0;  // constant function
      else
        nrm = std::pow(2.0 * z / M_PI, 0.75) * std::pow(4.0 * z, 0.5 * l) /
              std::sqrt(dfact(2 * e[0] - 1) * dfact(2 * e[1] - 1) * dfact(2 * e[2] - 1));
      s.sh_norm[(size_t)i * 6 + c] = nrm;
    }
    M += NCOMP[l];
  }
  s.M = M;
  s.lam.assign(in->orb_coef, in->orb_coef + (size_t)s.Norb * M);
  s.c_vb.assign(in->c_vb, in->c_vb + s.Nvb);
  s.terms.clear();
  for (int I = 0; I < s.Nvb; ++I) {
    std::vector<int> ina(in->inact + in->inact_off[I], in->inact + in->inact_off[I + 1]);
    std::vector<std::pair<int, int>> pr;
    for (int q = in->pair_off[I]; q < in->pair_off[I + 1]; ++q)
      pr.push_back({in->pairs[2 * q], in->pairs[2 * q + 1]});
    std::vector<int> un(in->unp + in->unp_off[I], in->unp + in->unp_off[I + 1]);
    size_t before = s.terms.size();
    expand_structure(I, ina, pr, un, s.terms);
    for (size_t t = before; t < s.terms.size(); ++t)
      if ((int)s.terms[t].up.size() != s.Nup || (int)s.terms[t].dn.size() != s.Ndn) return -2;
  }
  s.kappa = in->kappa;
  s.a.assign(in->jas_a, in->jas_a + 6 * s.n_elem);
  s.b.assign(in->jas_b, in->jas_b + 6);
  s.b1_anti = in->b1_anti; s.b1_par = in->b1_par;
  s.een_on = in->een_on;
  s.et = een_terms();
  een_null_basis(s.B, s.nfree);
  if (s.een_on) s.theta.assign(in->een_theta, in->een_theta + (size_t)s.n_elem * s.nfree);
  else s.theta.assign((size_t)s.n_elem * s.nfree, 0.0);
  s.cparam.assign(in->cparam, in->cparam + in->n_cparam);
  s.jas_param = in->jas_param;
  s.kap_k.clear(); s.kap_l.clear();
  for (int q = 0; q < in->n_kappa; ++q) {
    s.kap_k.push_back(in->kappa_kl[2 * q]);
    s.kap_l.push_back(in->kappa_kl[2 * q + 1]);
  }
  s.P = (int)s.cparam.size() + (s.jas_param ? (5 * s.n_elem + 5 + (s.een_on ? s.nfree * s.n_elem : 0)) : 0) +
        (int)s.kap_k.size();
  return 0;
}

// Parameter values and nucleus positions in scalar type T; 'dir' >= 0 puts a unit tangent on
// parameter dir (dir < P) or on nucleus coordinate dir - P.
template <class T> struct Params {
  std::vector<T> c, a, b, craw, lam;
  std::vector<T> nuc;  // [Nn][3] nucleus positions (basis centres, Jastrow e-n and e-e-n, V)
};

template <class T> static void set_tangent(T&, double) {}
template <class T> static void set_tangent(Dual<T>& x, double t) { x.d = T(t); }

template <class T> static Params<T> make_params(const Sys& s, int dir) {
  Params<T> P;
  P.c.resize(s.Nvb);
  for (int I = 0; I < s.Nvb; ++I) P.c[I] = T(s.c_vb[I]);
  P.a.resize(s.a.size());
  for (size_t i = 0; i < s.a.size(); ++i) P.a[i] = T(s.a[i]);
  P.b.resize(6);
  for (int i = 0; i < 6; ++i) P.b[i] = T(s.b[i]);
  int nt = (int)s.et.size();
  P.craw.assign((size_t)s.n_elem * nt, T(0.0));
  for (int e = 0; e < s.n_elem; ++e)
    for (int t = 0; t < nt; ++t) {
      double v = 0.0;
      for (int f = 0; f < s.nfree; ++f) v += s.B[(size_t)t * s.nfree + f] * s.theta[(size_t)e * s.nfree + f];
      P.craw[(size_t)e * nt + t] = T(v);
    }
  P.lam.resize(s.lam.size());
  for (size_t i = 0; i < s.lam.size(); ++i) P.lam[i] = T(s.lam[i]);
  P.nuc.resize(3 * (size_t)s.Nn);
  for (int i = 0; i < 3 * s.Nn; ++i) P.nuc[i] = T(s.nuc_xyz[i]);
  if (dir < 0) return P;
  // directions past the parameters: nucleus coordinate (dir - P) = 3 alpha + d
  if (dir >= s.P) { set_tangent(P.nuc[dir - s.P], 1.0); return P; }
  int j = dir;
  if (j < (int)s.cparam.size()) { set_tangent(P.c[s.cparam[j]], 1.0); return P; }
  j -= (int)s.cparam.size();
  if (s.jas_param) {
    if (j < 5 * s.n_elem) { set_tangent(P.a[(j / 5) * 6 + 1 + j % 5], 1.0); return P; }
    j -= 5 * s.n_elem;
    if (j < 5) { set_tangent(P.b[1 + j], 1.0); return P; }
    j -= 5;
    if (s.een_on) {
      if (j < s.nfree * s.n_elem) {
        int e = j / s.nfree, f = j % s.nfree;
        for (int t = 0; t < nt; ++t) set_tangent(P.craw[(size_t)e * nt + t], s.B[(size_t)t * s.nfree + f]);
        return P;
      }
      j -= s.nfree * s.n_elem;
    }
  }
  // orbital rotation kappa_kl: phi_l -> phi_l + eps phi_k
  int k = s.kap_k[j], l = s.kap_l[j];
  for (int mu = 0; mu < s.M; ++mu) set_tangent(P.lam[(size_t)l * s.M + mu], s.lam[(size_t)k * s.M + mu]);
  return P;
}

// Cartesian Gaussian values, gradients and Laplacians at point r (closed form):
// chi = N P(x) e^{-z r^2};  grad chi = N e (grad P - 2 z x P);
// lap chi = N e (lap P + P (4 z^2 r^2 - 6 z - 4 z l)).
// Slater shells: chi = N P(x) e^{-z r};  grad chi = N e (grad P - z x P / r);
// lap chi = N e (lap P + P (z^2 - 2 z (l + 1) / r))  (grad P . x = l P for the degree-l monomial).
// The centres are nuc (type T, so that a tangent on a nucleus position carries through).
template <class T>
static void basis_at(const Sys& s, const std::vector<T>& nuc, const double* r, T* chi, T* dchi, T* lchi) {
  for (int sh = 0; sh < s.S; ++sh) {
    int c = s.sh_center[sh], l = s.sh_l[sh];
    T x[3] = {r[0] - nuc[3 * c], r[1] - nuc[3 * c + 1], r[2] - nuc[3 * c + 2]};
    T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double z = s.sh_zeta[sh];
    const bool slater = s.sh_kind[sh] == 1;
    T rr = slater ? vsqrt(r2) : T(0.0);
    T e = slater ? vexp(rr * (-z)) : vexp(r2 * (-z));
    for (int q = 0; q < NCOMP[l]; ++q) {
      const int* ex = CART[CART_OFF[l] + q];
      double nrm = s.sh_norm[(size_t)sh * 6 + q];
      T P(1.0);
      for (int d = 0; d < 3; ++d) P = P * ipow(x[d], ex[d]);
      int mu = s.sh_first[sh] + q;
      chi[mu] = P * e * nrm;
      if (dchi) {
        for (int d = 0; d < 3; ++d) {
          T dP(0.0);
          if (ex[d] > 0) {
            dP = ipow(x[d], ex[d] - 1) * (double)ex[d];
            for (int o = 0; o < 3; ++o)
              if (o != d) dP = dP * ipow(x[o], ex[o]);
          }
          if (slater) dchi[3 * mu + d] = e * (dP - x[d] * P * z / rr) * nrm;
          else dchi[3 * mu + d] = e * (dP - x[d] * P * (2.0 * z)) * nrm;
        }
        T lapP(0.0);
        for (int d = 0; d < 3; ++d)
          if (ex[d] >= 2) {
            T t = ipow(x[d], ex[d] - 2) * (double)(ex[d] * (ex[d] - 1));
            for (int o = 0; o < 3; ++o)
              if (o != d) t = t * ipow(x[o], ex[o]);
            lapP = lapP + t;
          }
        if (slater) lchi[mu] = e * (lapP + P * (z * z - (2.0 * z * (l + 1)) / rr)) * nrm;
        else lchi[mu] = e * (lapP + P * (r2 * (4.0 * z * z) - (6.0 * z + 4.0 * z * l))) * nrm;
      }
    }
  }
}

// Determinant by LU with partial pivoting (ties: lowest row).
template <class T> static T det_lu(int n, std::vector<T> A) {
  T det(1.0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::fabs(val(A[(size_t)c * n + c]));
    for (int r = c + 1; r < n; ++r) {
      double v = std::fabs(val(A[(size_t)r * n + c]));
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0) return T(0.0);
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
      det = T(0.0) - det;
    }
    T piv = A[(size_t)c * n + c];
    det = det * piv;
    for (int r = c + 1; r < n; ++r) {
      T m = A[(size_t)r * n + c] / piv;
      for (int j = c + 1; j < n; ++j) A[(size_t)r * n + j] = A[(size_t)r * n + j] - m * A[(size_t)c * n + j];
    }
  }
  return det;
}

// Jastrow pieces (Sec. 2.1).  Positions of type S, parameters promoted from T.
template <class S, class T> static S f_en(const Sys& s, const Params<T>& P, const S* ri, int al) {
  S dx = ri[0] - S(P.nuc[3 * al]), dy = ri[1] - S(P.nuc[3 * al + 1]), dz = ri[2] - S(P.nuc[3 * al + 2]);
  S r = vsqrt(dx * dx + dy * dy + dz * dz);
  S R = r / (1.0 + s.kappa * r);
  const T* a = &P.a[(size_t)s.nuc_elem[al] * 6];
  S v = S(a[0]) * R / (1.0 + S(a[1]) * R);
  S Rp = R;
  for (int p = 2; p <= 5; ++p) { Rp = Rp * R; v = v + S(a[p]) * Rp; }
  return v;
}
template <class S, class T> static S f_ee(const Sys& s, const Params<T>& P, const S* ri, const S* rj, bool same) {
  S dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
  S r = vsqrt(dx * dx + dy * dy + dz * dz);
  S R = r / (1.0 + s.kappa * r);
  double b1 = same ? s.b1_par : s.b1_anti;
  S v = b1 * R / (1.0 + S(P.b[1]) * R);
  S Rp = R;
  for (int p = 2; p <= 5; ++p) { Rp = Rp * R; v = v + S(P.b[p]) * Rp; }
  return v;
}
template <class S, class T> static S f_een(const Sys& s, const Params<T>& P, const S* ri, const S* rj, int al) {
  const S A[3] = {S(P.nuc[3 * al]), S(P.nuc[3 * al + 1]), S(P.nuc[3 * al + 2])};
  S dij[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
  S dia[3] = {ri[0] - A[0], ri[1] - A[1], ri[2] - A[2]};
  S dja[3] = {rj[0] - A[0], rj[1] - A[1], rj[2] - A[2]};
  S rij = vsqrt(dij[0] * dij[0] + dij[1] * dij[1] + dij[2] * dij[2]);
  S ria = vsqrt(dia[0] * dia[0] + dia[1] * dia[1] + dia[2] * dia[2]);
  S rja = vsqrt(dja[0] * dja[0] + dja[1] * dja[1] + dja[2] * dja[2]);
  S u = 1.0 / (1.0 + s.kappa * rij);
  S sa = 1.0 / (1.0 + s.kappa * ria);
  S ta = 1.0 / (1.0 + s.kappa * rja);
  int nt = (int)s.et.size();
  const T* c = &P.craw[(size_t)s.nuc_elem[al] * nt];
  S v(0.0);
  for (int t = 0; t < nt; ++t) {
    const EenTerm& e = s.et[t];
    S term = ipow(u, e.k) * (ipow(sa, e.l) + ipow(ta, e.l)) * ipow(sa * ta, e.m);
    v = v + S(c[t]) * term;
  }
  return v;
}

template <class S, class T> static S lnJ_full(const Sys& s, const Params<T>& P, const S* pos) {
  S v(0.0);
  for (int i = 0; i < s.N; ++i)
    for (int al = 0; al < s.Nn; ++al) v = v + f_en(s, P, pos + 3 * i, al);
  for (int i = 0; i < s.N; ++i)
    for (int j = i + 1; j < s.N; ++j) {
      bool same = (i < s.Nup) == (j < s.Nup);
      v = v + f_ee(s, P, pos + 3 * i, pos + 3 * j, same);
      if (s.een_on)
        for (int al = 0; al < s.Nn; ++al) v = v + f_een(s, P, pos + 3 * i, pos + 3 * j, al);
    }
  return v;
}
// all terms of ln J that involve electron i
template <class S, class T> static S lnJ_of(const Sys& s, const Params<T>& P, const S* pos, int i) {
  S v(0.0);
  for (int al = 0; al < s.Nn; ++al) v = v + f_en(s, P, pos + 3 * i, al);
  for (int j = 0; j < s.N; ++j) {
    if (j == i) continue;
    bool same = (i < s.Nup) == (j < s.Nup);
    v = v + f_ee(s, P, pos + 3 * i, pos + 3 * j, same);
    if (s.een_on)
      for (int al = 0; al < s.Nn; ++al) v = v + f_een(s, P, pos + 3 * i, pos + 3 * j, al);
  }
  return v;
}

// V = V_en + V_ee + V_nn at electron positions R [N][3], nuclei at P.nuc.
template <class T> static T potential(const Sys& s, const Params<T>& P, const double* R) {
  T V(0.0);
  for (int i = 0; i < s.N; ++i)
    for (int al = 0; al < s.Nn; ++al) {
      T d[3] = {R[3 * i] - P.nuc[3 * al], R[3 * i + 1] - P.nuc[3 * al + 1], R[3 * i + 2] - P.nuc[3 * al + 2]};
      V = V - s.nuc_Z[al] / vsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  for (int i = 0; i < s.N; ++i)
    for (int j = i + 1; j < s.N; ++j) {
      double d[3] = {R[3 * i] - R[3 * j], R[3 * i + 1] - R[3 * j + 1], R[3 * i + 2] - R[3 * j + 2]};
      V = V + 1.0 / std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  for (int a = 0; a < s.Nn; ++a)
    for (int b = a + 1; b < s.Nn; ++b) {
      T d[3] = {P.nuc[3 * a] - P.nuc[3 * b], P.nuc[3 * a + 1] - P.nuc[3 * b + 1], P.nuc[3 * a + 2] - P.nuc[3 * b + 2]};
      V = V + s.nuc_Z[a] * s.nuc_Z[b] / vsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  return V;
}

template <class T> struct Eval {
  T logpsi;
  double sign;
  T eloc;
  std::vector<T> grad;  // grad ln|Psi| per electron [N][3]
};

// Evaluate ln|Psi|, sign and, if full, E_L and grad ln|Psi| at configuration R [N][3].
template <class T> static Eval<T> evaluate(const Sys& s, const Params<T>& P, const double* R, bool full) {
  const int N = s.N, M = s.M, No = s.Norb;
  std::vector<T> chi(M), dchi(3 * M), lchi(M);
  std::vector<T> phi((size_t)N * No), dphi(full ? (size_t)N * No * 3 : 0), lphi(full ? (size_t)N * No : 0);
  for (int e = 0; e < N; ++e) {
    basis_at(s, P.nuc, R + 3 * e, chi.data(), full ? dchi.data() : nullptr, full ? lchi.data() : nullptr);
    for (int k = 0; k < No; ++k) {
      T v(0.0), g0(0.0), g1(0.0), g2(0.0), lp(0.0);
      for (int mu = 0; mu < M; ++mu) {
        const T& lm = P.lam[(size_t)k * M + mu];
        v = v + lm * chi[mu];
        if (full) {
          g0 = g0 + lm * dchi[3 * mu];
          g1 = g1 + lm * dchi[3 * mu + 1];
          g2 = g2 + lm * dchi[3 * mu + 2];
          lp = lp + lm * lchi[mu];
        }
      }
      phi[(size_t)e * No + k] = v;
      if (full) {
        dphi[((size_t)e * No + k) * 3] = g0;
        dphi[((size_t)e * No + k) * 3 + 1] = g1;
        dphi[((size_t)e * No + k) * 3 + 2] = g2;
        lphi[(size_t)e * No + k] = lp;
      }
    }
  }
  // Slater part: Phi = sum_I c_I sum_k d_{I,k} det(A_up) det(A_dn)
  T Phi(0.0);
  std::vector<T> gPhi(full ? 3 * N : 0, T(0.0)), lPhi(full ? N : 0, T(0.0));
  for (const DetTerm& t : s.terms) {
    T Dsp[2];
    std::vector<T> gD[2], lD[2];
    for (int sp = 0; sp < 2; ++sp) {
      const std::vector<int>& occ = sp == 0 ? t.up : t.dn;
      int n = (int)occ.size(), e0 = sp == 0 ? 0 : s.Nup;
      std::vector<T> A((size_t)n * n);
      for (int e = 0; e < n; ++e)
        for (int o = 0; o < n; ++o) A[(size_t)e * n + o] = phi[(size_t)(e0 + e) * No + occ[o]];
      Dsp[sp] = det_lu(n, A);
      if (full) {
        gD[sp].assign(3 * n, T(0.0));
        lD[sp].assign(n, T(0.0));
        for (int e = 0; e < n; ++e) {
          for (int c = 0; c < 4; ++c) {
            std::vector<T> B = A;
            for (int o = 0; o < n; ++o)
              B[(size_t)e * n + o] = c < 3 ? dphi[((size_t)(e0 + e) * No + occ[o]) * 3 + c]
                                           : lphi[(size_t)(e0 + e) * No + occ[o]];
            T d = det_lu(n, B);
            if (c < 3) gD[sp][3 * e + c] = d;
            else lD[sp][e] = d;
          }
        }
      }
    }
    T coef = P.c[t.I] * t.d;
    Phi = Phi + coef * Dsp[0] * Dsp[1];
    if (full) {
      for (int sp = 0; sp < 2; ++sp) {
        int n = sp == 0 ? s.Nup : s.Ndn, e0 = sp == 0 ? 0 : s.Nup;
        T other = Dsp[1 - sp];
        for (int e = 0; e < n; ++e) {
          for (int c = 0; c < 3; ++c) gPhi[3 * (e0 + e) + c] = gPhi[3 * (e0 + e) + c] + coef * gD[sp][3 * e + c] * other;
          lPhi[e0 + e] = lPhi[e0 + e] + coef * lD[sp][e] * other;
        }
      }
    }
  }
  Eval<T> out;
  out.sign = val(Phi) > 0 ? 1.0 : (val(Phi) < 0 ? -1.0 : 0.0);
  // ln|Phi| with its tangent
  T absPhi = out.sign < 0 ? T(0.0) - Phi : Phi;
  std::vector<T> pos(3 * N);
  for (int i = 0; i < 3 * N; ++i) pos[i] = T(R[i]);
  T lnJ = lnJ_full(s, P, pos.data());
  out.logpsi = lnJ + vlog(absPhi);
  if (!full) return out;
  // Jastrow gradients and Laplacians with hyper-dual numbers, one coordinate at a time
  std::vector<HD<T>> hpos(3 * N);
  std::vector<T> G(3 * N, T(0.0)), LJ(N, T(0.0));
  for (int i = 0; i < N; ++i) {
    for (int d = 0; d < 3; ++d) {
      for (int q = 0; q < 3 * N; ++q) hpos[q] = HD<T>(pos[q]);
      hpos[3 * i + d] = HD<T>(pos[3 * i + d], T(1.0), T(1.0), T(0.0));
      HD<T> f = lnJ_of(s, P, hpos.data(), i);
      G[3 * i + d] = f.d1;
      LJ[i] = LJ[i] + f.d12;
    }
  }
  T kin(0.0);
  out.grad.assign(3 * N, T(0.0));
  for (int i = 0; i < N; ++i) {
    T dot(0.0), gg(0.0);
    for (int d = 0; d < 3; ++d) {
      T gphi = gPhi[3 * i + d] / Phi;
      dot = dot + G[3 * i + d] * gphi;
      gg = gg + G[3 * i + d] * G[3 * i + d];
      out.grad[3 * i + d] = G[3 * i + d] + gphi;
    }
    kin = kin + lPhi[i] / Phi + 2.0 * dot + LJ[i] + gg;
  }
  out.eloc = -0.5 * kin + potential(s, P, R);
  return out;
}

}  // namespace orc

using namespace orc;

template <class F> static void parallel_for(int n, int nthreads, F f) {
  if (nthreads <= 1 || n <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  nthreads = std::min(nthreads, n);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < n; i += nthreads) f(i);
    });
  for (auto& x : th) x.join();
}

extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

void orc_uniforms2(uint64_t seed, uint32_t walker, uint32_t step, uint32_t slot, uint32_t system, uint32_t purpose,
                   double* u) {
  uniforms2(seed, walker, step, slot, system, purpose, u);
}

int orc_num_params(const orc_system* in) {
  Sys s;
  if (build_sys(in, s)) return -1;
  return s.P;
}

int orc_basis_size(const orc_system* in) {
  Sys s;
  if (build_sys(in, s)) return -1;
  return s.M;
}

// e-e-n free-parameter basis B [23][nfree]; returns nfree
int orc_een_basis(double* B, int* nterms) {
  std::vector<double> b;
  int nf;
  een_null_basis(b, nf);
  std::vector<EenTerm> t = een_terms();
  *nterms = (int)t.size();
  std::copy(b.begin(), b.end(), B);
  return nf;
}

// e-e-n term exponents [nt][4] = (p, k, l, m)
int orc_een_terms(int* pklm) {
  std::vector<EenTerm> t = een_terms();
  for (size_t i = 0; i < t.size(); ++i) {
    pklm[4 * i] = t[i].p; pklm[4 * i + 1] = t[i].k; pklm[4 * i + 2] = t[i].l; pklm[4 * i + 3] = t[i].m;
  }
  return (int)t.size();
}

// Determinant expansion of all structures.  Returns the number of terms; fills
// str[t], d[t], up[t][Nup], dn[t][Ndn] for t < maxterms.
int orc_expand(const orc_system* in, int maxterms, int* str, double* d, int* up, int* dn) {
  Sys s;
  int rc = build_sys(in, s);
  if (rc) return rc;
  int nt = (int)s.terms.size();
  for (int t = 0; t < nt && t < maxterms; ++t) {
    str[t] = s.terms[t].I;
    d[t] = s.terms[t].d;
    for (int o = 0; o < s.Nup; ++o) up[(size_t)t * s.Nup + o] = s.terms[t].up[o];
    for (int o = 0; o < s.Ndn; ++o) dn[(size_t)t * s.Ndn + o] = s.terms[t].dn[o];
  }
  return nt;
}

int orc_basis_eval(const orc_system* in, const double* r, double* chi, double* dchi, double* lchi) {
  Sys s;
  if (build_sys(in, s)) return -1;
  basis_at(s, s.nuc_xyz, r, chi, dchi, lchi);
  return s.M;
}

double orc_det_lu(int n, const double* A) { return det_lu(n, std::vector<double>(A, A + (size_t)n * n)); }

// Leibniz formula: sum over permutations of sign * prod A[i][perm(i)] (small n only).
double orc_det_leibniz(int n, const double* A) {
  std::vector<int> p(n);
  for (int i = 0; i < n; ++i) p[i] = i;
  double tot = 0.0;
  do {
    int inv = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (p[i] > p[j]) ++inv;
    double prod = (inv & 1) ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) prod *= A[(size_t)i * n + p[i]];
    tot += prod;
  } while (std::next_permutation(p.begin(), p.end()));
  return tot;
}

// ln J alone (for tests of the Jastrow definition)
int orc_lnJ(const orc_system* in, int W, const double* R, double* out) {
  Sys s;
  if (build_sys(in, s)) return -1;
  Params<double> P = make_params<double>(s, -1);
  for (int w = 0; w < W; ++w) out[w] = lnJ_full(s, P, R + (size_t)w * 3 * s.N);
  return 0;
}

// Evaluate W walkers at R [W][N][3].  Optional outputs may be NULL:
//   grad [W][N][3] = grad ln|Psi|;  O [W][P] = dln|Psi|/dp;  dEL [W][P] = dE_L/dp.
int orc_eval(const orc_system* in, int W, const double* R, double* logpsi, double* sign, double* eloc,
             double* grad, double* O, double* dEL, int nthreads) {
  Sys s;
  int rc = build_sys(in, s);
  if (rc) return rc;
  const int N = s.N, P = s.P;
  Params<double> P0 = make_params<double>(s, -1);
  parallel_for(W, nthreads, [&](int w) {
    const double* Rw = R + (size_t)w * 3 * N;
    Eval<double> e = evaluate(s, P0, Rw, true);
    if (logpsi) logpsi[w] = e.logpsi;
    if (sign) sign[w] = e.sign;
    if (eloc) eloc[w] = e.eloc;
    if (grad)
      for (int q = 0; q < 3 * N; ++q) grad[(size_t)w * 3 * N + q] = e.grad[q];
    if (O || dEL) {
      for (int j = 0; j < P; ++j) {
        Params<Dual<double>> Pj = make_params<Dual<double>>(s, j);
        Eval<Dual<double>> ed = evaluate(s, Pj, Rw, dEL != nullptr);
        if (O) O[(size_t)w * P + j] = ed.logpsi.d;
        if (dEL) dEL[(size_t)w * P + j] = ed.eloc.d;
      }
    }
  });
  return 0;
}

// Nucleus-position derivatives at fixed electron positions R [W][N][3]: dlogpsi [W][Nn][3] =
// d ln|Psi| / dR_alpha and dEL [W][Nn][3] = d E_L / dR_alpha (either may be NULL).  The
// nucleus positions enter the basis centres, the e-n and e-e-n Jastrow terms and V; each of
// the 3 Nn coordinates gets one forward-mode tangent through the whole evaluation, as the
// parameters do for E_L,j (Sec. 2.3.1, the definition after Eq. H0j).
int orc_nuclear_derivs(const orc_system* in, int W, const double* R, double* dlogpsi, double* dEL, int nthreads) {
  Sys s;
  int rc = build_sys(in, s);
  if (rc) return rc;
  const int N = s.N, K = 3 * s.Nn;
  parallel_for(W, nthreads, [&](int w) {
    const double* Rw = R + (size_t)w * 3 * N;
    for (int q = 0; q < K; ++q) {
      Params<Dual<double>> Pq = make_params<Dual<double>>(s, s.P + q);
      Eval<Dual<double>> ed = evaluate(s, Pq, Rw, dEL != nullptr);
      if (dlogpsi) dlogpsi[(size_t)w * K + q] = ed.logpsi.d;
      if (dEL) dEL[(size_t)w * K + q] = ed.eloc.d;
    }
  });
  return 0;
}

// VMC (Sec. 2.3.1): nsweeps sweeps of single-electron Metropolis moves, r' = r + step*(2u-1)
// per coordinate, accepted when u_acc < |Psi(R')/Psi(R)|^2.  Random numbers: Philox keyed by
// seed, counter (walker_id, step0 + sweep, electron, (system << 8) | purpose), purpose 0 gives
// (u_x, u_y), purpose 1 gives (u_z, u_acc).
// Outputs (may be NULL): eloc_hist [nsweeps][W] E_L after each sweep; logpsi [W]; nacc [W].
int orc_vmc(const orc_system* in, int W, double* R, int nsweeps, double step, uint64_t seed, uint32_t step0,
            uint32_t system, const int* walker_id, double* eloc_hist, double* logpsi_out, int* nacc, int nthreads) {
  Sys s;
  int rc = build_sys(in, s);
  if (rc) return rc;
  const int N = s.N;
  Params<double> P0 = make_params<double>(s, -1);
  parallel_for(W, nthreads, [&](int w) {
    double* Rw = R + (size_t)w * 3 * N;
    uint32_t wid = walker_id ? (uint32_t)walker_id[w] : (uint32_t)w;
    double lp = evaluate(s, P0, Rw, false).logpsi;
    int acc = 0;
    std::vector<double> Rn(Rw, Rw + 3 * N);
    for (int sw = 0; sw < nsweeps; ++sw) {
      uint32_t st = step0 + (uint32_t)sw;
      for (int e = 0; e < N; ++e) {
        double u01[2], u23[2];
        uniforms2(seed, wid, st, (uint32_t)e, system, 0, u01);
        uniforms2(seed, wid, st, (uint32_t)e, system, 1, u23);
        double u[3] = {u01[0], u01[1], u23[0]};
        for (int d = 0; d < 3; ++d) {
          double dx = step * (2.0 * u[d] - 1.0);
          Rn[3 * e + d] = Rw[3 * e + d] + dx;
        }
        double lpn = evaluate(s, P0, Rn.data(), false).logpsi;
        double prob = std::exp(2.0 * (lpn - lp));
        if (u23[1] < prob) {
          for (int d = 0; d < 3; ++d) Rw[3 * e + d] = Rn[3 * e + d];
          lp = lpn;
          ++acc;
        } else {
          for (int d = 0; d < 3; ++d) Rn[3 * e + d] = Rw[3 * e + d];
        }
      }
      if (eloc_hist) eloc_hist[(size_t)sw * W + w] = evaluate(s, P0, Rw, true).eloc;
    }
    if (logpsi_out) logpsi_out[w] = lp;
    if (nacc) nacc[w] = acc;
  });
  return 0;
}

// Fixed-node DMC (Sec. 2.3.2) with the plain step described at the top of this file.
// Population in R [cap][N][3], weights are reset to 1 by branching.  For each step the
// random numbers are Philox with counter (walker index, step0 + step, slot, (system<<8)|purpose):
// slot e < N, purposes 2 and 3 give the four uniforms for the Box-Muller normals of electron e
// (purpose 2: z_x, z_y from (u0, u1); purpose 3: z_z from (u2, u3), cosine branch);
// slot N, purpose 4 gives (u_acc, u_branch).
// Outputs per step (may be NULL): sum_wE [nsteps], sum_w [nsteps], pop [nsteps] (after branching),
// e_trial [nsteps] (after update).  *W_io: population in/out.  Returns 0, or -3 if the
// population exceeds cap.
// The drift of Umrigar, Nightingale and Runge limited per electron (a = 1); returns the
// ratio |Vbar| / |V| of the whole walker (1 where V = 0).
static double limited_drift(int N, const double* v, double tau, double* vbar) {
  double n2 = 0.0, nb2 = 0.0;
  for (int e = 0; e < N; ++e) {
    const double* g = v + 3 * e;
    const double v2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const double x = v2 * tau;
    const double f = x > 0.0 ? (-1.0 + std::sqrt(1.0 + 2.0 * x)) / x : 1.0;
    for (int d = 0; d < 3; ++d) vbar[3 * e + d] = f * g[d];
    n2 += v2;
    nb2 += f * f * v2;
  }
  return n2 > 0.0 ? std::sqrt(nb2 / n2) : 1.0;
}

int orc_dmc(const orc_system* in, int cap, int* W_io, double* R, int nsteps, double tau, double* E_T_io,
            int target, uint64_t seed, uint32_t step0, uint32_t system, uint32_t walker_offset, double* sum_wE,
            double* sum_w, int* pop_out, double* et_out, int nthreads) {
  Sys s;
  int rc = build_sys(in, s);
  if (rc) return rc;
  const int N = s.N;
  Params<double> P0 = make_params<double>(s, -1);
  int W = *W_io;
  double E_T = *E_T_io;
  std::vector<double> Rnext;
  for (int k = 0; k < nsteps; ++k) {
    uint32_t st = step0 + (uint32_t)k;
    std::vector<double> wt(W), EL(W), EB(W);
    std::vector<int> copies(W);
    parallel_for(W, nthreads, [&](int w) {
      double* Rw = R + (size_t)w * 3 * N;
      const uint32_t wid = walker_offset + (uint32_t)w;
      Eval<double> e0 = evaluate(s, P0, Rw, true);
      std::vector<double> Rp(3 * N), vb0(3 * N), vb1(3 * N);
      const double lim0 = limited_drift(N, e0.grad.data(), tau, vb0.data());
      for (int e = 0; e < N; ++e) {
        double ua[2], ub[2];
        uniforms2(seed, wid, st, (uint32_t)e, system, 2, ua);
        uniforms2(seed, wid, st, (uint32_t)e, system, 3, ub);
        double ra = std::sqrt(-2.0 * std::log(1.0 - ua[0]));
        double rb = std::sqrt(-2.0 * std::log(1.0 - ub[0]));
        double z[3] = {ra * std::cos(2.0 * M_PI * ua[1]), ra * std::sin(2.0 * M_PI * ua[1]),
                       rb * std::cos(2.0 * M_PI * ub[1])};
        for (int d = 0; d < 3; ++d)
          Rp[3 * e + d] = Rw[3 * e + d] + tau * vb0[3 * e + d] + std::sqrt(tau) * z[d];
      }
      Eval<double> e1 = evaluate(s, P0, Rp.data(), true);
      const double lim1 = limited_drift(N, e1.grad.data(), tau, vb1.data());
      double uu[2];
      uniforms2(seed, wid, st, (uint32_t)N, system, 4, uu);
      bool accept = false;
      if (e1.sign == e0.sign && e1.sign != 0.0) {
        // -|R'-R-tau vbar(R)|^2/2tau and -|R-R'-tau vbar(R')|^2/2tau
        double lg_fwd = 0.0, lg_rev = 0.0;
        for (int q = 0; q < 3 * N; ++q) {
          double f = Rp[q] - Rw[q] - tau * vb0[q];
          double b = Rw[q] - Rp[q] - tau * vb1[q];
          lg_fwd += f * f;
          lg_rev += b * b;
        }
        double lnratio = 2.0 * (e1.logpsi - e0.logpsi) - lg_rev / (2.0 * tau) + lg_fwd / (2.0 * tau);
        accept = uu[0] < std::exp(lnratio);
      }
      double Enew = accept ? e1.eloc : e0.eloc;
      if (accept)
        for (int q = 0; q < 3 * N; ++q) Rw[q] = Rp[q];
      // branching energies limited in proportion to the drift, then cut off
      const double ecut = 0.2 * std::sqrt((double)N / tau);
      const double Eb0 = E_T + std::max(-ecut, std::min(ecut, (e0.eloc - E_T) * lim0));
      const double Eb1 = E_T + std::max(-ecut, std::min(ecut, (Enew - E_T) * (accept ? lim1 : lim0)));
      double w1 = std::exp(-tau * (0.5 * (Eb0 + Eb1) - E_T));
      wt[w] = w1;
      EL[w] = Enew;
      EB[w] = Eb1;
      int c = (int)std::floor(w1 + uu[1]);
      copies[w] = std::min(c, 3);
    });
    double swE = 0.0, sw = 0.0, swEb = 0.0;
    for (int w = 0; w < W; ++w) { swE += wt[w] * EL[w]; sw += wt[w]; swEb += wt[w] * EB[w]; }
    int total = 0;
    for (int w = 0; w < W; ++w) total += copies[w];
    if (total > cap) return -3;
    Rnext.assign((size_t)total * 3 * N, 0.0);
    int pos = 0;
    for (int w = 0; w < W; ++w)
      for (int c = 0; c < copies[w]; ++c, ++pos)
        std::copy(R + (size_t)w * 3 * N, R + (size_t)(w + 1) * 3 * N, Rnext.begin() + (size_t)pos * 3 * N);
    std::copy(Rnext.begin(), Rnext.end(), R);
    W = total;
    double Ebmean = sw > 0 ? swEb / sw : E_T;
    if (W > 0) E_T = Ebmean - (0.1 / tau) * std::log((double)W / (double)target);
    if (sum_wE) sum_wE[k] = swE;
    if (sum_w) sum_w[k] = sw;
    if (pop_out) pop_out[k] = W;
    if (et_out) et_out[k] = E_T;
    if (W == 0) break;
  }
  *W_io = W;
  *E_T_io = E_T;
  return 0;
}

}  // extern "C"
