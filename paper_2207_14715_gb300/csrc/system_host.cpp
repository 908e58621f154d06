// Host-side set-up of a JVB system: validation, basis normalisation, HLSP structure
// expansion into determinants (arXiv:2207.14715, Sec. 2.1, Eq. PhiI and the expansion
// after it), the cusp-preserving e-e-n parametrisation (Sec. 2.1, last paragraph) and the
// orbital-excitation tables (Sec. 2.2).
#include <algorithm>
#include <cmath>
#include <map>
#include <sstream>

#include "vbqmc_internal.h"

namespace vbq {

static const int kNcomp[3] = {1, 3, 6};
static const int kCart[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                 {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
static const int kCartOff[3] = {0, 1, 4};

std::vector<EenTerm> een_term_list() {
  std::vector<EenTerm> t;
  for (int p = 2; p <= 5; ++p)
    for (int k = 0; k < p; ++k) {
      const int lmax = k ? p - k : p - k - 2;
      for (int l = 0; l <= lmax; ++l)
        if ((p - k - l) % 2 == 0) t.push_back({p, k, l, (p - k - l) / 2});
    }
  return t;
}

// Linear conditions on the raw e-e-n coefficients that keep both cusps of the Jastrow.
// With u = Rbar(r_ij), s = Rbar(r_ia), t = Rbar(r_ja) and dRbar/dr(0) = -kappa:
//  * r_ij -> 0 (then s = t): d term / d r_ij = -2 kappa k s^(p-k), so for every power q
//    the coefficients with p - k = q satisfy sum k c = 0;
//  * r_ia -> 0 (then s = 1 and u = t): d term / d s = (l+m) t^(k+m) + m t^(k+l+m), so for
//    every power q of t the collected coefficients sum to zero.
// The free coefficients span the null space; B holds the basis read off the reduced row
// echelon form (free columns in ascending order), so c = B theta.
static void een_free_basis(std::vector<double>& B) {
  const std::vector<EenTerm> T = een_term_list();
  const int nt = (int)T.size();
  std::vector<std::vector<double>> rows;
  for (int q = 1; q <= 5; ++q) {
    std::vector<double> r(nt, 0.0);
    bool used = false;
    for (int i = 0; i < nt; ++i)
      if (T[i].k >= 1 && T[i].p - T[i].k == q) { r[i] = T[i].k; used = true; }
    if (used) rows.push_back(r);
  }
  for (int q = 0; q <= 6; ++q) {
    std::vector<double> r(nt, 0.0);
    bool used = false;
    for (int i = 0; i < nt; ++i) {
      double v = 0.0;
      if (T[i].k + T[i].m == q) v += T[i].l + T[i].m;
      if (T[i].k + T[i].l + T[i].m == q) v += T[i].m;
      if (v != 0.0) { r[i] = v; used = true; }
    }
    if (used) rows.push_back(r);
  }
  const int nr = (int)rows.size();
  std::vector<int> piv;
  int r = 0;
  for (int col = 0; col < nt && r < nr; ++col) {
    int best = -1;
    double bv = 1e-9;
    for (int i = r; i < nr; ++i)
      if (std::fabs(rows[i][col]) > bv) { bv = std::fabs(rows[i][col]); best = i; }
    if (best < 0) continue;
    std::swap(rows[r], rows[best]);
    const double pv = rows[r][col];
    for (double& x : rows[r]) x /= pv;
    for (int i = 0; i < nr; ++i) {
      if (i == r || rows[i][col] == 0.0) continue;
      const double f = rows[i][col];
      for (int j = 0; j < nt; ++j) rows[i][j] -= f * rows[r][j];
    }
    piv.push_back(col);
    ++r;
  }
  std::vector<int> is_free(nt, 1);
  for (int c : piv) is_free[c] = 0;
  std::vector<int> freecols;
  for (int j = 0; j < nt; ++j)
    if (is_free[j]) freecols.push_back(j);
  const int nf = (int)freecols.size();
  B.assign((size_t)nt * kNfree, 0.0);
  for (int f = 0; f < nf && f < kNfree; ++f) {
    B[(size_t)freecols[f] * kNfree + f] = 1.0;
    for (size_t i = 0; i < piv.size(); ++i) B[(size_t)piv[i] * kNfree + f] = -rows[i][freecols[f]];
  }
}

static double double_factorial(int n) {
  double r = 1.0;
  for (int i = n; i > 1; i -= 2) r *= i;
  return r;
}

// Parity of the permutation that sorts v ascending (v has distinct entries).
static int sort_parity(std::vector<int>& v) {
  int inv = 0;
  for (size_t i = 0; i < v.size(); ++i)
    for (size_t j = i + 1; j < v.size(); ++j)
      if (v[i] > v[j]) ++inv;
  std::sort(v.begin(), v.end());
  return inv & 1;
}

struct RawDet {
  std::vector<int> up, dn;
  double sign;
};

// All signed determinants of one HLSP structure.  A pair (i, j), i != j, contributes
// a+_{i up} a+_{j dn} - a+_{i dn} a+_{j up}; a self pair (i, i) contributes a+_{i up} a+_{i dn}
// (the factor 2 is dropped: structures are unnormalised).  Each product of creation
// operators is reordered to (up operators ascending)(down operators ascending); the
// permutation parity multiplies the sign.  Strings with a repeated spin orbital vanish.
static void expand_structure(const std::vector<int>& inact, const std::vector<std::pair<int, int>>& pairs,
                             const std::vector<int>& unp, std::vector<RawDet>& out) {
  const int np = (int)pairs.size();
  std::vector<int> choice(np, 0);
  for (;;) {
    std::vector<std::pair<int, int>> ops;  // (orbital, spin)
    double sgn = 1.0;
    for (int p : inact) { ops.push_back({p, 0}); ops.push_back({p, 1}); }
    for (int q = 0; q < np; ++q) {
      if (choice[q] == 0) { ops.push_back({pairs[q].first, 0}); ops.push_back({pairs[q].second, 1}); }
      else { ops.push_back({pairs[q].first, 1}); ops.push_back({pairs[q].second, 0}); sgn = -sgn; }
    }
    for (int q : unp) ops.push_back({q, 0});
    int crossings = 0, downs = 0;
    RawDet d;
    for (auto& o : ops) {
      if (o.second == 1) { ++downs; d.dn.push_back(o.first); }
      else { crossings += downs; d.up.push_back(o.first); }
    }
    if (crossings & 1) sgn = -sgn;
    if (sort_parity(d.up)) sgn = -sgn;
    if (sort_parity(d.dn)) sgn = -sgn;
    bool pauli = false;
    for (auto* v : {&d.up, &d.dn})
      for (size_t x = 1; x < v->size(); ++x)
        if ((*v)[x] == (*v)[x - 1]) pauli = true;
    d.sign = sgn;
    if (!pauli) out.push_back(d);
    int q = 0;
    for (; q < np; ++q) {
      const int nch = pairs[q].first == pairs[q].second ? 1 : 2;
      if (++choice[q] < nch) break;
      choice[q] = 0;
    }
    if (q == np) break;
  }
}

// Splits the nonzero coefficient ranges of the given orbitals into chunks so that 32 lanes
// finish together.  The chunk length L minimises the critical path of one warp:
//   ceil(chunks(L) / 32) * (L + 8)  [chunk loop, 8 ~ per-chunk overhead]
//   + ceil(orbitals / 32) * max chunks of one orbital  [per-orbital sum of the partials],
// with L >= 4.
static void make_chunks(const SysHost& s, const std::vector<int>& orbs, std::vector<int>& chunks,
                        std::vector<int>& off) {
  chunks.clear();
  off.assign(1, 0);
  int maxlen = 1;
  for (int k : orbs) maxlen = std::max(maxlen, s.orb_hi[k] - s.orb_lo[k]);
  int bestL = maxlen;
  long bestcost = -1;
  const long norb = (long)orbs.size();
  for (int L = std::min(4, maxlen); L <= maxlen; ++L) {
    long nch = 0, maxc = 1;
    for (int k : orbs) {
      const long c = std::max(1, (s.orb_hi[k] - s.orb_lo[k] + L - 1) / L);
      nch += c;
      maxc = std::max(maxc, c);
    }
    const long cost = ((nch + 31) / 32) * (L + 8) + ((norb + 31) / 32) * maxc;
    if (bestcost < 0 || cost < bestcost) { bestcost = cost; bestL = L; }
  }
  for (size_t q = 0; q < orbs.size(); ++q) {
    const int k = orbs[q], lo = s.orb_lo[k], hi = s.orb_hi[k], len = hi - lo;
    const int nc = std::max(1, (len + bestL - 1) / bestL);
    for (int c = 0; c < nc; ++c) {
      const int b = lo + (int)((long)len * c / nc), e = lo + (int)((long)len * (c + 1) / nc);
      chunks.insert(chunks.end(), {(int)q, b, e, s.orb_off[k] - lo});
    }
    off.push_back((int)(chunks.size() / 4));
  }
}

// Groups the evaluated orbitals for the contraction: width 1 (each orbital alone) or width 4
// (quads of orbitals with equal coefficient range, in order of first appearance, so that one
// basis-function load feeds four orbitals).  Each group's range is split into chunks of
// length L; the modelled critical path of one warp is
//   ceil(chunks / 32) * (c_mu L + 12)  [chunk loop; c_mu ~ instructions per mu: 8 or 23]
//   + ceil(orbitals / 32) * 5 * max chunks of one group  [per-orbital sum of the partials],
// and the width and L with the shorter path are taken.
static long plan_groups(const SysHost& s, int width, std::vector<std::vector<int>>& groups, int& bestL) {
  const std::vector<int>& orbs = s.ev_orb;
  groups.clear();
  std::vector<std::pair<int, int>> open_rng;
  std::vector<int> open_g;
  for (size_t q = 0; q < orbs.size(); ++q) {
    const std::pair<int, int> rng{s.orb_lo[orbs[q]], s.orb_hi[orbs[q]]};
    size_t g = 0;
    while (g < open_rng.size() && open_rng[g] != rng) ++g;
    if (g == open_rng.size()) {
      open_rng.push_back(rng);
      open_g.push_back(-1);
    }
    if (open_g[g] < 0 || (int)groups[open_g[g]].size() == width) {
      open_g[g] = (int)groups.size();
      groups.emplace_back();
    }
    groups[open_g[g]].push_back((int)q);
  }
  int maxlen = 1;
  for (auto& v : groups) maxlen = std::max(maxlen, s.orb_hi[orbs[v[0]]] - s.orb_lo[orbs[v[0]]]);
  const long cmu = width == 4 ? 23 : 8;
  long bestcost = -1;
  bestL = maxlen;
  for (int L = std::min(4, maxlen); L <= maxlen; ++L) {
    long nch = 0, maxc = 1;
    for (auto& v : groups) {
      const long c = std::max(1, (s.orb_hi[orbs[v[0]]] - s.orb_lo[orbs[v[0]]] + L - 1) / L);
      nch += c;
      maxc = std::max(maxc, c);
    }
    const long cost = ((nch + 31) / 32) * (cmu * L + 12) + (((long)orbs.size() + 31) / 32) * 5 * maxc;
    if (bestcost < 0 || cost < bestcost) { bestcost = cost; bestL = L; }
  }
  return bestcost;
}

static void make_quads(SysHost& s) {
  const std::vector<int>& orbs = s.ev_orb;
  std::vector<std::vector<int>> g1, g4;
  int L1 = 1, L4 = 1;
  const long c1 = plan_groups(s, 1, g1, L1), c4 = plan_groups(s, 4, g4, L4);
  const int width = c4 < c1 ? 4 : 1, bestL = width == 4 ? L4 : L1;
  const std::vector<std::vector<int>>& groups = width == 4 ? g4 : g1;
  s.evq_width = width;
  s.evq_slot.assign(orbs.size(), 0);
  s.evq_chunk.clear();
  s.evq_coef.clear();
  s.evq_chunk_off.assign(1, 0);
  for (size_t qd = 0; qd < groups.size(); ++qd) {
    const int k0 = orbs[groups[qd][0]], lo = s.orb_lo[k0], hi = s.orb_hi[k0], len = hi - lo;
    const int qoff = (int)s.evq_coef.size();
    s.evq_coef.resize(qoff + width * (size_t)len, 0.0);
    for (size_t t = 0; t < groups[qd].size(); ++t) {
      const int k = orbs[groups[qd][t]];
      s.evq_slot[groups[qd][t]] = 4 * (int)qd + (int)t;
      for (int mu = lo; mu < hi; ++mu) s.evq_coef[qoff + width * (mu - lo) + t] = s.orb_coef[s.orb_off[k] + mu - lo];
    }
    const int nc = std::max(1, (len + bestL - 1) / bestL);
    for (int c = 0; c < nc; ++c) {
      const int b = lo + (int)((long)len * c / nc), e = lo + (int)((long)len * (c + 1) / nc);
      s.evq_chunk.insert(s.evq_chunk.end(), {(int)qd, b, e, qoff - width * lo});
    }
    s.evq_chunk_off.push_back((int)(s.evq_chunk.size() / 4));
  }
}

#define VBQ_REQUIRE(cond, msg)                 \
  do {                                         \
    if (!(cond)) {                             \
      std::ostringstream os_;                  \
      os_ << msg;                              \
      err = os_.str();                         \
      return VBQMC_ERR_ARG;                    \
    }                                          \
  } while (0)

int build_system(const vbqmc_system_desc* d, SysHost& s, std::string& err) {
  VBQ_REQUIRE(d != nullptr, "null system description");
  VBQ_REQUIRE(d->Nn >= 1 && d->n_elem >= 1 && d->S >= 1 && d->Norb >= 1 && d->Nvb >= 1, "empty system");
  VBQ_REQUIRE(d->Nn < 65536, "more than 65535 nuclei");
  VBQ_REQUIRE(d->n_elem <= kMaxElem, "too many elements");
  VBQ_REQUIRE(d->Nup >= 0 && d->Ndn >= 0 && d->Nup + d->Ndn >= 1, "bad electron counts");
  if (d->Nup > kMaxSpinN || d->Ndn > kMaxSpinN || d->Nup + d->Ndn > kMaxN) {
    err = "electron count beyond kernel limits (N <= 64, per spin <= 32)";
    return VBQMC_ERR_CAPACITY;
  }
  VBQ_REQUIRE(d->nuc_xyz && d->nuc_Z && d->nuc_elem && d->sh_center && d->sh_l && d->sh_zeta && d->orb_coef &&
                  d->c_vb && d->inact_off && d->pair_off && d->unp_off && d->jas_a && d->jas_b,
              "missing array");
  s = SysHost();
  s.Nn = d->Nn; s.n_elem = d->n_elem; s.S = d->S; s.Norb = d->Norb; s.Nvb = d->Nvb;
  s.Nup = d->Nup; s.Ndn = d->Ndn; s.N = d->Nup + d->Ndn;
  s.nuc4.resize(4 * s.Nn);
  for (int a = 0; a < s.Nn; ++a) {
    for (int c = 0; c < 3; ++c) s.nuc4[4 * a + c] = d->nuc_xyz[3 * a + c];
    s.nuc4[4 * a + 3] = d->nuc_Z[a];
    VBQ_REQUIRE(d->nuc_elem[a] >= 0 && d->nuc_elem[a] < s.n_elem, "nucleus " << a << ": bad element id");
    VBQ_REQUIRE(std::isfinite(d->nuc_Z[a]), "non-finite nuclear charge");
  }
  s.nuc_elem.assign(d->nuc_elem, d->nuc_elem + s.Nn);
  // basis
  s.sh_center.assign(d->sh_center, d->sh_center + s.S);
  s.sh_l.assign(d->sh_l, d->sh_l + s.S);
  s.sh_zeta.assign(d->sh_zeta, d->sh_zeta + s.S);
  s.sh_first.resize(s.S);
  s.sh_norm.assign((size_t)6 * s.S, 0.0);
  int M = 0;
  for (int i = 0; i < s.S; ++i) {
    const int l = s.sh_l[i];
    VBQ_REQUIRE(l >= 0 && l <= 2, "shell " << i << ": l must be 0, 1 or 2");
    VBQ_REQUIRE(s.sh_center[i] >= 0 && s.sh_center[i] < s.Nn, "shell " << i << ": bad center");
    VBQ_REQUIRE(s.sh_zeta[i] >= 0.0 && std::isfinite(s.sh_zeta[i]), "shell " << i << ": bad exponent");
    const int kind = d->sh_kind ? d->sh_kind[i] : 0;
    VBQ_REQUIRE(kind == 0 || kind == 1, "shell " << i << ": kind must be 0 (Gaussian) or 1 (Slater)");
    VBQ_REQUIRE(kind == 0 || s.sh_zeta[i] > 0.0, "shell " << i << ": a Slater shell needs zeta > 0");
    s.sh_first[i] = M;
    const double z = s.sh_zeta[i];
    for (int c = 0; c < kNcomp[l]; ++c) {
      const int* e = kCart[kCartOff[l] + c];
      const double dfc = double_factorial(2 * e[0] - 1) * double_factorial(2 * e[1] - 1) *
                         double_factorial(2 * e[2] - 1);
      double nrm = 1.0;
      if (kind == 1) {
        // N^2 = (2 zeta)^(2l+3) (2l+1)!! / (4 pi (2l+2)! (2a-1)!!(2b-1)!!(2c-1)!!): the
        // monomial's angular integral times the radial integral of r^(2l+2) e^{-2 zeta r}
        double f = 1.0;
        for (int k = 2; k <= 2 * l + 2; ++k) f *= k;
        nrm = std::sqrt(std::pow(2.0 * z, 2 * l + 3) * double_factorial(2 * l + 1) / (4.0 * M_PI * f * dfc));
      } else if (z > 0.0) {
        nrm = std::pow(2.0 * z / M_PI, 0.75) * std::pow(4.0 * z, 0.5 * l) / std::sqrt(dfc);
      }
      s.sh_norm[(size_t)6 * i + c] = nrm;
    }
    // device encoding: a Slater shell carries its exponent negated (the kernels branch on the sign)
    if (kind == 1) {
      s.sh_zeta[i] = -z;
      s.has_slater = 1;
    }
    M += kNcomp[l];
  }
  s.sh_by_l.clear();
  for (int l = 0; l <= 2; ++l)
    for (int i = 0; i < s.S; ++i)
      if (s.sh_l[i] == l) s.sh_by_l.push_back(i);
  if (M > kMaxM) {
    err = "basis larger than 1024 functions";
    return VBQMC_ERR_CAPACITY;
  }
  s.M = M;
  // shells and basis functions of each nucleus: one contiguous run per nucleus
  s.nuc_sh.assign((size_t)4 * s.Nn, 0);
  s.max_nuc_mu = 0;
  for (int i = 0; i < s.S;) {
    const int a = s.sh_center[i];
    VBQ_REQUIRE(s.nuc_sh[4 * a + 1] == 0, "shells of nucleus " << a << " are not contiguous");
    int j = i;
    while (j < s.S && s.sh_center[j] == a) ++j;
    const int mu1 = j < s.S ? s.sh_first[j] : M;
    s.nuc_sh[4 * a] = i;
    s.nuc_sh[4 * a + 1] = j;
    s.nuc_sh[4 * a + 2] = s.sh_first[i];
    s.nuc_sh[4 * a + 3] = mu1;
    s.max_nuc_mu = std::max(s.max_nuc_mu, mu1 - s.sh_first[i]);
    i = j;
  }
  // orbital coefficient ranges
  s.orb_lo.resize(s.Norb);
  s.orb_hi.resize(s.Norb);
  s.orb_off.resize(s.Norb);
  for (int k = 0; k < s.Norb; ++k) {
    const double* row = d->orb_coef + (size_t)k * M;
    int lo = -1, hi = -1;
    for (int mu = 0; mu < M; ++mu) {
      VBQ_REQUIRE(std::isfinite(row[mu]), "orbital " << k << ": non-finite coefficient");
      if (row[mu] != 0.0) {
        if (lo < 0) lo = mu;
        hi = mu + 1;
      }
    }
    if (lo < 0) { lo = 0; hi = 0; }
    s.orb_lo[k] = lo;
    s.orb_hi[k] = hi;
    s.orb_off[k] = (int)s.orb_coef.size();
    for (int mu = lo; mu < hi; ++mu) s.orb_coef.push_back(row[mu]);
  }
  // structures -> determinants
  std::map<std::vector<int>, int> up_id, dn_id;
  std::vector<std::vector<int>> ups, dns;
  std::map<std::pair<int, int>, int> term_id;
  std::map<std::pair<int, int>, int> sterm_id;
  for (int I = 0; I < s.Nvb; ++I) {
    VBQ_REQUIRE(std::isfinite(d->c_vb[I]), "non-finite structure coefficient");
    std::vector<int> ina, unp;
    std::vector<std::pair<int, int>> prs;
    for (int q = d->inact_off[I]; q < d->inact_off[I + 1]; ++q) ina.push_back(d->inact[q]);
    for (int q = d->pair_off[I]; q < d->pair_off[I + 1]; ++q) prs.push_back({d->pairs[2 * q], d->pairs[2 * q + 1]});
    for (int q = d->unp_off[I]; q < d->unp_off[I + 1]; ++q) unp.push_back(d->unp[q]);
    for (int o : ina) VBQ_REQUIRE(o >= 0 && o < s.Norb, "structure " << I << ": bad orbital");
    for (int o : unp) VBQ_REQUIRE(o >= 0 && o < s.Norb, "structure " << I << ": bad orbital");
    for (auto& p : prs)
      VBQ_REQUIRE(p.first >= 0 && p.first < s.Norb && p.second >= 0 && p.second < s.Norb,
                  "structure " << I << ": bad orbital");
    VBQ_REQUIRE((int)(2 * ina.size() + 2 * prs.size() + unp.size()) == s.N,
                "structure " << I << ": electron count differs from Nup + Ndn");
    VBQ_REQUIRE((int)(ina.size() + prs.size() + unp.size()) == s.Nup, "structure " << I << ": spin count mismatch");
    std::vector<RawDet> raw;
    expand_structure(ina, prs, unp, raw);
    for (auto& r : raw) {
      auto iu = up_id.find(r.up);
      if (iu == up_id.end()) { iu = up_id.insert({r.up, (int)ups.size()}).first; ups.push_back(r.up); }
      auto idn = dn_id.find(r.dn);
      if (idn == dn_id.end()) { idn = dn_id.insert({r.dn, (int)dns.size()}).first; dns.push_back(r.dn); }
      std::pair<int, int> key(iu->second, idn->second);
      auto it = term_id.find(key);
      if (it == term_id.end()) {
        it = term_id.insert({key, (int)s.term_coef.size()}).first;
        s.term_det.push_back(key.first);
        s.term_det.push_back(key.second);
        s.term_coef.push_back(0.0);
      }
      s.term_coef[it->second] += d->c_vb[I] * r.sign;
      std::pair<int, int> sk(I, it->second);
      auto st = sterm_id.find(sk);
      if (st == sterm_id.end()) {
        sterm_id.insert({sk, (int)s.sterm_d.size()});
        s.sterm_I.push_back(I);
        s.sterm_k.push_back(it->second);
        s.sterm_d.push_back(r.sign);
      } else {
        s.sterm_d[st->second] += r.sign;
      }
    }
  }
  VBQ_REQUIRE(!s.term_coef.empty(), "every determinant vanishes");
  s.U[0] = (int)ups.size();
  s.U[1] = (int)dns.size();
  s.n[0] = s.Nup;
  s.n[1] = s.Ndn;
  // orbitals used by each spin; eval orbital list = det orbitals, then excitation targets
  std::vector<int> in_det(s.Norb, 0);
  for (int sp = 0; sp < 2; ++sp) {
    auto& sets = sp == 0 ? ups : dns;
    std::vector<int> used(s.Norb, 0);
    for (auto& v : sets)
      for (int o : v) used[o] = 1, in_det[o] = 1;
    for (int k = 0; k < s.Norb; ++k)
      if (used[k]) s.occ_list[sp].push_back(k);
  }
  std::vector<int> ev_of(s.Norb, -1);
  for (int k = 0; k < s.Norb; ++k)
    if (in_det[k]) { ev_of[k] = (int)s.ev_orb.size(); s.ev_orb.push_back(k); }
  s.n_ev_det = (int)s.ev_orb.size();
  s.n_kappa = d->n_kappa;
  for (int j = 0; j < s.n_kappa; ++j) {
    const int k = d->kappa_kl[2 * j], l = d->kappa_kl[2 * j + 1];
    VBQ_REQUIRE(k >= 0 && k < s.Norb && l >= 0 && l < s.Norb && k != l, "orbital excitation " << j << ": bad (k, l)");
    if (ev_of[k] < 0) { ev_of[k] = (int)s.ev_orb.size(); s.ev_orb.push_back(k); }
  }
  for (int sp = 0; sp < 2; ++sp) {
    auto& sets = sp == 0 ? ups : dns;
    std::vector<int> loc(s.Norb, -1);
    for (size_t q = 0; q < s.occ_list[sp].size(); ++q) loc[s.occ_list[sp][q]] = (int)q;
    for (auto& v : sets)
      for (int o : v) {
        s.det_loc[sp].push_back(loc[o]);
        s.det_ev[sp].push_back(ev_of[o]);
        s.det_glob[sp].push_back(o);
      }
    // excitation entries: phi_l -> phi_l + eps phi_k changes a determinant only if l is
    // occupied in it and k is not (otherwise two equal columns)
    s.kap_off[sp].push_back(0);
    for (size_t u = 0; u < sets.size(); ++u) {
      for (int j = 0; j < s.n_kappa; ++j) {
        const int k = d->kappa_kl[2 * j], l = d->kappa_kl[2 * j + 1];
        int slot = -1;
        bool has_k = false;
        for (int o = 0; o < (int)sets[u].size(); ++o) {
          if (sets[u][o] == l) slot = o;
          if (sets[u][o] == k) has_k = true;
        }
        if (slot < 0 || has_k) continue;
        s.kap_ent[sp].insert(s.kap_ent[sp].end(), {j, slot, ev_of[k], 0});
      }
      s.kap_off[sp].push_back((int)(s.kap_ent[sp].size() / 4));
    }
  }
  s.kap_x.assign(4 * (size_t)s.n_kappa, -1);
  for (int j = 0; j < s.n_kappa; ++j) {
    s.kap_x[4 * j + 2] = ev_of[d->kappa_kl[2 * j]];
    s.kap_x[4 * j + 3] = 0;
  }
  for (int sp = 0; sp < 2; ++sp)
    for (size_t t = 0; t < s.kap_ent[sp].size() / 4; ++t) {
      const int j = s.kap_ent[sp][4 * t];
      s.kap_x[4 * j + sp] = ev_of[d->kappa_kl[2 * j + 1]];
    }
  // reference-determinant tables: determinant u of a spin is the reference (u = 0) with the
  // slots S_u replaced by the orbitals Q_u (k_u <= kMaxExc each, ascending, paired in order),
  // up to the parity of the column permutation from that replaced column list to u's own
  // column order: D_u = sgn_u D_0 det(T[S_u, Q_u]) with T = A_0^-1 Phi.
  s.tab_ok = 1;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], U = s.U[sp];
    s.tab_x[sp].clear();
    s.tab_det[sp].assign((size_t)U * kTabStride, 0);
    if (n == 0) continue;
    const int* ref = s.det_ev[sp].data();
    std::vector<char> in_ref(s.ev_orb.size(), 0);
    for (int o = 0; o < n; ++o) in_ref[ref[o]] = 1;
    std::vector<int> xpos(s.ev_orb.size(), -1);
    for (int u = 0; u < U; ++u)
      for (int o = 0; o < n; ++o) {
        const int q = s.det_ev[sp][(size_t)u * n + o];
        if (!in_ref[q] && xpos[q] < 0) xpos[q] = 0;
      }
    for (size_t q = 0; q < xpos.size(); ++q)
      if (xpos[q] == 0) { xpos[q] = (int)s.tab_x[sp].size(); s.tab_x[sp].push_back((int)q); }
    s.tab_xl[sp].clear();
    for (int q : s.tab_x[sp]) {
      const int g = s.ev_orb[q];
      const int pos = (int)(std::find(s.occ_list[sp].begin(), s.occ_list[sp].end(), g) - s.occ_list[sp].begin());
      if (pos >= (int)s.occ_list[sp].size()) s.tab_ok = 0;  // every determinant orbital is in occ_list
      s.tab_xl[sp].push_back(pos);
    }
    for (int u = 0; u < U; ++u) {
      const int* cols = s.det_ev[sp].data() + (size_t)u * n;
      std::vector<char> in_u(s.ev_orb.size(), 0);
      for (int o = 0; o < n; ++o) in_u[cols[o]] = 1;
      std::vector<int> S, Q;
      for (int o = 0; o < n; ++o)
        if (!in_u[ref[o]]) S.push_back(o);
      for (int o = 0; o < n; ++o)
        if (!in_ref[cols[o]]) Q.push_back(cols[o]);
      std::sort(Q.begin(), Q.end());
      if ((int)S.size() > kMaxExc) { s.tab_ok = 0; continue; }
      // replaced column list and the parity of the permutation to u's order
      std::vector<int> rep(ref, ref + n);
      for (size_t j = 0; j < S.size(); ++j) rep[S[j]] = Q[j];
      std::vector<int> pos(n);
      for (int o = 0; o < n; ++o) pos[o] = (int)(std::find(rep.begin(), rep.end(), cols[o]) - rep.begin());
      int par = 0;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
          if (pos[i] > pos[j]) ++par;
      int* t = s.tab_det[sp].data() + (size_t)u * kTabStride;
      t[0] = (int)S.size();
      t[1] = (par & 1) ? -1 : 1;
      for (size_t j = 0; j < S.size(); ++j) {
        t[2 + j] = S[j];
        t[2 + kMaxExc + j] = xpos[Q[j]];
      }
    }
  }
  // contraction work chunks
  for (int sp = 0; sp < 2; ++sp) make_chunks(s, s.occ_list[sp], s.occ_chunk[sp], s.occ_chunk_off[sp]);
  make_quads(s);
  make_chunks(s, std::vector<int>(s.ev_orb.begin(), s.ev_orb.begin() + s.n_ev_det), s.det_chunk, s.det_chunk_off);
  // Jastrow
  s.kappa = d->kappa;
  s.b1_anti = d->b1_anti;
  s.b1_par = d->b1_par;
  s.een_on = d->een_on ? 1 : 0;
  s.jas_a.assign(d->jas_a, d->jas_a + 6 * s.n_elem);
  s.jas_b.assign(d->jas_b, d->jas_b + 6);
  een_free_basis(s.een_B);
  s.een_c.assign((size_t)s.n_elem * kNeen, 0.0);
  if (s.een_on) {
    VBQ_REQUIRE(d->een_theta != nullptr, "een_on without een_theta");
    for (int e = 0; e < s.n_elem; ++e)
      for (int t = 0; t < kNeen; ++t) {
        double v = 0.0;
        for (int f = 0; f < kNfree; ++f) v += s.een_B[(size_t)t * kNfree + f] * d->een_theta[e * kNfree + f];
        s.een_c[(size_t)e * kNeen + t] = v;
      }
  }
  // parameters
  s.cparam.assign(d->cparam, d->cparam + d->n_cparam);
  for (int I : s.cparam) VBQ_REQUIRE(I >= 0 && I < s.Nvb, "bad structure parameter index");
  s.cpar_off.assign(1, 0);
  s.cpar_st.clear();
  for (int I : s.cparam) {
    for (size_t t = 0; t < s.sterm_I.size(); ++t)
      if (s.sterm_I[t] == I) s.cpar_st.push_back((int)t);
    s.cpar_off.push_back((int)s.cpar_st.size());
  }
  {
    const int nterm = (int)s.term_coef.size();
    s.det_term_off.assign(1, 0);
    s.det_term.clear();
    for (int sp = 0; sp < 2; ++sp)
      for (int u = 0; u < s.U[sp]; ++u) {
        for (int k = 0; k < nterm; ++k)
          if (s.term_det[2 * k + sp] == u) s.det_term.push_back(k);
        s.det_term_off.push_back((int)s.det_term.size());
      }
  }
  s.jas_param = d->jas_param ? 1 : 0;
  s.P = (int)s.cparam.size() + (s.jas_param ? 5 * s.n_elem + 5 + (s.een_on ? kNfree * s.n_elem : 0) : 0) +
        s.n_kappa;
  // nucleus-nucleus repulsion
  double vnn = 0.0;
  for (int a = 0; a < s.Nn; ++a)
    for (int b = a + 1; b < s.Nn; ++b) {
      double r2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double x = s.nuc4[4 * a + c] - s.nuc4[4 * b + c];
        r2 += x * x;
      }
      VBQ_REQUIRE(r2 > 0.0, "coincident nuclei");
      vnn += s.nuc4[4 * a + 3] * s.nuc4[4 * b + 3] / std::sqrt(r2);
    }
  s.vnn = vnn;
  return VBQMC_OK;
}

}  // namespace vbq
