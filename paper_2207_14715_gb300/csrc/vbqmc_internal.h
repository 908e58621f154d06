// Internal data layout of the VB-QMC library: the host-side system tables built by
// vbqmc_set_system and the device image the kernels read.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vbqmc.h"

namespace vbq {

constexpr int kMaxN = 64;        // electrons
constexpr int kMaxSpinN = 32;    // electrons of one spin (Slater order <= one warp)
constexpr int kMaxM = 1024;      // basis functions
constexpr int kNeen = 23;        // e-e-n expansion terms per element (Sec. 2.1)
constexpr int kNfree = 15;       // free e-e-n coefficients per element after the cusp conditions
constexpr int kMaxElem = 16;
constexpr int kMaxExc = 4;                   // reference-determinant tables: excitation degree
constexpr int kTabStride = 2 + 2 * kMaxExc;  // per determinant: k, sign, S[kMaxExc], Q[kMaxExc]

// e-e-n terms (p, k, l, m): p = 2..5, k = 0..p-1, l = 0..lmax with lmax = p-k (k != 0) or
// p-k-2 (k = 0), kept when m = (p-k-l)/2 is an integer (Sec. 2.1, f_een).
struct EenTerm { int p, k, l, m; };
std::vector<EenTerm> een_term_list();

// Everything the kernels need, as host vectors (built by build_system).
struct SysHost {
  int N = 0, Nup = 0, Ndn = 0, Nn = 0, n_elem = 0, S = 0, M = 0, Norb = 0, Nvb = 0;
  std::vector<double> nuc4;            // [Nn][4] x y z Z
  std::vector<int> nuc_elem;
  std::vector<int> sh_center, sh_l, sh_first;
  std::vector<int> sh_by_l;            // shells in order of l (lanes of one round run one shell kind)
  std::vector<double> sh_zeta, sh_norm;  // norm [S][6]; zeta < 0: Slater shell with exponent -zeta
  int has_slater = 0;
  std::vector<int> nuc_sh;             // [Nn][4]: first shell, end shell, first and end basis function
  int max_nuc_mu = 0;                  // most basis functions on one nucleus
  // orbitals: nonzero range [lo, hi) per orbital, coefficients packed
  std::vector<int> orb_lo, orb_hi, orb_off;
  std::vector<double> orb_coef;
  // orbitals evaluated in a full evaluation: det orbitals first, then excitation targets
  std::vector<int> ev_orb;             // eval index -> global orbital
  int n_ev_det = 0;                    // first n_ev_det eval orbitals appear in determinants
  // per spin: orbitals appearing in its determinants (global ids, ascending)
  std::vector<int> occ_list[2];
  int U[2] = {0, 0};
  int n[2] = {0, 0};
  std::vector<int> det_loc[2];         // [U][n] index into occ_list[s]
  std::vector<int> det_ev[2];          // [U][n] eval index
  std::vector<int> det_glob[2];        // [U][n] global orbital id
  // reference-determinant tables (usable when tab_ok): eval indices of the determinant
  // orbitals outside the reference determinant u = 0, and per determinant [kTabStride]:
  // k, sign, reference slots S[kMaxExc], positions in tab_x of the new orbitals Q[kMaxExc]
  int tab_ok = 0;
  std::vector<int> tab_x[2];
  std::vector<int> tab_det[2];
  std::vector<int> tab_xl[2];          // [n_x] position of each tab_x orbital in occ_list[spin]
  // determinant terms: unique (up, dn) pairs with merged coefficients C_k = sum_I c_I d_{I,k}
  std::vector<int> term_det;           // [nterm][2]
  std::vector<double> term_coef;       // [nterm]
  // structure terms (I, term, d) for the c_I derivatives
  std::vector<int> sterm_I, sterm_k;
  std::vector<double> sterm_d;
  // the terms holding determinant ud (up u, then down U[0] + u): det_term[det_term_off[ud] ..
  // det_term_off[ud + 1]]; the structure terms of parameter q: cpar_st[cpar_off[q] .. [q + 1]]
  std::vector<int> det_term_off, det_term, cpar_off, cpar_st;
  // Jastrow
  double kappa = 0.8, b1_anti = 0.5, b1_par = 0.25, vnn = 0.0;
  int een_on = 0;
  std::vector<double> jas_a, jas_b;    // [n_elem][6], [6]
  std::vector<double> een_c;           // [n_elem][23] raw coefficients
  std::vector<double> een_B;           // [23][15] free-parameter basis
  // parameters
  int P = 0, jas_param = 0;
  std::vector<int> cparam;
  int n_kappa = 0;
  std::vector<int> kap_off[2];         // [U_s + 1]
  std::vector<int> kap_ent[2];         // [n_ent][4]: j, slot of l, eval index of k, 0
  // per excitation j: evaluation index of l for spin 0 and 1 (-1 where no determinant of the
  // spin holds l without k), evaluation index of k, 0
  std::vector<int> kap_x;
  // balanced work chunks of the orbital contraction phi_q = sum_mu lambda_{q,mu} chi_mu:
  // [n_chunk][4] = (orbital slot q, first mu, one-past-last mu, coefficient base so that the
  // coefficient of mu is orb_coef[base + mu]); chunk_off[q] .. chunk_off[q+1] are q's chunks.
  std::vector<int> occ_chunk[2], occ_chunk_off[2];   // per spin, over occ_list[spin]
  // groups of evq_width (4 or 1) evaluated orbitals with the same nonzero coefficient range,
  // contracted together (with width 4 one basis-function load feeds four orbitals):
  // evq_coef[qoff + width (mu - lo) + t] is the coefficient of mu in orbital t of the group (0
  // for the padding of a short group); evq_chunk [n][4] = (group, first mu, one-past-last mu,
  // qoff - width lo), evq_chunk_off[group] .. [group + 1] are the group's chunks;
  // evq_slot[q] = 4 group + t of evaluated orbital q.
  std::vector<int> evq_chunk, evq_chunk_off, evq_slot;
  std::vector<double> evq_coef;
  int evq_width = 4;
  std::vector<int> det_chunk, det_chunk_off;          // over the first n_ev_det evaluated orbitals
};

// Builds the tables; returns VBQMC_OK or an error code with a message in 'err'.
int build_system(const vbqmc_system_desc* d, SysHost& s, std::string& err);

// ---------------------------------------------------------------------------------------
// Device image: one contiguous allocation, POD view passed to every kernel by value.
// ---------------------------------------------------------------------------------------
struct SysDev {
  int N, Nup, Ndn, Nn, n_elem, S, M, Norb, Nvb;
  int n_ev, n_ev_det;
  int nocc[2], U[2], n[2];
  int nterm, nsterm;
  int P, n_cparam, jas_param, een_on, n_kappa;
  int p_off_a, p_off_b, p_off_theta, p_off_kappa;
  double kappa, b1_anti, b1_par, vnn;
  const double* nuc4;
  const int* nuc_elem;
  const int* sh_center;
  const int* sh_l;
  const int* sh_first;
  const int* sh_by_l;
  const int* sh_pack_f;                // [S][4] in the order of sh_by_l: center | l << 16, first function, shell, float bits of zeta
  const int* nuc_sh;                   // [Nn][4], see SysHost
  int max_nuc_mu;
  const double* sh_zeta;
  const double* sh_norm;
  const int* orb_lo;
  const int* orb_hi;
  const int* orb_off;
  const double* orb_coef;
  const float* orb_coef_f;
  const int* ev_orb;
  const int* occ_list[2];
  const int* det_loc[2];
  const int* det_ev[2];
  int msd;                             // determinant part through the reference-determinant tables
  int n_x[2];
  const int* tab_x[2];
  const int* tab_det[2];
  int tab_ksq;                         // sum over the determinants of both spins of k_u^2
  const int* tab_xl[2];
  const int* term_det;
  const double* term_coef;
  const int* sterm_I;
  const int* sterm_k;
  const double* sterm_d;
  const int* det_term_off;
  const int* det_term;
  const int* cpar_off;
  const int* cpar_st;
  const int* cparam;
  const double* jas_a;
  const double* jas_b;
  const double* een_c;
  const float* een_cf;
  const double* een_B;
  const int* kap_x;                    // [n_kappa][4]: eval index of l (spin 0, spin 1; -1: none), of k, 0
  int n_occ_chunk[2], n_evq_chunk, n_det_chunk, evq_width;
  const int* occ_chunk[2];
  const int* occ_chunk_off[2];
  const int* evq_chunk;
  const int* evq_chunk_off;
  const int* evq_slot;
  const double* evq_coef;
  const float* evq_coef_f;
  const int* det_chunk;
  const int* det_chunk_off;
  int state_doubles;                   // persistent walker state: inverses, ln|det|, signs
  // float-float copies (hi, lo) for the mixed form's double-accurate values
  const float* sh_zeta_ds;             // [S][2]
  const float* sh_norm_ds;             // [S][6][2]
  const float* orb_coef_ds;            // like orb_coef, [.][2]
  const float* nuc_ds;                 // [Nn][3][2] nucleus coordinates
  const float* nuc_zf;                 // [Nn] nuclear charges
  // float copies for the mixed form's bulk arithmetic
  const float* sh_zeta_f;              // [S]
  const float* sh_norm_f;              // [S][6]
  const float* jas_af;                 // like jas_a
  const float* jas_bf;                 // like jas_b
  const float* een_Bf;                 // like een_B
  float kappa_f, b1_anti_f, b1_par_f;
  // float-float copies for the mixed form's e-n and e-e Jastrow values and Rbar (they set ln J)
  const float* jas_a_ds;               // [n_elem][6][2]
  const float* jas_b_ds;               // [6][2]
  const float* een_c_ds;               // [n_elem][23][2] e-e-n coefficients
  float kappa_ds[2], b1_anti_ds[2], b1_par_ds[2];
};

// Records the calling thread's error message (read by vbqmc_last_error) and returns 'code';
// the CUDA form takes a cudaError_t value and returns VBQMC_ERR_CUDA.  Defined with the
// other entry points.
int set_error(int code, const std::string& msg);
int set_cuda_error(int cuda_error, const char* what);

}  // namespace vbq
