// Launch-side view of the VB-QMC kernels: per-warp shared-memory layouts and launchers.
#pragma once

#include <cuda_runtime.h>

#include "vbqmc_internal.h"

namespace vbq {

// The evaluation runs as four kernels, each with the occupancy its own working set allows:
//   jastrow     warp per walker: geometry tables, ln J, grad_i ln J, lap_i ln J, potential
//   orbitals    warp per (walker, electron): basis functions and orbital values/derivatives
//   det         warp per walker: Slater LU + inverses, structure sum, E_L, grad ln|Psi|,
//               structure-coefficient and orbital-excitation derivatives, walker state
//   jastrow_d   warp per walker: Jastrow-parameter derivatives (needs grad ln|Psi|)
// connected through a device workspace (eval_workspace_bytes).  Offsets are bytes from the
// start of a warp's shared-memory region.
struct JasLayout {
  int wpb = 0, warp_bytes = 0;
  int R, vg, red, geo;
  int jas_P, jas_S;  // lanes: electron = lane % jas_P, group = lane / jas_P (jas_S groups)
  // nw > 1: the Jastrow kernel runs one walker per block of nw warps (wide_bytes of shared
  // memory: the walker's tables, then the warps' partial sums at wred and wred2)
  int nw = 1, wide_bytes = 0, wred = 0, wred2 = 0;
};

struct OrbLayout {
  int wpb = 0, warp_bytes = 0;
  int bas, bds, ctab, part, partd;
};

struct DetLayout {
  int wpb = 0, warp_bytes = 0;
  int vg, G, LJ, PhiD, Lphi, Gphi, Bt0, Bt1, ldet, dsg, tdet, Wdet, Tdet, rk, scratch;
  int G0, G1;  // lane-group size per spin for the LU
};

// Determinant part through the reference-determinant tables (eval_dettab.cu), warp per walker.
struct DetTabLayout {
  int wpb = 0, warp_bytes = 0;
  int vg, G, B0, B1, T0, T1, Y0, Y1, A, Bs, perm, Ls, ldet, dsg, tdet, Wdet, rk, Minv, Gam;
};

struct EvalLayout {
  JasLayout jas;
  OrbLayout orb;
  DetLayout det;
  DetLayout detc;  // the same kernel from carried inverses: no LU scratch
  DetTabLayout tab;  // used instead of det when the system's msd flag is set
};

// VMC sweep, warp per walker.  With per-determinant inverses (tab = 0): Binv0/Binv1 hold the
// inverse of every unique determinant of each spin, wk the term ratios D_k/Phi.  With the
// reference-determinant tables (tab = 1, systems whose per-determinant inverses do not fit):
// Binv0/Binv1 hold the reference inverse B of each spin, T0/T1 the tables T = B Phi_X
// [n][n_x], wk the replacement determinants q_u = D_u/D_0 of both spins [U0 + U1], qn the
// proposed q_u of the moving electron's spin, cx the vector c_x of the move.
struct SweepLayout {
  int wpb = 0, warp_bytes = 0;
  int R, Rds, rtab, rtds, Binv0, Binv1, ldet, dsg, wk, PhiO, bas, vrow, part, rho, rinv, cvec, scratch, geo, geom;
  int T0 = 0, T1 = 0, qn = 0, cx = 0;
  int tab = 0;
  int nocc_max;
  int G0, G1;    // lanes per determinant of the LU and Sherman-Morrison (power of two >= n)
  int RG0, RG1;  // lanes per determinant of the move's ratios (power of two <= G)
};

// Nucleus-derivative kernel (eval_forces.cu), one block per walker with one warp per nucleus.
// Block-shared (offsets from the block's base): positions, determinant weights, grad ln J,
// pair distances and unit vectors, orbital gradients, dressed Laplacians, inverses B_u and
// Z_u = B_u L_u B_u.  Per warp (offsets from shared_bytes + warp * warp_bytes): the orbital
// tangents D [N][n_ev_det][6], basis derivatives of Ec electrons at a time bd
// [Ec][max_mu][12], the Jastrow tangents dG [N][3][3] and dLJ [N][3], distances to the
// warp's nucleus sN [N][4] and the scratch Y of Z_u.
struct ForceLayout {
  int nwarps = 0, shared_bytes = 0, warp_bytes = 0, block_bytes = 0;
  int R, wt, G, uE, uH, Gphi, Ld, B, Z;
  int D, bd, dG, dLJ, sN, Y;
  int Ec, max_mu;
};

int make_eval_layout(const SysDev& s, int bulk_bytes, int max_smem, EvalLayout& L);
int make_det_layout(const SysDev& s, int bulk_bytes, int max_smem, DetLayout& L, bool carried = false);
int make_dettab_layout(const SysDev& s, int bulk_bytes, int max_smem, DetTabLayout& L);
template <class Tb>
cudaError_t launch_dettab(const SysDev& s, const DetTabLayout& L, int W, const Tb* JG, const Tb* JL, const double* JS,
                          const Tb* OB, const double* OD, double* logpsi, double* sign, double* eloc, double* vg_ws,
                          double* grad, Tb* O, Tb* dEL, cudaStream_t st);
int make_force_layout(const SysDev& s, int bulk_bytes, int max_smem, ForceLayout& L);
int make_sweep_layout(const SysDev& s, int bulk_bytes, int max_smem, SweepLayout& L);

// Device workspace of one evaluation of W walkers (bytes, 256-aligned pieces).
size_t eval_workspace_bytes(const SysDev& s, int bulk_bytes, int W);

// Pieces of the evaluation workspace (carve_eval_ws): JG [W][N][3] and JL [W][N] grad and
// Laplacian of ln J (bulk type), JS [W][2] ln J and V, OB [W][N][5][n_ev] orbital values,
// gradients and Laplacians (bulk type), OD [W][N][n_ev_det] double orbital values, VG
// [W][N][3] grad ln|Psi|.
struct EvalWs {
  void *JG, *JL, *OB;
  double *JS, *OD, *VG;
};
EvalWs carve_eval_ws(const SysDev& s, int bulk_bytes, int W, void* ws);

// Evaluation of W walkers; ws: eval_workspace_bytes(s, bulk, W) bytes of device memory.
// *nlaunch receives the number of kernels launched.  If ev is not null, ev[0..4] are recorded
// on st before the Jastrow kernel and after the Jastrow, orbital, determinant and
// Jastrow-derivative kernels (the last right after the determinant kernel when it is skipped).
// If aux is not null, the determinant kernel writes per walker [2 U + 1] doubles: the
// marginal weights W_u and T_u of every unique determinant (both spins, U = U_up + U_dn)
// and K[Phi]/Phi (see eval_det.cu), which the nucleus-derivative kernel reads.
constexpr int kEvalKernels = 4;
// If carry is not null (a walker state written by a sweep at R), the determinant kernel takes the
// inverses, term ratios and ln|Phi| from it instead of factorising, and the orbital kernel skips
// the double-accuracy determinant-orbital values that only the factorisation reads.
cudaError_t launch_eval(int precision, const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                        double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out, void* ws,
                        cudaStream_t st, int* nlaunch, cudaEvent_t* ev = nullptr, double* aux = nullptr,
                        const double* carry = nullptr);
// Evaluation followed by the nucleus-derivative kernel: logpsi, sign, eloc as launch_eval,
// dlp [W][Nn][3] = d ln|Psi|/dR_a, dEL [W][Nn][3] = dE_L/dR_a (may be null).  ws: evaluation
// workspace; fws: force_workspace_bytes(s, W) bytes (walker state and determinant weights).
size_t force_workspace_bytes(const SysDev& s, int W);
cudaError_t launch_nuclear_derivs(int precision, const SysDev& s, const EvalLayout& LE, const ForceLayout& LF, int W,
                                  const double* R, double* logpsi, double* sign, double* eloc, double* dlp,
                                  double* dEL, void* ws, void* fws, cudaStream_t st, int* nlaunch);
// out[k] = sum_w (ga[w] Ja[w][k] + gb[w] Jb[w][k]) (gradient.cu); J element type double
// (jtype 0) or float (jtype 1), gb/Jb may be null; part: colsum_slices(W) * K doubles.
int colsum_slices(int W);
cudaError_t launch_weighted_colsum(int W, int K, int jtype, const double* ga, const void* Ja, const double* gb,
                                   const void* Jb, double* out, double* part, cudaStream_t st);
// Structure overlap (gradient.cu): out[pair] = sum_m w_m R_i R_j over the upper triangle i <= j
// of the columns 0..nvb, column nvb being 1 (so the last pairs hold sum w R_i and sum w);
// R_I = O[m][col[I]] for col[I] >= 0, else (1 - sum_J c_J R_J) / c_I.  O element type double
// (otype 0) or float (otype 1), row stride ldo; part: overlap_part_doubles(M, nvb) doubles.
constexpr int kOvMaxStruct = 32;
struct OverlapMap {
  int nvb;
  int col[kOvMaxStruct];
  double c[kOvMaxStruct];
};
size_t overlap_part_doubles(int M, int nvb);
cudaError_t launch_structure_overlap(int M, int ldo, int otype, const void* O, const double* wts, const OverlapMap& map,
                                     double* part, double* out, cudaStream_t st);
// VMC sweeps; state (may be null): read when state_valid, written after the last sweep with the
// carried inverses, term ratios and ln|Phi| (its ln|det| entries are left as they were).
cudaError_t launch_sweep(int precision, const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps,
                         int refresh, double* state, int state_valid, double step, uint64_t seed, uint32_t step0,
                         uint32_t tag, uint32_t woff, int* nacc, cudaStream_t st);

// Per-kernel launchers of the evaluation (eval_jastrow.cu, eval_orbitals.cu, eval_det.cu).
template <class Tb>
cudaError_t launch_jastrow(const SysDev& s, const JasLayout& L, int W, const double* R, Tb* JG, Tb* JL, double* JS,
                           cudaStream_t st);
template <class Tb>
cudaError_t launch_jastrow_deriv(const SysDev& s, const JasLayout& L, int W, const double* R, const double* vg, Tb* O,
                                 Tb* dEL, cudaStream_t st);
template <class Tb>
cudaError_t launch_orbitals(const SysDev& s, const OrbLayout& L, int W, const double* R, Tb* OB, double* OD,
                            cudaStream_t st);
int make_jas_layout(const SysDev& s, int bulk_bytes, int max_smem, JasLayout& L);
int make_orb_layout(const SysDev& s, int bulk_bytes, int max_smem, OrbLayout& L);

}  // namespace vbq
