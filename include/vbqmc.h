/*
 * vbqmc.h -- C ABI of the GB300 (sm_103a) Valence-Bond quantum Monte Carlo hot path.
 *
 * The library evaluates Jastrow-Valence-Bond (JVB) trial wave functions over a population
 * of walkers and moves the walkers with VMC Metropolis sweeps, following Radenkovic,
 * Domin, Toulouse and Braida, "The Valence-Bond Quantum Monte Carlo Method"
 * (arXiv:2207.14715):
 *
 *   Psi(p) = J(alpha) exp(kappa_hat) sum_I c_I Phi_I          Sec. 2.1 Eq. PsiJVBSCF, Sec. 2.2 Eq. PsiJVBp
 *   Phi_I  = HLSP structure (inactive pairs, singlet pairs,   Sec. 2.1 Eq. PhiI, expanded into
 *            unpaired up electrons)                           2^Npairs determinants
 *   J      = exp(f_en + f_ee + f_een), kappa = 0.8            Sec. 2.1, Jastrow expansions
 *   E_L    = (H Psi)/Psi                                      Sec. 2.3.1
 *   O_j    = Psi_j/Psi,  E_L,j = dE_L/dp_j                    Sec. 2.3.1, Eqs. Hi0..Sij
 *
 * Conventions
 *   - Electrons 0..n_up-1 are spin up, n_up..N-1 spin down (spins fixed, Sec. 2.3.1).
 *   - Basis: uncontracted normalised cartesian Gaussians N x^a y^b z^c e^{-zeta r^2} or, per
 *     shell (sh_kind), Slater functions N x^a y^b z^c e^{-zeta r} (the paper's all-electron
 *     basis, Sec. 2.1, whose 1s shells carry the nuclear cusp so that a_1 = 0); a shell of
 *     angular momentum l (0, 1, 2) contributes 1, 3, 6 functions in the order s; x y z;
 *     xx yy zz xy xz yz.  A Gaussian zeta = 0 denotes the constant function 1.
 *   - Walker positions R are walker-major: R[w][i][d] (double), w < W, i < N, d < 3.
 *     Per-walker outputs are [W]; parameter derivatives are [W][P] (double).
 *   - Parameters p, in this order: c_I for I in cparam; if jas_param: a_2..a_6 per
 *     element, b_2..b_6, then (if een_on) 15 free e-e-n parameters theta per element;
 *     then one kappa_kl per orbital excitation (k, l).
 *   - All device pointers are borrowed for the duration of the call and must stay valid
 *     until the work enqueued on 'stream' has completed.  Host arrays are copied.
 *   - 'stream' is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous
 *     with respect to the host unless stated otherwise.
 *   - Return value: VBQMC_OK (0) or a negative error code; vbqmc_last_error() gives a
 *     message for the calling thread.  No function aborts or traps.
 */
#ifndef VBQMC_H
#define VBQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VBQMC_OK 0
#define VBQMC_ERR_ARG -1          /* invalid argument or inconsistent system description */
#define VBQMC_ERR_CUDA -2         /* a CUDA runtime call failed */
#define VBQMC_ERR_NOSYS -3        /* no system loaded under that id */
#define VBQMC_ERR_CAPACITY -4     /* a size exceeds what the kernels support */
#define VBQMC_ERR_UNSUPPORTED -5  /* option not implemented */

#define VBQMC_FP64 0   /* every step in double precision */
#define VBQMC_MIXED 1  /* basis, orbitals, Jastrow and bulk derivatives in float; Slater LU,
                          inverses, ratios, structure sums and energy accumulation in double */

#define VBQMC_MAX_SYSTEMS 64

typedef struct vbqmc_ctx vbqmc_ctx;  /* opaque; owned by the library */

/* System description: the inputs of Eqs. PsiJVBSCF, PhiI and PsiJVBp (Sec. 2.1-2.2).
 * Every pointer is a host array, read during vbqmc_set_system only. */
typedef struct vbqmc_system_desc {
  int Nn, n_elem;          /* 1 <= Nn < 65536 */
  const double* nuc_xyz;   /* [Nn][3] bohr */
  const double* nuc_Z;     /* [Nn] */
  const int* nuc_elem;     /* [Nn] element index in [0, n_elem); Jastrow a and theta are per element */
  int S;
  const int* sh_center;    /* [S] nucleus of each shell; shells of one nucleus must be contiguous */
  const int* sh_l;         /* [S] 0, 1 or 2 */
  const double* sh_zeta;   /* [S] exponent >= 0 */
  int Norb;
  const double* orb_coef;  /* [Norb][M] lambda_{p,mu}, M = number of basis functions */
  int Nup, Ndn;            /* electrons of each spin (Nup >= Ndn) */
  int Nvb;
  const double* c_vb;      /* [Nvb] structure coefficients c_I */
  const int* inact_off;    /* [Nvb+1] offsets into inact */
  const int* inact;        /* inactive (doubly occupied) orbitals of each structure */
  const int* pair_off;     /* [Nvb+1] offsets into pairs */
  const int* pairs;        /* [npairs][2] singlet-coupled active orbital pairs (i, j), i = j allowed */
  const int* unp_off;      /* [Nvb+1] offsets into unp */
  const int* unp;          /* unpaired (spin up) active orbitals */
  double kappa;            /* Jastrow scaling parameter (0.8 in the paper) */
  const double* jas_a;     /* [n_elem][6] a_1..a_6 of f_en */
  const double* jas_b;     /* [6] b_1 (ignored) and b_2..b_6 of f_ee */
  double b1_anti, b1_par;  /* b_1 for antiparallel and parallel pairs (1/2 and 1/4 give the cusps) */
  int een_on;              /* include f_een */
  const double* een_theta; /* [n_elem][15] free e-e-n parameters (cusp-preserving subspace) */
  int n_cparam;
  const int* cparam;       /* structure indices whose c_I are parameters */
  int jas_param;           /* nonzero: Jastrow parameters are parameters */
  int n_kappa;
  const int* kappa_kl;     /* [n_kappa][2] orbital excitations (k, l): phi_l -> phi_l + kappa phi_k */
  const int* sh_kind;      /* [S] 0 Gaussian, 1 Slater (N x^a y^b z^c e^{-zeta r}, zeta > 0), or NULL:
                              all Gaussian */
} vbqmc_system_desc;

/* Creates a context on CUDA device 'device' (the calling thread's current device is
 * restored on return).  *out receives the handle; release with vbqmc_destroy.  A context
 * owns device workspaces that its calls share (grown on demand): calls on one context must
 * not overlap in time (use one stream per context, or order the streams). */
int vbqmc_create(vbqmc_ctx** out, int device);

/* Releases every device allocation of the context.  Waits for the device. */
void vbqmc_destroy(vbqmc_ctx* ctx);

/* Message of the last error raised on the calling thread (static storage, valid until the
 * next failing call on this thread). */
const char* vbqmc_last_error(void);

/* Loads a system under sys_id (0 <= sys_id < VBQMC_MAX_SYSTEMS), replacing any previous one.
 * Host-side set-up (Sec. 2.1-2.2): validates the description, expands every structure into
 * signed determinants (Eq. PhiI and the expansion after it: 2^Npairs terms, self pairs
 * i = j give one term), merges identical determinants, derives the cusp-preserving e-e-n
 * coefficients c = B theta (the coefficients held fixed so that the cusp conditions
 * still hold, Sec. 2.1), builds the orbital-excitation tables (Sec. 2.2), chooses per-
 * determinant inverses or reference-determinant tables for the determinant part (see
 * vbqmc_use_tables) and uploads everything to the device.  Synchronous.  Errors: VBQMC_ERR_ARG for inconsistent input,
 * VBQMC_ERR_CAPACITY if a size exceeds the kernels' limits (N <= 64, n_up <= 32, M <= 1024). */
int vbqmc_set_system(vbqmc_ctx* ctx, int sys_id, const vbqmc_system_desc* desc);

/* Host-only variant of the set-up above for inspection: no device is touched.
 * info[0..11] = N, P, M, Norb, number of determinant terms, unique up determinants,
 * unique down determinants, structure terms, orbitals evaluated per walker, orbital
 * excitation entries, n_up, n_dn.  If terms != NULL it receives up to max_terms rows of
 * [n_up + n_dn + 2] ints: up orbitals (ascending), down orbitals (ascending), structure
 * index, sign (+1/-1) of that structure's term.  If een_B != NULL it receives the 23x15
 * e-e-n free-parameter basis (row-major).  Returns VBQMC_OK or an error code. */
int vbqmc_inspect_system(const vbqmc_system_desc* desc, int* info, int* terms, int max_terms, double* een_B);

/* Per-walker persistent state: the inverse of every unique Slater matrix, its ln|det| and
 * sign, the ratio D_k/Phi of every determinant term, ln|Phi| and its sign, as written by the
 * evaluation (or carried by the sweeps) and read by the next VMC sweep so that a sweep starts
 * without a fresh LU.  *ndoubles receives the number of doubles per walker; a state buffer
 * for W walkers holds W * ndoubles doubles, walker-major.  The layout is private to the
 * library and valid only together with the positions it was computed at. */
int vbqmc_walker_state_size(vbqmc_ctx* ctx, int sys_id, int* ndoubles);

/* Evaluates the trial wave function at W walker positions (Sec. 2.1; Sec. 2.3.1 for E_L,
 * O_j and E_L,j).  The element type of O and dEL is double for VBQMC_FP64 and float for
 * VBQMC_MIXED (the form's bulk type).
 *   R         [W][N][3] device, in
 *   logpsi    [W] device, out: ln|Psi|       sign [W] device, out: sign of Psi (0 if singular)
 *   eloc      [W] device, out: E_L = (H Psi)/Psi, Hamiltonian with nucleus-nucleus repulsion
 *   grad      [W][N][3] device or NULL, out: grad_i ln|Psi|
 *   O         [W][P] device or NULL, out: Psi_j/Psi
 *   dEL       [W][P] device or NULL, out: dE_L/dp_j (requires O != NULL)
 *   state_out [W][ndoubles] device or NULL, out: walker state at R (see above)
 * precision: VBQMC_FP64 or VBQMC_MIXED.  W may be 0. */
int vbqmc_eval_walkers(vbqmc_ctx* ctx, int sys_id, int precision, int W, const double* R, double* logpsi,
                       double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out,
                       void* stream);

/* Derivatives with respect to the nucleus positions R_a at fixed electron positions: the
 * derivative of E_L defined after Eq. H0j (Sec. 2.3.1), E_L,j = dE_L/dp_j, taken with p_j a
 * nucleus coordinate, and the matching O_j = d ln|Psi|/dp_j.  Moving a nucleus moves the
 * basis functions centred on it (Sec. 2.1, orbital expansion), its e-n and e-e-n Jastrow
 * terms and the potential.  These give the usual force estimate
 *   F_a = -<dE_L/dR_a> - 2 <(E_L - <E_L>) d ln|Psi|/dR_a>.
 * The walkers are evaluated as by vbqmc_eval_walkers (no parameter derivatives), then one
 * more kernel forms the derivatives.
 *   R           [W][N][3] device, in
 *   logpsi, sign, eloc  [W] device, out (as vbqmc_eval_walkers)
 *   dlogpsi_dR  [W][Nn][3] device double, out: d ln|Psi| / dR_a
 *   dEL_dR      [W][Nn][3] device double or NULL, out: dE_L / dR_a
 * precision: VBQMC_FP64, or VBQMC_MIXED (bulk arithmetic in float as in the evaluation, the
 * sums over determinants and the potential term in double).  W may be 0.  Errors:
 * VBQMC_ERR_CAPACITY if the per-walker tables do not fit in shared memory;
 * VBQMC_ERR_UNSUPPORTED for systems with Slater shells or on reference-determinant tables. */
int vbqmc_eval_nuclear_derivs(vbqmc_ctx* ctx, int sys_id, int precision, int W, const double* R, double* logpsi,
                              double* sign, double* eloc, double* dlogpsi_dR, double* dEL_dR, void* stream);

/* Weighted sums over walkers of derivative rows, in double with a fixed summation order:
 *   out[k] = sum_w (ga[w] Ja[w][k] + gb[w] Jb[w][k]),  k < K.
 * With Ja = O, Jb = dEL (vbqmc_eval_walkers), ga = 2 (E_L - <E_L>)/W and gb = 1/W this is the
 * energy gradient of Eq. H0j (Sec. 2.3.1) up to its factor 2 convention; with the walkers'
 * upstream gradients as ga, gb it is the vector-Jacobian product of (ln|Psi|, E_L), and with
 * the [W][Nn*3] nucleus derivatives (vbqmc_eval_nuclear_derivs) it gives forces.
 *   Ja, Jb  [W][K] device, element type double (jtype 0) or float (jtype 1); gb and Jb are
 *           both NULL or both given
 *   ga, gb  [W] device double
 *   out     [K] device double (zero when W = 0)
 * The context's calls must not overlap (a grow-only workspace of the context is used). */
int vbqmc_weighted_colsum(vbqmc_ctx* ctx, int W, int K, int jtype, const double* ga, const void* Ja,
                          const double* gb, const void* Jb, double* out, void* stream);

/* VMC (Sec. 2.3.1): nsweeps sweeps of single-electron Metropolis moves over every walker,
 * electron i moved to r_i + step*(2u - 1) per coordinate and accepted when
 * u_acc < |Psi(R')/Psi(R)|^2.  Determinant ratios and Sherman-Morrison updates of the
 * inverses are double in both precision modes (the mixed mode forms the proposed orbital row
 * in float).  The inverses at the start come from 'state' when state_valid != 0 (written by
 * a previous evaluation or sweep at the current R), else from a fresh double-precision LU;
 * within the call they are refreshed by LU every 'refresh' sweeps (0: never).  The sweeps carry
 * the inverses, the determinant-term ratios and ln|Phi| through their moves and, when state is
 * given, write them back after the last sweep.
 * Random numbers: Philox4x32-10 keyed by seed, counter (walker_offset + w, step0 + sweep,
 * electron, (system_tag << 8) | purpose) with purpose 0 -> (u_x, u_y) and 1 -> (u_z, u_acc),
 * each uniform (x >> 11) * 2^-53 of one 64-bit half of the output.
 *   R     [W][N][3] device, in/out
 *   state [W][ndoubles] device or NULL, in (if state_valid) and out
 *   nacc  [W] device int or NULL, out: accepted moves (accumulated over the sweeps)
 * After the last sweep, if logpsi/sign/eloc/O/dEL are non-NULL, the walkers are evaluated as
 * by vbqmc_eval_walkers (one walker-step = one sweep + that evaluation).  With a state and
 * nsweeps > 0 the evaluation takes the carried inverses instead of factorising the Slater
 * matrices, except when step0 + nsweeps is a multiple of refresh (refresh > 0): then it
 * factorises afresh and rewrites the state (refresh = 1: always).  Systems on the
 * reference-determinant tables (vbqmc_use_tables) carry the reference inverse, the tables and
 * the minors through the moves instead (Sherman-Morrison on the reference, a rank-1 update of
 * the tables), refreshed the same way; they keep no state (state must be NULL). */
int vbqmc_vmc_steps(vbqmc_ctx* ctx, int sys_id, int precision, int W, double* R, int nsweeps, double step,
                    uint64_t seed, uint32_t step0, uint32_t system_tag, uint32_t walker_offset, int refresh,
                    double* state, int state_valid, int* nacc, double* logpsi, double* sign, double* eloc,
                    void* O, void* dEL, void* stream);

/* Fixed-node diffusion Monte Carlo steps (Sec. 2.3.2; mixed estimator Eq. E0DMCweights).  The
 * paper runs the algorithm of Umrigar, Nightingale and Runge (J. Chem. Phys. 99, 2865 (1993))
 * without printing it; the step here is an all-electron move that keeps that algorithm's
 * limits on the drift and on the branching energy near the nodes.  Per walker:
 *   vbar_i = v_i (-1 + sqrt(1 + 2 |v_i|^2 tau)) / (|v_i|^2 tau) per electron, v = grad ln|Psi|;
 *   R' = R + tau vbar(R) + sqrt(tau) z  (z standard normal per coordinate);
 *   rejected if sign Psi(R') != sign Psi(R), else accepted with probability
 *   min(1, exp(2 (ln|Psi(R')| - ln|Psi(R)|)) G(R <- R') / G(R' <- R)),
 *   G(R' <- R) = exp(-|R' - R - tau vbar(R)|^2 / (2 tau));
 *   E_b = E_T + clamp((E_L - E_T) |Vbar| / |V|, -E_cut, E_cut) at R and at the kept point (V, Vbar
 *   the whole-walker drift vectors; E_cut = 0.2 sqrt(N / tau), the energy cutoff of Zen, Sorella,
 *   Gillan, Michaelides and Alfe, Phys. Rev. B 93, 241118(R) (2016));
 *   weight w = exp(-tau ((E_b(R) + E_b(R_kept)) / 2 - E_T)); copies = min(floor(w + u), 3),
 *   children in parent order (weights are 1 after branching);
 *   then E_T = sum(w E_b) / sum(w) - (0.1 / tau) ln(population / target), E_b at the kept points
 *   (the energies that set the weights, so that the population settles at the target; the
 *   estimator returned in sum_wE / sum_w uses the raw E_L).
 * Random numbers: Philox4x32-10 keyed by seed, counter (walker_offset + walker index in the
 * current population, step0 + step, slot, (system_tag << 8) | purpose): slot e < N, purpose 2 ->
 * (u0, u1) giving z_x = r cos(2 pi u1), z_y = r sin(2 pi u1) with r = sqrt(-2 ln(1 - u0)); purpose
 * 3 -> z_z from the cosine branch of its pair; slot N, purpose 4 -> (u_acc, u_branch).  Uniforms as
 * in vbqmc_vmc_steps.  Ranks of a multi-GPU run pass disjoint walker_offset ranges (e.g. rank x
 * cap) so that their streams differ.  The evaluation at R' computes E_L and grad ln|Psi| in the
 * given precision mode; acceptance, weights and sums are double in both modes.
 *   W_io     host, in/out: population (0 <= W <= cap)
 *   R        [cap][N][3] device, in/out: walkers (the first W rows are the population)
 *   E_T_io   host, in/out: trial energy
 *   sum_wE, sum_w, sum_wEb [nsteps] host double or NULL: per step, sums of the pre-branching
 *            weights times E_L, of the weights (the estimator is sum_wE / sum_w) and of the weights
 *            times E_b (what the trial-energy update averages)
 *   pop [nsteps] host int or NULL: population after branching; e_trial [nsteps] host or NULL:
 *            E_T after its update;  accepted: host or NULL, accepted moves over the call.
 * The call synchronizes 'stream' once per step (to read the population and the sums) and keeps
 * a device workspace for 'cap' walkers in the context (grown on demand).  A population of 0
 * ends the call early.  Returns VBQMC_ERR_CAPACITY if branching would exceed 'cap': the moves of
 * that step are applied, its branching is not, and W_io holds the population before it. */
int vbqmc_dmc_steps(vbqmc_ctx* ctx, int sys_id, int precision, int* W_io, int cap, double* R, int nsteps, double tau,
                    double* E_T_io, int target, uint64_t seed, uint32_t step0, uint32_t system_tag,
                    uint32_t walker_offset, double* sum_wE, double* sum_w, double* sum_wEb, int* pop, double* e_trial,
                    int64_t* accepted, void* stream);

/* Linear-method estimators from M samples (Sec. 2.3.1, Eqs. Hi0, H0j, Hij, Sij, feeding the
 * generalized eigenproblem Eq. geneigeqM).  With weights w (NULL: all 1), averages
 * <x> = sum w x / sum w and Ot = O - <O>, the outputs are
 *   E0 = <E_L>,  gL_i = 2 <Ot_i E_L>,  gR_j = 2 (<Ot_j E_L> + <E_L,j>),
 *   S[i][j] = <Ot_i Ot_j>,  H[i][j] = <Ot_i (E_L Ot_j + E_L,j)>,
 * which equal the printed sums of averages term by term.
 *   O, dEL  [M][P] device, element type double (VBQMC_FP64) or float (VBQMC_MIXED)
 *   eloc    [M] device double;  weights [M] device double or NULL
 *   E0 [1], gL [P], gR [P], S [P][P], H [P][P]: device double, out
 * Column sums are double (fixed-order block partials); the centred values, times sqrt(w) and a
 * power-of-two scale per parameter that bounds them by 2^14, are split into high and low FP16
 * halves (22 significant bits); the products run on the tensor cores (tcgen05 kind::f16,
 * three MMAs per product: hi*hi + hi*lo + lo*hi, FP32 accumulators in TMEM drained every 64
 * samples into FP32 registers) over chunks of samples, and the chunk partials are summed in
 * double and unscaled.  The context keeps a device workspace (grown on demand, synchronizing
 * 'stream' when it grows). */
int vbqmc_accumulate_lin_matrices(vbqmc_ctx* ctx, int precision, int P, int64_t M, const void* O, const void* dEL,
                                  const double* eloc, const double* weights, double* E0, double* gL, double* gR,
                                  double* S, double* H, void* stream);

/* Parameter update of the linear method (Sec. 2.3.1, Eq. geneigeqM): the generalized
 * eigenproblem A v = E B v of the (P+1) x (P+1) matrices
 *   A = [[E0, gR^T / 2], [gL / 2, H + shift I]],   B = [[1, 0], [0, S]]
 * (the outputs of vbqmc_accumulate_lin_matrices; shift >= 0 stabilises the step).  The answer
 * is the lowest real eigenvalue E whose eigenvector v has |v_0| >= 1e-3 |v|, with v scaled to
 * v_0 = 1: dp[j] = v_{j+1}, *e_lin = E.  Host routine in double (no device is touched):
 * S's eigendecomposition (directions with eigenvalues <= P eps max are dropped as redundant
 * parameters), the pencil reduced with S^-1/2 to a standard nonsymmetric problem, its
 * eigenvalues by Hessenberg reduction and Francis double-shift QR, the eigenvectors by inverse
 * iteration.  All arrays are host, row-major: gL, gR [P], H, S [P][P] in; dp [P] out.
 * Errors: VBQMC_ERR_ARG for bad or non-finite input, an S with no positive eigenvalue, a QR
 * iteration that does not converge or no admissible eigenvector (message in vbqmc_last_error). */
int vbqmc_lin_solve(int P, double E0, const double* gL, const double* gR, const double* H, const double* S,
                    double shift, double* dp, double* e_lin);

/* Merges linear-method estimators computed on disjoint parts of a sample (e.g. the walkers of
 * several ranks) into the estimators of the whole sample, as vbqmc_accumulate_lin_matrices
 * defines them (Sec. 2.3.1, Eqs. Hi0..Sij).  Part r has weight sum wsum[r] (its sample count for
 * unit weights), mean derivative row mean[r] = <O>_r, and E0, gL, gR, S, H centred on its own
 * mean.  With the global mean mu = sum_r wsum_r mean_r / sum_r wsum_r and d_r = mean_r - mu, the
 * parts are re-centred exactly (no cancellation) and averaged with weights wsum_r:
 *   S = <S_r + d d^T>,  gL = <gL_r + 2 d E0_r>,  gR = gL + 2 <(gR_r - gL_r) / 2>,
 *   H_ij = <H_r,ij + (d_j gL_r,i + d_i gL_r,j) / 2 + d_i d_j E0_r + d_i (gR_r,j - gL_r,j) / 2>.
 * Host routine, double.  In (host): wsum [nparts], mean [nparts][P], E0 [nparts],
 * gL, gR [nparts][P], S, H [nparts][P][P].  Out (host): E0_out [1], mean_out [P] (or NULL),
 * gL_out, gR_out [P], S_out, H_out [P][P].  Errors: VBQMC_ERR_ARG. */
int vbqmc_lin_merge(int nparts, int P, const double* wsum, const double* mean, const double* E0, const double* gL,
                    const double* gR, const double* S, const double* H, double* E0_out, double* mean_out,
                    double* gL_out, double* gR_out, double* S_out, double* H_out);

/* Overlap matrix of the JVB structures (Sec. 2.4) over M samples:
 *   S_IJ = <(Psi_I/Psi_0)(Psi_J/Psi_0)>,  <x> = sum_m w_m x_m / sum_m w_m,
 * with Psi_I = J c_I-derivative of Eq. PsiJVBp, i.e. Psi_I/Psi_0 = Phi_I/Phi: the c_I
 * derivatives that vbqmc_eval_walkers writes as the first n_cparam columns of O.  A structure
 * missing from cparam (at most one; its c_I must be nonzero) is rebuilt at every sample from
 * the identity sum_I c_I Psi_I/Psi_0 = 1.  Products and sums are double, in a fixed order,
 * for either element type of O.
 *   O        [M][ldo] device, element type double (VBQMC_FP64) or float (VBQMC_MIXED), in
 *   weights  [M] device double or NULL (all 1)
 *   c_vb     [nvb] host: structure coefficients; cparam [n_cparam] host: structure of each
 *            leading column of O (n_cparam >= nvb - 1, nvb <= 32)
 *   S        [nvb][nvb] host double, out
 * Synchronizes 'stream' (the result is copied to the host).  Uses the context's reduction
 * workspace (grown on demand).  Errors: VBQMC_ERR_ARG, VBQMC_ERR_CAPACITY (nvb > 32),
 * VBQMC_ERR_CUDA. */
int vbqmc_structure_overlap(vbqmc_ctx* ctx, int precision, int M, int ldo, const void* O, const double* weights,
                            int nvb, const double* c_vb, int n_cparam, const int* cparam, double* S, void* stream);

/* Weights of the JVB structures from their overlap S (Sec. 2.4), host double:
 *   Chirgwin-Coulson  w_I = c_I (S c)_I / (c^T S c);
 *   Loewdin           w_I = (S^1/2 c)_I^2 / |S^1/2 c|^2,
 * S^1/2 through the eigendecomposition of the symmetric part of S (negative eigenvalues of
 * rounding size taken as 0).  S [nvb][nvb], c [nvb] in; w_cc, w_lowdin [nvb] out (either may
 * be NULL).  Errors: VBQMC_ERR_ARG for bad or non-finite input or a vanishing norm. */
int vbqmc_structure_weights(int nvb, const double* S, const double* c, double* w_cc, double* w_lowdin);

/* Measured ALU throughput of a device (diagnostics; the paper has no counterpart): the
 * denominators of the walker kernels' rooflines.  out[0] FP32 FMA TFLOP/s, out[1] FP64 FMA
 * TFLOP/s, out[2] special-function exponentials in 10^12 per second, out[3] SM count; *n = 4.
 * Each probe runs independent FMA (or exponential) chains over 8 x 256 threads per SM and is
 * timed with CUDA events (best of three launches after one warm-up).  Synchronous; allocates
 * nothing; the calling thread's current device is restored. */
int vbqmc_measure_alu_peaks(int device, double* out, int max, int* n);

/* Scratch size of vbqmc_accumulate_lin_matrices_noalloc, bytes per device (64 MiB). */
#define VBQMC_NOALLOC_SCRATCH_BYTES (64u << 20)

/* The same estimators as vbqmc_accumulate_lin_matrices, computed by the same kernels, without
 * any device memory allocation (the paper has no counterpart: this is a library service).
 * For callers that must not have the library allocate: applications that give the whole
 * device to their own allocator or a fixed budget, or latency-critical paths where an
 * allocation's implicit synchronization or failure is unacceptable.  Arguments, layouts and
 * outputs are those of vbqmc_accumulate_lin_matrices, without a context: the call works on
 * the calling thread's current device, and 'stream' must belong to it.
 * Workspace: one fixed device array of VBQMC_NOALLOC_SCRATCH_BYTES per device, created when
 * the library's module is loaded.  The first call with a device current looks up its address
 * (set-up work; make that call before any stream capture begins).  Each call clears, on
 * 'stream', the parts of the array that must start at zero; the array keeps the last call's
 * contents otherwise.  Calls on one device whose executions overlap (other streams, other
 * threads) race on the array and give wrong results: order them on one stream.
 * Errors: VBQMC_ERR_CAPACITY when (P, M) needs more scratch than the fixed size (about
 * 8 bytes x M x P rounded up to 128, plus chunk partials; a 16384 x 216 call needs 40 MiB);
 * VBQMC_ERR_ARG for bad precision, P < 1, M < 1 or a NULL required pointer;
 * VBQMC_ERR_CUDA when a CUDA call or launch fails.  Message in vbqmc_last_error(). */
int vbqmc_accumulate_lin_matrices_noalloc(int precision, int P, int64_t M, const void* O, const void* dEL,
                                          const double* eloc, const double* weights, double* E0, double* gL,
                                          double* gR, double* S, double* H, void* stream);

/* ---- Batched systems (many small molecules of uneven size in one launch per step) ----
 * A batch holds several systems already loaded in the context (each with its own walker
 * count W[k]) in one precision mode.  A step is one persistent launch: its blocks take
 * (system, tile of walkers) work items, ordered by estimated cost, from a device queue and run
 * the sweep and every evaluation phase on each tile (the tuner may instead pick one launch per
 * kernel type over per-kind work items, when that measures faster); the step is captured in a
 * CUDA graph on first use (per call shape: with or without sweeps, evaluation and derivatives)
 * and replayed.  Results equal those of the
 * per-system calls with system_tag = the system id and walker_offset = 0.  A batch keeps a
 * copy of the systems' tables: recreate it after reloading one of its systems.  The paper has
 * no counterpart (it runs one molecule per calculation); this serves many small systems at
 * once. */
typedef struct vbqmc_batch vbqmc_batch;
/* Creates a batch of nsys distinct loaded systems sys_ids[k] with W[k] >= 1 walkers each;
 * allocates the evaluation workspace of all of them.  Errors: VBQMC_ERR_NOSYS,
 * VBQMC_ERR_CAPACITY (a system's per-walker state does not fit in shared memory),
 * VBQMC_ERR_ARG, VBQMC_ERR_CUDA. */
int vbqmc_batch_create(vbqmc_ctx* ctx, int nsys, const int* sys_ids, const int* W, int precision, vbqmc_batch** out);
void vbqmc_batch_destroy(vbqmc_batch* batch);
/* vbqmc_vmc_steps for every system of the batch; every pointer argument is a host array of
 * nsys device pointers (R, and state/nacc/logpsi/sign/eloc/O/dEL when not NULL), each laid out
 * as in vbqmc_vmc_steps for its own system.  The call copies its arguments through pinned
 * staging buffers: it waits until the previous call's graph has read them. */
int vbqmc_batch_vmc_steps(vbqmc_batch* batch, double* const* R, int nsweeps, double step, uint64_t seed,
                          uint32_t step0, int refresh, double* const* state, int state_valid, int* const* nacc,
                          double* const* logpsi, double* const* sign, double* const* eloc, void* const* O,
                          void* const* dEL, void* stream);
/* Launch-shape tuner: times the evaluation on the walkers R (outputs written to
 * logpsi/sign/eloc), for the per-kind kernels with one-block-per-item and persistent grids and
 * with and without a cap on walkers per block, and for the one-launch step over tile shapes
 * (8, 12 or 16 warps per block, tiles capped at 4 walkers or not, 1 or 2 x the resident blocks);
 * keeps the fastest shapes and the faster launch style, and drops captured graphs.
 * Synchronizes 'stream'. */
int vbqmc_batch_tune(vbqmc_batch* batch, double* const* R, double* const* logpsi, double* const* sign,
                     double* const* eloc, void* stream);
/* Launch shapes: out[5 k + 0..4] = work items, grid, warps per block, persistence (0: one
 * block per item, p: p x resident blocks), walkers-per-block cap (0: none) for kernel k in
 * the order sweep, Jastrow, Jastrow derivatives, orbitals, determinants, then k = 5 the
 * one-launch step; out[30] = 1 when steps run as one launch, out[31] and out[32] the tuner's
 * evaluation times in microseconds of the per-kind launches and of the one-launch step
 * (0 before tuning).  out holds 33 ints. */
int vbqmc_batch_info(vbqmc_batch* batch, int* out);

/* Per-kernel timing of the evaluation (diagnostics; the paper has no counterpart).  With
 * timing on, every evaluation (vbqmc_eval_walkers, and the evaluation at the end of
 * vbqmc_vmc_steps) records CUDA events on its stream around each of its kernels; the
 * evaluation runs as four kernels in this order: Jastrow factor, orbitals, determinants
 * (with E_L, structure and excitation derivatives), Jastrow-parameter derivatives (skipped
 * when no derivatives are asked for: time 0).  vbqmc_accumulate_lin_matrices records the same
 * four intervals around its phases: column sums (with the scales), centring and splitting,
 * tensor-core products, final reduction. */
int vbqmc_set_kernel_timing(vbqmc_ctx* ctx, int on);
/* Durations in ms of the four intervals of the last timed call (evaluation or linear-method
 * accumulation), in the order above: ms[0..min(max, 4) - 1]; *n = 4.  Waits for that call to
 * finish.  Error if no timed call has been recorded since timing was switched on. */
int vbqmc_kernel_times(vbqmc_ctx* ctx, double* ms, int max, int* n);

/* Launch shape of the walker kernels for a loaded system: out[0..3] = walkers (warps) per
 * thread block and shared-memory bytes per walker of the evaluation's determinant kernel, then
 * the same two numbers for the sweep kernel, for the given precision mode; out[4] = 1 when the
 * system is on reference-determinant tables (vbqmc_use_tables).  out holds 5 ints. */
int vbqmc_launch_info(vbqmc_ctx* ctx, int sys_id, int precision, int* out);

/* Chooses how the determinant part of a loaded system is carried (Sec. 2.1: the determinants
 * of a spin share the inactive orbitals and differ from the first one by a few active
 * columns).  on = 0: every unique determinant's inverse (walker state, orbital-excitation and
 * nucleus derivatives available); on = 1: the first determinant of each spin as reference, its
 * inverse B and the tables T = B Phi_X, every other determinant as a k x k minor (k <= 4):
 * VMC sweeps and evaluations keep no walker state, orbital-excitation and nucleus derivatives
 * are refused.  vbqmc_set_system takes the tables when the per-determinant inverses of one
 * walker do not fit in shared memory, and, for systems without orbital-excitation parameters,
 * when the per-determinant sweep region of a walker exceeds 48 KB, or 32 KB with 16 or more
 * unique determinants of a spin (few walkers per SM: the measured crossover on molecules of
 * 2-32 electrons).  Errors: VBQMC_ERR_NOSYS, VBQMC_ERR_UNSUPPORTED (a
 * determinant differs from the reference in more than 4 columns), VBQMC_ERR_CAPACITY (on = 0
 * but the inverses do not fit). */
int vbqmc_use_tables(vbqmc_ctx* ctx, int sys_id, int on);

/* Number of kernel launches enqueued by the last successful call on this context. */
int vbqmc_last_launch_count(vbqmc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VBQMC_H */
