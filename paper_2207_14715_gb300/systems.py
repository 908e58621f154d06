"""Seeded synthetic inputs: molecular systems and initial walker positions.

This module only draws inputs.  It holds none of the method's arithmetic: no basis
function, determinant, Jastrow or energy is evaluated here.  The same SystemSpec feeds
both the CUDA library and the CPU oracle; each side derives everything else (structure
expansion, cusp-constrained Jastrow coefficients, tables) on its own.

The system descriptions follow the inputs of the JVB wave function (arXiv:2207.14715,
Sec. 2.1, Eqs. PsiJVBSCF and PhiI; Sec. 2.2, Eq. PsiJVBp):
  nuclei (positions, charges, element ids), uncontracted cartesian Gaussian shells,
  orbital coefficients lambda[p][mu], VB structures as (inactive, pairs, unpaired) lists
  with coefficients c_I, Jastrow parameters (a per element, b, e-e-n free parameters
  theta per element), and the optimisable-parameter selection (structure coefficients,
  Jastrow, orbital excitations (k, l)).

Electron ordering: electrons 0..n_up-1 are spin up, n_up..N-1 spin down.
Basis-function ordering: shells in the given order; components s; x y z; xx yy zz xy xz yz.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NCOMP = (1, 3, 6)
EEN_NFREE = 15  # free e-e-n parameters per element (23 terms, rank-8 cusp conditions)


@dataclasses.dataclass
class SystemSpec:
    name: str
    nuc_xyz: np.ndarray      # (Nn, 3) float64, bohr
    nuc_Z: np.ndarray        # (Nn,) float64
    nuc_elem: np.ndarray     # (Nn,) int32 element index
    n_elem: int
    sh_center: np.ndarray    # (S,) int32
    sh_l: np.ndarray         # (S,) int32 in {0, 1, 2}
    sh_zeta: np.ndarray      # (S,) float64 (0 means the constant function 1)
    orb_coef: np.ndarray     # (Norb, M) float64
    orb_class: np.ndarray    # (Norb,) int32 localisation class (center index, -1 delocalised)
    orb_kind: np.ndarray     # (Norb,) int32 0 inactive, 1 active, 2 virtual
    n_up: int
    n_dn: int
    c_vb: np.ndarray         # (Nvb,) float64
    inact_off: np.ndarray    # (Nvb+1,) int32
    inact: np.ndarray        # int32
    pair_off: np.ndarray     # (Nvb+1,) int32
    pairs: np.ndarray        # (npairs, 2) int32
    unp_off: np.ndarray      # (Nvb+1,) int32
    unp: np.ndarray          # int32
    jas_a: np.ndarray        # (n_elem, 6) a1..a6
    jas_b: np.ndarray        # (6,) b1 (unused: b1 fixed by spin), b2..b6
    b1_anti: float = 0.5
    b1_par: float = 0.25
    kappa: float = 0.8
    een_on: bool = False
    een_theta: np.ndarray | None = None   # (n_elem, 15)
    cparam: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    jas_param: bool = False
    kappa_kl: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 2), np.int32))
    step: float = 0.3        # VMC step size (bohr)
    sh_kind: np.ndarray | None = None  # (S,) int32: 0 Gaussian, 1 Slater (None: all Gaussian)

    @property
    def N(self) -> int:
        return self.n_up + self.n_dn

    @property
    def Nn(self) -> int:
        return int(self.nuc_xyz.shape[0])

    @property
    def M(self) -> int:
        return int(sum(NCOMP[int(l)] for l in self.sh_l))

    @property
    def Norb(self) -> int:
        return int(self.orb_coef.shape[0])

    @property
    def Nvb(self) -> int:
        return int(self.c_vb.shape[0])

    @property
    def n_params(self) -> int:
        p = len(self.cparam) + len(self.kappa_kl)
        if self.jas_param:
            p += 5 * self.n_elem + 5 + (EEN_NFREE * self.n_elem if self.een_on else 0)
        return p

    def theta(self) -> np.ndarray:
        if self.een_theta is None:
            return np.zeros((self.n_elem, EEN_NFREE))
        return np.ascontiguousarray(self.een_theta, dtype=np.float64)


def _structures(lst):
    """lst: list of (inactive list, pair list, unpaired list)."""
    io, ina, po, prs, uo, un = [0], [], [0], [], [0], []
    for inactive, pairs, unpaired in lst:
        ina += list(inactive)
        io.append(len(ina))
        prs += [list(p) for p in pairs]
        po.append(len(prs))
        un += list(unpaired)
        uo.append(len(un))
    pairs_arr = np.array(prs, np.int32).reshape(-1, 2)
    return (np.array(io, np.int32), np.array(ina, np.int32), np.array(po, np.int32), pairs_arr,
            np.array(uo, np.int32), np.array(un, np.int32))


def structure_subset(spec: SystemSpec, keep) -> SystemSpec:
    """The same system with only the VB structures `keep` (in that order, with their
    coefficients): the wave function of a "diabatic" state restricted to a subset of Lewis
    structures, whose VMC energy minus that of the full expansion is a resonance energy (Sec. 2.4,
    Sec. 3).  Structure-coefficient parameters follow their structures (those of dropped
    structures are removed)."""
    keep = [int(I) for I in keep]
    lst = []
    for I in keep:
        ina = spec.inact[spec.inact_off[I]:spec.inact_off[I + 1]]
        prs = spec.pairs[spec.pair_off[I]:spec.pair_off[I + 1]]
        un = spec.unp[spec.unp_off[I]:spec.unp_off[I + 1]]
        lst.append((list(ina), [tuple(p) for p in prs], list(un)))
    io, ina, po, prs, uo, un = _structures(lst)
    new_index = {I: k for k, I in enumerate(keep)}
    cparam = np.array([new_index[int(I)] for I in spec.cparam if int(I) in new_index], np.int32)
    return dataclasses.replace(spec, name=spec.name + "_subset", c_vb=np.asarray(spec.c_vb, np.float64)[keep].copy(),
                               inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un, cparam=cparam)


def _center_shells(rng, elem_of_center, shell_ls, zeta_lo=0.1, zeta_hi=20.0):
    """Shells per center with exponents log-uniform in [zeta_lo, zeta_hi], drawn once per element."""
    zeta_elem = {}
    sc, sl, sz = [], [], []
    for c, e in enumerate(elem_of_center):
        if e not in zeta_elem:
            zeta_elem[e] = np.exp(rng.uniform(math.log(zeta_lo), math.log(zeta_hi), size=len(shell_ls)))
        for l, z in zip(shell_ls, zeta_elem[e]):
            sc.append(c)
            sl.append(l)
            sz.append(z)
    return np.array(sc, np.int32), np.array(sl, np.int32), np.array(sz, np.float64)


def _basis_ranges(sh_center, sh_l, Nn):
    """First and one-past-last basis index per center (shells are grouped by center)."""
    lo = np.full(Nn, -1, np.int64)
    hi = np.zeros(Nn, np.int64)
    mu = 0
    for c, l in zip(sh_center, sh_l):
        if lo[c] < 0:
            lo[c] = mu
        mu += NCOMP[int(l)]
        hi[c] = mu
    return lo, hi


def _local_orbital(rng, M, lo, hi, sh_center, sh_l, center, s_positive=True, scale=1.0):
    v = np.zeros(M)
    mu = 0
    for c, l in zip(sh_center, sh_l):
        n = NCOMP[int(l)]
        if c == center:
            if l == 0 and s_positive:
                v[mu:mu + n] = rng.uniform(0.0, 1.0, n)
            else:
                v[mu:mu + n] = rng.uniform(-1.0, 1.0, n)
        mu += n
    return v * scale


def _shaped_orbital(rng, M, sh_center, sh_l, center, k, admix=0.15):
    """The k-th orbital placed on a centre, with a distinct angular character per k so that the
    orbitals sharing a centre are far from linearly dependent: k = 0 s-like (every s shell
    positive), k = 1..3 the x, y, z components of the p shells, k >= 4 the (k - 4)-th d
    component; every other function of the centre gets a seeded admixture of size 'admix'."""
    v = np.zeros(M)
    mu = 0
    for c, l in zip(sh_center, sh_l):
        n = NCOMP[int(l)]
        if c == center:
            v[mu:mu + n] = admix * rng.uniform(-1.0, 1.0, n)
            if k == 0 and l == 0:
                v[mu] = rng.uniform(0.5, 1.0)
            elif 1 <= k <= 3 and l == 1:
                v[mu + k - 1] = rng.uniform(0.5, 1.0)
            elif k >= 4 and l == 2:
                v[mu + (k - 4) % 6] = rng.uniform(0.5, 1.0)
        mu += n
    return v


# ----------------------------------------------------------------------------------
# Tiny systems with closed-form answers (used by the physics pins of the oracle).
# ----------------------------------------------------------------------------------
def one_electron(Z: float, zeta: float, a1: float = 0.0, a2: float = 0.0, name: str = "hydrogenic") -> SystemSpec:
    """One nucleus of charge Z, one spin-up electron, one s Gaussian orbital exp(-zeta r^2).

    With zeta = 0 the orbital is the constant 1; with a1 = -Z, a2 = -kappa the e-n Jastrow
    term a1 R/(1 + a2 R) equals -Z r, so Psi = exp(-Z r) (hydrogen-like 1s)."""
    io, ina, po, prs, uo, un = _structures([([], [], [0])])
    return SystemSpec(
        name=name, nuc_xyz=np.zeros((1, 3)), nuc_Z=np.array([float(Z)]), nuc_elem=np.zeros(1, np.int32), n_elem=1,
        sh_center=np.zeros(1, np.int32), sh_l=np.zeros(1, np.int32), sh_zeta=np.array([float(zeta)]),
        orb_coef=np.ones((1, 1)), orb_class=np.zeros(1, np.int32), orb_kind=np.ones(1, np.int32),
        n_up=1, n_dn=0, c_vb=np.ones(1), inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.array([[a1, a2, 0, 0, 0, 0]], np.float64), jas_b=np.zeros(6), b1_anti=0.0, b1_par=0.0)


def slater_1s(Z: float, zeta: float) -> SystemSpec:
    """One nucleus of charge Z, one electron in a 1s Slater orbital exp(-zeta r), no Jastrow
    (a1 = 0, the paper's choice with cusp-correct orbitals).  zeta = Z is the exact ground
    state: E_L = -Z^2/2 everywhere."""
    io, ina, po, prs, uo, un = _structures([([], [], [0])])
    return SystemSpec(
        name="slater_1s", nuc_xyz=np.zeros((1, 3)), nuc_Z=np.array([float(Z)]), nuc_elem=np.zeros(1, np.int32),
        n_elem=1, sh_center=np.zeros(1, np.int32), sh_l=np.zeros(1, np.int32), sh_zeta=np.array([float(zeta)]),
        orb_coef=np.ones((1, 1)), orb_class=np.zeros(1, np.int32), orb_kind=np.ones(1, np.int32),
        n_up=1, n_dn=0, c_vb=np.ones(1), inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.zeros((1, 6)), jas_b=np.zeros(6), b1_anti=0.0, b1_par=0.0, sh_kind=np.ones(1, np.int32))


def slater_h2(seed: int = 20220728 + 7) -> SystemSpec:
    """H2 at R = 1.4 bohr on Slater shells (the paper's all-electron practice, Sec. 2.1): per
    center a 1s (zeta 1.0), a 2s-like s (zeta 0.6), a p and a d Slater shell, Heitler-London and
    two ionic structures, e-n Jastrow a1 = 0 (the 1s shells carry the nuclear cusp), e-e Pade,
    e-e-n terms; c_2, c_3 and the Jastrow parameters are parameters."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, -0.7], [0.0, 0.0, 0.7]])
    sc, sl, sz = [], [], []
    for c in range(2):
        for l, z in ((0, 1.0), (0, 0.6), (1, 0.9), (2, 1.3)):
            sc.append(c), sl.append(l), sz.append(z)
    sc, sl, sz = np.array(sc, np.int32), np.array(sl, np.int32), np.array(sz)
    M = int(sum(NCOMP[l] for l in sl))
    orb = np.zeros((2, M))
    half = M // 2
    for c in range(2):
        orb[c, c * half:(c + 1) * half] = rng.uniform(-0.3, 0.3, half)
        orb[c, c * half] = 1.0                      # the 1s shell carries the cusp
    io, ina, po, prs, uo, un = _structures([([], [(0, 1)], []), ([], [(0, 0)], []), ([], [(1, 1)], [])])
    jas_a = np.array([[0.0, 1.0, 0.02, -0.01, 0.0, 0.0]])
    return SystemSpec(
        name="slater_h2", nuc_xyz=xyz, nuc_Z=np.ones(2), nuc_elem=np.zeros(2, np.int32), n_elem=1, sh_center=sc,
        sh_l=sl, sh_zeta=sz, orb_coef=orb, orb_class=np.array([0, 1], np.int32), orb_kind=np.ones(2, np.int32),
        n_up=1, n_dn=1, c_vb=np.array([1.0, 0.3, 0.3]), inact_off=io, inact=ina, pair_off=po, pairs=prs,
        unp_off=uo, unp=un, jas_a=jas_a, jas_b=np.array([0.0, 1.0, 0.01, 0.0, 0.0, 0.0]), een_on=True,
        een_theta=rng.uniform(-0.02, 0.02, (1, EEN_NFREE)), cparam=np.array([1, 2], np.int32), jas_param=True,
        sh_kind=np.ones(len(sl), np.int32))


def two_electron_product(Z: float, zeta: float) -> SystemSpec:
    """He-like singlet: both electrons in one s Gaussian on a nucleus of charge Z, no Jastrow."""
    io, ina, po, prs, uo, un = _structures([([0], [], [])])
    return SystemSpec(
        name="two_electron", nuc_xyz=np.zeros((1, 3)), nuc_Z=np.array([float(Z)]), nuc_elem=np.zeros(1, np.int32),
        n_elem=1, sh_center=np.zeros(1, np.int32), sh_l=np.zeros(1, np.int32), sh_zeta=np.array([float(zeta)]),
        orb_coef=np.ones((1, 1)), orb_class=np.zeros(1, np.int32), orb_kind=np.zeros(1, np.int32),
        n_up=1, n_dn=1, c_vb=np.ones(1), inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.zeros((1, 6)), jas_b=np.zeros(6), b1_anti=0.0, b1_par=0.0)


def two_structure_1s(Z: float, zeta: float, c2: float) -> SystemSpec:
    """One electron, Psi = J (Phi_1 + c2 Phi_2) with Phi_1 = constant orbital, Phi_2 = s Gaussian,
    J = exp(-Z r).  The exact ground state lies in the span of Psi and dPsi/dc2 (at c2 -> the
    exact point the Gaussian is not needed), which is the strong zero-variance case."""
    io, ina, po, prs, uo, un = _structures([([], [], [0]), ([], [], [1])])
    kap = 0.8
    return SystemSpec(
        name="two_structure_1s", nuc_xyz=np.zeros((1, 3)), nuc_Z=np.array([float(Z)]),
        nuc_elem=np.zeros(1, np.int32), n_elem=1, sh_center=np.zeros(2, np.int32), sh_l=np.zeros(2, np.int32),
        sh_zeta=np.array([0.0, float(zeta)]), orb_coef=np.eye(2), orb_class=np.zeros(2, np.int32),
        orb_kind=np.ones(2, np.int32), n_up=1, n_dn=0, c_vb=np.array([1.0, float(c2)]),
        inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.array([[-float(Z), -kap, 0, 0, 0, 0]]), jas_b=np.zeros(6), b1_anti=0.0, b1_par=0.0,
        cparam=np.array([1], np.int32))


def h2_nodeless(R: float = 1.4, zetas=(0.2, 0.6, 1.8), weights=(1.0, 0.5, 0.2)) -> SystemSpec:
    """H2 at bond length R with a nodeless singlet: one positive s combination per atom,
    covalent + two ionic structures with positive c, cusp-correct Pade e-n and e-e Jastrow."""
    xyz = np.array([[0, 0, -R / 2], [0, 0, R / 2]], np.float64)
    sc = np.array([0] * len(zetas) + [1] * len(zetas), np.int32)
    sl = np.zeros(2 * len(zetas), np.int32)
    sz = np.array(list(zetas) * 2, np.float64)
    w = np.asarray(weights, np.float64)
    orb = np.zeros((2, 2 * len(zetas)))
    orb[0, :len(zetas)] = w
    orb[1, len(zetas):] = w
    io, ina, po, prs, uo, un = _structures([([], [(0, 1)], []), ([], [(0, 0)], []), ([], [(1, 1)], [])])
    return SystemSpec(
        name="h2_nodeless", nuc_xyz=xyz, nuc_Z=np.array([1.0, 1.0]), nuc_elem=np.zeros(2, np.int32), n_elem=1,
        sh_center=sc, sh_l=sl, sh_zeta=sz, orb_coef=orb, orb_class=np.array([0, 1], np.int32),
        orb_kind=np.ones(2, np.int32), n_up=1, n_dn=1, c_vb=np.array([1.0, 0.25, 0.25]),
        inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.array([[-1.0, 1.0, 0, 0, 0, 0]]), jas_b=np.array([0.0, 1.0, 0, 0, 0, 0]), step=0.6)


# ----------------------------------------------------------------------------------
# Workload systems.
# ----------------------------------------------------------------------------------
def h2_vb(seed: int = 20220728 + 0) -> SystemSpec:
    """Two H nuclei at (0, 0, +-0.7) bohr, 1 up + 1 down electron; per center 4 s + 1 p
    Gaussians with exponents log-uniform in [0.1, 20]; two atom-localised orbitals; three
    structures (Heitler-London covalent pair + two ionic), 4 determinants; Pade e-e
    (b1 = 1/2, b2 = 1) and e-n (a1 = -Z, a2 = 1) Jastrow; step 0.3 bohr."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0, 0, -0.7], [0, 0, 0.7]], np.float64)
    sc, sl, sz = _center_shells(rng, [0, 0], [0, 0, 0, 0, 1])
    M = int(sum(NCOMP[l] for l in sl))
    lo, hi = _basis_ranges(sc, sl, 2)
    orb = np.stack([_local_orbital(rng, M, lo, hi, sc, sl, c) for c in (0, 1)])
    io, ina, po, prs, uo, un = _structures([([], [(0, 1)], []), ([], [(0, 0)], []), ([], [(1, 1)], [])])
    return SystemSpec(
        name="h2_vb", nuc_xyz=xyz, nuc_Z=np.array([1.0, 1.0]), nuc_elem=np.zeros(2, np.int32), n_elem=1,
        sh_center=sc, sh_l=sl, sh_zeta=sz, orb_coef=orb, orb_class=np.array([0, 1], np.int32),
        orb_kind=np.ones(2, np.int32), n_up=1, n_dn=1, c_vb=np.array([1.0, 0.3, 0.3]),
        inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=np.array([[-1.0, 1.0, 0, 0, 0, 0]]), jas_b=np.array([0.0, 1.0, 0, 0, 0, 0]), step=0.3)


def _kappa_pairs_same_class(orb_class, orb_kind, active_skip=()):
    """Orbital excitations (k <- l) within one localisation class: inactive->active,
    inactive->virtual, active->virtual, active->active (both directions, except the
    pairs listed in active_skip, which map structures onto each other)."""
    pairs = []
    n = len(orb_class)
    for l in range(n):
        for k in range(n):
            if k == l or orb_class[k] != orb_class[l]:
                continue
            kl, kk = orb_kind[l], orb_kind[k]
            if kl == 0 and kk in (1, 2):
                pairs.append((k, l))
            elif kl == 1 and kk == 2:
                pairs.append((k, l))
            elif kl == 1 and kk == 1 and (k, l) not in active_skip and (l, k) not in active_skip:
                pairs.append((k, l))
    return np.array(pairs, np.int32).reshape(-1, 2)


def ethylene_vb(seed: int = 20220728 + 1, n_virt_center: int = 15, n_virt_deloc: int = 8,
                params: bool = True) -> SystemSpec:
    """Ethylene-shaped 16-electron system (8 up / 8 down), six nuclei Z = {6, 6, 1, 1, 1, 1}
    planar: C at (+-1.265, 0, 0), H 2.05 bohr from each C at +-121.5 degrees from the C-C axis.
    Per center 6 s, 3 p, 1 d Gaussians (M = 126).  Orbitals: 2 C cores (localised), 4 C-H
    (delocalised), 6 active localised (sigma_a, sigma_b, pi_a, pi'_a, pi_b, pi'_b), virtuals.
    Six structures: (sigma_a, sigma_b) pair x one split-pi pair; 24 determinants, 8 unique per
    spin.  Jastrow e-n, e-e, e-e-n.  Parameters: c_2..c_6, Jastrow (45), orbital excitations."""
    rng = np.random.default_rng(seed)
    cx, dch, ang = 1.265, 2.05, math.radians(180.0 - 121.5)
    xyz = [[-cx, 0, 0], [cx, 0, 0]]
    for sgn in (-1, 1):
        for sy in (1, -1):
            xyz.append([sgn * (cx + dch * math.cos(ang)), sy * dch * math.sin(ang), 0.0])
    xyz = np.array(xyz, np.float64)
    Z = np.array([6, 6, 1, 1, 1, 1], np.float64)
    elem = np.array([0, 0, 1, 1, 1, 1], np.int32)
    sc, sl, sz = _center_shells(rng, list(elem), [0] * 6 + [1] * 3 + [2])
    M = int(sum(NCOMP[l] for l in sl))
    lo, hi = _basis_ranges(sc, sl, 6)
    orbs, ocls, okind = [], [], []

    def add(v, cls, kind):
        orbs.append(v); ocls.append(cls); okind.append(kind)

    for c in (0, 1):                                  # 0, 1: cores
        add(_local_orbital(rng, M, lo, hi, sc, sl, c), c, 0)
    for _ in range(4):                                # 2..5: C-H bonds, delocalised
        add(rng.uniform(-1, 1, M) / math.sqrt(6.0), -1, 0)
    for c in (0, 1):                                  # 6, 7: sigma_a, sigma_b
        add(_local_orbital(rng, M, lo, hi, sc, sl, c), c, 1)
    for c in (0, 0, 1, 1):                            # 8, 9: pi_a, pi'_a ; 10, 11: pi_b, pi'_b
        add(_local_orbital(rng, M, lo, hi, sc, sl, c), c, 1)
    for c in (0, 1):
        for _ in range(n_virt_center):
            add(_local_orbital(rng, M, lo, hi, sc, sl, c, s_positive=False), c, 2)
    for _ in range(n_virt_deloc):
        add(rng.uniform(-1, 1, M) / math.sqrt(6.0), -1, 2)
    orb = np.stack(orbs)
    pi_pairs = [(8, 10), (9, 11), (8, 11), (9, 10), (8, 9), (10, 11)]
    strs = [([0, 1, 2, 3, 4, 5], [(6, 7), p], []) for p in pi_pairs]
    io, ina, po, prs, uo, un = _structures(strs)
    c_vb = np.concatenate([[1.0], rng.uniform(0.1, 0.6, 5)])
    jas_a = np.zeros((2, 6))
    jas_a[:, 0] = -np.array([6.0, 1.0])
    jas_a[:, 1] = 1.0
    jas_a[:, 2:] = rng.uniform(-0.05, 0.05, (2, 4))
    jas_b = np.zeros(6)
    jas_b[1] = 1.0
    jas_b[2:] = rng.uniform(-0.05, 0.05, 4)
    theta = rng.uniform(-0.02, 0.02, (2, EEN_NFREE))
    skip = [(8, 9), (10, 11)]
    kap = _kappa_pairs_same_class(np.array(ocls), np.array(okind), active_skip=skip) if params else np.zeros((0, 2), np.int32)
    return SystemSpec(
        name="ethylene_vb", nuc_xyz=xyz, nuc_Z=Z, nuc_elem=elem, n_elem=2, sh_center=sc, sh_l=sl, sh_zeta=sz,
        orb_coef=orb, orb_class=np.array(ocls, np.int32), orb_kind=np.array(okind, np.int32),
        n_up=8, n_dn=8, c_vb=c_vb, inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        jas_a=jas_a, jas_b=jas_b, een_on=True, een_theta=theta,
        cparam=np.arange(1, 6, dtype=np.int32) if params else np.zeros(0, np.int32),
        jas_param=params, kappa_kl=kap, step=0.3)


def bovb(spec: SystemSpec, eps: float = 0.05, seed: int = 20220728 + 9) -> SystemSpec:
    """Breathing-orbital VB form of a VBSCF system (Sec. 2.2, Eq. PsiJBOVB): every structure
    gets its own copy of the orbitals it uses (inactive, paired and unpaired), so that each
    structure's orbitals can relax on their own.  The original orbitals stay in the list first
    (no structure uses them: they are excitation targets); structure I's copies follow in a
    block.  Each copy's nonzero coefficients are scaled by (1 + eps u), u ~ U(-1, 1) seeded (eps = 0:
    exact copies, the wave function is the VBSCF one).  Every VBSCF orbital excitation (k, l)
    becomes one excitation per structure I that uses l: (k_I, l_I) with k_I = I's copy of k when
    I uses k, else the original k."""
    rng = np.random.default_rng(seed)
    nvb = spec.Nvb
    orbs = [spec.orb_coef[q] for q in range(spec.Norb)]
    cls = list(spec.orb_class)
    kind = list(spec.orb_kind)
    copy = []                                        # per structure: original -> copy index
    strs = []
    for I in range(nvb):
        ina = [int(x) for x in spec.inact[spec.inact_off[I]:spec.inact_off[I + 1]]]
        prs = [tuple(int(v) for v in p) for p in spec.pairs[spec.pair_off[I]:spec.pair_off[I + 1]]]
        unp = [int(x) for x in spec.unp[spec.unp_off[I]:spec.unp_off[I + 1]]]
        used = sorted(set(ina) | {v for p in prs for v in p} | set(unp))
        m = {}
        for q in used:
            v = spec.orb_coef[q].copy()
            nz = v != 0.0
            v[nz] *= 1.0 + eps * rng.uniform(-1.0, 1.0, int(nz.sum()))
            m[q] = len(orbs)
            orbs.append(v)
            cls.append(spec.orb_class[q])
            kind.append(spec.orb_kind[q])
        copy.append(m)
        strs.append(([m[q] for q in ina], [(m[a], m[b]) for a, b in prs], [m[q] for q in unp]))
    io, ina, po, prs, uo, un = _structures(strs)
    kap = []
    for k, l in spec.kappa_kl:
        for I in range(nvb):
            if int(l) in copy[I]:
                kap.append((copy[I].get(int(k), int(k)), copy[I][int(l)]))
    return dataclasses.replace(
        spec, name=spec.name + "_bovb", orb_coef=np.stack(orbs), orb_class=np.array(cls, np.int32),
        orb_kind=np.array(kind, np.int32), inact_off=io, inact=ina, pair_off=po, pairs=prs, unp_off=uo, unp=un,
        kappa_kl=np.array(kap, np.int32).reshape(-1, 2))


def ethylene_bovb(eps: float = 0.05) -> SystemSpec:
    """The ethylene-shaped workload in breathing-orbital form: six structures with their own
    10 orbitals each (24 determinants, none shared between structures)."""
    return bovb(ethylene_vb(), eps=eps)


def ethylene_vb_p400(seed: int = 20220728 + 4) -> SystemSpec:
    """The ethylene-shaped system with enough virtual orbitals for exactly 400 parameters
    (5 structure coefficients, 45 Jastrow, 350 orbital excitations), for the linear-method
    accumulation at scale."""
    return ethylene_vb(seed=seed, n_virt_center=30, n_virt_deloc=24, params=True)


def small_open_shell(seed: int = 11, params: bool = True, een: bool = True) -> SystemSpec:
    """Small test system: 3 nuclei (Z = 3, 1, 1), 5 electrons (3 up, 2 down, one unpaired),
    s/s/p/d shells per center, one localised core, four active orbitals, three virtuals; four
    structures mixing a self-pair, distinct pairs and unpaired electrons."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, 0.0], [2.1, 0.4, -0.3], [-0.8, 1.9, 0.6]])
    Z = np.array([3.0, 1.0, 1.0])
    elem = np.array([0, 1, 1], np.int32)
    sc, sl, sz = _center_shells(rng, list(elem), [0, 0, 1, 2], 0.2, 8.0)
    M = int(sum(NCOMP[l] for l in sl))
    lo, hi = _basis_ranges(sc, sl, 3)
    orbs, ocls, okind = [], [], []
    for c, kind in [(0, 0), (0, 1), (1, 1), (2, 1), (0, 1), (0, 2), (1, 2), (2, 2)]:
        orbs.append(_local_orbital(rng, M, lo, hi, sc, sl, c, s_positive=(kind != 2)))
        ocls.append(c)
        okind.append(kind)
    strs = [([0], [(1, 2)], [3]), ([0], [(2, 3)], [1]), ([0], [(1, 1)], [2]), ([0], [(4, 2)], [3])]
    io, ina, po, prs, uo, un = _structures(strs)
    jas_a = np.zeros((2, 6))
    jas_a[:, 0] = [-3.0, -1.0]
    jas_a[:, 1] = [1.2, 0.9]
    jas_a[:, 2:] = rng.uniform(-0.1, 0.1, (2, 4))
    jas_b = np.zeros(6)
    jas_b[1] = 0.8
    jas_b[2:] = rng.uniform(-0.1, 0.1, 4)
    kap = np.array([(4, 1), (1, 4), (5, 1), (5, 0), (4, 0), (6, 2), (7, 3), (5, 4), (3, 2)], np.int32)
    return SystemSpec(
        name="small_open_shell", nuc_xyz=xyz, nuc_Z=Z, nuc_elem=elem, n_elem=2, sh_center=sc, sh_l=sl, sh_zeta=sz,
        orb_coef=np.stack(orbs), orb_class=np.array(ocls, np.int32), orb_kind=np.array(okind, np.int32),
        n_up=3, n_dn=2, c_vb=np.array([1.0, 0.4, -0.3, 0.25]), inact_off=io, inact=ina, pair_off=po, pairs=prs,
        unp_off=uo, unp=un, jas_a=jas_a, jas_b=jas_b, een_on=een,
        een_theta=rng.uniform(-0.05, 0.05, (2, EEN_NFREE)),
        cparam=np.array([1, 2, 3], np.int32) if params else np.zeros(0, np.int32), jas_param=params,
        kappa_kl=kap if params else np.zeros((0, 2), np.int32), step=0.4)


def dmc48(seed: int = 20220728 + 3) -> SystemSpec:
    """48-electron system for DMC at scale: 12 nuclei C2 N2 O2 H6 (sum Z = 48) at seeded positions
    at least 1.8 bohr apart; per center 5 s, 3 p, 2 d Gaussians (M = 312), exponents per element
    log-uniform in [0.1, 20].  24 electrons per spin occupy 20 inactive orbitals and 4 of 8
    active orbitals (localised on the nuclei where the initial walkers start; the orbitals of
    one centre take s, p_x, p_y, p_z and d characters in turn, so that they stay well apart).
    20 structures:
    12 pair the 8 active orbitals into 4 distinct singlet pairs (16 determinants each), 8 use 3
    distinct pairs and one doubly occupied active orbital (8 determinants each): 256
    determinants, up to C(8,4) = 70 unique determinants per spin.  Jastrow e-n, e-e, e-e-n; no
    optimisable parameters (the system is for DMC)."""
    rng = np.random.default_rng(seed)
    Z = np.array([6, 6, 7, 7, 8, 8, 1, 1, 1, 1, 1, 1], np.float64)
    Nn = len(Z)
    box = 1.8 * (Nn ** (1.0 / 3.0)) + 1.0
    xyz = []
    while len(xyz) < Nn:
        p = rng.uniform(-box, box, 3)
        if all(np.linalg.norm(p - q) >= 1.8 for q in xyz):
            xyz.append(p)
    xyz = np.array(xyz, np.float64)
    elems = [1, 6, 7, 8]
    elem = np.array([elems.index(int(z)) for z in Z], np.int32)
    sc, sl, sz = _center_shells(rng, list(elem), [0] * 5 + [1] * 3 + [2] * 2)
    M = int(sum(NCOMP[l] for l in sl))
    lo, hi = _basis_ranges(sc, sl, Nn)
    slots = []
    for a, z in enumerate(Z):
        slots += [a] * int(round(z))
    n_inact, n_act = 20, 8
    orbs, ocls, okind = [], [], []
    per_center = {}
    for q in range(n_inact + n_act):
        c = slots[(2 * q) % len(slots)] if q < n_inact else slots[(2 * n_inact + (q - n_inact)) % len(slots)]
        k = per_center.get(c, 0)
        per_center[c] = k + 1
        orbs.append(_shaped_orbital(rng, M, sc, sl, c, k))
        ocls.append(c)
        okind.append(0 if q < n_inact else 1)
    orb = np.stack(orbs)
    inactive = list(range(n_inact))
    act = list(range(n_inact, n_inact + n_act))
    strs, seen = [], set()
    while len(strs) < 12:                      # 4 distinct pairs
        perm = [int(x) for x in rng.permutation(act)]
        prs = tuple(sorted((min(perm[2 * q], perm[2 * q + 1]), max(perm[2 * q], perm[2 * q + 1])) for q in range(4)))
        if prs not in seen:
            seen.add(prs)
            strs.append((inactive, list(prs), []))
    while len(strs) < 20:                      # 3 distinct pairs + 1 doubly occupied active orbital
        perm = [int(x) for x in rng.permutation(act)]
        prs = [(min(perm[2 * q], perm[2 * q + 1]), max(perm[2 * q], perm[2 * q + 1])) for q in range(3)]
        prs = tuple(sorted(prs + [(perm[6], perm[6])]))
        if prs not in seen:
            seen.add(prs)
            strs.append((inactive, list(prs), []))
    io, ina, po, prs_arr, uo, un = _structures(strs)
    c_vb = np.concatenate([[1.0], rng.uniform(0.1, 0.6, len(strs) - 1)])
    jas_a = np.zeros((len(elems), 6))
    jas_a[:, 0] = -np.array(elems, np.float64)
    jas_a[:, 1] = 1.0
    jas_a[:, 2:] = rng.uniform(-0.05, 0.05, (len(elems), 4))
    jas_b = np.zeros(6)
    jas_b[1] = 1.0
    jas_b[2:] = rng.uniform(-0.05, 0.05, 4)
    return SystemSpec(
        name="dmc48", nuc_xyz=xyz, nuc_Z=Z, nuc_elem=elem, n_elem=len(elems), sh_center=sc, sh_l=sl, sh_zeta=sz,
        orb_coef=orb, orb_class=np.array(ocls, np.int32), orb_kind=np.array(okind, np.int32), n_up=24, n_dn=24,
        c_vb=c_vb, inact_off=io, inact=ina, pair_off=po, pairs=prs_arr, unp_off=uo, unp=un, jas_a=jas_a,
        jas_b=jas_b, een_on=True, een_theta=rng.uniform(-0.02, 0.02, (len(elems), EEN_NFREE)), step=0.3)


def random_molecule(seed: int, max_electrons: int = 32) -> SystemSpec:
    """One system of the batched workload of many small uneven molecules: 2-10 nuclei with Z in
    {1, 3, 6, 7, 8, 9} at random positions at least 1.8 bohr apart, N = sum Z rounded up to
    even and clamped to [2, max_electrons] (resampled while sum Z > max_electrons + 2), Sz = 0.
    Per center 4-12 Gaussian shells split s:p:d about 5:3:2 (at least one s), exponents per
    element log-uniform in [0.1, 20].  Orbitals: N/2 - k doubly occupied and 2k active
    localised orbitals, placed on the nuclei in proportion to their charges, k = 0..4 distinct pairs per structure
    (at most n);
    2-16 structures drawn as random pairings of the active orbitals (covalent or ionic, duplicates
    removed).  Jastrow e-n, e-e and e-e-n with small random polynomial parts; parameters: the
    structure coefficients after the first and the Jastrow."""
    rng = np.random.default_rng(seed)
    zs = [1, 3, 6, 7, 8, 9]
    while True:
        Nn = int(rng.integers(2, 11))
        Z = rng.choice(zs, size=Nn)
        if Z.sum() <= max_electrons + 2:
            break
    N = int(min(max(2, Z.sum() + (Z.sum() % 2)), max_electrons))
    n = N // 2
    # positions: rejection sampling in a box that grows with the number of nuclei
    box = 1.8 * (Nn ** (1.0 / 3.0)) + 1.0
    xyz = []
    while len(xyz) < Nn:
        p = rng.uniform(-box, box, 3)
        if all(np.linalg.norm(p - q) >= 1.8 for q in xyz):
            xyz.append(p)
    xyz = np.array(xyz, np.float64)
    elems = sorted(set(int(z) for z in Z))
    elem = np.array([elems.index(int(z)) for z in Z], np.int32)
    # shells per element: 4-12 primitives, s:p:d about 5:3:2
    shell_ls_elem = {}
    for e in range(len(elems)):
        nsh = int(rng.integers(4, 13))
        nd = int(round(0.2 * nsh))
        npp = int(round(0.3 * nsh))
        ns = max(1, nsh - nd - npp)
        shell_ls_elem[e] = [0] * ns + [1] * npp + [2] * nd
    zeta_elem = {e: np.exp(rng.uniform(math.log(0.1), math.log(20.0), size=len(v))) for e, v in shell_ls_elem.items()}
    sc, sl, sz = [], [], []
    for c in range(Nn):
        e = int(elem[c])
        for l, z in zip(shell_ls_elem[e], zeta_elem[e]):
            sc.append(c); sl.append(l); sz.append(z)
    sc, sl, sz = np.array(sc, np.int32), np.array(sl, np.int32), np.array(sz, np.float64)
    M = int(sum(NCOMP[l] for l in sl))
    lo, hi = _basis_ranges(sc, sl, Nn)
    # distinct pairs per structure (up to 4: 16 determinants); systems whose unique determinants
    # do not fit the per-determinant kernels run on reference-determinant tables
    k = min(int(rng.integers(0, 5)), n)
    n_inact = n - k
    # orbital q sits on the nucleus that initial_walkers() places electrons 2q and 2q + 1 near
    # (nuclei listed round(Z) times each), so that starting configurations are well conditioned
    slots = []
    for a, z in enumerate(Z):
        slots += [a] * max(1, int(round(z)))
    orbs, ocls, okind = [], [], []
    for q in range(n_inact):
        c = slots[(2 * q) % len(slots)]
        orbs.append(_local_orbital(rng, M, lo, hi, sc, sl, c)); ocls.append(c); okind.append(0)
    act = []
    for q in range(2 * k):
        c = slots[(2 * n_inact + q) % len(slots)]
        act.append(len(orbs))
        orbs.append(_local_orbital(rng, M, lo, hi, sc, sl, c)); ocls.append(c); okind.append(1)
    orb = np.stack(orbs)
    inactive = list(range(n_inact))
    target = int(rng.integers(2, 17))
    strs, seen = [], set()
    for _ in range(200):
        if len(strs) >= target:
            break
        perm = list(rng.permutation(act)) if k else []
        prs = []
        for q in range(k):
            a, b = int(perm[2 * q]), int(perm[2 * q + 1])
            if rng.uniform() < 0.2:   # ionic: both electrons of the pair on one orbital
                b = a
            prs.append((min(a, b), max(a, b)))
        key = tuple(sorted(prs))
        if key in seen:
            continue
        seen.add(key)
        strs.append((inactive, prs, []))
    io, ina, po, prs_arr, uo, un = _structures(strs)
    nvb = len(strs)
    c_vb = np.concatenate([[1.0], rng.uniform(0.1, 0.6, nvb - 1)])
    n_elem = len(elems)
    jas_a = np.zeros((n_elem, 6))
    jas_a[:, 0] = -np.array(elems, np.float64)
    jas_a[:, 1] = 1.0
    jas_a[:, 2:] = rng.uniform(-0.05, 0.05, (n_elem, 4))
    jas_b = np.zeros(6)
    jas_b[1] = 1.0
    jas_b[2:] = rng.uniform(-0.05, 0.05, 4)
    return SystemSpec(
        name="random_molecule_%d" % seed, nuc_xyz=xyz, nuc_Z=Z.astype(np.float64), nuc_elem=elem, n_elem=n_elem,
        sh_center=sc, sh_l=sl, sh_zeta=sz, orb_coef=orb, orb_class=np.array(ocls, np.int32),
        orb_kind=np.array(okind, np.int32), n_up=n, n_dn=n, c_vb=c_vb, inact_off=io, inact=ina, pair_off=po,
        pairs=prs_arr, unp_off=uo, unp=un, jas_a=jas_a, jas_b=jas_b, een_on=True,
        een_theta=rng.uniform(-0.02, 0.02, (n_elem, EEN_NFREE)),
        cparam=np.arange(1, nvb, dtype=np.int32), jas_param=True, step=0.3)


def batched_workload(n_systems: int = 64, seed: int = 20220728 + 2, w_lo: int = 256, w_hi: int = 4096):
    """The batched workload: n_systems random molecules with walker counts drawn log-uniform
    in [w_lo, w_hi] (rounded to multiples of 32).  Returns (specs, walker counts)."""
    rng = np.random.default_rng(seed)
    specs = [random_molecule(seed * 1000 + i) for i in range(n_systems)]
    W = [int(round(math.exp(rng.uniform(math.log(w_lo), math.log(w_hi))) / 32.0)) * 32 for _ in range(n_systems)]
    return specs, [max(32, w) for w in W]


def initial_walkers(spec: SystemSpec, W: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Walker positions (W, N, 3): electron e placed Gaussian(sigma) around a nucleus chosen
    round-robin over a list holding each nucleus round(Z) times; up and down electrons
    alternate through that list."""
    rng = np.random.default_rng(seed)
    slots = []
    for a, z in enumerate(spec.nuc_Z):
        slots += [a] * max(1, int(round(z)))
    centers = np.empty(spec.N, np.int64)
    for i in range(spec.n_up):
        centers[i] = slots[(2 * i) % len(slots)]
    for i in range(spec.n_dn):
        centers[spec.n_up + i] = slots[(2 * i + 1) % len(slots)]
    R = spec.nuc_xyz[centers][None, :, :] + sigma * rng.standard_normal((W, spec.N, 3))
    return np.ascontiguousarray(R, dtype=np.float64)
