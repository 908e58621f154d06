"""Resonance energies on the GPU (Sec. 2.4 and the diabatic states of Sec. 3): the VMC energy of
the wave function restricted to a subset of the VB structures minus that of the full expansion,
each from an independent VMC run, with its statistical error.

Error bars: VMC walkers never interact, so the time averages of disjoint walker groups are
independent; sigma of each energy from 32 groups, sigma of a difference of independent runs
sigma^2 = sigma_sub^2 + sigma_full^2.  The reblocked error of the walker-averaged series is
printed beside it.
  H2 (covalent structure only vs covalent + two ionic): the GPU's resonance energy (mixed form)
     agrees with the oracle's within 2 sigma (the two sigmas combined).
  Ethylene-shaped system (four of the six split-pi structures vs all six): the mixed and FP64
     forms on the GPU, from different random streams, agree within 2 sigma."""
import numpy as np
import pytest

from paper_2207_14715_gb300 import systems as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GROUPS = 32


@pytest.fixture(scope="module")
def vb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14715_gb300 import build, vbqmc
    build.build()
    ctx = vbqmc.create(0)
    yield vbqmc, ctx
    ctx.close()


def _groups(E):
    g = E.reshape(E.shape[0], GROUPS, -1).mean(axis=(0, 2))
    return g.mean(), g.std(ddof=1) / np.sqrt(GROUPS)


def gpu_energy(vb, spec, W, nequil, nsteps, seed, precision):
    """Mean E_L of a VMC run and its error from independent walker groups; the series of walker
    averages for reblocking."""
    mod, ctx = vb
    ctx.set_system(0, spec)
    Rt = torch.tensor(S.initial_walkers(spec, W, seed), device="cuda")
    lp = torch.zeros(W, dtype=torch.float64, device="cuda")
    sg, el = torch.zeros_like(lp), torch.zeros_like(lp)
    ctx.vmc_steps(0, precision, Rt, nequil, spec.step, seed, step0=0)
    es = []
    for k in range(nsteps):
        ctx.vmc_steps(0, precision, Rt, 1, spec.step, seed, step0=100000 + k, logpsi=lp, sign=sg, eloc=el)
        es.append(el.cpu().numpy().copy())
    E = np.array(es)
    m, e = _groups(E)
    return m, e, E.mean(axis=1)


def oracle_energy(orc, spec, W, nequil, nsteps, seed):
    R, _, _, _ = orc.vmc(spec, S.initial_walkers(spec, W, seed), nequil, spec.step, seed=seed, eloc=False)
    _, hist, _, _ = orc.vmc(spec, R, nsteps, spec.step, seed=seed, step0=100000)
    E = np.asarray(hist)
    m, e = _groups(E)
    return m, e, E.mean(axis=1)


def test_h2_resonance_energy_matches_oracle(vb, orc):
    full = S.h2_vb()
    sub = S.structure_subset(full, [0])
    gs, es, ts = gpu_energy(vb, sub, 65536, 100, 400, 11, 1)
    gf, ef, tf = gpu_energy(vb, full, 65536, 100, 400, 12, 1)
    os_, eos, _ = oracle_energy(orc, sub, 16384, 100, 400, 13)
    of, eof, _ = oracle_energy(orc, full, 16384, 100, 400, 14)
    dg, sg = gs - gf, np.hypot(es, ef)
    do, so = os_ - of, np.hypot(eos, eof)
    rb = np.hypot(orc.reblock(ts)[1], orc.reblock(tf)[1])
    print("H2: E(covalent) GPU %.5f +- %.5f, oracle %.5f +- %.5f; E(all) GPU %.5f +- %.5f, oracle %.5f +- %.5f"
          % (gs, es, os_, eos, gf, ef, of, eof))
    print("H2 resonance energy: GPU %.5f +- %.5f (reblocked %.5f), oracle %.5f +- %.5f"
          % (dg, sg, rb, do, so))
    assert np.isfinite(dg) and sg > 0
    assert abs(dg - do) <= 2.0 * np.hypot(sg, so)


def test_ethylene_resonance_energy_mixed_vs_fp64(vb, orc):
    full = S.ethylene_vb()
    sub = S.structure_subset(full, [0, 1, 2, 3])
    res = {}
    for precision, seeds in ((1, (21, 22)), (0, (23, 24))):
        W = 16384 if precision else 4096
        gs, es, ts = gpu_energy(vb, sub, W, 200, 200, seeds[0], precision)
        gf, ef, tf = gpu_energy(vb, full, W, 200, 200, seeds[1], precision)
        rb = np.hypot(orc.reblock(ts)[1], orc.reblock(tf)[1])
        res[precision] = (gs - gf, np.hypot(es, ef))
        print("ethylene resonance energy (%s): E(4 structures) %.4f +- %.4f, E(6) %.4f +- %.4f, "
              "difference %.4f +- %.4f (reblocked %.4f)"
              % ("mixed" if precision else "fp64", gs, es, gf, ef, gs - gf, np.hypot(es, ef), rb))
    (dm, sm), (dd, sd) = res[1], res[0]
    assert np.isfinite(dm) and np.isfinite(dd)
    assert abs(dm - dd) <= 2.0 * np.hypot(sm, sd)
