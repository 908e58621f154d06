"""The allocation-free linear-method accumulation against the context's accumulation.

Both run the same kernels; only where the workspace lives differs (a fixed device array that
keeps the previous call's contents, against a context-owned allocation).  Two calls in a row
with different sizes, precisions and weights, then a repeat of the first, each compared with
the context's entry point within the linear-method tests' tolerance (1e-5 of the matrix scale
for float inputs, 2e-6 for double inputs).  This file is collected last on purpose: it must
pass after everything else has used the device, as well as alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14715_gb300 import build, vbqmc
    build.build()
    ctx = vbqmc.create(0)
    yield vbqmc, ctx
    ctx.close()


def inputs(M, P, seed, precision, weights):
    rng = np.random.default_rng(seed)
    mix = rng.normal(size=(P, P)) / np.sqrt(P)
    O = rng.normal(size=(M, P)) @ mix + rng.normal(size=P)
    dE = rng.normal(size=(M, P)) * 0.3
    E = -10.0 + rng.normal(size=M) + 0.5 * O[:, 0]
    w = rng.uniform(0.2, 1.8, M) if weights else None
    dt = torch.float32 if precision == 1 else torch.float64
    dev = lambda x, d=torch.float64: None if x is None else torch.tensor(x, dtype=d, device="cuda")
    return dev(O, dt), dev(dE, dt), dev(E), dev(w)


def outputs(P, fill):
    f = lambda *shape: torch.full(shape, fill, dtype=torch.float64, device="cuda")
    return {"E0": f(1), "gL": f(P), "gR": f(P), "S": f(P, P), "H": f(P, P)}


def compare(got, ref, precision):
    tol = 1e-5 if precision == 1 else 2e-6
    for k in ("S", "H", "gL", "gR"):
        g, r = got[k].cpu().numpy(), ref[k].cpu().numpy()
        scale = max(1.0, np.abs(r).max())
        assert np.isfinite(g).all(), k
        assert np.abs(g - r).max() / scale < tol, (k, np.abs(g - r).max() / scale)
    e0, r0 = float(got["E0"][0]), float(ref["E0"][0])
    assert abs(e0 - r0) < 1e-12 * max(1.0, abs(r0))


CASES = [  # (M, P, precision, weights, seed)
    (16384, 216, 1, True, 1),   # one block of the ethylene-shaped run: 16384 walkers, 216 parameters
    (3001, 37, 0, False, 2),    # smaller, double inputs: stale contents of the first call must not leak
]


def test_noalloc_matches_context_accumulation(vb):
    mod, ctx = vb
    results = []
    for (M, P, prec, weights, seed) in CASES + CASES[:1]:
        O, dE, E, w = inputs(M, P, seed, prec, weights)
        ref = ctx.accumulate_lin_matrices(prec, O, dE, E, w)
        got = outputs(P, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        mod.accumulate_lin_matrices_noalloc(prec, O, dE, E, w, got["E0"], got["gL"], got["gR"], got["S"], got["H"])
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        compare(got, ref, prec)
        results.append((got, free0, free1))
    # the repeat of the first case: same answer as the first call, and no device memory taken
    first, again = results[0][0], results[2][0]
    compare(again, first, CASES[0][2])
    assert results[2][1] == results[2][2]


def test_noalloc_rejects_sizes_beyond_its_scratch(vb):
    mod, _ = vb
    M, P = 65536, 400  # needs ~256 MiB of centred values
    O = torch.zeros((M, P), dtype=torch.float32, device="cuda")
    dE = torch.zeros_like(O)
    E = torch.zeros(M, dtype=torch.float64, device="cuda")
    out = outputs(P, 0.0)
    with pytest.raises(mod.VbqmcError, match="fixed maximum"):
        mod.accumulate_lin_matrices_noalloc(1, O, dE, E, None, out["E0"], out["gL"], out["gR"], out["S"], out["H"])
