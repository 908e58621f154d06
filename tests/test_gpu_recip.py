"""Direct test of the device reciprocal recip_dd (the LU pivot and U-diagonal reciprocals of the
Slater-matrix factorisation): the float reciprocal of the mantissa refined by two Newton steps
and scaled by the exponent, with the division for zero, subnormal, huge and non-finite inputs.

Against IEEE division 1/x over the whole normal exponent range, both signs, mantissas near 1
and near 2, and the edges of the fast branch: at most 2 ulp (two Newton steps from a correctly
rounded float seed leave an error far below an ulp before the last two roundings); the
division branch is exact (zero, subnormals, the largest exponents, infinities, NaN)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2207_14715_gb300", "csrc")

PROBE = r"""
#include "wf_device.cuh"
__global__ void recip_probe(const double* x, double* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = vbq::recip_dd(x[i]);
}
extern "C" int run_recip(const double* x, double* y, int n) {
  double *dx = nullptr, *dy = nullptr;
  cudaError_t e = cudaMalloc(&dx, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    recip_probe<<<(n + 255) / 256, 256>>>(dx, dy, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  return (int)e;
}
"""


@pytest.fixture(scope="module")
def recip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = tempfile.mkdtemp(prefix="recip_probe_")
    src, so = os.path.join(d, "probe.cu"), os.path.join(d, "probe.so")
    with open(src, "w") as f:
        f.write(PROBE)
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.run_recip.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]

    def run(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        assert lib.run_recip(x.ctypes.data, y.ctypes.data, x.size) == 0
        return y
    return run


def _ulps(a, b):
    """Distance in units in the last place between finite doubles of one sign."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_recip_dd_normal_range(recip):
    rng = np.random.default_rng(7)
    n = 1 << 20
    # exponents over the fast branch (biased 2..2044), random mantissas, both signs
    e = rng.integers(2, 2045, size=n)
    m = rng.integers(0, 1 << 52, size=n, dtype=np.int64)
    bits = (e.astype(np.int64) << 52) | m
    x = bits.view(np.float64) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # mantissas next to 1 and next to 2 at a few exponents, and the branch edges
    edge = []
    for ex in (2, 3, 1022, 1023, 1024, 2043, 2044):
        base = ex << 52
        for k in range(64):
            edge += [base + k, base + (1 << 52) - 1 - k]
    xe = np.array(edge, dtype=np.int64).view(np.float64)
    tiny = np.finfo(np.float64).tiny
    x = np.concatenate([x, xe, -xe, [1.0, -1.0, 0.5, 2.0, 3.0, 1.0 / 3.0, 7.0, 1e-300, 1e300, 2 * tiny, 3 * tiny]])
    y = recip(x)
    ref = 1.0 / x
    assert np.all(np.sign(y) == np.sign(ref))
    u = _ulps(np.abs(y), np.abs(ref))
    print("recip_dd: %d inputs, worst %d ulp, %.4f%% not correctly rounded" % (x.size, u.max(), 100.0 * np.mean(u > 0)))
    assert u.max() <= 2


def test_recip_dd_division_branch(recip):
    tiny = np.finfo(np.float64).tiny
    # biased exponents 0 and 1, and 2045 and 2046: the division
    sub = np.array([5e-324, 1e-310, tiny / 3.0, tiny, 1.5 * tiny], dtype=np.float64)
    big = np.array([np.finfo(np.float64).max, 1.5e308, 2.0 ** 1022, 2.0 ** 1023], dtype=np.float64)
    x = np.concatenate([sub, -sub, big, -big, [0.0, -0.0, np.inf, -np.inf]])
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    y = recip(x)
    np.testing.assert_array_equal(y, ref)
    assert np.isnan(recip(np.array([np.nan]))[0])
