"""Direct tests of the sweep's bit-pattern helpers (wf_device.cuh): f2d_bits (float -> double by
moving the bits, with the conversion for zero, subnormal and non-finite values) against the
exact IEEE widening, and less_nonneg (a < b for a >= 0 and b >= 0 or NaN, compared on the bit
patterns) against the floating-point comparison, over random and special values."""
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
__global__ void f2d_probe(const float* x, double* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = vbq::f2d_bits(x[i]);
}
__global__ void less_probe(const double* a, const double* b, int* r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = vbq::less_nonneg(a[i], b[i]) ? 1 : 0;
}
template <class T>
static cudaError_t up(T** d, const T* h, int n) {
  cudaError_t e = cudaMalloc(d, sizeof(T) * (n > 0 ? n : 1));
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice);
  return e;
}
extern "C" int run_f2d(const float* x, double* y, int n) {
  float* dx = nullptr;
  double* dy = nullptr;
  cudaError_t e = up(&dx, x, n);
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(double) * n);
  if (e == cudaSuccess) {
    f2d_probe<<<(n + 255) / 256, 256>>>(dx, dy, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  return (int)e;
}
extern "C" int run_less(const double* a, const double* b, int* r, int n) {
  double *da = nullptr, *db = nullptr;
  int* dr = nullptr;
  cudaError_t e = up(&da, a, n);
  if (e == cudaSuccess) e = up(&db, b, n);
  if (e == cudaSuccess) e = cudaMalloc(&dr, sizeof(int) * n);
  if (e == cudaSuccess) {
    less_probe<<<(n + 255) / 256, 256>>>(da, db, dr, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(r, dr, sizeof(int) * n, cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dr);
  return (int)e;
}
"""


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = tempfile.mkdtemp(prefix="bitconv_probe_")
    src, so = os.path.join(d, "probe.cu"), os.path.join(d, "probe.so")
    with open(src, "w") as f:
        f.write(PROBE)
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.run_f2d.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.run_less.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def test_f2d_bits_is_the_exact_widening(probe):
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 1 << 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x807fffff, 0x00800000, 0x7f7fffff, 0xff7fffff,
                        0x3f800000, 0x7f800000, 0xff800000, 0x7fc00000, 0x3effffff], dtype=np.uint32)
    x = np.concatenate([bits, special]).view(np.float32)
    y = np.empty(x.size, dtype=np.float64)
    assert probe.run_f2d(x.ctypes.data, y.ctypes.data, x.size) == 0
    with np.errstate(invalid="ignore"):  # signalling NaNs among the random patterns
        ref = x.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(y), nan)
    np.testing.assert_array_equal(y[~nan].view(np.int64), ref[~nan].view(np.int64))


def test_less_nonneg_is_the_comparison(probe):
    rng = np.random.default_rng(12)
    n = 1 << 18
    a = rng.random(n)  # acceptance uniforms in [0, 1)
    tiny = np.finfo(np.float64).tiny
    pool = np.array([0.0, 5e-324, tiny, 0.5, 1.0 - 2.0 ** -53, 1.0, 2.0, 1e300, np.inf, np.nan])
    b = np.where(rng.random(n) < 0.5, rng.random(n) * 2.0, pool[rng.integers(0, pool.size, n)])
    # equal pairs and neighbours one ulp apart
    a[:1000] = b[:1000] = rng.random(1000)
    b[1000:2000] = np.nextafter(a[1000:2000], 2.0)
    b[2000:3000] = np.nextafter(a[2000:3000], -1.0)
    a[3000:3100] = 0.0
    b[3000:3100] = 0.0
    r = np.empty(n, dtype=np.int32)
    assert probe.run_less(a.ctypes.data, b.ctypes.data, r.ctypes.data, n) == 0
    with np.errstate(invalid="ignore"):
        ref = (a < b).astype(np.int32)
    np.testing.assert_array_equal(r, ref)
