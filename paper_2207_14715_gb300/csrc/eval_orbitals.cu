// Orbitals at every electron (arXiv:2207.14715, Sec. 2.1: phi_p = sum_mu lambda_{p mu} chi_mu):
// basis functions with gradients and Laplacians, then the contraction in balanced chunks of
// the nonzero coefficients, four orbitals of equal coefficient range at a time.  One warp per (walker, electron), so that many warps share each
// SM; results go to the evaluation workspace:
//   OB [W][N][5][n_ev] bulk type: phi, d/dx, d/dy, d/dz, lap phi of the evaluated orbitals
//   OD [W][N][n_det_ev] double: values of the orbitals that enter determinants; in the mixed
//      form these come from float-float basis values and coefficients, and OB holds them
//      rounded to float.

#include "orbital_body.cuh"

namespace vbq {

namespace {
template <class Tb>
__global__ void __launch_bounds__(32 * kOrbWarps, 4) orbital_kernel(const SysDev s, const OrbLayout L, int W,
                                                                     const double* __restrict__ Rg,
                                                                     Tb* __restrict__ OB, double* __restrict__ OD) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kOrbWarps + wl;
  if (gw >= (long long)W * s.N) return;
  orbital_body<Tb>(s, L, gw, smem + wl * L.warp_bytes, Rg, OB, OD);
}

template <class Tb>
__global__ void __launch_bounds__(32 * kOrbWarps, 4)
    orbital_batch_kernel(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items, int nitems) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    orbital_body<Tb>(b.dev, b.lay.orb, (long long)item.first + wl, smem + wl * b.lay.orb.warp_bytes, b.R,
                     static_cast<Tb*>(b.OB), b.OD);
  }
}

}  // namespace

int make_orb_layout(const SysDev& s, int tb, int max_smem, OrbLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int M = s.M;
  L.bas = take(5 * M * tb);
  L.bds = take(tb == 4 ? 8 * M : 16);
  L.ctab = take(tb == 4 ? 8 * 4 * s.Nn : 16);
  L.part = take(5 * s.evq_width * tb * std::max(s.n_evq_chunk, 1));
  L.partd = take(tb == 4 ? 8 * std::max(s.n_det_chunk, 1) : 16);
  L.warp_bytes = off;
  L.wpb = kOrbWarps;
  if (kOrbWarps * off > max_smem) return VBQMC_ERR_CAPACITY;
  return VBQMC_OK;
}

template <class Tb>
cudaError_t launch_orbitals(const SysDev& s, const OrbLayout& L, int W, const double* R, Tb* OB, double* OD,
                            cudaStream_t st) {
  const int smem = kOrbWarps * L.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(orbital_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long warps = (long long)W * s.N;
  orbital_kernel<Tb><<<(unsigned)((warps + kOrbWarps - 1) / kOrbWarps), 32 * kOrbWarps, smem, st>>>(s, L, W, R, OB,
                                                                                                    OD);
  return cudaGetLastError();
}

template <class Tb>
cudaError_t launch_orbitals_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps,
                                  int smem, cudaStream_t st) {
  orbital_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems);
  return cudaGetLastError();
}
int orbital_batch_grid(int is_float, int nitems, int warps, int smem, int persist) {
  return batch_grid(is_float ? (const void*)orbital_batch_kernel<float> : (const void*)orbital_batch_kernel<double>,
                    nitems, warps, smem, persist);
}
template cudaError_t launch_orbitals_batch<float>(const BatchSys*, const BatchItem*, int, int, int, int, cudaStream_t);
template cudaError_t launch_orbitals_batch<double>(const BatchSys*, const BatchItem*, int, int, int, int, cudaStream_t);

template cudaError_t launch_orbitals<float>(const SysDev&, const OrbLayout&, int, const double*, float*, double*,
                                            cudaStream_t);
template cudaError_t launch_orbitals<double>(const SysDev&, const OrbLayout&, int, const double*, double*, double*,
                                             cudaStream_t);

}  // namespace vbq
