// Jastrow part of the evaluation (arXiv:2207.14715, Sec. 2.1, Jastrow factor; Sec. 2.3.1):
//   jastrow_kernel        ln J, grad_i ln J, lap_i ln J and the Coulomb potential per walker
//   jastrow_deriv_kernel  O_alpha = d ln J/d alpha and E_L,alpha = -1/2 sum_i (lap_i g_alpha +
//                         2 grad_i g_alpha . grad_i ln|Psi|) for every Jastrow parameter alpha
// One warp per walker; the geometry tables of the walker live in shared memory.
#include "jastrow_body.cuh"

namespace vbq {

namespace {

template <class Tb>
__global__ void __launch_bounds__(256, JasBounds<Tb>::min_blocks)
    jastrow_kernel(const SysDev s, const JasLayout L, int W, const double* __restrict__ Rg, Tb* __restrict__ JG,
                   Tb* __restrict__ JL, double* __restrict__ JS) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  jastrow_body<Tb>(s, L, w, smem + wl * L.warp_bytes, Rg, JG, JL, JS);
}

// one block (L.nw warps) per walker, for systems whose per-walker tables leave few warps per SM
template <class Tb>
__global__ void __launch_bounds__(256, JasBounds<Tb>::min_blocks)
    jastrow_wide_kernel(const SysDev s, const JasLayout L, const double* __restrict__ Rg, Tb* __restrict__ JG,
                        Tb* __restrict__ JL, double* __restrict__ JS) {
  extern __shared__ __align__(16) unsigned char smem[];
  jastrow_body<Tb, true>(s, L, blockIdx.x, smem, Rg, JG, JL, JS);
}

template <class Tb>
__global__ void __launch_bounds__(256, JasBounds<Tb>::min_blocks)
    jastrow_batch_kernel(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items, int nitems) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    jastrow_body<Tb>(b.dev, b.lay.jas, item.first + wl, smem + wl * b.lay.jas.warp_bytes, b.R,
                     static_cast<Tb*>(b.JG), static_cast<Tb*>(b.JL), b.JS);
  }
}

template <class Tb>
__global__ void __launch_bounds__(256, JasBounds<Tb>::min_blocks)
    jastrow_deriv_kernel(const SysDev s, const JasLayout L, int W, const double* __restrict__ Rg,
                         const double* __restrict__ vgg, Tb* __restrict__ Og, Tb* __restrict__ dELg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  jastrow_deriv_body<Tb>(s, L, w, smem + wl * L.warp_bytes, Rg, vgg, Og, dELg);
}

template <class Tb>
__global__ void __launch_bounds__(256, JasBounds<Tb>::min_blocks)
    jastrow_deriv_batch_kernel(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items, int nitems) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    if (!b.O || !b.dev.jas_param) continue;
    jastrow_deriv_body<Tb>(b.dev, b.lay.jas, item.first + wl, smem + wl * b.lay.jas.warp_bytes, b.R, b.VG,
                           static_cast<Tb*>(b.O), static_cast<Tb*>(b.dEL));
  }
}

}  // namespace

int make_jas_layout(const SysDev& s, int tb, int max_smem, JasLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N;
  L.R = take(8 * 3 * N);
  L.vg = take(8 * 3 * N);
  L.red = take(8 * 2 * kNeen);
  L.geo = take(tb * geo_elems<float>(N, s.Nn));
  {
    int P = 1;
    while (P < N && P < 32) P <<= 1;
    L.jas_P = P;
    L.jas_S = 32 / P;
  }
  L.warp_bytes = off;
  int wpb = std::min(8, max_smem / off);
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  // few walkers per block: the Jastrow kernel runs one walker per block of eight warps that
  // share its tables (the derivative kernel keeps one warp per walker)
  L.nw = 1;
  if (wpb < 4) {
    const int nw = 8;
    L.wred = take(tb * 4 * L.jas_P * nw);
    L.wred2 = take(8 * 2 * nw);
    L.wide_bytes = off;
    if (off <= max_smem) L.nw = nw;
  }
  return VBQMC_OK;
}

template <class K>
static cudaError_t set_smem(K kernel, int smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class Tb>
cudaError_t launch_jastrow(const SysDev& s, const JasLayout& L, int W, const double* R, Tb* JG, Tb* JL, double* JS,
                           cudaStream_t st) {
  if (L.nw > 1) {
    cudaError_t e = set_smem(jastrow_wide_kernel<Tb>, L.wide_bytes);
    if (e != cudaSuccess) return e;
    jastrow_wide_kernel<Tb><<<W, 32 * L.nw, L.wide_bytes, st>>>(s, L, R, JG, JL, JS);
    return cudaGetLastError();
  }
  const int smem = L.wpb * L.warp_bytes;
  cudaError_t e = set_smem(jastrow_kernel<Tb>, smem);
  if (e != cudaSuccess) return e;
  jastrow_kernel<Tb><<<(W + L.wpb - 1) / L.wpb, 32 * L.wpb, smem, st>>>(s, L, W, R, JG, JL, JS);
  return cudaGetLastError();
}

template <class Tb>
cudaError_t launch_jastrow_deriv(const SysDev& s, const JasLayout& L, int W, const double* R, const double* vg, Tb* O,
                                 Tb* dEL, cudaStream_t st) {
  const int smem = L.wpb * L.warp_bytes;
  cudaError_t e = set_smem(jastrow_deriv_kernel<Tb>, smem);
  if (e != cudaSuccess) return e;
  jastrow_deriv_kernel<Tb><<<(W + L.wpb - 1) / L.wpb, 32 * L.wpb, smem, st>>>(s, L, W, R, vg, O, dEL);
  return cudaGetLastError();
}

template <class Tb>
cudaError_t launch_jastrow_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps, int smem,
                                 cudaStream_t st) {
  jastrow_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems);
  return cudaGetLastError();
}
template <class Tb>
cudaError_t launch_jastrow_deriv_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps,
                                       int smem, cudaStream_t st) {
  jastrow_deriv_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems);
  return cudaGetLastError();
}
int jastrow_batch_grid(int is_float, int deriv, int nitems, int warps, int smem, int persist) {
  const void* fn = deriv ? (is_float ? (const void*)jastrow_deriv_batch_kernel<float>
                                     : (const void*)jastrow_deriv_batch_kernel<double>)
                         : (is_float ? (const void*)jastrow_batch_kernel<float> : (const void*)jastrow_batch_kernel<double>);
  return batch_grid(fn, nitems, warps, smem, persist);
}
#define VBQ_INST(T)                                                                                                  \
  template cudaError_t launch_jastrow_batch<T>(const BatchSys*, const BatchItem*, int, int, int, int, cudaStream_t); \
  template cudaError_t launch_jastrow_deriv_batch<T>(const BatchSys*, const BatchItem*, int, int, int, int,         \
                                                     cudaStream_t);
VBQ_INST(float)
VBQ_INST(double)
#undef VBQ_INST

template cudaError_t launch_jastrow<float>(const SysDev&, const JasLayout&, int, const double*, float*, float*,
                                           double*, cudaStream_t);
template cudaError_t launch_jastrow<double>(const SysDev&, const JasLayout&, int, const double*, double*, double*,
                                            double*, cudaStream_t);
template cudaError_t launch_jastrow_deriv<float>(const SysDev&, const JasLayout&, int, const double*, const double*,
                                                 float*, float*, cudaStream_t);
template cudaError_t launch_jastrow_deriv<double>(const SysDev&, const JasLayout&, int, const double*, const double*,
                                                  double*, double*, cudaStream_t);

}  // namespace vbq
