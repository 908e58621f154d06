// VMC sweep kernel for sm_103a (arXiv:2207.14715, Sec. 2.3.1): one warp per walker, the
// walker's inverses and tables in shared memory.  (The evaluation kernels are in
// eval_jastrow.cu, eval_orbitals.cu and eval_det.cu.)
//
// Precision: template parameter Tb is the bulk type (proposal rows and Jastrow changes); the
// determinant ratios and Sherman-Morrison updates of the inverses are always double.
#include "sweep_body.cuh"

namespace vbq {

template <class Tb, bool TAB>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const SysDev s, const SweepLayout L, int W, double* __restrict__ Rg,
                                                    int nsweeps, int refresh, double* __restrict__ state, int state_valid,
                                                    double step, uint64_t seed, uint32_t step0, uint32_t tag,
                                                    uint32_t woff, int* __restrict__ nacc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  sweep_body<Tb, TAB>(s, L, w, smem + wl * L.warp_bytes, Rg, nsweeps, refresh, state, state_valid, step, seed, step0,
                      tag, woff, nacc);
}

// All systems of a batch: blocks loop over work items; warp wl takes walker first + wl.
template <class Tb>
__global__ void __launch_bounds__(512, 1) sweep_batch_kernel(const BatchSys* __restrict__ sys,
                                                          const BatchItem* __restrict__ items, int nitems,
                                                          const BatchCall* __restrict__ call) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    sweep_body<Tb, false>(b.dev, b.sweep, item.first + wl, smem + wl * b.sweep.warp_bytes, b.R, call->nsweeps,
                          call->refresh,
                   b.state, call->state_valid, call->step, call->seed, call->step0, b.tag, 0u, b.nacc);
  }
}

// =====================================================================================
// layouts and launchers
// =====================================================================================
int make_sweep_layout(const SysDev& s, int tb, int max_smem, SweepLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1];
  L.tab = s.msd ? 1 : 0;
  L.G0 = group_size(s.n[0]);
  L.G1 = group_size(s.n[1]);
  // a double instruction costs the same whatever the number of active lanes: the ratios take
  // the lane-group size with the fewest double instructions per move (passes over the
  // determinants times the products per lane plus the reduction levels)
  auto ratio_group = [](int n, int U, int G) {
    int best = G, bc = 1 << 30;
    for (int g = 1, lg = 0; g <= G; g <<= 1, ++lg) {
      const int per = 32 / g, c = ((U + per - 1) / per) * ((n + g - 1) / g + lg);
      if (c < bc) {
        bc = c;
        best = g;
      }
    }
    return best;
  };
  L.RG0 = ratio_group(s.n[0], s.U[0], L.G0);
  L.RG1 = ratio_group(s.n[1], s.U[1], L.G1);
  L.nocc_max = std::max(std::max(s.nocc[0], s.nocc[1]), 1);
  L.R = take(8 * 3 * N);
  L.Rds = take(tb == 4 ? 8 * 3 * N : 16);
  if (L.tab) {  // reference inverse and tables per spin, q_u of both spins, proposed q_u, c_x
    L.Binv0 = take(8 * s.n[0] * s.n[0]);
    L.Binv1 = take(8 * s.n[1] * s.n[1]);
    L.T0 = take(8 * std::max(s.n[0] * s.n_x[0], 1));
    L.T1 = take(8 * std::max(s.n[1] * s.n_x[1], 1));
    L.wk = take(8 * std::max(Ut, 1));
    L.qn = take(8 * std::max(std::max(s.U[0], s.U[1]), 1));
    L.cx = take(8 * std::max(std::max(s.n_x[0], s.n_x[1]), 1));
  } else {
    L.Binv0 = take(8 * s.U[0] * s.n[0] * s.n[0]);
    L.Binv1 = take(8 * s.U[1] * s.n[1] * s.n[1]);
    L.wk = take(8 * s.nterm);
  }
  // a refactorisation's ln|det|, signs and orbital matrix overlay the sweep's proposals and
  // the move-only geometry (the refactorisation runs before the proposals are formed, and its
  // outputs are consumed by the term ratios before the moves start)
  const int over0 = off;
  L.rtab = take(8 * 4 * N);
  L.rtds = take(tb == 4 ? 8 * 3 * N : 16);
  L.geom = take(tb * (2 * N + s.Nn + 6 * s.Nn + 10 * (N + 1)));
  const int moves_end = off;
  off = over0;
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.PhiO = take(8 * N * L.nocc_max);
  off = std::max(off, moves_end);
  int cv = 0, scr = 0;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], G = sp ? L.G1 : L.G0, ng = L.tab ? 1 : 32 / G;
    cv = std::max(cv, 8 * (L.tab ? 1 : 2) * ng * n);  // Sherman-Morrison stages two passes' columns
    scr = std::max(scr, ng * (8 * n * n + 4 * n) + 16);
  }
  // the LU scratch of a refactorisation shares its space with the buffers of the moves (the
  // basis values and partial sums that build PhiO are consumed before the LU starts)
  const int shared0 = off;
  L.bas = take(8 * s.M);
  L.vrow = take(8 * L.nocc_max);
  L.part = take(8 * std::max(std::max(s.n_occ_chunk[0], s.n_occ_chunk[1]), 1));
  L.rho = take(8 * std::max(s.U[0], s.U[1]));
  L.rinv = take(8 * (std::max(s.U[0], s.U[1]) + 1));
  L.cvec = take(std::max(cv, 8));
  L.scratch = shared0;
  off = std::max(off, align16(shared0 + std::max(scr, 16)));
  L.geo = take(tb * (N * s.Nn + (N + 1) * s.Nn));
  L.warp_bytes = off;
  int wpb = max_smem / off;
  if (wpb > 16) wpb = 16;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

template <class Tb>
static cudaError_t launch_sweep_t(const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps, int refresh,
                                  double* state, int state_valid, double step, uint64_t seed, uint32_t step0, uint32_t tag,
                                  uint32_t woff, int* nacc, cudaStream_t st) {
  // walkers per block: the most that fit, unless one or two fewer need no more waves of
  // blocks over the SMs (a wave costs about 3 % more per extra warp on the SM, measured on the
  // ethylene-shaped system; an idle part of the last wave costs its full share)
  SweepLayout Lw = L;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                               cudaSuccess && sms > 0 && W > 0) {
    auto cost = [&](int p) {
      const long waves = ((long)W + (long)p * sms - 1) / ((long)p * sms);
      return waves * (100 + 3 * p);
    };
    for (int p = L.wpb - 1; p >= std::max(1, L.wpb - 2); --p)
      if (cost(p) < cost(Lw.wpb)) Lw.wpb = p;
  }
  const int smem = Lw.wpb * Lw.warp_bytes;
  const void* fn = Lw.tab ? (const void*)sweep_kernel<Tb, true> : (const void*)sweep_kernel<Tb, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = (W + Lw.wpb - 1) / Lw.wpb;
  if (Lw.tab)
    sweep_kernel<Tb, true><<<blocks, 32 * Lw.wpb, smem, st>>>(s, Lw, W, R, nsweeps, refresh, nullptr, 0, step, seed,
                                                              step0, tag, woff, nacc);
  else
    sweep_kernel<Tb, false><<<blocks, 32 * Lw.wpb, smem, st>>>(s, Lw, W, R, nsweeps, refresh, state, state_valid, step,
                                                               seed, step0, tag, woff, nacc);
  return cudaGetLastError();
}

template <class Tb>
cudaError_t launch_sweep_batch(const BatchSys* sys, const BatchItem* items, int nitems, const BatchCall* call,
                               int grid, int warps, int smem, cudaStream_t st) {
  sweep_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems, call);
  return cudaGetLastError();
}
int batch_grid(const void* fn, int nitems, int warps, int smem, int persist) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return -1;
  if (persist <= 0) return nitems;
  int bps = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 32 * warps, smem) != cudaSuccess) return -1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1;
  const long long g = (long long)persist * std::max(bps, 1) * sms;
  return (int)std::max<long long>(1, std::min<long long>(g, nitems));
}
int sweep_batch_grid(int is_float, int nitems, int warps, int smem, int persist) {
  return batch_grid(is_float ? (const void*)sweep_batch_kernel<float> : (const void*)sweep_batch_kernel<double>, nitems,
                    warps, smem, persist);
}

template cudaError_t launch_sweep_batch<float>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                               cudaStream_t);
template cudaError_t launch_sweep_batch<double>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                                cudaStream_t);

cudaError_t launch_sweep(int precision, const SysDev& s, const SweepLayout& L, int W, double* R, int nsweeps,
                         int refresh, double* state, int state_valid, double step, uint64_t seed, uint32_t step0, uint32_t tag,
                         uint32_t woff, int* nacc, cudaStream_t st) {
  if (precision == VBQMC_MIXED)
    return launch_sweep_t<float>(s, L, W, R, nsweeps, refresh, state, state_valid, step, seed, step0, tag, woff, nacc,
                                 st);
  return launch_sweep_t<double>(s, L, W, R, nsweeps, refresh, state, state_valid, step, seed, step0, tag, woff, nacc,
                                st);
}

}  // namespace vbq
