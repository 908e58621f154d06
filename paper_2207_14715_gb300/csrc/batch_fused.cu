// One persistent launch per batched step (many small systems of uneven size): each block takes
// work items (system, tile of walkers) from a device queue and runs every phase of the walker
// step on its tile in turn (Sec. 2.3.1: sweep of single-electron Metropolis moves, then the
// evaluation of ln|Psi|, E_L and the parameter derivatives), with block barriers between the
// phases: the VMC sweep (warp per walker), the Jastrow factor (warp per walker), the orbitals
// (warps over the tile's (walker, electron) pairs), the determinant part (warp per walker) and
// the Jastrow-parameter derivatives (warp per walker); systems on reference-determinant tables
// take the table forms of the sweep and of the determinant part.  The phases exchange their results
// through the systems' evaluation workspaces in global memory, written and read by the same
// block.  Items are ordered by estimated cost (largest first) so that the queue ends with
// small items.
#include "det_body.cuh"
#include "dettab_body.cuh"
#include "jastrow_body.cuh"
#include "orbital_body.cuh"
#include "sweep_body.cuh"

namespace vbq {

namespace {

// MAXT: the block size the registers are allocated for (256: up to 255 registers per thread,
// 384: 168, 512: 128).
template <class Tb, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) batch_fused_kernel(const BatchSys* __restrict__ sys,
                                                          const BatchItem* __restrict__ items, int nitems,
                                                          const BatchCall* __restrict__ call, int* __restrict__ queue,
                                                          int sweep, int eval, int derivs) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const int wl = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned dsmem;  // this launch's dynamic shared memory: no warp's region may pass its end
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
  auto fit = [&](int c, int bytes) { return min(c, (int)(dsmem / (unsigned)max(bytes, 1))); };
  for (;;) {
    __syncthreads();  // every warp is done with the previous item's shared memory
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const BatchItem item = items[it];
    const BatchSys& b = sys[item.sys];
    // per-walker phases: warp wl < c takes walkers wl, wl + c, ... of the tile
    const int cs = fit(b.cw[0], b.sweep.warp_bytes), cj = fit(b.cw[1], b.lay.jas.warp_bytes),
              cd = fit(b.cw[2], b.dev.msd ? b.lay.tab.warp_bytes : b.lay.det.warp_bytes),
              co = fit(nw, b.lay.orb.warp_bytes);
    // systems on reference-determinant tables (many determinants per structure) carry the
    // reference inverse and tables through their moves and keep no walker state
    if (sweep && wl < cs)
      for (int r = wl; r < item.count; r += cs) {
        const int w = item.first + r;
        if (b.dev.msd)
          sweep_body<Tb, true>(b.dev, b.sweep, w, smem + wl * b.sweep.warp_bytes, b.R, call->nsweeps, call->refresh,
                               nullptr, 0, call->step, call->seed, call->step0, b.tag, 0u, b.nacc);
        else
          sweep_body<Tb, false>(b.dev, b.sweep, w, smem + wl * b.sweep.warp_bytes, b.R, call->nsweeps,
                                call->refresh, b.state, call->state_valid, call->step, call->seed, call->step0, b.tag,
                                0u, b.nacc);
      }
    if (!eval) continue;
    __syncthreads();
    if (wl < cj)
      for (int r = wl; r < item.count; r += cj)
        jastrow_body<Tb>(b.dev, b.lay.jas, item.first + r, smem + wl * b.lay.jas.warp_bytes, b.R,
                         static_cast<Tb*>(b.JG), static_cast<Tb*>(b.JL), b.JS);
    __syncthreads();
    const int npair = item.count * b.dev.N;
    if (wl < co)
      for (int p = wl; p < npair; p += co)
        orbital_body<Tb>(b.dev, b.lay.orb, (long long)item.first * b.dev.N + p, smem + wl * b.lay.orb.warp_bytes,
                         b.R, static_cast<Tb*>(b.OB), b.OD);
    __syncthreads();
    const bool d = derivs && b.O && b.dev.P > 0;
    if (wl < cd)
      for (int r = wl; r < item.count; r += cd) {
        const int w = item.first + r;
        if (b.dev.msd)
          dettab_body<Tb>(b.dev, b.lay.tab, w, smem + wl * b.lay.tab.warp_bytes, static_cast<const Tb*>(b.JG),
                          static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD, b.logpsi, b.sign,
                          b.eloc, b.VG, nullptr, d ? static_cast<Tb*>(b.O) : nullptr,
                          d ? static_cast<Tb*>(b.dEL) : nullptr);
        else
          det_body<Tb>(b.dev, b.lay.det, w, smem + wl * b.lay.det.warp_bytes, static_cast<const Tb*>(b.JG),
                       static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD, b.logpsi, b.sign,
                       b.eloc, b.VG, nullptr, d ? static_cast<Tb*>(b.O) : nullptr,
                       d ? static_cast<Tb*>(b.dEL) : nullptr, b.state, nullptr, nullptr);
      }
    if (d && b.dev.jas_param) {
      __syncthreads();
      if (wl < cj)
        for (int r = wl; r < item.count; r += cj)
          jastrow_deriv_body<Tb>(b.dev, b.lay.jas, item.first + r, smem + wl * b.lay.jas.warp_bytes, b.R, b.VG,
                                 static_cast<Tb*>(b.O), static_cast<Tb*>(b.dEL));
    }
  }
}

}  // namespace

cudaError_t launch_batch_fused(int is_float, const BatchSys* sys, const BatchItem* items, int nitems,
                               const BatchCall* call, int* queue, bool sweep, bool eval, bool derivs, int grid,
                               int warps, int smem, cudaStream_t st) {
#define VBQ_FUSED(T, MT) \
  batch_fused_kernel<T, MT><<<grid, 32 * warps, smem, st>>>(sys, items, nitems, call, queue, sweep, eval, derivs)
  if (warps <= 8) {
    if (is_float) VBQ_FUSED(float, 256);
    else VBQ_FUSED(double, 256);
  } else if (warps <= 12) {
    if (is_float) VBQ_FUSED(float, 384);
    else VBQ_FUSED(double, 384);
  } else {
    if (is_float) VBQ_FUSED(float, 512);
    else VBQ_FUSED(double, 512);
  }
#undef VBQ_FUSED
  return cudaGetLastError();
}

int batch_fused_grid(int is_float, int warps, int smem, int persist) {
  const void* fn = warps <= 8    ? (is_float ? (const void*)batch_fused_kernel<float, 256>
                                             : (const void*)batch_fused_kernel<double, 256>)
                   : warps <= 12 ? (is_float ? (const void*)batch_fused_kernel<float, 384>
                                             : (const void*)batch_fused_kernel<double, 384>)
                                 : (is_float ? (const void*)batch_fused_kernel<float, 512>
                                             : (const void*)batch_fused_kernel<double, 512>);
  return batch_grid(fn, 1 << 30, warps, smem, persist);
}

}  // namespace vbq
