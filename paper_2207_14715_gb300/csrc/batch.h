// Batched launches over several systems (uneven electron counts and walker populations):
// one launch per kernel type covers every system, through a table of work items.
#pragma once

#include "kernels.h"

namespace vbq {

// Work item: walkers first .. first + count - 1 of system sys (for the orbital kernel:
// (walker, electron) pairs in the same walker-major order).  One warp per walker (pair).
struct BatchItem {
  int sys, first, count, pad;
};

// Per-call scalars (device copy read by the kernels).
struct BatchCall {
  double step;
  uint64_t seed;
  uint32_t step0;
  int nsweeps, refresh, state_valid, derivs;
};

// Per-system tables, layouts, caller buffers and evaluation workspace (device copy).
struct BatchSys {
  SysDev dev;
  EvalLayout lay;
  SweepLayout sweep;
  int W;
  uint32_t tag;
  double* R;
  double* state;
  int* nacc;
  double* logpsi;
  double* sign;
  double* eloc;
  void* O;
  void* dEL;
  void* JG;
  void* JL;
  void* OB;
  double* JS;
  double* OD;
  double* VG;
  int cw[3];  // one-launch step: walkers run at once in the sweep, Jastrow and determinant phases
};

// Launchers: 'warps' warps per block, 'smem' dynamic shared memory, 'grid' blocks, each
// looping over items blockIdx.x, blockIdx.x + grid, ...
template <class Tb>
cudaError_t launch_sweep_batch(const BatchSys* sys, const BatchItem* items, int nitems, const BatchCall* call,
                               int grid, int warps, int smem, cudaStream_t st);
template <class Tb>
cudaError_t launch_jastrow_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps, int smem,
                                 cudaStream_t st);
template <class Tb>
cudaError_t launch_jastrow_deriv_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps,
                                       int smem, cudaStream_t st);
template <class Tb>
cudaError_t launch_orbitals_batch(const BatchSys* sys, const BatchItem* items, int nitems, int grid, int warps,
                                  int smem, cudaStream_t st);
template <class Tb>
cudaError_t launch_det_batch(const BatchSys* sys, const BatchItem* items, int nitems, const BatchCall* call, int grid,
                             int warps, int smem, cudaStream_t st);
// The whole step in one persistent launch (batch_fused.cu): blocks take items (system, tile of
// walkers) from the device counter *queue (zero before the launch) and run the sweep (if sweep),
// the evaluation kernels' bodies (if eval) and the Jastrow-parameter derivatives (if derivs) on
// each tile in turn.  Every item's count fits the block's warps; in the per-walker phases of
// system s, warps 0 .. s.cw[phase] - 1 take the tile's walkers in turn (cw[phase] regions of
// that phase fit the shared memory smem), and the orbital phase spreads the tile's (walker,
// electron) pairs over all warps.
cudaError_t launch_batch_fused(int is_float, const BatchSys* sys, const BatchItem* items, int nitems,
                               const BatchCall* call, int* queue, bool sweep, bool eval, bool derivs, int grid,
                               int warps, int smem, cudaStream_t st);
int batch_fused_grid(int is_float, int warps, int smem, int persist);
// Grid of each batched kernel for nitems items: one block per item (persist = 0), or
// persist x the blocks that fit on all SMs at once (persistent blocks looping over items);
// -1 on a CUDA error.  Also sets the kernel's dynamic shared-memory limit, so call these
// outside stream capture.
int batch_grid(const void* fn, int nitems, int warps, int smem, int persist);
int sweep_batch_grid(int is_float, int nitems, int warps, int smem, int persist);
int jastrow_batch_grid(int is_float, int deriv, int nitems, int warps, int smem, int persist);
int orbital_batch_grid(int is_float, int nitems, int warps, int smem, int persist);
int det_batch_grid(int is_float, int nitems, int warps, int smem, int persist);

}  // namespace vbq
