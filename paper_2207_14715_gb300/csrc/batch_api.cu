// Batched VMC steps over many loaded systems (C ABI in include/vbqmc.h).  A step is one
// persistent launch (batch_fused.cu) over a device queue of (system, walker tile) work items
// that runs every phase of the step on each tile; the launch (with the reset of the queue
// counter and the staging copies) is captured once per call shape in a CUDA graph and replayed.
// The tile shape (warps per block, walkers per tile) and the persistence of the grid are chosen
// by timing the candidates on the batch itself.  One launch per kernel type over per-kind
// work items remains as the alternative the tuner compares against.
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "batch.h"
#include "ctx_internal.h"

using vbq::BatchCall;
using vbq::BatchItem;
using vbq::BatchSys;

namespace {

constexpr int kKinds = 5;  // 0 sweep, 1 Jastrow, 2 Jastrow derivatives, 3 orbitals, 4 determinants
const char* const kKindName[kKinds] = {"sweep", "jastrow", "jastrow_deriv", "orbitals", "det"};
constexpr int kFused = kKinds;  // plan index of the one-launch step

struct KernelPlan {
  int persist = 1;  // 0: one block per item; k: k x the blocks resident at once
  int cap = 0;      // cap on walkers per block (0: none)
  int warps = 1, smem = 0, grid = 0, nitems = 0;
  BatchItem* d_items = nullptr;
};

}  // namespace

struct vbqmc_batch {
  vbqmc_ctx* ctx = nullptr;
  int precision = 0, n = 0;
  std::vector<int> ids, W;
  std::vector<BatchSys> sys;  // host template (tables, layouts, workspace pointers)
  KernelPlan plan[kKinds + 1];  // per kind, then the one-launch step
  bool fused = true;             // steps as one launch (else one launch per kind)
  bool tables = false;           // a system on reference-determinant tables: one-launch steps only
  int* d_queue = nullptr;        // work-queue counter of the one-launch step
  BatchSys* d_sys = nullptr;
  BatchCall* d_call = nullptr;
  BatchSys* h_sys = nullptr;  // pinned staging copied by the graph
  BatchCall* h_call = nullptr;
  void* ws = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[8] = {};
  cudaEvent_t staged = nullptr;  // the last graph launch has read the staging buffers
  bool tuned = false;
  float tune_ms[2] = {0.0f, 0.0f};  // evaluation per launch style at the tuned shapes
};

namespace {

int fail(int code, const std::string& msg) { return vbq::set_error(code, msg); }
int cuda_fail(cudaError_t e, const char* what) { return vbq::set_cuda_error((int)e, what); }

// per-walker cost estimate used to order the work items (largest first)
double walker_cost(const vbq::SysDev& s) {
  return (double)s.N * s.M * 5.0 + (double)s.N * s.N * s.Nn * 10.0 + (double)(s.U[0] + s.U[1]) * s.n[0] * s.n[0] * s.n[0];
}

void drop_graphs(vbqmc_batch* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Builds the work items and launch shape of one kernel kind from the systems' layouts.
int build_plan(vbqmc_batch* b, int kind) {
  KernelPlan& p = b->plan[kind];
  const bool f = b->precision == VBQMC_MIXED;
  auto wpb_of = [&](const BatchSys& s) {
    switch (kind) {
      case 0: return s.sweep.wpb;
      case 1:
      case 2: return s.lay.jas.wpb;
      case 3: return s.lay.orb.wpb;
      default: return s.lay.det.wpb;
    }
  };
  auto bytes_of = [&](const BatchSys& s) {
    switch (kind) {
      case 0: return s.sweep.warp_bytes;
      case 1:
      case 2: return s.lay.jas.warp_bytes;
      case 3: return s.lay.orb.warp_bytes;
      default: return s.lay.det.warp_bytes;
    }
  };
  int warps = 1, smem = 0;
  for (const auto& s : b->sys) {
    int w = wpb_of(s);
    if (p.cap > 0) w = std::max(1, std::min(w, p.cap));
    warps = std::max(warps, w);
    smem = std::max(smem, w * bytes_of(s));
  }
  struct It {
    BatchItem item;
    double cost;
  };
  std::vector<It> its;
  for (int k = 0; k < b->n; ++k) {
    const BatchSys& s = b->sys[k];
    // walkers per block for this system: as many as the block's warps and shared memory allow
    const int per = std::max(1, std::min(warps, smem / std::max(bytes_of(s), 1)));
    const long long units = (kind == 3) ? (long long)s.W * s.dev.N : s.W;
    const double c = walker_cost(s.dev);
    for (long long f0 = 0; f0 < units; f0 += per) {
      It t;
      t.item.sys = k;
      t.item.first = (int)f0;
      t.item.count = (int)std::min<long long>(per, units - f0);
      t.item.pad = 0;
      t.cost = c * t.item.count;
      its.push_back(t);
    }
  }
  std::stable_sort(its.begin(), its.end(), [](const It& a, const It& c) { return a.cost > c.cost; });
  std::vector<BatchItem> items(its.size());
  for (size_t i = 0; i < its.size(); ++i) items[i] = its[i].item;
  if (p.d_items) cudaFree(p.d_items);
  p.d_items = nullptr;
  cudaError_t e = cudaMalloc(&p.d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch items)");
  e = cudaMemcpy(p.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch items)");
  p.nitems = (int)items.size();
  p.warps = warps;
  p.smem = smem;
  int g = -1;
  switch (kind) {
    case 0: g = vbq::sweep_batch_grid(f, p.nitems, warps, smem, p.persist); break;
    case 1: g = vbq::jastrow_batch_grid(f, 0, p.nitems, warps, smem, p.persist); break;
    case 2: g = vbq::jastrow_batch_grid(f, 1, p.nitems, warps, smem, p.persist); break;
    case 3: g = vbq::orbital_batch_grid(f, p.nitems, warps, smem, p.persist); break;
    default: g = vbq::det_batch_grid(f, p.nitems, warps, smem, p.persist); break;
  }
  if (g < 0) return fail(VBQMC_ERR_CUDA, std::string("launch setup of the batched ") + kKindName[kind] + " kernel");
  p.grid = g;
  return VBQMC_OK;
}

// Work items and shape of the one-launch step: with p.warps warps per block, tiles of T = p.warps
// walkers (p.cap > 0: at most p.cap); one block per SM holds the opt-in shared memory, and in each
// per-walker phase of system s as many walkers run at once as that phase's per-walker regions
// fit it (cw, at most T); the orbital phase gives every warp its own region.
int build_fused_plan(vbqmc_batch* b) {
  KernelPlan& p = b->plan[kFused];
  const bool f = b->precision == VBQMC_MIXED;
  const int smax = b->ctx->max_smem;
  const int warps = std::max(1, std::min(p.warps, 16));
  const int T = p.cap > 0 ? std::max(1, std::min(warps, p.cap)) : warps;
  const int smem = smax - 128;  // the kernel's static shared memory (the item index) takes the rest
  std::vector<int> per(b->n);
  for (int k = 0; k < b->n; ++k) {
    BatchSys& s = b->sys[k];
    const int bytes[3] = {s.sweep.warp_bytes, s.lay.jas.warp_bytes,
                          s.dev.msd ? s.lay.tab.warp_bytes : s.lay.det.warp_bytes};
    for (int q = 0; q < 3; ++q) {
      if (bytes[q] > smem) return fail(VBQMC_ERR_CAPACITY, "per-walker region of a batched system");
      s.cw[q] = std::max(1, std::min(T, smem / std::max(bytes[q], 1)));
    }
    if (warps * s.lay.orb.warp_bytes > smem) return fail(VBQMC_ERR_CAPACITY, "orbital tables of a batched system");
    per[k] = T;
  }
  struct It {
    BatchItem item;
    double cost;
  };
  std::vector<It> its;
  for (int k = 0; k < b->n; ++k) {
    const double c = walker_cost(b->sys[k].dev);
    for (int f0 = 0; f0 < b->sys[k].W; f0 += per[k]) {
      It t;
      t.item = BatchItem{k, f0, std::min(per[k], b->sys[k].W - f0), 0};
      t.cost = c * t.item.count;
      its.push_back(t);
    }
  }
  std::stable_sort(its.begin(), its.end(), [](const It& a, const It& c) { return a.cost > c.cost; });
  std::vector<BatchItem> items(its.size());
  for (size_t i = 0; i < its.size(); ++i) items[i] = its[i].item;
  if (p.d_items) cudaFree(p.d_items);
  p.d_items = nullptr;
  cudaError_t e = cudaMalloc(&p.d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1));
  if (e == cudaSuccess) e = cudaMemcpy(p.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch items");
  p.nitems = (int)items.size();
  p.warps = warps;
  p.smem = smem;
  const int g = vbq::batch_fused_grid(f, warps, smem, std::max(p.persist, 1));
  if (g < 0) return fail(VBQMC_ERR_CUDA, "launch setup of the one-launch batched step");
  p.grid = std::min(g, std::max(p.nitems, 1));
  return VBQMC_OK;
}

cudaError_t launch_kind(vbqmc_batch* b, int kind, cudaStream_t st) {
  const KernelPlan& p = b->plan[kind];
  if (p.nitems == 0) return cudaSuccess;
  const bool f = b->precision == VBQMC_MIXED;
  switch (kind) {
    case 0:
      return f ? vbq::launch_sweep_batch<float>(b->d_sys, p.d_items, p.nitems, b->d_call, p.grid, p.warps, p.smem, st)
               : vbq::launch_sweep_batch<double>(b->d_sys, p.d_items, p.nitems, b->d_call, p.grid, p.warps, p.smem, st);
    case 1:
      return f ? vbq::launch_jastrow_batch<float>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st)
               : vbq::launch_jastrow_batch<double>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st);
    case 2:
      return f ? vbq::launch_jastrow_deriv_batch<float>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st)
               : vbq::launch_jastrow_deriv_batch<double>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st);
    case 3:
      return f ? vbq::launch_orbitals_batch<float>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st)
               : vbq::launch_orbitals_batch<double>(b->d_sys, p.d_items, p.nitems, p.grid, p.warps, p.smem, st);
    default:
      return f ? vbq::launch_det_batch<float>(b->d_sys, p.d_items, p.nitems, b->d_call, p.grid, p.warps, p.smem, st)
               : vbq::launch_det_batch<double>(b->d_sys, p.d_items, p.nitems, b->d_call, p.grid, p.warps, p.smem, st);
  }
}

cudaError_t launch_fused(vbqmc_batch* b, bool sweep, bool eval, bool derivs, cudaStream_t st) {
  const KernelPlan& p = b->plan[kFused];
  if (p.nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return vbq::launch_batch_fused(b->precision == VBQMC_MIXED, b->d_sys, p.d_items, p.nitems, b->d_call, b->d_queue,
                                 sweep, eval, derivs, p.grid, p.warps, p.smem, st);
}

// The launches of one call shape: staging copy, then the one-launch step or the sweep and/or
// evaluation kernels.
cudaError_t record_step(vbqmc_batch* b, bool sweep, bool eval, bool derivs, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(b->d_sys, b->h_sys, sizeof(BatchSys) * b->n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_call, b->h_call, sizeof(BatchCall), cudaMemcpyHostToDevice, st);
  if (b->fused) return e == cudaSuccess ? launch_fused(b, sweep, eval, derivs, st) : e;
  if (e == cudaSuccess && sweep) e = launch_kind(b, 0, st);
  if (e == cudaSuccess && eval) e = launch_kind(b, 1, st);
  if (e == cudaSuccess && eval) e = launch_kind(b, 3, st);
  if (e == cudaSuccess && eval) e = launch_kind(b, 4, st);
  if (e == cudaSuccess && derivs) e = launch_kind(b, 2, st);
  return e;
}

int launch_count(const vbqmc_batch* b, bool sweep, bool eval, bool derivs) {
  if (b->fused) return (sweep || eval) && b->plan[kFused].nitems ? 1 : 0;
  int n = 0;
  if (sweep && b->plan[0].nitems) ++n;
  if (eval) n += (b->plan[1].nitems ? 1 : 0) + (b->plan[3].nitems ? 1 : 0) + (b->plan[4].nitems ? 1 : 0);
  if (derivs && b->plan[2].nitems) ++n;
  return n;
}

// Fills the pinned staging buffers for one call (after the previous graph launch read them).
int stage_call(vbqmc_batch* b, double* const* R, int nsweeps, double step, uint64_t seed, uint32_t step0, int refresh,
               double* const* state, int state_valid, int* const* nacc, double* const* logpsi, double* const* sign,
               double* const* eloc, void* const* O, void* const* dEL) {
  cudaError_t e = cudaEventSynchronize(b->staged);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  for (int k = 0; k < b->n; ++k) {
    BatchSys s = b->sys[k];
    s.R = R[k];
    s.state = state ? state[k] : nullptr;
    s.nacc = nacc ? nacc[k] : nullptr;
    s.logpsi = logpsi ? logpsi[k] : nullptr;
    s.sign = sign ? sign[k] : nullptr;
    s.eloc = eloc ? eloc[k] : nullptr;
    s.O = O ? O[k] : nullptr;
    s.dEL = dEL ? dEL[k] : nullptr;
    b->h_sys[k] = s;
  }
  BatchCall c{};
  c.step = step;
  c.seed = seed;
  c.step0 = step0;
  c.nsweeps = nsweeps;
  c.refresh = refresh;
  c.state_valid = state_valid;
  c.derivs = O ? 1 : 0;
  *b->h_call = c;
  return VBQMC_OK;
}

void free_batch(vbqmc_batch* b) {
  drop_graphs(b);
  for (auto& p : b->plan)
    if (p.d_items) cudaFree(p.d_items);
  if (b->d_sys) cudaFree(b->d_sys);
  if (b->d_call) cudaFree(b->d_call);
  if (b->h_sys) cudaFreeHost(b->h_sys);
  if (b->h_call) cudaFreeHost(b->h_call);
  if (b->ws) cudaFree(b->ws);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->staged) cudaEventDestroy(b->staged);
  delete b;
}

}  // namespace

extern "C" {

int vbqmc_batch_create(vbqmc_ctx* ctx, int nsys, const int* sys_ids, const int* W, int precision, vbqmc_batch** out) {
  if (!ctx || !out || !sys_ids || !W) return fail(VBQMC_ERR_ARG, "null argument");
  *out = nullptr;
  if (nsys < 1) return fail(VBQMC_ERR_ARG, "need at least one system");
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return fail(VBQMC_ERR_ARG, "bad precision mode");
  for (int k = 0; k < nsys; ++k) {
    const int id = sys_ids[k];
    if (id < 0 || id >= VBQMC_MAX_SYSTEMS || !ctx->sys[id].loaded)
      return fail(VBQMC_ERR_NOSYS, "no system loaded under id " + std::to_string(id));
    if (W[k] < 1) return fail(VBQMC_ERR_ARG, "every system needs at least one walker");
    if (ctx->sys[id].lay_rc_eval[precision] || ctx->sys[id].lay_rc_sweep[precision])
      return fail(VBQMC_ERR_CAPACITY, "per-walker state of system " + std::to_string(id) + " exceeds shared memory");
    for (int q = 0; q < k; ++q)
      if (sys_ids[q] == id) return fail(VBQMC_ERR_ARG, "a system appears twice in the batch");
  }
  vbq::DeviceGuard g(ctx->device);
  vbqmc_batch* b = new vbqmc_batch();
  b->ctx = ctx;
  b->precision = precision;
  b->n = nsys;
  b->ids.assign(sys_ids, sys_ids + nsys);
  b->W.assign(W, W + nsys);
  const int tb = precision == VBQMC_MIXED ? 4 : 8;
  // evaluation workspace of every system, one allocation
  std::vector<size_t> off(nsys + 1, 0);
  for (int k = 0; k < nsys; ++k)
    off[k + 1] = off[k] + ((vbq::eval_workspace_bytes(ctx->sys[sys_ids[k]].dev, tb, W[k]) + 255) & ~size_t(255));
  cudaError_t e = cudaMalloc(&b->ws, std::max<size_t>(off[nsys], 256));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sys, sizeof(BatchSys) * nsys);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_call, sizeof(BatchCall));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_sys, sizeof(BatchSys) * nsys);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_call, sizeof(BatchCall));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "batch allocation");
  }
  b->sys.resize(nsys);
  for (int k = 0; k < nsys; ++k) {
    const vbq::LoadedSystem& L = ctx->sys[sys_ids[k]];
    BatchSys s{};
    s.dev = L.dev;
    s.lay = L.lay_eval[precision];
    s.sweep = L.lay_sweep[precision];
    s.W = W[k];
    s.tag = (uint32_t)sys_ids[k];
    // carve this system's evaluation workspace as the single-system evaluation does
    unsigned char* p = static_cast<unsigned char*>(b->ws) + off[k];
    auto take = [&](size_t bytes) {
      unsigned char* q = p;
      p += (bytes + 255) & ~size_t(255);
      return q;
    };
    const size_t N = L.dev.N, Wz = W[k];
    s.JG = take(Wz * 3 * N * tb);
    s.JL = take(Wz * N * tb);
    s.JS = reinterpret_cast<double*>(take(Wz * 2 * 8));
    s.OB = take(Wz * N * 5 * L.dev.n_ev * tb);
    s.OD = reinterpret_cast<double*>(take(Wz * N * std::max(L.dev.n_ev_det, 1) * 8));
    s.VG = reinterpret_cast<double*>(take(Wz * 3 * N * 8));
    b->sys[k] = s;
  }
  for (int k = 0; k < nsys; ++k) b->tables = b->tables || ctx->sys[sys_ids[k]].dev.msd;
  for (int kind = 0; kind < kKinds && !b->tables; ++kind) {  // the per-kind kernels have no table forms
    const int rc = build_plan(b, kind);
    if (rc) {
      free_batch(b);
      return rc;
    }
  }
  b->plan[kFused].warps = 16;
  const int rcf = build_fused_plan(b);
  if (rcf) {
    free_batch(b);
    return rcf;
  }
  *out = b;
  return VBQMC_OK;
}

void vbqmc_batch_destroy(vbqmc_batch* b) {
  if (!b) return;
  vbq::DeviceGuard g(b->ctx->device);
  cudaDeviceSynchronize();
  free_batch(b);
}

int vbqmc_batch_vmc_steps(vbqmc_batch* b, double* const* R, int nsweeps, double step, uint64_t seed, uint32_t step0,
                          int refresh, double* const* state, int state_valid, int* const* nacc, double* const* logpsi,
                          double* const* sign, double* const* eloc, void* const* O, void* const* dEL, void* stream) {
  if (!b || !R) return fail(VBQMC_ERR_ARG, "null batch or positions");
  if (nsweeps < 0 || !(step > 0.0) || refresh < 0) return fail(VBQMC_ERR_ARG, "bad sweep count, step or refresh");
  if (state_valid && !state) return fail(VBQMC_ERR_ARG, "state_valid without state");
  const bool eval = logpsi || sign || eloc || O || dEL;
  if (eval && (!logpsi || !sign || !eloc)) return fail(VBQMC_ERR_ARG, "evaluation needs logpsi, sign and eloc");
  if (dEL && !O) return fail(VBQMC_ERR_ARG, "dEL requires O");
  for (int k = 0; k < b->n; ++k) {
    if (!R[k]) return fail(VBQMC_ERR_ARG, "null positions of a system");
    if (eval && (!logpsi[k] || !sign[k] || !eloc[k])) return fail(VBQMC_ERR_ARG, "null evaluation output");
    if (state_valid && !state[k]) return fail(VBQMC_ERR_ARG, "null state of a system");
  }
  vbq::DeviceGuard g(b->ctx->device);
  int rc = stage_call(b, R, nsweeps, step, seed, step0, refresh, state, state_valid, nacc, logpsi, sign, eloc, O, dEL);
  if (rc) return rc;
  const bool sweep = nsweeps > 0, derivs = O != nullptr;
  const int key = (sweep ? 1 : 0) | (eval ? 2 : 0) | (derivs ? 4 : 0);
  cudaError_t e = cudaSuccess;
  if (!b->graph[key]) {
    cudaGraph_t gr = nullptr;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const cudaError_t er = record_step(b, sweep, eval, derivs, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &gr);
    if (er != cudaSuccess || e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return cuda_fail(er != cudaSuccess ? er : e, "capturing the batched step");
    }
    e = cudaGraphInstantiate(&b->graph[key], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      b->graph[key] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  e = cudaGraphLaunch(b->graph[key], (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->staged, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batched step launch");
  b->ctx->last_launches = launch_count(b, sweep, eval, derivs);
  return VBQMC_OK;
}

// The per-phase walker counts of a new one-launch plan into the staged and device copies of the
// system table (the tuner launches from the copy staged at its start), after the previous
// launches have read it.
static cudaError_t refresh_walker_counts(vbqmc_batch* b, cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < b->n; ++k)
    for (int q = 0; q < 3; ++q) b->h_sys[k].cw[q] = b->sys[k].cw[q];
  return cudaMemcpyAsync(b->d_sys, b->h_sys, sizeof(BatchSys) * b->n, cudaMemcpyHostToDevice, st);
}

int vbqmc_batch_tune(vbqmc_batch* b, double* const* R, double* const* logpsi, double* const* sign, double* const* eloc,
                     void* stream) {
  if (!b || !R || !logpsi || !sign || !eloc) return fail(VBQMC_ERR_ARG, "null argument");
  vbq::DeviceGuard g(b->ctx->device);
  const cudaStream_t st = (cudaStream_t)stream;
  int rc = stage_call(b, R, 0, 1.0, 0, 0, 0, nullptr, 0, nullptr, logpsi, sign, eloc, nullptr, nullptr);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  e = cudaMemcpyAsync(b->d_sys, b->h_sys, sizeof(BatchSys) * b->n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_call, b->h_call, sizeof(BatchCall), cudaMemcpyHostToDevice, st);
  // evaluation kernels in order (each reads what the previous one wrote); for each, try
  // one-block-per-item and persistent grids with and without a cap on walkers per block
  const int kinds[3] = {1, 3, 4};
  for (int kk = 0; kk < 3 && e == cudaSuccess && rc == VBQMC_OK && !b->tables; ++kk) {
    const int kind = kinds[kk];
    KernelPlan& p = b->plan[kind];
    int best_persist = p.persist, best_cap = p.cap;
    float best = 1e30f;
    const int full = p.warps;
    const int caps[2] = {0, std::max(1, full / 2)};
    const int persists[3] = {0, 1, 2};
    for (int ci = 0; ci < 2 && rc == VBQMC_OK; ++ci)
      for (int pi = 0; pi < 3 && rc == VBQMC_OK; ++pi) {
        if (ci == 1 && caps[1] == full) continue;
        p.cap = caps[ci];
        p.persist = persists[pi];
        rc = build_plan(b, kind);
        if (rc) break;
        e = launch_kind(b, kind, st);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_kind(b, kind, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms < best) {
          best = ms;
          best_persist = p.persist;
          best_cap = p.cap;
        }
      }
    p.persist = best_persist;
    p.cap = best_cap;
    if (rc == VBQMC_OK && e == cudaSuccess) rc = build_plan(b, kind);
  }
  // the sweep and the Jastrow derivatives follow the determinant kernel's grid choice
  if (rc == VBQMC_OK && e == cudaSuccess && !b->tables) {
    b->plan[0].persist = b->plan[2].persist = b->plan[4].persist;
    rc = build_plan(b, 0);
    if (rc == VBQMC_OK) rc = build_plan(b, 2);
  }
  // the per-kind evaluation at its best shapes, then the one-launch step over tile shapes
  // (warps per block, walkers per tile) and grid persistence
  float best_kinds = 1e30f;
  if (rc == VBQMC_OK && e == cudaSuccess && !b->tables) {
    b->fused = false;
    auto run = [&]() {
      cudaError_t r = cudaSuccess;
      for (int kind : {1, 3, 4})
        if (r == cudaSuccess) r = launch_kind(b, kind, st);
      return r;
    };
    e = run();
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&best_kinds, e0, e1);
  }
  float best_fused = 1e30f;
  if (rc == VBQMC_OK && e == cudaSuccess) {
    KernelPlan& p = b->plan[kFused];
    int bw = p.warps, bc = p.cap, bp = p.persist;
    for (int warps : {8, 12, 16})
      for (int cap : {0})
        for (int persist : {1}) {
          if (rc != VBQMC_OK || e != cudaSuccess) break;
          p.warps = warps;
          p.cap = cap;
          p.persist = persist;
          rc = build_fused_plan(b);
          if (rc) break;
          e = refresh_walker_counts(b, st);
          if (e == cudaSuccess) e = launch_fused(b, false, true, false, st);
          if (e == cudaSuccess) e = cudaEventRecord(e0, st);
          for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_fused(b, false, true, false, st);
          if (e == cudaSuccess) e = cudaEventRecord(e1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e == cudaSuccess && ms < best_fused) {
            best_fused = ms;
            bw = warps;
            bc = cap;
            bp = persist;
          }
        }
    p.warps = bw;
    p.cap = bc;
    p.persist = bp;
    if (rc == VBQMC_OK && e == cudaSuccess) rc = build_fused_plan(b);
    if (rc == VBQMC_OK && e == cudaSuccess) e = refresh_walker_counts(b, st);
    b->fused = best_fused <= best_kinds;
  }
  b->tune_ms[0] = best_kinds / 3.0f;
  b->tune_ms[1] = best_fused / 3.0f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "batch tuning");
  if (rc) return rc;
  drop_graphs(b);
  b->tuned = true;
  return cudaEventRecord(b->staged, st) == cudaSuccess ? VBQMC_OK : fail(VBQMC_ERR_CUDA, "cudaEventRecord");
}

int vbqmc_batch_info(vbqmc_batch* b, int* out) {
  if (!b || !out) return fail(VBQMC_ERR_ARG, "null argument");
  for (int k = 0; k <= kKinds; ++k) {
    out[5 * k] = b->plan[k].nitems;
    out[5 * k + 1] = b->plan[k].grid;
    out[5 * k + 2] = b->plan[k].warps;
    out[5 * k + 3] = b->plan[k].persist;
    out[5 * k + 4] = b->plan[k].cap;
  }
  out[5 * (kKinds + 1)] = b->fused ? 1 : 0;
  out[5 * (kKinds + 1) + 1] = (int)(1000.0f * b->tune_ms[0]);
  out[5 * (kKinds + 1) + 2] = (int)(1000.0f * b->tune_ms[1]);
  return VBQMC_OK;
}

}  // extern "C"
