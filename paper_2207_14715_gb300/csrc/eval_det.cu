// Determinant part of the evaluation and the evaluation driver (arXiv:2207.14715, Sec. 2.1,
// Sec. 2.2, Sec. 2.3.1).  One warp per walker:
//   C  Slater LU + inverses of every unique determinant (double), structure sum in the log
//      domain, E_L and grad ln|Psi|; optionally the walker state (inverses, ln|det|, signs)
//   D1 structure-coefficient derivatives; D3 orbital-excitation derivatives
// from the Jastrow and orbital results in the evaluation workspace.  The inverses are kept in
// shared memory in the bulk type only (the double inverses go straight to the walker state).

#include "det_body.cuh"

namespace vbq {

namespace {
template <class Tb>
__global__ void __launch_bounds__(EvalBounds<Tb>::threads, 1)
    det_kernel(const SysDev s, const DetLayout L, int W, const Tb* __restrict__ JG, const Tb* __restrict__ JL,
               const double* __restrict__ JS, const Tb* __restrict__ OB, const double* __restrict__ OD,
               double* __restrict__ logpsi, double* __restrict__ sgn_out, double* __restrict__ eloc,
               double* __restrict__ vg_ws, double* __restrict__ grad, Tb* __restrict__ Og, Tb* __restrict__ dELg,
               double* __restrict__ state_out, double* __restrict__ aux, const double* __restrict__ carry) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  det_body<Tb>(s, L, w, smem + wl * L.warp_bytes, JG, JL, JS, OB, OD, logpsi, sgn_out, eloc, vg_ws, grad, Og, dELg,
               state_out, aux, carry);
}

template <class Tb>
__global__ void __launch_bounds__(EvalBounds<Tb>::threads, 1)
    det_batch_kernel(const BatchSys* __restrict__ sys, const BatchItem* __restrict__ items, int nitems,
                     const BatchCall* __restrict__ call) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the warps' shared-memory regions depend on the item's system: start together
    __syncthreads();
    const BatchItem item = items[it];
    if (wl >= item.count) continue;
    const BatchSys& b = sys[item.sys];
    const bool d = call->derivs && b.O && b.dev.P > 0;
    det_body<Tb>(b.dev, b.lay.det, item.first + wl, smem + wl * b.lay.det.warp_bytes, static_cast<const Tb*>(b.JG),
                 static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD, b.logpsi, b.sign, b.eloc, b.VG,
                 nullptr, d ? static_cast<Tb*>(b.O) : nullptr, d ? static_cast<Tb*>(b.dEL) : nullptr, b.state,
                 nullptr, nullptr);
  }
}

}  // namespace

int make_det_layout(const SysDev& s, int tb, int max_smem, DetLayout& L, bool carried) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1];
  L.G0 = group_size(s.n[0]);
  L.G1 = group_size(s.n[1]);
  L.vg = take(8 * 3 * N);
  L.G = take(tb * 3 * N);
  L.LJ = take(tb * N);
  L.PhiD = take(8 * N * std::max(s.n_ev_det, 1));
  L.Lphi = take(tb * N * s.n_ev);
  L.Gphi = take(tb * N * s.n_ev_det * 3);
  L.Bt0 = take(tb * s.U[0] * s.n[0] * s.n[0]);
  L.Bt1 = take(tb * s.U[1] * s.n[1] * s.n[1]);
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.tdet = take(8 * Ut);
  L.Wdet = take(8 * Ut);
  L.Tdet = take(8 * Ut);
  L.rk = take(8 * s.nterm);
  int scr = 16;
  for (int sp = 0; sp < 2; ++sp) {
    const int n = s.n[sp], G = sp ? L.G1 : L.G0, ng = 32 / G;
    if (!carried) scr = std::max(scr, ng * (16 * n * n + 4 * n) + 16);  // LU: A, inverse, pivots per group
    scr = std::max(scr, 8 * s.U[sp] * n);                  // carried state: trace partials
  }
  // Gam and Aux rows of both spins, one product B_u L_u
  scr = std::max(scr, tb * (2 * std::max(s.n_ev_det, 1) * N + std::max(s.n[0] * s.n[0], s.n[1] * s.n[1])));
  L.scratch = take(scr);
  L.warp_bytes = off;
  int wpb = max_smem / off;
  const int cap = (tb == 8 ? EvalBounds<double>::threads : EvalBounds<float>::threads) / 32;
  if (wpb > cap) wpb = cap;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

namespace {
inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

EvalWs carve_eval_ws(const SysDev& s, int tb, int W, void* ws) {
  const size_t N = s.N, Wz = W;
  unsigned char* p = static_cast<unsigned char*>(ws);
  EvalWs r;
  auto take = [&](size_t b) {
    unsigned char* q = p;
    p += al256(b);
    return q;
  };
  r.JG = take(Wz * 3 * N * tb);
  r.JL = take(Wz * N * tb);
  r.JS = reinterpret_cast<double*>(take(Wz * 2 * 8));
  r.OB = take(Wz * N * 5 * s.n_ev * tb);
  r.OD = reinterpret_cast<double*>(take(Wz * N * std::max(s.n_ev_det, 1) * 8));
  r.VG = reinterpret_cast<double*>(take(Wz * 3 * N * 8));
  return r;
}

namespace {

template <class Tb>
cudaError_t launch_eval_t(const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi, double* sign,
                          double* eloc, double* grad, Tb* O, Tb* dEL, double* state_out, void* ws, cudaStream_t st,
                          int* nlaunch, cudaEvent_t* ev, double* aux, const double* carry) {
  const EvalWs b = carve_eval_ws(s, (int)sizeof(Tb), W, ws);
  *nlaunch = 0;
  auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], st) : cudaSuccess; };
  cudaError_t e = mark(0);
  if (e != cudaSuccess) return e;
  e = launch_jastrow<Tb>(s, L.jas, W, R, static_cast<Tb*>(b.JG), static_cast<Tb*>(b.JL), b.JS, st);
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(1)) != cudaSuccess) return e;
  e = launch_orbitals<Tb>(s, L.orb, W, R, static_cast<Tb*>(b.OB), carry ? nullptr : b.OD, st);
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(2)) != cudaSuccess) return e;
  if (s.msd) {
    e = launch_dettab<Tb>(s, L.tab, W, static_cast<const Tb*>(b.JG), static_cast<const Tb*>(b.JL), b.JS,
                          static_cast<const Tb*>(b.OB), b.OD, logpsi, sign, eloc, b.VG, grad, O, dEL, st);
  } else {
    const DetLayout& D = carry ? L.detc : L.det;
    const int smem = D.wpb * D.warp_bytes;
    e = cudaFuncSetAttribute(det_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    det_kernel<Tb><<<(W + D.wpb - 1) / D.wpb, 32 * D.wpb, smem, st>>>(
        s, D, W, static_cast<const Tb*>(b.JG), static_cast<const Tb*>(b.JL), b.JS, static_cast<const Tb*>(b.OB), b.OD,
        logpsi, sign, eloc, b.VG, grad, O, dEL, carry ? nullptr : state_out, aux, carry);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if ((e = mark(3)) != cudaSuccess) return e;
  if (O && s.jas_param) {
    e = launch_jastrow_deriv<Tb>(s, L.jas, W, R, b.VG, O, dEL, st);
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return mark(4);
}

}  // namespace

template <class Tb>
cudaError_t launch_det_batch(const BatchSys* sys, const BatchItem* items, int nitems, const BatchCall* call, int grid,
                             int warps, int smem, cudaStream_t st) {
  det_batch_kernel<Tb><<<grid, 32 * warps, smem, st>>>(sys, items, nitems, call);
  return cudaGetLastError();
}
int det_batch_grid(int is_float, int nitems, int warps, int smem, int persist) {
  return batch_grid(is_float ? (const void*)det_batch_kernel<float> : (const void*)det_batch_kernel<double>, nitems,
                    warps, smem, persist);
}
template cudaError_t launch_det_batch<float>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_det_batch<double>(const BatchSys*, const BatchItem*, int, const BatchCall*, int, int, int,
                                              cudaStream_t);

int make_eval_layout(const SysDev& s, int tb, int max_smem, EvalLayout& L) {
  int rc = make_jas_layout(s, tb, max_smem, L.jas);
  if (rc == VBQMC_OK) rc = make_orb_layout(s, tb, max_smem, L.orb);
  if (rc == VBQMC_OK)
    rc = s.msd ? make_dettab_layout(s, tb, max_smem, L.tab) : make_det_layout(s, tb, max_smem, L.det);
  if (rc == VBQMC_OK && !s.msd) rc = make_det_layout(s, tb, max_smem, L.detc, true);
  return rc;
}

size_t eval_workspace_bytes(const SysDev& s, int tb, int W) {
  const size_t N = s.N, Wz = std::max(W, 1);
  return al256(Wz * 3 * N * tb) + al256(Wz * N * tb) + al256(Wz * 2 * 8) + al256(Wz * N * 5 * s.n_ev * tb) +
         al256(Wz * N * std::max(s.n_ev_det, 1) * 8) + al256(Wz * 3 * N * 8);
}

cudaError_t launch_eval(int precision, const SysDev& s, const EvalLayout& L, int W, const double* R, double* logpsi,
                        double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out, void* ws,
                        cudaStream_t st, int* nlaunch, cudaEvent_t* ev, double* aux, const double* carry) {
  if (precision == VBQMC_MIXED)
    return launch_eval_t<float>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<float*>(O),
                                static_cast<float*>(dEL), state_out, ws, st, nlaunch, ev, aux, carry);
  return launch_eval_t<double>(s, L, W, R, logpsi, sign, eloc, grad, static_cast<double*>(O),
                               static_cast<double*>(dEL), state_out, ws, st, nlaunch, ev, aux, carry);
}

}  // namespace vbq
