// Determinant part of the evaluation through a reference determinant and tables
// (arXiv:2207.14715, Sec. 2.1: every determinant of a spin shares the inactive orbitals and
// differs from the others by a few active columns), for systems whose per-determinant
// inverses do not fit in shared memory.  One warp per walker.  Per spin:
//   A_0 = reference determinant (u = 0), B = A_0^-1 by the lane-group LU (double);
//   T = B Phi_X, Yhat = B L_X - (B L_0) T   over the orbitals X outside the reference;
//   determinant u replaces the reference slots S_u by the orbitals Q_u (k_u <= 4):
//     D_u = sgn_u D_0 det M_u,   M_u = T[S_u, Q_u]                (k x k, pivoted elimination)
//     t_u = tr(A_u^-1 L_u) = tr(B L_0) + tr(M_u^-1 Yhat[S_u, Q_u])
//     grad_i ln D_u = sum_o B[o][i] grad phi_o(r_i) + tr(M_u^-1 B[S_u][i] c_i[Q_u]),
//     c_i[x] = grad phi_x(r_i) - sum_o grad phi_{ref o}(r_i) T[o][x],
// where L is the Jastrow-dressed Laplacian lap phi + 2 grad ln J . grad phi.  The weighted sum
// over determinants of the gradient term goes through Gamma[x][o] = sum_u W_u (M_u^-1)[x][o].
// The structure sum, E_L and the structure-coefficient derivatives follow the direct kernel.
#include "dettab_body.cuh"

namespace vbq {

namespace {
template <class Tb>
__global__ void __launch_bounds__(256, 1)
    dettab_kernel(const SysDev s, const DetTabLayout L, int W, const Tb* __restrict__ JG, const Tb* __restrict__ JL,
                  const double* __restrict__ JS, const Tb* __restrict__ OB, const double* __restrict__ OD,
                  double* __restrict__ logpsi, double* __restrict__ sgn_out, double* __restrict__ eloc,
                  double* __restrict__ vg_ws, double* __restrict__ grad, Tb* __restrict__ Og, Tb* __restrict__ dELg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * L.wpb + wl;
  if (w >= W) return;
  dettab_body<Tb>(s, L, w, smem + wl * L.warp_bytes, JG, JL, JS, OB, OD, logpsi, sgn_out, eloc, vg_ws, grad, Og,
                  dELg);
}

}  // namespace

int make_dettab_layout(const SysDev& s, int tb, int max_smem, DetTabLayout& L) {
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off = align16(off + bytes);
    return o;
  };
  const int N = s.N, Ut = s.U[0] + s.U[1], nevd = std::max(s.n_ev_det, 1);
  const int nmax = std::max(std::max(s.n[0], s.n[1]), 1);
  const int nxmax = std::max(std::max(s.n_x[0], s.n_x[1]), 1);
  L.vg = take(8 * 3 * N);
  L.G = take(tb * 3 * N);
  L.B0 = take(8 * std::max(s.n[0] * s.n[0], 1));
  L.B1 = take(8 * std::max(s.n[1] * s.n[1], 1));
  L.T0 = take(8 * std::max(s.n[0] * s.n_x[0], 1));
  L.T1 = take(8 * std::max(s.n[1] * s.n_x[1], 1));
  L.Y0 = take(8 * std::max(s.n[0] * s.n_x[0], 1));
  L.Y1 = take(8 * std::max(s.n[1] * s.n_x[1], 1));
  L.A = take(8 * std::max(nmax * nmax, nxmax * nmax));
  L.Bs = take(8 * nxmax * nmax);
  L.perm = take(4 * nmax);
  L.Ls = take(8 * nmax * nevd);
  L.ldet = take(8 * Ut);
  L.dsg = take(8 * Ut);
  L.tdet = take(8 * Ut);
  L.Wdet = take(8 * Ut);
  L.rk = take(8 * std::max(s.nterm, 1));
  L.Minv = take(8 * std::max(s.tab_ksq, 1));  // the k_u x k_u minor inverses, packed
  L.Gam = take(8 * nxmax * nmax);
  L.warp_bytes = off;
  int wpb = max_smem / off;
  if (wpb > 8) wpb = 8;
  if (wpb < 1) return VBQMC_ERR_CAPACITY;
  L.wpb = wpb;
  return VBQMC_OK;
}

template <class Tb>
cudaError_t launch_dettab(const SysDev& s, const DetTabLayout& L, int W, const Tb* JG, const Tb* JL, const double* JS,
                          const Tb* OB, const double* OD, double* logpsi, double* sign, double* eloc, double* vg_ws,
                          double* grad, Tb* O, Tb* dEL, cudaStream_t st) {
  const int smem = L.wpb * L.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(dettab_kernel<Tb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dettab_kernel<Tb><<<(W + L.wpb - 1) / L.wpb, 32 * L.wpb, smem, st>>>(s, L, W, JG, JL, JS, OB, OD, logpsi, sign, eloc,
                                                                      vg_ws, grad, O, dEL);
  return cudaGetLastError();
}
template cudaError_t launch_dettab<float>(const SysDev&, const DetTabLayout&, int, const float*, const float*,
                                          const double*, const float*, const double*, double*, double*, double*,
                                          double*, double*, float*, float*, cudaStream_t);
template cudaError_t launch_dettab<double>(const SysDev&, const DetTabLayout&, int, const double*, const double*,
                                           const double*, const double*, const double*, double*, double*, double*,
                                           double*, double*, double*, double*, cudaStream_t);

}  // namespace vbq
