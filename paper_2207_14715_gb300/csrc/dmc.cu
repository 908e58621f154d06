// Fixed-node diffusion Monte Carlo step (arXiv:2207.14715, Sec. 2.3.2, Eq. E0DMCweights).
//
// The paper runs the algorithm of Umrigar, Nightingale and Runge (J. Chem. Phys. 99, 2865
// (1993)) without printing it.  The step here is an all-electron drift-diffusion move with
// Metropolis acceptance that keeps that algorithm's two limits near the nodes, where the
// drift and E_L diverge:
//   vbar_i = v_i (-1 + sqrt(1 + 2 a |v_i|^2 tau)) / (a |v_i|^2 tau), a = 1, v_i = grad_i ln|Psi|;
//   R' = R + tau vbar(R) + sqrt(tau) z,   z ~ N(0, 1) per coordinate;
//   rejected when sign Psi(R') != sign Psi(R) (fixed node), else accepted with probability
//   min(1, Psi(R')^2 G(R <- R') / (Psi(R)^2 G(R' <- R))), G(R' <- R) = exp(-|R' - R - tau vbar(R)|^2 / 2 tau);
//   branching energy E_b = E_T + clamp((E_L - E_T) |Vbar| / |V|, -E_cut, E_cut) (whole-walker drift
//   vectors), E_cut = 0.2 sqrt(N / tau): the energy cutoff of Zen, Sorella, Gillan, Michaelides and
//   Alfe (Phys. Rev. B 93, 241118(R) (2016)), which keeps walkers at a huge |E_L| away from any
//   node from multiplying without bound;
//   weight w = exp(-tau [ (E_b(R) + E_b(R_new)) / 2 - E_T ]) with R_new the position kept;
//   copies = min(floor(w + u), 3), children stored in parent order (exclusive prefix sum);
//   E_T <- sum w E_b / sum w - (0.1 / tau) ln(population / target) after branching, E_b at the kept
//   positions (the energies that set the weights: the population settles at the target); the
//   reported estimator is sum w E_L / sum w with the raw E_L.
// Random numbers: Philox4x32-10 with counter (walker_offset + walker index in the current
// population, step, slot, (system << 8) | purpose): slot e < N, purposes 2 and 3 -> Box-Muller
// normals of electron e (purpose 2: z_x, z_y from the cosine and sine branches; purpose 3: z_z
// from the cosine branch); slot N, purpose 4 -> (u_acc, u_branch).
//
// Kernels per step: dmc_propose (thread per electron), the evaluation kernel at R' with the
// gradient, dmc_accept (warp per walker), dmc_scan (one block: prefix sum of the copies and
// the weight sums in a fixed order, so results do not depend on scheduling) and dmc_branch
// (warp per parent).
#include "dmc.h"
#include "wf_device.cuh"

namespace vbq {

namespace {

// Limiting factor of one electron's drift: vbar = f v with f = (-1 + sqrt(1 + 2x)) / x,
// x = |v|^2 tau (a = 1), written as 2 / (1 + sqrt(1 + 2x)) (no cancellation at small x).
__device__ __forceinline__ double drift_factor(double v2, double tau) {
  return 2.0 / (1.0 + sqrt(fma(2.0 * tau, v2, 1.0)));
}

__global__ void dmc_propose_kernel(int W, int N, const double* __restrict__ R, const double* __restrict__ grad,
                                   double tau, double sqtau, uint64_t seed, uint32_t step, uint32_t tag, uint32_t woff,
                                   double* __restrict__ Rp) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)W * N) return;
  const int w = (int)(t / N), e = (int)(t % N);
  double ua0, ua1, ub0, ub1;
  uniforms2(seed, woff + (uint32_t)w, step, (uint32_t)e, tag, 2, ua0, ua1);
  uniforms2(seed, woff + (uint32_t)w, step, (uint32_t)e, tag, 3, ub0, ub1);
  const double ra = sqrt(-2.0 * log(1.0 - ua0));
  const double rb = sqrt(-2.0 * log(1.0 - ub0));
  double sa, ca;
  sincospi(2.0 * ua1, &sa, &ca);
  const double z[3] = {ra * ca, ra * sa, rb * cospi(2.0 * ub1)};
  const size_t o = (size_t)t * 3;
  const double g0 = grad[o], g1 = grad[o + 1], g2 = grad[o + 2];
  const double f = drift_factor(g0 * g0 + g1 * g1 + g2 * g2, tau);
  const double g[3] = {g0, g1, g2};
#pragma unroll
  for (int d = 0; d < 3; ++d) Rp[o + d] = R[o + d] + tau * (f * g[d]) + sqtau * z[d];
}

// Acceptance, weight and copy count per walker; the accepted move is written into the carried
// walker (R, ln|Psi|, sign, E_L, grad) in place.
__global__ void dmc_accept_kernel(int W, int N, double* __restrict__ R, double* __restrict__ lp,
                                  double* __restrict__ sg, double* __restrict__ el, double* __restrict__ grad,
                                  const double* __restrict__ Rp, const double* __restrict__ lp1,
                                  const double* __restrict__ sg1, const double* __restrict__ el1,
                                  const double* __restrict__ grad1, double tau, double E_T, uint64_t seed,
                                  uint32_t step, uint32_t tag, uint32_t woff, double* __restrict__ wt,
                                  double* __restrict__ wE, double* __restrict__ wEb, int* __restrict__ copies,
                                  int* __restrict__ acc) {
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = lane_id();
  if (w >= W) return;
  const int n3 = 3 * N;
  const size_t base = (size_t)w * n3;
  // per electron: limited drifts at R and R', the Green's function exponents, and the squared
  // norms of the raw and limited whole-walker drifts at both points
  double f = 0.0, b = 0.0, n0 = 0.0, nb0 = 0.0, n1 = 0.0, nb1 = 0.0;
  for (int e = lane; e < N; e += 32) {
    const size_t o = base + 3 * (size_t)e;
    double g0[3], g1[3];
    double v0 = 0.0, v1 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      g0[d] = grad[o + d];
      g1[d] = grad1[o + d];
      v0 = fma(g0[d], g0[d], v0);
      v1 = fma(g1[d], g1[d], v1);
    }
    const double f0 = drift_factor(v0, tau), f1 = drift_factor(v1, tau);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double r = R[o + d], p = Rp[o + d];
      const double fq = p - r - tau * (f0 * g0[d]);
      const double bq = r - p - tau * (f1 * g1[d]);
      f = fma(fq, fq, f);
      b = fma(bq, bq, b);
    }
    n0 += v0;
    nb0 += f0 * f0 * v0;
    n1 += v1;
    nb1 += f1 * f1 * v1;
  }
  f = warp_sum(f);
  b = warp_sum(b);
  n0 = warp_sum(n0);
  nb0 = warp_sum(nb0);
  n1 = warp_sum(n1);
  nb1 = warp_sum(nb1);
  int accept = 0;
  if (lane == 0) {
    double uacc, ubr;
    uniforms2(seed, woff + (uint32_t)w, step, (uint32_t)N, tag, 4, uacc, ubr);
    const double s0 = sg[w], s1 = sg1[w];
    if (s1 == s0 && s1 != 0.0) {
      const double lnr = 2.0 * (lp1[w] - lp[w]) - b / (2.0 * tau) + f / (2.0 * tau);
      accept = uacc < exp(lnr);
    }
    const double e0 = el[w];
    const double en = accept ? el1[w] : e0;
    // branching energies limited in proportion to the drift, |Vbar| / |V| at each point
    const double q0 = n0 > 0.0 ? sqrt(nb0 / n0) : 1.0, q1 = n1 > 0.0 ? sqrt(nb1 / n1) : 1.0;
    const double ecut = 0.2 * sqrt((double)N / tau);
    const double eb0 = E_T + fmin(ecut, fmax(-ecut, (e0 - E_T) * q0));
    const double eb1 = E_T + fmin(ecut, fmax(-ecut, (en - E_T) * (accept ? q1 : q0)));
    const double ww = exp(-tau * (0.5 * (eb0 + eb1) - E_T));
    const double x = ww + ubr;
    const int c = (x >= 3.0) ? 3 : (x >= 0.0 ? (int)floor(x) : 0);  // NaN weights die
    wt[w] = ww;
    wE[w] = ww * en;
    wEb[w] = ww * eb1;
    copies[w] = c;
    acc[w] = accept;
    if (accept) {
      lp[w] = lp1[w];
      sg[w] = s1;
      el[w] = en;
    }
  }
  accept = __shfl_sync(kFull, accept, 0);
  if (accept)
    for (int q = lane; q < n3; q += 32) {
      R[base + q] = Rp[base + q];
      grad[base + q] = grad1[base + q];
    }
}

constexpr int kScanThreads = 1024;

// One block: exclusive prefix sum of the copies (children offsets), population after
// branching, and the weight sums, each thread summing a fixed stride of walkers, then a fixed
// reduction tree.
__global__ void __launch_bounds__(kScanThreads) dmc_scan_kernel(int W, const int* __restrict__ copies,
                                                                const double* __restrict__ wt,
                                                                const double* __restrict__ wE,
                                                                const double* __restrict__ wEb,
                                                                const int* __restrict__ acc,
                                                                int* __restrict__ offsets, DmcTotals* out) {
  __shared__ int wsum[32];
  __shared__ double rs[3][32];
  __shared__ int ra[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  long long running = 0;
  double sw = 0.0, swe = 0.0, sweb = 0.0;
  int na = 0;
  for (int base = 0; base < W; base += kScanThreads) {
    const int i = base + tid;
    const int c = i < W ? copies[i] : 0;
    if (i < W) {
      sw += wt[i];
      swe += wE[i];
      sweb += wEb[i];
      na += acc[i];
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
      }
      wsum[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const int warp_off = wid ? wsum[wid - 1] : 0;
    if (i < W) offsets[i] = (int)(running + warp_off + incl - c);
    running += wsum[31];
    __syncthreads();
  }
  sw = warp_sum(sw);
  swe = warp_sum(swe);
  sweb = warp_sum(sweb);
  na = warp_sum(na);
  if (lane == 0) {
    rs[0][wid] = sw;
    rs[1][wid] = swe;
    rs[2][wid] = sweb;
    ra[wid] = na;
  }
  __syncthreads();
  if (wid == 0) {
    double a = rs[0][lane], e = rs[1][lane], eb = rs[2][lane];
    int n = ra[lane];
    a = warp_sum(a);
    e = warp_sum(e);
    eb = warp_sum(eb);
    n = warp_sum(n);
    if (lane == 0) {
      out->total = running;
      out->sum_w = a;
      out->sum_wE = e;
      out->sum_wEb = eb;
      out->accepted = n;
    }
  }
}

// Children of each parent, in parent order, into the second buffer set (skipped when the new
// population would exceed the capacity; the host reports that).
__global__ void dmc_branch_kernel(int W, int N, int cap, const int* __restrict__ copies,
                                  const int* __restrict__ offsets, const DmcTotals* __restrict__ tot,
                                  const double* __restrict__ R, const double* __restrict__ lp,
                                  const double* __restrict__ sg, const double* __restrict__ el,
                                  const double* __restrict__ grad, double* __restrict__ Rb, double* __restrict__ lpb,
                                  double* __restrict__ sgb, double* __restrict__ elb, double* __restrict__ gradb) {
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = lane_id();
  if (w >= W || tot->total > cap) return;
  const int c = copies[w], o = offsets[w], n3 = 3 * N;
  for (int k = 0; k < c; ++k) {
    const size_t src = (size_t)w * n3, dst = (size_t)(o + k) * n3;
    for (int q = lane; q < n3; q += 32) {
      Rb[dst + q] = R[src + q];
      gradb[dst + q] = grad[src + q];
    }
    if (lane == 0) {
      lpb[o + k] = lp[w];
      sgb[o + k] = sg[w];
      elb[o + k] = el[w];
    }
  }
}

}  // namespace

cudaError_t launch_dmc_propose(int W, int N, const double* R, const double* grad, double tau, uint64_t seed,
                               uint32_t step, uint32_t tag, uint32_t woff, double* Rp, cudaStream_t st) {
  const long long n = (long long)W * N;
  dmc_propose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, N, R, grad, tau, sqrt(tau), seed, step, tag,
                                                                    woff, Rp);
  return cudaGetLastError();
}

cudaError_t launch_dmc_accept(int W, int N, double* R, double* lp, double* sg, double* el, double* grad,
                              const double* Rp, const double* lp1, const double* sg1, const double* el1,
                              const double* grad1, double tau, double E_T, uint64_t seed, uint32_t step, uint32_t tag,
                              uint32_t woff, double* wt, double* wE, double* wEb, int* copies, int* acc,
                              cudaStream_t st) {
  const long long threads = (long long)W * 32;
  dmc_accept_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(W, N, R, lp, sg, el, grad, Rp, lp1, sg1, el1,
                                                                        grad1, tau, E_T, seed, step, tag, woff, wt, wE,
                                                                        wEb, copies, acc);
  return cudaGetLastError();
}

cudaError_t launch_dmc_scan(int W, const int* copies, const double* wt, const double* wE, const double* wEb,
                            const int* acc, int* offsets, DmcTotals* out, cudaStream_t st) {
  dmc_scan_kernel<<<1, kScanThreads, 0, st>>>(W, copies, wt, wE, wEb, acc, offsets, out);
  return cudaGetLastError();
}

cudaError_t launch_dmc_branch(int W, int N, int cap, const int* copies, const int* offsets, const DmcTotals* tot,
                              const double* R, const double* lp, const double* sg, const double* el,
                              const double* grad, double* Rb, double* lpb, double* sgb, double* elb, double* gradb,
                              cudaStream_t st) {
  const long long threads = (long long)W * 32;
  dmc_branch_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(W, N, cap, copies, offsets, tot, R, lp, sg,
                                                                        el, grad, Rb, lpb, sgb, elb, gradb);
  return cudaGetLastError();
}

}  // namespace vbq
