// Per-(walker, electron) body of the orbital kernel (arXiv:2207.14715, Sec. 2.1, orbital
// expansion): basis functions and orbital values, gradients and Laplacians; shared by the
// single-system, batched and fused batch kernels.
#pragma once

#include "batch.h"
#include "walker_common.cuh"

namespace vbq {

namespace {

constexpr int kOrbWarps = 8;

// Chunks c = lane, lane + 32, ... of the contraction with groups of WD orbitals (coefficients
// interleaved, stride WD): partial sums of phi, grad phi and lap phi over the chunk's basis
// functions into part[(5 t + k) nch + c].  Basis layout as written by orbital_body.
template <class Tb, int WD>
__device__ __forceinline__ void contract_groups(const SysDev& s, int lane, int nch, const Tb* __restrict__ cq,
                                                const Tb* bv, Tb* part) {
  const int M = s.M;
  for (int c = lane; c < nch; c += 32) {
    const int4 ch = __ldg(reinterpret_cast<const int4*>(s.evq_chunk) + c);
    Tb a[WD][5];
#pragma unroll
    for (int t = 0; t < WD; ++t)
#pragma unroll
      for (int k = 0; k < 5; ++k) a[t][k] = (Tb)0;
    for (int mu = ch.y; mu < ch.z; ++mu) {
      Tb cm[WD], b[5];
      if constexpr (WD == 4 && kSameType<Tb, double>) {
        const double2 c01 = __ldg(reinterpret_cast<const double2*>(cq + ch.w + 4 * mu));
        const double2 c23 = __ldg(reinterpret_cast<const double2*>(cq + ch.w + 4 * mu) + 1);
        cm[0] = c01.x; cm[1] = c01.y; cm[2] = c23.x; cm[3] = c23.y;
      } else if constexpr (WD == 4) {
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(cq + ch.w + 4 * mu));
        cm[0] = c4.x; cm[1] = c4.y; cm[2] = c4.z; cm[3] = c4.w;
      } else {
        cm[0] = __ldg(cq + ch.w + mu);
      }
      if constexpr (kSameType<Tb, double>) {
        b[0] = bv[mu]; b[1] = bv[M + mu]; b[2] = bv[2 * M + mu]; b[3] = bv[3 * M + mu]; b[4] = bv[4 * M + mu];
      } else {
        const float4 b4 = reinterpret_cast<const float4*>(bv)[mu];
        b[0] = b4.x; b[1] = b4.y; b[2] = b4.z; b[3] = b4.w;
        b[4] = reinterpret_cast<const float*>(bv)[4 * M + mu];
      }
#pragma unroll
      for (int t = 0; t < WD; ++t)
#pragma unroll
        for (int k = 0; k < 5; ++k) a[t][k] += cm[t] * b[k];
    }
#pragma unroll
    for (int t = 0; t < WD; ++t)
#pragma unroll
      for (int k = 0; k < 5; ++k) part[(5 * t + k) * nch + c] = a[t][k];
  }
}

// One warp, (walker, electron) pair gw (walker gw / N, electron gw % N).
template <class Tb>
__device__ __forceinline__ void orbital_body(const SysDev& s, const OrbLayout& L, long long gw, unsigned char* base,
                                             const double* Rg, Tb* __restrict__ OB,
                                             double* __restrict__ OD) {
  const int lane = threadIdx.x & 31;
  const int nev = s.n_ev, nevd = s.n_ev_det, M = s.M;
  Tb* bv = reinterpret_cast<Tb*>(base + L.bas);
  Tb* bx = bv + M;
  Tb* by = bx + M;
  Tb* bz = by + M;
  Tb* bl = bz + M;
  dsf* bds = reinterpret_cast<dsf*>(base + L.bds);
  dsf* ctab = reinterpret_cast<dsf*>(base + L.ctab);
  Tb* part = reinterpret_cast<Tb*>(base + L.part);
  dsf* partds = reinterpret_cast<dsf*>(base + L.partd);
  const double* r = Rg + (size_t)gw * 3;
  const Tb* cf = orb_coefs<Tb>(s);
  if constexpr (kSameType<Tb, double>) {
    basis_at<double, true>(s, lane, r[0], r[1], r[2], bv, bx, by, bz, bl);
  } else {
    // float form: value and gradient of a basis function interleaved as one float4 (one
    // shared-memory load per function and coefficient), Laplacians after them
    // lane d < 3 converts coordinate d (the conversion runs on the double pipe), then a broadcast
    const dsf rl = lane < 3 ? ds_from_double(r[lane]) : dsf{0.0f, 0.0f};
    dsf r3[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) r3[d] = dsf{__shfl_sync(kFull, rl.hi, d), __shfl_sync(kFull, rl.lo, d)};
    basis_at_f<true, true>(s, lane, r3, bv, nullptr, nullptr, nullptr, bv + 4 * M);
    if (OD) basis_values_ds(s, lane, r3, ctab, bds);
  }
  __syncwarp();
  // contraction by groups of orbitals sharing a coefficient range (quads: one basis-function
  // load feeds four orbitals); partials component-major, part[(5 t + k) nch + chunk]
  const int nch = s.n_evq_chunk;
  const Tb* cq = kSameType<Tb, double> ? reinterpret_cast<const Tb*>(s.evq_coef)
                                       : reinterpret_cast<const Tb*>(s.evq_coef_f);
  if (s.evq_width == 4)
    contract_groups<Tb, 4>(s, lane, nch, cq, bv, part);
  else
    contract_groups<Tb, 1>(s, lane, nch, cq, bv, part);
  if (!kSameType<Tb, double> && OD)
    for (int c = lane; c < s.n_det_chunk; c += 32) {
      const int4 ch = __ldg(reinterpret_cast<const int4*>(s.det_chunk) + c);
      const float2* cb = reinterpret_cast<const float2*>(s.orb_coef_ds) + ch.w;
      dsf acc = {0.0f, 0.0f};
      for (int mu = ch.y; mu < ch.z; ++mu) {
        const float2 lm = __ldg(cb + mu);
        acc = ds_add(acc, ds_mul(dsf{lm.x, lm.y}, bds[mu]));
      }
      partds[c] = acc;
    }
  __syncwarp();
  Tb* out = OB + (size_t)gw * 5 * nev;
  for (int q = lane; q < nev; q += 32) {
    const int qs = __ldg(s.evq_slot + q), qd = qs >> 2;
    const int c0 = __ldg(s.evq_chunk_off + qd), c1 = __ldg(s.evq_chunk_off + qd + 1);
    const Tb* pp = part + 5 * (qs & 3) * nch;
    Tb v = 0, gx = 0, gy = 0, gz = 0, lp = 0;
    for (int c = c0; c < c1; ++c) {
      v += pp[c]; gx += pp[nch + c]; gy += pp[2 * nch + c]; gz += pp[3 * nch + c]; lp += pp[4 * nch + c];
    }
    if (q < nevd && OD) {  // OD null: the determinant-orbital values in double are not needed
      double vd = 0.0;
      if (kSameType<Tb, double>) {
        vd = (double)v;
      } else {
        const int d0 = __ldg(s.det_chunk_off + q), d1 = __ldg(s.det_chunk_off + q + 1);
        dsf acc = {0.0f, 0.0f};
        for (int c = d0; c < d1; ++c) acc = ds_add(acc, partds[c]);
        vd = ds_to_double(acc);
      }
      OD[(size_t)gw * nevd + q] = vd;
      v = (Tb)vd;
    }
    out[q] = v;
    out[nev + q] = gx;
    out[2 * nev + q] = gy;
    out[3 * nev + q] = gz;
    out[4 * nev + q] = lp;
  }
}

}  // namespace

}  // namespace vbq
