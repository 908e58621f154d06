// C ABI of the VB-QMC library (declared in include/vbqmc.h): context, system upload and
// the walker entry points.
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <cmath>

#include "dmc.h"
#include "kernels.h"
#include "linmethod.h"
#include "ctx_internal.h"
#include "vbqmc_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return VBQMC_ERR_CUDA;
}

// Packs host arrays into one 16-byte-aligned blob and records where each one went.
struct BlobBuilder {
  std::vector<unsigned char> bytes;
  template <class T> size_t add(const std::vector<T>& v) {
    size_t off = (bytes.size() + 15) & ~size_t(15);
    bytes.resize(off + std::max<size_t>(v.size() * sizeof(T), 16), 0);
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

}  // namespace

using vbq::DeviceGuard;
using vbq::LoadedSystem;

namespace vbq {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
int set_cuda_error(int cuda_error, const char* what) { return cuda_fail((cudaError_t)cuda_error, what); }
}  // namespace vbq

static void make_layouts(const vbqmc_ctx* ctx, LoadedSystem& ls) {
  for (int p = 0; p < 2; ++p) {
    const int tb = p == VBQMC_MIXED ? 4 : 8;
    ls.lay_rc_eval[p] = vbq::make_eval_layout(ls.dev, tb, ctx->max_smem, ls.lay_eval[p]);
    ls.lay_rc_sweep[p] = vbq::make_sweep_layout(ls.dev, tb, ctx->max_smem, ls.lay_sweep[p]);
    ls.lay_rc_force[p] = vbq::make_force_layout(ls.dev, tb, ctx->max_smem, ls.lay_force[p]);
  }
}

static void free_system(LoadedSystem& s) {
  if (s.blob) cudaFree(s.blob);
  s = LoadedSystem();
}

extern "C" {

const char* vbqmc_last_error(void) { return g_err.c_str(); }

int vbqmc_create(vbqmc_ctx** out, int device) {
  if (!out) return fail(VBQMC_ERR_ARG, "null output handle");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(VBQMC_ERR_ARG, "device index out of range");
  DeviceGuard g(device);
  if (!g.ok) return fail(VBQMC_ERR_CUDA, "cudaSetDevice failed");
  int smem = 0;
  e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  vbqmc_ctx* c = new vbqmc_ctx();
  c->device = device;
  c->max_smem = smem;
  *out = c;
  return VBQMC_OK;
}

void vbqmc_destroy(vbqmc_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto& s : ctx->sys) free_system(s);
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->dmc_work) cudaFree(ctx->dmc_work);
  if (ctx->eval_work) cudaFree(ctx->eval_work);
  if (ctx->force_work) cudaFree(ctx->force_work);
  if (ctx->red_work) cudaFree(ctx->red_work);
  for (auto& ev : ctx->tev)
    if (ev) cudaEventDestroy(ev);
  delete ctx;
}

int vbqmc_inspect_system(const vbqmc_system_desc* desc, int* info, int* terms, int max_terms, double* een_B) {
  vbq::SysHost h;
  std::string err;
  int rc = vbq::build_system(desc, h, err);
  if (rc) return fail(rc, err);
  if (info) {
    int ent = (int)((h.kap_ent[0].size() + h.kap_ent[1].size()) / 4);
    int v[12] = {h.N, h.P, h.M, h.Norb, (int)h.term_coef.size(), h.U[0], h.U[1], (int)h.sterm_d.size(),
                 (int)h.ev_orb.size(), ent, h.Nup, h.Ndn};
    std::memcpy(info, v, sizeof(v));
  }
  if (terms) {
    const int row = h.Nup + h.Ndn + 2;
    const int nst = (int)h.sterm_d.size();
    for (int t = 0; t < nst && t < max_terms; ++t) {
      const int k = h.sterm_k[t];
      const int a = h.term_det[2 * k], b = h.term_det[2 * k + 1];
      int* r = terms + (size_t)t * row;
      for (int o = 0; o < h.Nup; ++o) r[o] = h.det_glob[0][a * h.Nup + o];
      for (int o = 0; o < h.Ndn; ++o) r[h.Nup + o] = h.det_glob[1][b * h.Ndn + o];
      r[h.Nup + h.Ndn] = h.sterm_I[t];
      r[h.Nup + h.Ndn + 1] = (int)h.sterm_d[t];
    }
  }
  if (een_B) std::memcpy(een_B, h.een_B.data(), h.een_B.size() * sizeof(double));
  return VBQMC_OK;
}

int vbqmc_set_system(vbqmc_ctx* ctx, int sys_id, const vbqmc_system_desc* desc) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  if (sys_id < 0 || sys_id >= VBQMC_MAX_SYSTEMS) return fail(VBQMC_ERR_ARG, "sys_id out of range");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(VBQMC_ERR_CUDA, "cudaSetDevice failed");
  LoadedSystem ls;
  std::string err;
  int rc = vbq::build_system(desc, ls.host, err);
  if (rc) return fail(rc, err);
  const vbq::SysHost& h = ls.host;
  BlobBuilder bb;
  std::vector<float> coef_f(h.orb_coef.begin(), h.orb_coef.end());
  std::vector<float> evq_f(h.evq_coef.begin(), h.evq_coef.end());
  std::vector<int> sh_pack;
  for (int sh : h.sh_by_l) {
    const float z = (float)h.sh_zeta[sh];
    int zb;
    std::memcpy(&zb, &z, sizeof(zb));
    sh_pack.insert(sh_pack.end(), {h.sh_center[sh] | (h.sh_l[sh] << 16), h.sh_first[sh], sh, zb});
  }
  std::vector<float> een_cf(h.een_c.begin(), h.een_c.end());
  auto split = [](const std::vector<double>& v) {
    std::vector<float> o(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float hi = (float)v[i];
      o[2 * i] = hi;
      o[2 * i + 1] = (float)(v[i] - (double)hi);
    }
    return o;
  };
  const std::vector<float> zeta_ds = split(h.sh_zeta), norm_ds = split(h.sh_norm), coef_ds = split(h.orb_coef);
  std::vector<double> nuc_xyz;
  for (size_t a = 0; a < h.nuc4.size() / 4; ++a)
    for (int d = 0; d < 3; ++d) nuc_xyz.push_back(h.nuc4[4 * a + d]);
  const std::vector<float> nuc_ds = split(nuc_xyz);
  std::vector<float> nuc_zf;
  for (size_t a = 0; a < h.nuc4.size() / 4; ++a) nuc_zf.push_back((float)h.nuc4[4 * a + 3]);
  const std::vector<float> zeta_f(h.sh_zeta.begin(), h.sh_zeta.end()), norm_f(h.sh_norm.begin(), h.sh_norm.end()),
      jas_af(h.jas_a.begin(), h.jas_a.end()), jas_bf(h.jas_b.begin(), h.jas_b.end()),
      een_Bf(h.een_B.begin(), h.een_B.end());
  const size_t o_nuc4 = bb.add(h.nuc4), o_nuc_elem = bb.add(h.nuc_elem), o_sh_center = bb.add(h.sh_center),
               o_sh_l = bb.add(h.sh_l), o_sh_first = bb.add(h.sh_first), o_sh_zeta = bb.add(h.sh_zeta),
               o_sh_norm = bb.add(h.sh_norm), o_orb_lo = bb.add(h.orb_lo), o_orb_hi = bb.add(h.orb_hi),
               o_orb_off = bb.add(h.orb_off), o_orb_coef = bb.add(h.orb_coef), o_orb_coef_f = bb.add(coef_f),
               o_ev_orb = bb.add(h.ev_orb), o_occ0 = bb.add(h.occ_list[0]), o_occ1 = bb.add(h.occ_list[1]),
               o_dl0 = bb.add(h.det_loc[0]), o_dl1 = bb.add(h.det_loc[1]), o_de0 = bb.add(h.det_ev[0]),
               o_de1 = bb.add(h.det_ev[1]), o_term_det = bb.add(h.term_det), o_term_coef = bb.add(h.term_coef),
               o_sI = bb.add(h.sterm_I), o_sk = bb.add(h.sterm_k), o_sd = bb.add(h.sterm_d), o_dto = bb.add(h.det_term_off), o_dt = bb.add(h.det_term),
               o_cpo = bb.add(h.cpar_off), o_cps = bb.add(h.cpar_st),
               o_cparam = bb.add(h.cparam), o_jas_a = bb.add(h.jas_a), o_jas_b = bb.add(h.jas_b),
               o_een_c = bb.add(h.een_c), o_een_cf = bb.add(een_cf), o_een_B = bb.add(h.een_B),
               o_kx = bb.add(h.kap_x), o_oc0 = bb.add(h.occ_chunk[0]), o_oc1 = bb.add(h.occ_chunk[1]),
               o_oco0 = bb.add(h.occ_chunk_off[0]), o_oco1 = bb.add(h.occ_chunk_off[1]), o_evc = bb.add(h.evq_chunk),
               o_evco = bb.add(h.evq_chunk_off), o_evs = bb.add(h.evq_slot), o_evq = bb.add(h.evq_coef),
               o_evqf = bb.add(evq_f), o_dc = bb.add(h.det_chunk), o_dco = bb.add(h.det_chunk_off),
               o_zds = bb.add(zeta_ds), o_nds = bb.add(norm_ds), o_cds = bb.add(coef_ds), o_nucds = bb.add(nuc_ds),
               o_zf = bb.add(zeta_f), o_nf = bb.add(norm_f), o_jaf = bb.add(jas_af), o_jbf = bb.add(jas_bf),
               o_ebf = bb.add(een_Bf), o_nzf = bb.add(nuc_zf), o_nsh = bb.add(h.nuc_sh), o_sbl = bb.add(h.sh_by_l), o_shp = bb.add(sh_pack),
               o_jads = bb.add(split(h.jas_a)), o_jbds = bb.add(split(h.jas_b)), o_ecds = bb.add(split(h.een_c)), o_tx0 = bb.add(h.tab_x[0]),
               o_tx1 = bb.add(h.tab_x[1]), o_td0 = bb.add(h.tab_det[0]), o_td1 = bb.add(h.tab_det[1]),
               o_txl0 = bb.add(h.tab_xl[0]), o_txl1 = bb.add(h.tab_xl[1]);
  cudaError_t e = cudaMalloc(&ls.blob, bb.bytes.size());
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(system tables)");
  ls.blob_bytes = bb.bytes.size();
  e = cudaMemcpy(ls.blob, bb.bytes.data(), bb.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(ls.blob);
    return cuda_fail(e, "cudaMemcpy(system tables)");
  }
  const unsigned char* B = static_cast<const unsigned char*>(ls.blob);
  vbq::SysDev& d = ls.dev;
  d.N = h.N; d.Nup = h.Nup; d.Ndn = h.Ndn; d.Nn = h.Nn; d.n_elem = h.n_elem; d.S = h.S; d.M = h.M;
  d.Norb = h.Norb; d.Nvb = h.Nvb;
  d.n_ev = (int)h.ev_orb.size(); d.n_ev_det = h.n_ev_det;
  for (int sp = 0; sp < 2; ++sp) {
    d.nocc[sp] = (int)h.occ_list[sp].size();
    d.U[sp] = h.U[sp];
    d.n[sp] = h.n[sp];
  }
  d.nterm = (int)h.term_coef.size();
  d.nsterm = (int)h.sterm_d.size();
  d.P = h.P; d.n_cparam = (int)h.cparam.size(); d.jas_param = h.jas_param; d.een_on = h.een_on;
  d.n_kappa = h.n_kappa;
  d.p_off_a = d.n_cparam;
  d.p_off_b = d.p_off_a + (h.jas_param ? 5 * h.n_elem : 0);
  d.p_off_theta = d.p_off_b + (h.jas_param ? 5 : 0);
  d.p_off_kappa = d.p_off_theta + (h.jas_param && h.een_on ? vbq::kNfree * h.n_elem : 0);
  d.kappa = h.kappa; d.b1_anti = h.b1_anti; d.b1_par = h.b1_par; d.vnn = h.vnn;
  d.nuc4 = (const double*)(B + o_nuc4);
  d.nuc_elem = (const int*)(B + o_nuc_elem);
  d.sh_center = (const int*)(B + o_sh_center);
  d.sh_l = (const int*)(B + o_sh_l);
  d.sh_first = (const int*)(B + o_sh_first);
  d.nuc_sh = (const int*)(B + o_nsh);
  d.sh_by_l = (const int*)(B + o_sbl);
  d.sh_pack_f = (const int*)(B + o_shp);
  d.max_nuc_mu = h.max_nuc_mu;
  d.sh_zeta = (const double*)(B + o_sh_zeta);
  d.sh_norm = (const double*)(B + o_sh_norm);
  d.orb_lo = (const int*)(B + o_orb_lo);
  d.orb_hi = (const int*)(B + o_orb_hi);
  d.orb_off = (const int*)(B + o_orb_off);
  d.orb_coef = (const double*)(B + o_orb_coef);
  d.orb_coef_f = (const float*)(B + o_orb_coef_f);
  d.ev_orb = (const int*)(B + o_ev_orb);
  d.occ_list[0] = (const int*)(B + o_occ0);
  d.occ_list[1] = (const int*)(B + o_occ1);
  d.det_loc[0] = (const int*)(B + o_dl0);
  d.det_loc[1] = (const int*)(B + o_dl1);
  d.det_ev[0] = (const int*)(B + o_de0);
  d.det_ev[1] = (const int*)(B + o_de1);
  d.tab_x[0] = (const int*)(B + o_tx0);
  d.tab_x[1] = (const int*)(B + o_tx1);
  d.tab_det[0] = (const int*)(B + o_td0);
  d.tab_det[1] = (const int*)(B + o_td1);
  d.tab_ksq = 0;
  for (int sp = 0; sp < 2; ++sp)
    for (size_t u = 0; u * vbq::kTabStride < h.tab_det[sp].size(); ++u) {
      const int k = h.tab_det[sp][u * vbq::kTabStride];
      d.tab_ksq += k * k;
    }
  d.tab_xl[0] = (const int*)(B + o_txl0);
  d.tab_xl[1] = (const int*)(B + o_txl1);
  d.n_x[0] = (int)h.tab_x[0].size();
  d.n_x[1] = (int)h.tab_x[1].size();
  d.term_det = (const int*)(B + o_term_det);
  d.term_coef = (const double*)(B + o_term_coef);
  d.sterm_I = (const int*)(B + o_sI);
  d.sterm_k = (const int*)(B + o_sk);
  d.sterm_d = (const double*)(B + o_sd);
  d.det_term_off = (const int*)(B + o_dto);
  d.det_term = (const int*)(B + o_dt);
  d.cpar_off = (const int*)(B + o_cpo);
  d.cpar_st = (const int*)(B + o_cps);
  d.cparam = (const int*)(B + o_cparam);
  d.jas_a = (const double*)(B + o_jas_a);
  d.jas_b = (const double*)(B + o_jas_b);
  d.een_c = (const double*)(B + o_een_c);
  d.een_cf = (const float*)(B + o_een_cf);
  d.een_B = (const double*)(B + o_een_B);
  d.kap_x = (const int*)(B + o_kx);
  for (int sp = 0; sp < 2; ++sp) d.n_occ_chunk[sp] = (int)(h.occ_chunk[sp].size() / 4);
  d.n_evq_chunk = (int)(h.evq_chunk.size() / 4);
  d.evq_width = h.evq_width;
  d.n_det_chunk = (int)(h.det_chunk.size() / 4);
  d.occ_chunk[0] = (const int*)(B + o_oc0);
  d.occ_chunk[1] = (const int*)(B + o_oc1);
  d.occ_chunk_off[0] = (const int*)(B + o_oco0);
  d.occ_chunk_off[1] = (const int*)(B + o_oco1);
  d.evq_chunk = (const int*)(B + o_evc);
  d.evq_chunk_off = (const int*)(B + o_evco);
  d.evq_slot = (const int*)(B + o_evs);
  d.evq_coef = (const double*)(B + o_evq);
  d.evq_coef_f = (const float*)(B + o_evqf);
  d.det_chunk = (const int*)(B + o_dc);
  d.det_chunk_off = (const int*)(B + o_dco);
  // walker state: inverses, ln|det| and signs per unique determinant, r_k = D_k/Phi per term,
  // ln|Phi| and its sign
  d.state_doubles = h.U[0] * h.n[0] * h.n[0] + h.U[1] * h.n[1] * h.n[1] + 2 * (h.U[0] + h.U[1]) +
                    (int)h.term_coef.size() + 2;
  d.sh_zeta_ds = (const float*)(B + o_zds);
  d.sh_norm_ds = (const float*)(B + o_nds);
  d.orb_coef_ds = (const float*)(B + o_cds);
  d.nuc_ds = (const float*)(B + o_nucds);
  d.nuc_zf = (const float*)(B + o_nzf);
  d.sh_zeta_f = (const float*)(B + o_zf);
  d.sh_norm_f = (const float*)(B + o_nf);
  d.jas_af = (const float*)(B + o_jaf);
  d.jas_bf = (const float*)(B + o_jbf);
  d.een_Bf = (const float*)(B + o_ebf);
  d.kappa_f = (float)d.kappa;
  d.b1_anti_f = (float)d.b1_anti;
  d.b1_par_f = (float)d.b1_par;
  d.jas_a_ds = (const float*)(B + o_jads);
  d.jas_b_ds = (const float*)(B + o_jbds);
  d.een_c_ds = (const float*)(B + o_ecds);
  {
    const std::vector<float> sc = split(std::vector<double>{d.kappa, d.b1_anti, d.b1_par});
    d.kappa_ds[0] = sc[0]; d.kappa_ds[1] = sc[1];
    d.b1_anti_ds[0] = sc[2]; d.b1_anti_ds[1] = sc[3];
    d.b1_par_ds[0] = sc[4]; d.b1_par_ds[1] = sc[5];
  }
  // determinants through the reference-determinant tables when the per-determinant inverses of
  // one walker do not fit in shared memory, or when they hold so much of it that few walkers
  // share an SM: a sweep region above 48 KB, or above 32 KB with 16 or more unique
  // determinants of a spin (the measured crossover on molecules of 2-32 electrons; systems with
  // orbital-excitation parameters keep the per-determinant form, whose derivatives they need)
  d.msd = 0;
  {
    vbq::DetLayout probe;
    if (h.tab_ok && vbq::make_det_layout(d, 8, ctx->max_smem, probe) != VBQMC_OK) d.msd = 1;
  }
  make_layouts(ctx, ls);
  if (!d.msd && h.tab_ok && d.n_kappa == 0 && ls.lay_rc_sweep[VBQMC_MIXED] == VBQMC_OK) {
    const int bytes = ls.lay_sweep[VBQMC_MIXED].warp_bytes, U = std::max(d.U[0], d.U[1]);
    if (bytes > 48 * 1024 || (bytes > 32 * 1024 && U >= 16)) {
      d.msd = 1;
      make_layouts(ctx, ls);
    }
  }
  ls.loaded = true;
  free_system(ctx->sys[sys_id]);
  ctx->sys[sys_id] = ls;
  return VBQMC_OK;
}

int vbqmc_last_launch_count(vbqmc_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

int vbqmc_use_tables(vbqmc_ctx* ctx, int sys_id, int on) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  if (sys_id < 0 || sys_id >= VBQMC_MAX_SYSTEMS || !ctx->sys[sys_id].loaded)
    return fail(VBQMC_ERR_NOSYS, "no system loaded under this id");
  LoadedSystem& ls = ctx->sys[sys_id];
  if (on) {
    if (!ls.host.tab_ok)
      return fail(VBQMC_ERR_UNSUPPORTED, "a determinant differs from the reference by more than 4 orbitals");
    ls.dev.msd = 1;
  } else {
    vbq::DetLayout probe;
    if (vbq::make_det_layout(ls.dev, 8, ctx->max_smem, probe) != VBQMC_OK)
      return fail(VBQMC_ERR_CAPACITY, "per-determinant inverses of one walker exceed shared memory");
    ls.dev.msd = 0;
  }
  make_layouts(ctx, ls);
  return VBQMC_OK;
}

int vbqmc_launch_info(vbqmc_ctx* ctx, int sys_id, int precision, int* out) {
  if (!ctx || !out) return fail(VBQMC_ERR_ARG, "null argument");
  if (sys_id < 0 || sys_id >= VBQMC_MAX_SYSTEMS || !ctx->sys[sys_id].loaded)
    return fail(VBQMC_ERR_NOSYS, "no system loaded under this id");
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return fail(VBQMC_ERR_ARG, "bad precision mode");
  const LoadedSystem& s = ctx->sys[sys_id];
  out[0] = s.dev.msd ? s.lay_eval[precision].tab.wpb : s.lay_eval[precision].det.wpb;
  out[1] = s.dev.msd ? s.lay_eval[precision].tab.warp_bytes : s.lay_eval[precision].det.warp_bytes;
  out[2] = s.lay_sweep[precision].wpb;
  out[3] = s.lay_sweep[precision].warp_bytes;
  out[4] = s.dev.msd ? 1 : 0;
  return VBQMC_OK;
}

static int check_call(vbqmc_ctx* ctx, int sys_id, int precision, int W) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  if (sys_id < 0 || sys_id >= VBQMC_MAX_SYSTEMS || !ctx->sys[sys_id].loaded)
    return fail(VBQMC_ERR_NOSYS, "no system loaded under this id");
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return fail(VBQMC_ERR_ARG, "bad precision mode");
  if (W < 0) return fail(VBQMC_ERR_ARG, "negative walker count");
  return VBQMC_OK;
}

int vbqmc_walker_state_size(vbqmc_ctx* ctx, int sys_id, int* ndoubles) {
  if (!ctx || !ndoubles) return fail(VBQMC_ERR_ARG, "null argument");
  if (sys_id < 0 || sys_id >= VBQMC_MAX_SYSTEMS || !ctx->sys[sys_id].loaded)
    return fail(VBQMC_ERR_NOSYS, "no system loaded under this id");
  *ndoubles = ctx->sys[sys_id].dev.state_doubles;
  return VBQMC_OK;
}

// Events for a timed evaluation (null when timing is off; creates them on first use).
static cudaEvent_t* timing_events(vbqmc_ctx* ctx) {
  if (!ctx->timing) return nullptr;
  for (auto& ev : ctx->tev)
    if (!ev && cudaEventCreate(&ev) != cudaSuccess) return nullptr;
  ctx->tev_valid = true;
  return ctx->tev;
}

// Grows the context's evaluation workspace to hold W walkers of the system (synchronizing
// 'stream' first when it grows, since earlier work on it may still use the old buffer).
static int ensure_eval_ws(vbqmc_ctx* ctx, const LoadedSystem& s, int precision, int W, cudaStream_t st) {
  const size_t need = vbq::eval_workspace_bytes(s.dev, precision == VBQMC_MIXED ? 4 : 8, W);
  if (need <= ctx->eval_bytes) return VBQMC_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (ctx->eval_work) cudaFree(ctx->eval_work);
  ctx->eval_work = nullptr;
  ctx->eval_bytes = 0;
  e = cudaMalloc(&ctx->eval_work, need);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(evaluation workspace)");
  ctx->eval_bytes = need;
  return VBQMC_OK;
}

int vbqmc_eval_walkers(vbqmc_ctx* ctx, int sys_id, int precision, int W, const double* R, double* logpsi,
                       double* sign, double* eloc, double* grad, void* O, void* dEL, double* state_out,
                       void* stream) {
  int rc = check_call(ctx, sys_id, precision, W);
  if (rc) return rc;
  ctx->last_launches = 0;
  if (W == 0) return VBQMC_OK;
  if (!R || !logpsi || !sign || !eloc) return fail(VBQMC_ERR_ARG, "null required pointer");
  if (dEL && !O) return fail(VBQMC_ERR_ARG, "dEL requires O");
  LoadedSystem& s = ctx->sys[sys_id];
  if (s.lay_rc_eval[precision]) return fail(s.lay_rc_eval[precision], "per-walker state exceeds shared memory");
  if ((O || dEL) && s.dev.P == 0) O = dEL = nullptr;
  if (s.dev.msd && state_out)
    return fail(VBQMC_ERR_UNSUPPORTED, "walker state: this system's determinants go through reference tables");
  if (s.dev.msd && O && s.dev.n_kappa > 0)
    return fail(VBQMC_ERR_UNSUPPORTED, "orbital-excitation derivatives with reference-determinant tables");
  DeviceGuard g(ctx->device);
  rc = ensure_eval_ws(ctx, s, precision, W, (cudaStream_t)stream);
  if (rc) return rc;
  int nl = 0;
  cudaError_t e = vbq::launch_eval(precision, s.dev, s.lay_eval[precision], W, R, logpsi, sign, eloc, grad, O, dEL,
                                   state_out, ctx->eval_work, (cudaStream_t)stream, &nl, timing_events(ctx));
  ctx->last_launches = nl;
  if (e != cudaSuccess) return cuda_fail(e, "evaluation kernel launch");
  return VBQMC_OK;
}

int vbqmc_eval_nuclear_derivs(vbqmc_ctx* ctx, int sys_id, int precision, int W, const double* R, double* logpsi,
                              double* sign, double* eloc, double* dlogpsi_dR, double* dEL_dR, void* stream) {
  int rc = check_call(ctx, sys_id, precision, W);
  if (rc) return rc;
  ctx->last_launches = 0;
  if (W == 0) return VBQMC_OK;
  if (!R || !logpsi || !sign || !eloc || !dlogpsi_dR) return fail(VBQMC_ERR_ARG, "null required pointer");
  LoadedSystem& s = ctx->sys[sys_id];
  if (s.lay_rc_eval[precision]) return fail(s.lay_rc_eval[precision], "per-walker state exceeds shared memory");
  if (s.dev.msd) return fail(VBQMC_ERR_UNSUPPORTED, "nucleus derivatives with reference-determinant tables");
  if (s.host.has_slater) return fail(VBQMC_ERR_UNSUPPORTED, "nucleus derivatives of Slater shells");
  if (s.lay_rc_force[precision])
    return fail(s.lay_rc_force[precision], "nucleus-derivative tables exceed shared memory");
  DeviceGuard g(ctx->device);
  const cudaStream_t st = (cudaStream_t)stream;
  rc = ensure_eval_ws(ctx, s, precision, W, st);
  if (rc) return rc;
  const size_t need = vbq::force_workspace_bytes(s.dev, W);
  if (need > ctx->force_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->force_work) cudaFree(ctx->force_work);
    ctx->force_work = nullptr;
    ctx->force_bytes = 0;
    e = cudaMalloc(&ctx->force_work, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(nucleus-derivative workspace)");
    ctx->force_bytes = need;
  }
  int nl = 0;
  cudaError_t e = vbq::launch_nuclear_derivs(precision, s.dev, s.lay_eval[precision], s.lay_force[precision], W, R,
                                             logpsi, sign, eloc, dlogpsi_dR, dEL_dR, ctx->eval_work,
                                             ctx->force_work, st, &nl);
  ctx->last_launches = nl;
  if (e != cudaSuccess) return cuda_fail(e, "nucleus-derivative kernel launch");
  return VBQMC_OK;
}

int vbqmc_weighted_colsum(vbqmc_ctx* ctx, int W, int K, int jtype, const double* ga, const void* Ja,
                          const double* gb, const void* Jb, double* out, void* stream) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  ctx->last_launches = 0;
  if (W < 0 || K < 0) return fail(VBQMC_ERR_ARG, "negative size");
  if (jtype != 0 && jtype != 1) return fail(VBQMC_ERR_ARG, "jtype must be 0 (double) or 1 (float)");
  if (K == 0) return VBQMC_OK;
  if (!out) return fail(VBQMC_ERR_ARG, "null out");
  if ((gb == nullptr) != (Jb == nullptr)) return fail(VBQMC_ERR_ARG, "gb and Jb must both be given or both NULL");
  DeviceGuard g(ctx->device);
  const cudaStream_t st = (cudaStream_t)stream;
  if (W == 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)K * sizeof(double), st);
    return e == cudaSuccess ? VBQMC_OK : cuda_fail(e, "cudaMemsetAsync");
  }
  if (!ga || !Ja) return fail(VBQMC_ERR_ARG, "null ga or Ja");
  const size_t need = (size_t)vbq::colsum_slices(W) * K * sizeof(double);
  if (need > ctx->red_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->red_work) cudaFree(ctx->red_work);
    ctx->red_work = nullptr;
    ctx->red_bytes = 0;
    e = cudaMalloc(&ctx->red_work, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(column-sum workspace)");
    ctx->red_bytes = need;
  }
  cudaError_t e =
      vbq::launch_weighted_colsum(W, K, jtype, ga, Ja, gb, Jb, out, static_cast<double*>(ctx->red_work), st);
  if (e != cudaSuccess) return cuda_fail(e, "column-sum kernel launch");
  ctx->last_launches = 2;
  return VBQMC_OK;
}

int vbqmc_structure_overlap(vbqmc_ctx* ctx, int precision, int M, int ldo, const void* O, const double* weights,
                            int nvb, const double* c_vb, int n_cparam, const int* cparam, double* S, void* stream) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  ctx->last_launches = 0;
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return fail(VBQMC_ERR_ARG, "bad precision mode");
  if (M < 1 || nvb < 1 || !c_vb || !S) return fail(VBQMC_ERR_ARG, "structure_overlap: bad size or null pointer");
  if (nvb > vbq::kOvMaxStruct) return fail(VBQMC_ERR_CAPACITY, "structure_overlap: more than 32 structures");
  if (n_cparam < 0 || n_cparam > nvb || n_cparam < nvb - 1 || (n_cparam > 0 && (!cparam || !O)) || ldo < n_cparam)
    return fail(VBQMC_ERR_ARG, "structure_overlap: cparam must list every structure but at most one");
  vbq::OverlapMap map{};
  map.nvb = nvb;
  for (int I = 0; I < nvb; ++I) {
    map.col[I] = -1;
    map.c[I] = c_vb[I];
  }
  for (int k = 0; k < n_cparam; ++k) {
    const int I = cparam[k];
    if (I < 0 || I >= nvb || map.col[I] >= 0) return fail(VBQMC_ERR_ARG, "structure_overlap: bad or repeated cparam entry");
    map.col[I] = k;
  }
  for (int I = 0; I < nvb; ++I)
    if (map.col[I] < 0 && !(c_vb[I] != 0.0))
      return fail(VBQMC_ERR_ARG, "structure_overlap: the structure left out of cparam needs c_I != 0");
  DeviceGuard g(ctx->device);
  const cudaStream_t st = (cudaStream_t)stream;
  const int np = (nvb + 1) * (nvb + 2) / 2;
  const size_t need = (vbq::overlap_part_doubles(M, nvb) + np) * sizeof(double);
  if (need > ctx->red_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->red_work) cudaFree(ctx->red_work);
    ctx->red_work = nullptr;
    ctx->red_bytes = 0;
    e = cudaMalloc(&ctx->red_work, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(overlap workspace)");
    ctx->red_bytes = need;
  }
  double* part = static_cast<double*>(ctx->red_work);
  double* out = part + vbq::overlap_part_doubles(M, nvb);
  cudaError_t e = vbq::launch_structure_overlap(M, ldo, precision == VBQMC_MIXED ? 1 : 0, O, weights, map, part, out, st);
  if (e != cudaSuccess) return cuda_fail(e, "structure overlap kernel launch");
  ctx->last_launches = 2;
  std::vector<double> sums(np);
  e = cudaMemcpyAsync(sums.data(), out, np * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "structure overlap result copy");
  const double wsum = sums[np - 1];
  if (!(wsum > 0.0)) return fail(VBQMC_ERR_ARG, "structure_overlap: the weights do not sum to a positive value");
  int t = 0;
  for (int i = 0; i <= nvb; ++i)
    for (int j = i; j <= nvb; ++j, ++t)
      if (i < nvb && j < nvb) S[(size_t)i * nvb + j] = S[(size_t)j * nvb + i] = sums[t] / wsum;
  return VBQMC_OK;
}

int vbqmc_vmc_steps(vbqmc_ctx* ctx, int sys_id, int precision, int W, double* R, int nsweeps, double step,
                    uint64_t seed, uint32_t step0, uint32_t system_tag, uint32_t walker_offset, int refresh,
                    double* state, int state_valid, int* nacc, double* logpsi, double* sign, double* eloc, void* O,
                    void* dEL, void* stream) {
  int rc = check_call(ctx, sys_id, precision, W);
  if (rc) return rc;
  ctx->last_launches = 0;
  if (nsweeps < 0 || !(step > 0.0) || refresh < 0) return fail(VBQMC_ERR_ARG, "bad sweep count, step or refresh");
  if (state_valid && !state) return fail(VBQMC_ERR_ARG, "state_valid without state");
  if (system_tag > 0xffffffu) return fail(VBQMC_ERR_ARG, "system_tag must fit in 24 bits");
  if (W == 0) return VBQMC_OK;
  if (!R) return fail(VBQMC_ERR_ARG, "null R");
  LoadedSystem& s = ctx->sys[sys_id];
  if (s.dev.msd && (state || state_valid))
    return fail(VBQMC_ERR_UNSUPPORTED, "systems on reference-determinant tables keep no walker state (pass NULL)");
  if (s.lay_rc_sweep[precision]) return fail(s.lay_rc_sweep[precision], "per-walker state exceeds shared memory");
  const bool do_eval = logpsi || sign || eloc || O || dEL;
  if (do_eval && (!logpsi || !sign || !eloc)) return fail(VBQMC_ERR_ARG, "evaluation needs logpsi, sign and eloc");
  if (dEL && !O) return fail(VBQMC_ERR_ARG, "dEL requires O");
  DeviceGuard g(ctx->device);
  int launches = 0;
  if (nsweeps > 0) {
    cudaError_t e = vbq::launch_sweep(precision, s.dev, s.lay_sweep[precision], W, R, nsweeps, refresh, state,
                                      state_valid, step, seed, step0, system_tag, walker_offset, nacc,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sweep kernel launch");
    ++launches;
  }
  if (do_eval) {
    if (s.lay_rc_eval[precision]) return fail(s.lay_rc_eval[precision], "per-walker state exceeds shared memory");
    if ((O || dEL) && s.dev.P == 0) O = dEL = nullptr;
    rc = ensure_eval_ws(ctx, s, precision, W, (cudaStream_t)stream);
    if (rc) return rc;
    int nl = 0;
    // the evaluation takes the inverses the sweeps carried, except at global step counts that are
    // multiples of 'refresh', where it factorises afresh and rewrites the state
    const bool carried = state && nsweeps > 0 && !(refresh > 0 && (step0 + (uint32_t)nsweeps) % (uint32_t)refresh == 0);
    cudaError_t e = vbq::launch_eval(precision, s.dev, s.lay_eval[precision], W, R, logpsi, sign, eloc, nullptr, O,
                                     dEL, carried ? nullptr : state, ctx->eval_work, (cudaStream_t)stream, &nl,
                                     timing_events(ctx), nullptr, carried ? state : nullptr);
    launches += nl;
    if (e != cudaSuccess) {
      ctx->last_launches = launches;
      return cuda_fail(e, "evaluation kernel launch");
    }
  }
  ctx->last_launches = launches;
  return VBQMC_OK;
}

int vbqmc_dmc_steps(vbqmc_ctx* ctx, int sys_id, int precision, int* W_io, int cap, double* R, int nsteps, double tau,
                    double* E_T_io, int target, uint64_t seed, uint32_t step0, uint32_t system_tag,
                    uint32_t walker_offset, double* sum_wE, double* sum_w, double* sum_wEb, int* pop, double* e_trial,
                    int64_t* accepted, void* stream) {
  if (!W_io || !E_T_io) return fail(VBQMC_ERR_ARG, "null W_io or E_T_io");
  int rc = check_call(ctx, sys_id, precision, *W_io);
  if (rc) return rc;
  ctx->last_launches = 0;
  int W = *W_io;
  if (cap < 1 || W > cap) return fail(VBQMC_ERR_ARG, "need 1 <= cap and W <= cap");
  if (nsteps < 0 || !(tau > 0.0) || target < 1) return fail(VBQMC_ERR_ARG, "bad step count, tau or target");
  if (system_tag > 0xffffffu) return fail(VBQMC_ERR_ARG, "system_tag must fit in 24 bits");
  if (accepted) *accepted = 0;
  if (W == 0 || nsteps == 0) return VBQMC_OK;
  if (!R) return fail(VBQMC_ERR_ARG, "null R");
  LoadedSystem& s = ctx->sys[sys_id];
  if (s.lay_rc_eval[precision]) return fail(s.lay_rc_eval[precision], "per-walker state exceeds shared memory");
  DeviceGuard g(ctx->device);
  const cudaStream_t st = (cudaStream_t)stream;
  const int N = s.dev.N, n3 = 3 * N;
  // workspace: Rp, grad A, grad1, R B, grad B ([cap][3N] each), 11 per-walker doubles, 3 ints, totals
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t vec = al(sizeof(double) * (size_t)cap * n3), sca = al(sizeof(double) * (size_t)cap),
               ints = al(sizeof(int) * (size_t)cap);
  const size_t need = 5 * vec + 12 * sca + 3 * ints + al(sizeof(vbq::DmcTotals));
  if (need > ctx->dmc_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->dmc_work) cudaFree(ctx->dmc_work);
    ctx->dmc_work = nullptr;
    ctx->dmc_bytes = 0;
    e = cudaMalloc(&ctx->dmc_work, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(DMC workspace)");
    ctx->dmc_bytes = need;
  }
  unsigned char* p = static_cast<unsigned char*>(ctx->dmc_work);
  auto take = [&](size_t b) {
    unsigned char* r = p;
    p += b;
    return r;
  };
  struct Set {
    double *R, *lp, *sg, *el, *grad;
  };
  double* Rp = reinterpret_cast<double*>(take(vec));
  double* grad1 = reinterpret_cast<double*>(take(vec));
  Set cur, nxt;
  cur.R = R;
  cur.grad = reinterpret_cast<double*>(take(vec));
  nxt.R = reinterpret_cast<double*>(take(vec));
  nxt.grad = reinterpret_cast<double*>(take(vec));
  cur.lp = reinterpret_cast<double*>(take(sca));
  cur.sg = reinterpret_cast<double*>(take(sca));
  cur.el = reinterpret_cast<double*>(take(sca));
  nxt.lp = reinterpret_cast<double*>(take(sca));
  nxt.sg = reinterpret_cast<double*>(take(sca));
  nxt.el = reinterpret_cast<double*>(take(sca));
  double* lp1 = reinterpret_cast<double*>(take(sca));
  double* sg1 = reinterpret_cast<double*>(take(sca));
  double* el1 = reinterpret_cast<double*>(take(sca));
  double* wt = reinterpret_cast<double*>(take(sca));
  double* wE = reinterpret_cast<double*>(take(sca));
  double* wEb = reinterpret_cast<double*>(take(sca));
  int* copies = reinterpret_cast<int*>(take(ints));
  int* offsets = reinterpret_cast<int*>(take(ints));
  int* acc = reinterpret_cast<int*>(take(ints));
  vbq::DmcTotals* tot = reinterpret_cast<vbq::DmcTotals*>(take(al(sizeof(vbq::DmcTotals))));
  int launches = 0;
  double E_T = *E_T_io;
  int64_t nacc = 0;
  rc = ensure_eval_ws(ctx, s, precision, cap, st);
  if (rc) return rc;
  // the walkers' values at R, carried from step to step
  int nl = 0;
  cudaError_t e = vbq::launch_eval(precision, s.dev, s.lay_eval[precision], W, cur.R, cur.lp, cur.sg, cur.el, cur.grad,
                                   nullptr, nullptr, nullptr, ctx->eval_work, st, &nl);
  if (e != cudaSuccess) return cuda_fail(e, "evaluation kernel launch");
  launches += nl;
  int rcode = VBQMC_OK;
  for (int k = 0; k < nsteps; ++k) {
    const uint32_t stp = step0 + (uint32_t)k;
    e = vbq::launch_dmc_propose(W, N, cur.R, cur.grad, tau, seed, stp, system_tag, walker_offset, Rp, st);
    if (e == cudaSuccess)
      e = vbq::launch_eval(precision, s.dev, s.lay_eval[precision], W, Rp, lp1, sg1, el1, grad1, nullptr, nullptr,
                           nullptr, ctx->eval_work, st, &nl);
    if (e == cudaSuccess)
      e = vbq::launch_dmc_accept(W, N, cur.R, cur.lp, cur.sg, cur.el, cur.grad, Rp, lp1, sg1, el1, grad1, tau, E_T,
                                 seed, stp, system_tag, walker_offset, wt, wE, wEb, copies, acc, st);
    if (e == cudaSuccess) e = vbq::launch_dmc_scan(W, copies, wt, wE, wEb, acc, offsets, tot, st);
    if (e == cudaSuccess)
      e = vbq::launch_dmc_branch(W, N, cap, copies, offsets, tot, cur.R, cur.lp, cur.sg, cur.el, cur.grad, nxt.R,
                                 nxt.lp, nxt.sg, nxt.el, nxt.grad, st);
    vbq::DmcTotals h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rcode = cuda_fail(e, "DMC step");
      break;
    }
    launches += 4 + nl;
    nacc += h.accepted;
    if (h.total > cap) {
      rcode = fail(VBQMC_ERR_CAPACITY, "DMC population " + std::to_string(h.total) + " exceeds capacity " +
                                           std::to_string(cap) + " at step " + std::to_string(k) +
                                           " (moves of that step applied, branching not done)");
      break;
    }
    std::swap(cur, nxt);
    W = (int)h.total;
    const double Ebmean = h.sum_w > 0.0 ? h.sum_wEb / h.sum_w : E_T;
    if (W > 0) E_T = Ebmean - (0.1 / tau) * std::log((double)W / (double)target);
    if (sum_wE) sum_wE[k] = h.sum_wE;
    if (sum_w) sum_w[k] = h.sum_w;
    if (sum_wEb) sum_wEb[k] = h.sum_wEb;
    if (pop) pop[k] = W;
    if (e_trial) e_trial[k] = E_T;
    if (W == 0) break;
  }
  // the population lives in the caller's R at return
  if (cur.R != R && W > 0) {
    e = cudaMemcpyAsync(R, cur.R, sizeof(double) * (size_t)W * n3, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && rcode == VBQMC_OK) rcode = cuda_fail(e, "DMC population copy");
  }
  *W_io = W;
  *E_T_io = E_T;
  if (accepted) *accepted = nacc;
  ctx->last_launches = launches;
  return rcode;
}

int vbqmc_set_kernel_timing(vbqmc_ctx* ctx, int on) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  ctx->timing = on ? 1 : 0;
  ctx->tev_valid = false;
  return VBQMC_OK;
}

int vbqmc_kernel_times(vbqmc_ctx* ctx, double* ms, int max, int* n) {
  if (!ctx || !ms || !n) return fail(VBQMC_ERR_ARG, "null argument");
  if (!ctx->tev_valid) return fail(VBQMC_ERR_ARG, "no timed evaluation recorded");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaEventSynchronize(ctx->tev[vbq::kEvalKernels]);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
  *n = vbq::kEvalKernels;
  for (int k = 0; k < vbq::kEvalKernels && k < max; ++k) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, ctx->tev[k], ctx->tev[k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms[k] = t;
  }
  return VBQMC_OK;
}

int vbqmc_accumulate_lin_matrices(vbqmc_ctx* ctx, int precision, int P, int64_t M, const void* O, const void* dEL,
                                  const double* eloc, const double* weights, double* E0, double* gL, double* gR,
                                  double* S, double* H, void* stream) {
  if (!ctx) return fail(VBQMC_ERR_ARG, "null context");
  if (precision != VBQMC_FP64 && precision != VBQMC_MIXED) return fail(VBQMC_ERR_ARG, "bad precision mode");
  if (P < 1 || M < 1) return fail(VBQMC_ERR_ARG, "need P >= 1 and M >= 1");
  if (!O || !dEL || !eloc || !E0 || !gL || !gR || !S || !H) return fail(VBQMC_ERR_ARG, "null required pointer");
  DeviceGuard g(ctx->device);
  ctx->last_launches = 0;
  const int nsm = vbq::lin_sms();
  const size_t need = vbq::lin_workspace_bytes(P, M, nsm);
  if (need > ctx->work_bytes) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->work) cudaFree(ctx->work);
    ctx->work = nullptr;
    ctx->work_bytes = 0;
    e = cudaMalloc(&ctx->work, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(linear-method workspace)");
    ctx->work_bytes = need;
  }
  int nl = 0;
  cudaError_t e = vbq::launch_lin(precision == VBQMC_MIXED, P, (long long)M, O, dEL, eloc, weights, ctx->work,
                                  ctx->work_bytes, nsm, E0, gL, gR, S, H, (cudaStream_t)stream, &nl,
                                  timing_events(ctx));
  if (e != cudaSuccess) return cuda_fail(e, "linear-method kernels");
  ctx->last_launches = nl;
  return VBQMC_OK;
}

}  // extern "C"
