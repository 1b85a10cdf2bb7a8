// libmrcm C ABI: set-up, MRCM-OS preconditioner application and restarted GMRES (Algorithm 1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace mrcm;

namespace mrcm {
static std::atomic<long long> g_launches{0};
// this thread's launches: a phase counts only the kernels its own thread launched, although request
// workers launch from several threads at once
static thread_local long long t_launches = 0;
void count_launch(int kernels) {
  g_launches.fetch_add(kernels, std::memory_order_relaxed);
  t_launches += kernels;
}
}  // namespace mrcm

static thread_local std::string g_last_error;

namespace mrcm {
void set_thread_error(const std::string& msg) { g_last_error = msg; }
}  // namespace mrcm

namespace {

// NVTX range names of the phases (for profilers; without one attached a range is a no-op)
const char* const kPhaseName[MRCM_PHASES] = {
    "mrcm assemble", "mrcm factor ohat robin", "mrcm informed spaces", "mrcm factor omega", "mrcm basis",
    "mrcm coupling factor", "mrcm factor ohat dirichlet", "mrcm particular", "mrcm coupling solve",
    "mrcm reconstruct", "mrcm residual", "mrcm schwarz", "mrcm krylov", "mrcm stage fp32 rhs"};

// Phase brackets: an NVTX range always, and a (start, stop) event pair per kernel group while
// profiling is enabled.
struct Phase {
  mrcm_handle h;
  int ph;
  cudaStream_t st;
  long long l0;
  long long slot = -1;  // this phase's event pair (reserved at construction, so phases may nest)
  Phase(mrcm_handle h_, int ph_, cudaStream_t st_) : h(h_), ph(ph_), st(st_), l0(t_launches) {
    nvtxRangePushA(kPhaseName[ph]);
    if (!h->prof || !((h->prof_mask >> ph) & 1u)) return;
    if (h->ph_seen[ph]++ % h->prof_every != 0) return;
    const size_t need = 2 * (h->ev_used + 1);
    while (h->ev_pool.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        h->prof = false;
        return;
      }
      h->ev_pool.push_back(e);
    }
    if (h->ev_phase.size() < h->ev_used + 1) h->ev_phase.resize(h->ev_used + 1);
    slot = (long long)h->ev_used++;
    h->ev_phase[slot] = ph;
    cudaEventRecord(h->ev_pool[2 * slot], st);
  }
  ~Phase() {
    nvtxRangePop();
    if (slot < 0) return;
    cudaEventRecord(h->ev_pool[2 * slot + 1], st);
    h->ph_launch[ph] += t_launches - l0;
  }
};

mrcm_status fail(mrcm_handle h, mrcm_status s, const std::string& msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  return s;
}

#define CK(h, x)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) return fail((h), MRCM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
T* at(mrcm_handle h, size_t off) {
  return reinterpret_cast<T*>(h->ws + off);
}

struct Tables {
  int* iface;
  int* home;
  int* off;
  int* rank;
  int* cidx;
};

Tables tables(mrcm_handle h) {
  const Plan& P = h->plan;
  int* base = at<int>(h, h->lay.tab);
  Tables t;
  t.iface = base;
  t.home = t.iface + 3 * P.E;
  t.off = t.home + P.E2;
  t.rank = t.off + P.S;
  t.cidx = t.rank + 6 * P.S;
  return t;
}

Geo geo(mrcm_handle h) {
  Geo g;
  const Plan& P = h->plan;
  g.nx = P.n[0];
  g.ny = P.n[1];
  g.sx = P.sub[0];
  g.sy = P.sub[1];
  g.mx = P.m[0];
  g.my = P.m[1];
  g.l = P.l;
  g.smax = h->lay.smax;
  g.nq = P.nq;
  g.hx = h->h[0];
  g.hy = h->h[1];
  g.hz = h->h[2];
  g.alpha = h->prm.alpha;
  g.K = at<double>(h, h->lay.K);
  g.Ky = at<double>(h, h->lay.Ky);
  g.Tx = at<double>(h, h->lay.Tx);
  g.Ty = at<double>(h, h->lay.Ty);
  g.gtr = at<double>(h, h->lay.gtr);
  if (h->plan.dim == 2) {
    g.rto = h->plan.l > 0 ? at<double>(h, h->lay.rto) : nullptr;
    g.rtl = at<double>(h, h->lay.rtl);
    g.rlo = std::max(h->lay.wo, h->lay.ho);
    g.rll = std::max(h->lay.wl, h->lay.hl);
  }
  return g;
}

CoarseDev coarse(mrcm_handle h) {
  CoarseDev c;
  const Plan& P = h->plan;
  Tables t = tables(h);
  c.n = P.NC;
  c.nq = P.nq;
  c.kl = P.kl;
  c.ku = P.ku;
  c.ldab = h->lay.ldab;
  c.ab = at<double>(h, h->lay.G);
  c.ipiv = at<int>(h, h->lay.ipiv);
  c.rdiag = at<double>(h, h->lay.rdiag);
  c.nbk = P.NC > COARSE_DENSE_MAX ? (P.NC + GBB_NB - 1) / GBB_NB : 0;
  c.ML = at<double>(h, h->lay.gbML);
  c.MU = at<double>(h, h->lay.gbMU);
  c.X = at<double>(h, h->lay.gbX);
  c.Y = at<double>(h, h->lay.gbY);
  c.F = at<double>(h, h->lay.gbF);
  c.C = at<double>(h, h->lay.gbC);
  c.g = at<double>(h, h->lay.gc);
  c.iface = t.iface;
  c.home = t.home;
  c.off = t.off;
  c.rank = t.rank;
  return c;
}

MfDev mfdev(mrcm_handle h) {
  MfDev m;
  const Layout& L = h->lay;
  const Plan& P = h->plan;
  m.fr = at<MfFront>(h, L.mf_fr);
  m.order = at<int>(h, L.mf_ord);
  m.lvl = at<int>(h, L.mf_lvl);
  m.idx = at<int>(h, L.mf_idx);
  m.asmv = at<int2>(h, L.mf_asm);
  m.map = at<int>(h, L.mf_map);
  m.task = at<int4>(h, L.mf_task);
  m.F = at<double>(h, L.mf_F);
  m.V = at<double>(h, L.mf_V);
  m.scr = at<unsigned>(h, L.mf_scr);
  m.done = at<unsigned>(h, L.mf_done);
  m.nfront = (int)P.mf_front.size();
  m.levels = P.mf_level.empty() ? 0 : (int)P.mf_level.size() - 1;
  m.max_f = P.mf_max_f;
  m.mcap = P.mf_mcap;
  return m;
}

size_t ncell(mrcm_handle h) { return (size_t)h->n[0] * h->n[1] * h->n[2]; }

std::string supported(const mrcm_problem& p, const mrcm_params& q) {
  if (p.dim != 2) return "the GPU path implements dim == 2";
  if (q.sub[0] + 2 * q.oversample > 64 || q.sub[1] + 2 * q.oversample > 64)
    return "the GPU path needs sub + 2 * oversample <= 64 on x and y";
  return std::string();
}

mrcm_status copy_problem(mrcm_handle h, const mrcm_problem* p, cudaStream_t st) {
  const size_t n = ncell(h);
  if (!p->K) return fail(h, MRCM_ERR_INVALID_ARG, "problem->K is null");
  CK(h, cudaMemcpyAsync(at<double>(h, h->lay.K), p->K, 8 * n, cudaMemcpyDeviceToDevice, st));
  h->iso = p->K_y == nullptr;
  CK(h, cudaMemcpyAsync(at<double>(h, h->lay.Ky), h->iso ? p->K : p->K_y, 8 * n, cudaMemcpyDeviceToDevice, st));
  h->has_f = p->f != nullptr;
  if (p->f) CK(h, cudaMemcpyAsync(at<double>(h, h->lay.f), p->f, 8 * n, cudaMemcpyDeviceToDevice, st));
  const size_t len = std::max(h->n[0], h->n[1]);
  double* bcv = at<double>(h, h->lay.bcv);
  for (int s = 0; s < 4; ++s) {
    h->has_bc[s] = p->bc_val[s] != nullptr;
    const size_t cnt = s < 2 ? (size_t)h->n[1] : (size_t)h->n[0];
    if (p->bc_val[s]) CK(h, cudaMemcpyAsync(bcv + s * len, p->bc_val[s], 8 * cnt, cudaMemcpyDeviceToDevice, st));
  }
  h->factored = false;
  return MRCM_OK;
}

__global__ void k_check_positive(const double* K, size_t n, int* flags) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = K[i];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(flags, FLAG_NONFINITE);
  }
}

__global__ void k_set(double* p, double v) { *p = v; }

void bc_ptrs(mrcm_handle h, const double* ptrs[4]) {
  const size_t len = std::max(h->n[0], h->n[1]);
  const double* bcv = at<double>(h, h->lay.bcv);
  for (int s = 0; s < 4; ++s) ptrs[s] = h->has_bc[s] ? bcv + s * len : nullptr;
}

}  // namespace

extern "C" {

void mrcm_autotune(int32_t mode) { mrcm::autotune_mode(mode); }

mrcm_status mrcm_autotune_table(double* buf, size_t cap, size_t* len) {
  if (!len) return MRCM_ERR_INVALID_ARG;
  const std::vector<double> t = mrcm::autotune_table();
  *len = t.size();
  if (buf) std::memcpy(buf, t.data(), sizeof(double) * std::min(cap, t.size()));
  return MRCM_OK;
}

const char* mrcm_status_string(mrcm_status s) {
  switch (s) {
    case MRCM_OK: return "ok";
    case MRCM_ERR_INVALID_ARG: return "invalid argument";
    case MRCM_ERR_OOM: return "workspace too small";
    case MRCM_ERR_SINGULAR: return "singular factorisation";
    case MRCM_ERR_NOT_CONVERGED: return "not converged";
    case MRCM_ERR_TIMEOUT: return "device wait timed out";
    case MRCM_ERR_CUDA: return "CUDA error";
    case MRCM_ERR_BUSY: return "busy";
    case MRCM_ERR_UNSUPPORTED: return "unsupported on the GPU path";
    case MRCM_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* mrcm_last_error(mrcm_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

mrcm_status mrcm_plan_export(const mrcm_problem* problem, const mrcm_params* params, int32_t* buf, size_t cap,
                             size_t* len) {
  if (!problem || !params || !len) return fail(nullptr, MRCM_ERR_INVALID_ARG, "null argument");
  Plan P;
  std::string why = make_plan(*problem, *params, P);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_INVALID_ARG, why);
  std::vector<int32_t> out = export_plan(P);
  *len = out.size();
  if (buf) std::memcpy(buf, out.data(), sizeof(int32_t) * std::min(cap, out.size()));
  return MRCM_OK;
}

mrcm_status mrcm_plan_mf_export(const mrcm_problem* problem, const mrcm_params* params, int32_t* buf, size_t cap,
                                size_t* len) {
  if (!problem || !params || !len) return fail(nullptr, MRCM_ERR_INVALID_ARG, "null argument");
  Plan P;
  std::string why = make_plan(*problem, *params, P);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_INVALID_ARG, why);
  const int nf = (int)P.mf_front.size();
  const int levels = P.mf_level.empty() ? 0 : (int)P.mf_level.size() - 1;
  std::vector<int32_t> out = {P.mf ? 1 : 0, nf, levels, P.NC, P.kl, P.ku};
  std::vector<int> lev(nf, 0);
  for (int L = 0; L < levels; ++L)
    for (int i = P.mf_level[L]; i < P.mf_level[L + 1]; ++i) lev[P.mf_order[i]] = L;
  for (int f = 0; f < nf; ++f) {
    const MfFront& fr = P.mf_front[f];
    out.insert(out.end(), {fr.np, fr.nu, lev[f], fr.nch, fr.nch > 0 ? fr.ch[0] : -1, fr.nch > 1 ? fr.ch[1] : -1,
                           fr.par});
  }
  for (int f = 0; f < nf; ++f) {
    const MfFront& fr = P.mf_front[f];
    out.insert(out.end(), P.mf_idx.begin() + fr.io, P.mf_idx.begin() + fr.io + fr.np + fr.nu);
  }
  // assembly pairs back to (row, column): the band offset is kl + ku + row - col + col ldab
  const long long kv = (long long)P.kl + P.ku, ldab = 2LL * P.kl + P.ku + 1;
  for (int f = 0; f < nf; ++f) {
    const MfFront& fr = P.mf_front[f];
    out.push_back(fr.na);
    for (int t = 0; t < fr.na; ++t) {
      const long long src = P.mf_asm[2 * (fr.ao + t) + 1];
      const long long col = src / ldab, row = src % ldab - kv + col;
      out.push_back((int32_t)row);
      out.push_back((int32_t)col);
    }
  }
  *len = out.size();
  if (buf) std::memcpy(buf, out.data(), sizeof(int32_t) * std::min(cap, out.size()));
  return MRCM_OK;
}

mrcm_status mrcm_footprint(const mrcm_problem* problem, const mrcm_params* params, size_t* bytes) {
  if (!problem || !params || !bytes) return fail(nullptr, MRCM_ERR_INVALID_ARG, "null argument");
  Plan P;
  std::string why = make_plan(*problem, *params, P);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_INVALID_ARG, why);
  why = supported(*problem, *params);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_UNSUPPORTED, why);
  *bytes = make_layout(P, *params).total;
  return MRCM_OK;
}

mrcm_status mrcm_setup(const mrcm_problem* problem, const mrcm_params* params, void* workspace, size_t workspace_bytes,
                       void* stream, mrcm_handle* out) {
  if (!problem || !params || !out) return fail(nullptr, MRCM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  Plan P;
  std::string why = make_plan(*problem, *params, P);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_INVALID_ARG, why);
  why = supported(*problem, *params);
  if (!why.empty()) return fail(nullptr, MRCM_ERR_UNSUPPORTED, why);
  Layout L = make_layout(P, *params);
  if (!workspace) return fail(nullptr, MRCM_ERR_INVALID_ARG, "workspace is null");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(nullptr, MRCM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(nullptr, MRCM_ERR_OOM, "workspace smaller than mrcm_footprint(): need " + std::to_string(L.total) + " bytes");
  mrcm_handle h = new (std::nothrow) mrcm_ctx();
  if (!h) return fail(nullptr, MRCM_ERR_OOM, "host allocation failed");
  h->plan = P;
  h->lay = L;
  h->prm = *params;
  h->dim = problem->dim;
  for (int a = 0; a < 3; ++a) {
    h->n[a] = problem->n[a];
    h->h[a] = problem->h[a];
  }
  for (int s = 0; s < 6; ++s) h->bc_kind[s] = problem->bc_kind[s];
  h->ws = static_cast<char*>(workspace);
  h->ws_bytes = workspace_bytes;
  h->coarse_n = P.E2;
  if (cudaGetDevice(&h->device) != cudaSuccess) h->device = -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mrcm_status rc = copy_problem(h, problem, st);
  if (rc != MRCM_OK) {
    g_last_error = h->err;
    delete h;
    return rc;
  }
  // plan tables to the device
  std::vector<int> tab;
  tab.insert(tab.end(), P.iface.begin(), P.iface.end());
  tab.insert(tab.end(), P.row_home.begin(), P.row_home.end());
  tab.insert(tab.end(), P.off.begin(), P.off.end());
  tab.insert(tab.end(), P.rank.begin(), P.rank.end());
  for (int s = 0; s < P.S; ++s)
    for (int k = 0; k < 4; ++k) tab.push_back(P.rank[6 * s + k] >= 0 ? P.off[s] + P.rank[6 * s + k] : -1);
  h->tab_host = tab;
  cudaError_t e = cudaMemcpyAsync(at<int>(h, L.tab), h->tab_host.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, st);
  if (P.mf) {   // multifrontal tables (the host copies live in h->plan)
    const Plan& HP = h->plan;
    auto up = [&](size_t off, const void* src, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(h->ws + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    up(L.mf_fr, HP.mf_front.data(), sizeof(MfFront) * HP.mf_front.size());
    up(L.mf_ord, HP.mf_order.data(), 4 * HP.mf_order.size());
    up(L.mf_lvl, HP.mf_level.data(), 4 * HP.mf_level.size());
    up(L.mf_idx, HP.mf_idx.data(), 4 * HP.mf_idx.size());
    up(L.mf_asm, HP.mf_asm.data(), 4 * HP.mf_asm.size());
    up(L.mf_map, HP.mf_map.data(), 4 * HP.mf_map.size());
    up(L.mf_task, HP.mf_task.data(), 4 * HP.mf_task.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.mf_scr, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.mf_done, 0, 8 * HP.mf_front.size(), st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(at<unsigned char>(h, L.red), 0, 8 * RED_DOUBLES + 64, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<int>(h, L.flags), 0, 4 * 64, st);
  if (e != cudaSuccess) {
    g_last_error = std::string("set-up copies: ") + cudaGetErrorString(e);
    delete h;
    return MRCM_ERR_CUDA;
  }
  *out = h;
  return MRCM_OK;
}

mrcm_status mrcm_update_problem(mrcm_handle h, const mrcm_problem* problem, void* stream) {
  if (!h || !problem) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (problem->dim != h->dim) return fail(h, MRCM_ERR_INVALID_ARG, "dimension differs from set-up");
  for (int a = 0; a < 3; ++a)
    if (problem->n[a] != h->n[a] || problem->h[a] != h->h[a]) return fail(h, MRCM_ERR_INVALID_ARG, "grid differs from set-up");
  for (int s = 0; s < 6; ++s)
    if (problem->bc_kind[s] != h->bc_kind[s]) return fail(h, MRCM_ERR_INVALID_ARG, "boundary kinds differ from set-up");
  return copy_problem(h, problem, static_cast<cudaStream_t>(stream));
}

mrcm_status mrcm_factor_local(mrcm_handle h, void* stream) {
  if (!h) return fail(h, MRCM_ERR_INVALID_ARG, "null handle");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout& L = h->lay;
  const Plan& P = h->plan;
  const bool fp32 = h->prm.local_prec == MRCM_PREC_FP32;
  int* flags = at<int>(h, L.flags);
  CK(h, cudaMemsetAsync(flags, 0, 4 * 64, st));
  const size_t n = ncell(h);
  k_check_positive<<<256, 256, 0, st>>>(at<double>(h, L.K), n, flags);
  k_check_positive<<<256, 256, 0, st>>>(at<double>(h, L.Ky), n, flags);
  CK(h, cudaGetLastError());
  Geo g = geo(h);
  const double* bcp[4];
  bc_ptrs(h, bcp);
  {
    Phase ph(h, MRCM_PH_ASSEMBLE, st);
    CK(h, launch_assemble(g, h->bc_kind, bcp, h->has_f ? at<double>(h, L.f) : nullptr, at<double>(h, L.Tx),
                          at<double>(h, L.Ty), at<double>(h, L.b), st));
    CK(h, launch_gamma_coef(g, st));
    // both tables before the fork: a table launch queued on the second stream waits behind the
    // oversampled factor's CTAs and delays the subdomain factor
    if (P.l > 0) CK(h, launch_robin_tab(g, true, at<double>(h, L.rto), st));
    CK(h, launch_robin_tab(g, false, at<double>(h, L.rtl), st));
  }
  // The factorisations depend only on A and are latency-bound (a barrier per column), so
  // independent ones share the SMs: the local Robin factors of MRCM-OS step 3 and then the
  // Dirichlet factors of the oversampled regions (the smoothing of step 4) run on a second stream
  // beside the oversampled Robin factors and the informed spaces of step 2; the basis solves wait
  // for the first, the end of the set-up for the second.  The two chains take about the same time,
  // so the second stream is done by the time the coupling factorisation (a cooperative launch
  // holding one CTA on every SM) starts.
  if (!h->side) {
    CK(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    CK(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    CK(h, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
    CK(h, cudaEventCreateWithFlags(&h->omega_ev, cudaEventDisableTiming));
  }
  CK(h, cudaEventRecord(h->fork_ev, st));
  CK(h, cudaStreamWaitEvent(h->side, h->fork_ev, 0));
  // MRCM-OS step 2: informed multiplier spaces from the oversampled Robin problems (Eq. 15); the
  // oversampled factors are submitted first, since the informed spaces wait for them
  CK(h, cudaMemsetAsync(at<double>(h, L.phi), 0, 8 * (size_t)P.S * 16 * P.nq * L.smax, st));
  // FP32 set-up solves refined once against the FP64 box operators (refine_setup)
  const bool refine = fp32 && h->prm.refine_setup != 0;           // the basis solves
  const bool refine_inf = fp32 && h->prm.refine_setup == 1;        // and the informed spaces
  if (P.l > 0) {
    Phase ph(h, MRCM_PH_FACTOR_OHAT_ROBIN, st);
    CK(h, launch_factor(g, BOX_OHAT_ROBIN, L.wo, L.ho, L.LSo, at<void>(h, L.Linv_ohat_r), fp32, flags, st,
                        refine_inf ? at<double>(h, L.coef_o) : nullptr));
  }
  const bool smooth = h->prm.smooth_steps > 0;
  {
    Phase ph(h, MRCM_PH_FACTOR_OMEGA, h->side);
    CK(h, launch_factor(g, BOX_OMEGA_ROBIN, L.wl, L.hl, L.LSl, at<void>(h, L.Linv_loc), fp32, flags, h->side,
                        refine ? at<double>(h, L.coef_l) : nullptr));
  }
  CK(h, cudaEventRecord(h->omega_ev, h->side));
  if (smooth) {
    Phase ph(h, MRCM_PH_FACTOR_OHAT_DIRICHLET, h->side);
    CK(h, launch_factor(g, BOX_OHAT_DIRICHLET, L.wo, L.ho, L.LSo, at<void>(h, L.Linv_ohat_d), fp32, flags, h->side));
  }
  CK(h, cudaEventRecord(h->join_ev, h->side));
  {
    Phase ph(h, MRCM_PH_INFORMED, st);
    for (int q = 0; q < P.nq; ++q)
      CK(h, launch_informed(g, at<void>(h, L.Linv_ohat_r), L.LSo, fp32, at<double>(h, L.phi), q, at<int>(h, L.flags), st,
                            refine_inf ? at<double>(h, L.coef_o) : nullptr));
  }
  // MRCM-OS step 3: multiscale basis functions from the local Robin factors
  CK(h, cudaStreamWaitEvent(st, h->omega_ev, 0));
  {
    Phase ph(h, MRCM_PH_BASIS, st);
    for (int q = 0; q < P.nq; ++q)
      CK(h, launch_basis(g, at<void>(h, L.Linv_loc), L.LSl, fp32, at<double>(h, L.phi), q, at<double>(h, L.psi),
                         at<double>(h, L.mom), at<int>(h, L.flags), st,
                         refine ? at<double>(h, L.coef_l) : nullptr));
  }
  // coupling system (Eq. 13-14): band LU without row interchanges over the whole GPU first; the
  // pivoted factorisation only if that one reports a zero pivot or element growth (or if the
  // caller asks for pivoting)
  CoarseDev c = coarse(h);
  unsigned* np_scratch = reinterpret_cast<unsigned*>(flags + 16);
  // partial pivoting: the variants give identical factors, and the autotuner times each once per
  // band shape (re-assembling G before every run, since the factorisation works in place)
  auto pivoted = [&]() -> mrcm_status {
    int vars[COARSE_FACTOR_MAX_VARIANTS];
    const int nv = coarse_factor_variants(c, vars);
    const int key[6] = {c.n, c.kl, c.ku, 0, 0, 0};
    cudaError_t terr = cudaSuccess;
    const int pick = autotune(TUNE_COARSE_FACTOR, key, nv, st, [&](int i) {
      const cudaError_t e = launch_coarse_assemble(c, at<double>(h, L.mom), P.E, st);
      return e != cudaSuccess ? e : launch_coarse_factor(c, flags, st, vars[i]);
    }, &terr);
    CK(h, terr);
    CK(h, launch_coarse_assemble(c, at<double>(h, L.mom), P.E, st));
    CK(h, launch_coarse_factor(c, flags, st, pick >= 0 ? vars[pick] : -1));
    return MRCM_OK;
  };
  h->coarse_pivoted = h->prm.coarse_pivoting != 0;
  h->coarse_mf = P.mf && !h->coarse_pivoted;
  {
    Phase ph(h, MRCM_PH_COARSE_FACTOR, st);
    if (h->coarse_pivoted) {
      const mrcm_status rc = pivoted();
      if (rc != MRCM_OK) return rc;
    } else if (h->coarse_mf) {   // nested-dissection multifrontal LU (k_mf.cu), G read from the band copy
      CK(h, launch_coarse_assemble(c, at<double>(h, L.mom), P.E, st));
      CK(h, launch_mf_factor(mfdev(h), P, c.ab, flags, st));
    } else {
      CK(h, launch_coarse_assemble(c, at<double>(h, L.mom), P.E, st));
      CK(h, launch_coarse_factor_nopiv(c, flags, np_scratch, st));
    }
  }
  {
    Phase ph(h, MRCM_PH_COARSE_FACTOR, st);
    if (h->coarse_mf) {
    } else if (P.NC <= COARSE_DENSE_MAX) {
      CK(h, launch_coarse_invert(c, at<double>(h, L.Ginv), st));
    } else {
      CK(h, launch_coarse_blocks(c, st));
    }
  }
  CK(h, cudaStreamWaitEvent(st, h->join_ev, 0));
  int hf = 0;
  CK(h, cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if ((hf & FLAG_NOPIV_REJECTED) && !(hf & (FLAG_NONFINITE | FLAG_SINGULAR_LOCAL | FLAG_TIMEOUT))) {
    Phase ph(h, MRCM_PH_COARSE_FACTOR, st);
    CK(h, cudaMemsetAsync(flags, 0, sizeof(int), st));
    const mrcm_status rc = pivoted();
    if (rc != MRCM_OK) return rc;
    if (P.NC <= COARSE_DENSE_MAX) CK(h, launch_coarse_invert(c, at<double>(h, L.Ginv), st));
    else CK(h, launch_coarse_blocks(c, st));
    CK(h, cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    h->coarse_pivoted = true;
    h->coarse_mf = false;
  }
  if (hf & FLAG_NONFINITE) return fail(h, MRCM_ERR_INVALID_ARG, "K must be positive and finite");
  if (hf & FLAG_SINGULAR_LOCAL) return fail(h, MRCM_ERR_SINGULAR, "non-positive pivot in a local factorisation");
  if (hf & FLAG_SINGULAR_COARSE) return fail(h, MRCM_ERR_SINGULAR, "zero pivot in the coupling system");
  if (hf & FLAG_TIMEOUT) return fail(h, MRCM_ERR_TIMEOUT, "a bounded device wait gave up (local solve line copy)");
  h->factored = true;
  return MRCM_OK;
}

static mrcm_status apply_T(mrcm_handle h, const double* r, double* z, cudaStream_t st) {
  const Layout& L = h->lay;
  const Plan& P = h->plan;
  const bool fp32 = h->prm.local_prec == MRCM_PREC_FP32;
  Geo g = geo(h);
  // particular solutions and their side moments
  float* rho32 = fp32 ? at<float>(h, L.rho) : nullptr;   // FP32 right-hand sides, formed on the grid
  if (fp32) {
    Phase ph(h, MRCM_PH_STAGE, st);
    CK(h, launch_stage32(g, r, nullptr, rho32, st));
  }
  {
    Phase ph(h, MRCM_PH_PARTICULAR, st);
    // on the extended regions' Robin factors when l > 0 (the source term's basis function is built
    // there), on the subdomains' own Robin factors when l = 0
    const bool ext = P.l > 0;
    CK(h, launch_particular(g, at<void>(h, ext ? L.Linv_ohat_r : L.Linv_loc), ext ? L.LSo : L.LSl, fp32, r,
                            at<double>(h, L.psi0), at<double>(h, L.mom0), at<int>(h, L.flags), st, rho32));
  }
  // coupling system
  CoarseDev c = coarse(h);
  {
    Phase ph(h, MRCM_PH_COARSE_SOLVE, st);
    if (h->coarse_mf) {
      CK(h, launch_mf_solve(mfdev(h), c, at<double>(h, L.mom0), P.E, at<int>(h, L.flags), st));
    } else if (P.NC <= COARSE_DENSE_MAX) {
      CK(h, launch_coarse_apply(c, at<double>(h, L.Ginv), at<double>(h, L.mom0), P.E, st));
    } else {
      CK(h, launch_coarse_solve(c, at<double>(h, L.mom0), P.E, st));
    }
  }
  // reconstruction, into the buffer that makes the last smoothing sweep land in z: each sweep
  // reads one buffer (its residual needs the neighbours' values) and writes the other
  const int s = h->prm.smooth_steps;
  const bool mult = h->prm.smooth_kind == MRCM_SMOOTH_MULTIPLICATIVE;
  double* zb[2] = {z, at<double>(h, L.zt)};
  double* z_rec = mult ? z : zb[s & 1];
  {
    Phase ph(h, MRCM_PH_RECONSTRUCT, st);
    CK(h, launch_reconstruct(g, at<double>(h, L.psi0), at<double>(h, L.psi), tables(h).cidx, at<double>(h, L.gc),
                             z_rec, st));
  }
  if (h->keep_z0) CK(h, cudaMemcpyAsync(at<double>(h, L.z0), z_rec, 8 * ncell(h), cudaMemcpyDeviceToDevice, st));
  // smoothing sweeps (residual fused into the local solve): additive, all boxes from one residual
  // (ping-pong buffers); or multiplicative multicolour, one launch per colour updating z in place
  for (int it = 0; it < s; ++it) {
    if (mult) {
      Phase ph(h, MRCM_PH_SCHWARZ, st);
      for (int colour = 0; colour < (1 << P.dim); ++colour)
        CK(h, launch_schwarz(g, at<void>(h, L.Linv_ohat_d), L.LSo, fp32, r, z, z, at<int>(h, L.flags), colour, st));
    } else {
      const double* zin = zb[(s - it) & 1];
      double* zout = zb[(s - it - 1) & 1];
      if (fp32) {   // additive: every box from the same residual, r - A z formed once on the grid
        Phase ph(h, MRCM_PH_STAGE, st);
        CK(h, launch_stage32(g, r, zin, rho32, st));
      }
      Phase ph(h, MRCM_PH_SCHWARZ, st);
      CK(h, launch_schwarz(g, at<void>(h, L.Linv_ohat_d), L.LSo, fp32, r, zin, zout, at<int>(h, L.flags), -1, st,
                           rho32));
    }
  }
  return MRCM_OK;
}

mrcm_status mrcm_apply_precond(mrcm_handle h, const double* r, double* z, void* stream) {
  if (!h || !r || !z) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (!h->factored) return fail(h, MRCM_ERR_INVALID_ARG, "mrcm_factor_local has not completed");
  if (r == z) return fail(h, MRCM_ERR_INVALID_ARG, "r and z must not overlap");
  return apply_T(h, r, z, static_cast<cudaStream_t>(stream));
}

mrcm_status mrcm_apply_operator(mrcm_handle h, const double* v, double* w, void* stream) {
  if (!h || !v || !w) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (!h->factored) return fail(h, MRCM_ERR_INVALID_ARG, "mrcm_factor_local has not completed");
  CK(h, launch_matvec(geo(h), v, w, static_cast<cudaStream_t>(stream)));
  return MRCM_OK;
}

mrcm_status mrcm_rhs(mrcm_handle h, double* b, void* stream) {
  if (!h || !b) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (!h->factored) return fail(h, MRCM_ERR_INVALID_ARG, "mrcm_factor_local has not completed");
  CK(h, cudaMemcpyAsync(b, at<double>(h, h->lay.b), 8 * ncell(h), cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return MRCM_OK;
}

mrcm_status mrcm_gmres_solve(mrcm_handle h, const double* b, double* p, double* ux, double* uy, double* uz,
                             mrcm_result* result, void* stream) {
  if (!h || !p || !result) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (!h->factored) return fail(h, MRCM_ERR_INVALID_ARG, "mrcm_factor_local has not completed");
  (void)uz;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout& L = h->lay;
  const size_t n = ncell(h);
  const int m = h->prm.restart, ldh = m + 1;
  Geo g = geo(h);
  const double* bb = b ? b : at<double>(h, L.b);
  double* V = at<double>(h, L.V);
  double* Z = at<double>(h, L.Z);
  double* w = at<double>(h, L.w);
  double* Hs = at<double>(h, L.Hs);
  double* H = Hs;
  double* cs = H + (size_t)ldh * m;
  double* sn = cs + m;
  double* gv = sn + m;
  double* out = gv + (m + 1);        // [0..3]
  double* wn2 = out + 4;
  double* beta_d = wn2 + 1;
  double* bnorm_d = beta_d + 1;
  double* partials = at<double>(h, L.red);
  unsigned* counter = reinterpret_cast<unsigned*>(partials + RED_DOUBLES);
  unsigned* bar = counter + 1;
  int* flags = at<int>(h, L.flags);
  bool fused = true;  // fused Arnoldi kernel, unless the vector is too long for one co-resident wave
  if (!h->rb) {
    CK(h, cudaHostAlloc(reinterpret_cast<void**>(&h->rb), 2 * sizeof(mrcm_ctx::StepReadback), cudaHostAllocDefault));
    for (cudaEvent_t& e : h->rb_ev) CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  std::vector<double> hist;
  result->iterations = 0;
  result->restarts = 0;
  result->status = MRCM_OK;
  result->latency_ms = 0.0;
  result->queue_ms = 0.0;
  double hb[2] = {0, 0};
  CK(h, launch_norm2(bb, n, partials, counter, bnorm_d, st));
  CK(h, cudaMemcpyAsync(hb, bnorm_d, 8, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const double bnorm = hb[0];
  result->bnorm = bnorm;
  const bool rel = h->prm.tol_relative != 0;
  if (rel && bnorm == 0.0) {
    CK(h, cudaMemsetAsync(p, 0, 8 * n, st));
    result->abs_res = result->rel_res = 0.0;
    result->history_len = 0;
    if (ux || uy) {
      const double* bcp[4];
      bc_ptrs(h, bcp);
      CK(h, launch_fluxes(g, h->bc_kind, bcp, p, ux, uy, st));
    }
    CK(h, cudaStreamSynchronize(st));
    return MRCM_OK;
  }
  const double tol_abs = rel ? h->prm.tol * bnorm : h->prm.tol;
  CK(h, launch_residual_norm(g, bb, p, V, partials, counter, beta_d, st));
  double beta = 0.0;
  CK(h, cudaMemcpyAsync(&beta, beta_d, 8, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  hist.push_back(beta);
  int it = 0;
  mrcm_status status = MRCM_OK;
  while (true) {
    if (beta <= tol_abs) break;
    if (it >= h->prm.max_iter) {
      status = MRCM_ERR_NOT_CONVERGED;
      break;
    }
    CK(h, launch_scale(V, beta_d, n, V, st));
    CK(h, cudaMemsetAsync(gv, 0, 8 * (m + 1), st));
    k_set<<<1, 1, 0, st>>>(gv, beta);
    CK(h, cudaGetLastError());
    // Steps are pipelined by one: step j+1 is enqueued before the host reads step j's residual
    // estimate, so the device never waits for the host.  When step j ends the cycle, the extra step
    // has only written V_{j+2}, Z_{j+1}, column j+1 of H, rotation j+1 and g_{j+1..j+2}, none of
    // which the solution update over columns 0..j reads.
    int k = 0;
    int pend = -1;  // step whose read-back is in flight
    for (int j = 0; j <= m; ++j) {
      const bool launch = j < m && it + (pend >= 0 ? 1 : 0) < h->prm.max_iter;
      if (launch) {
        double* vj = V + (size_t)j * n;
        double* zj = Z + (size_t)j * n;
        mrcm_status rc = apply_T(h, vj, zj, st);
        if (rc != MRCM_OK) return rc;
        double* col = H + (size_t)j * ldh;
        {
          Phase ph(h, MRCM_PH_KRYLOV, st);
          cudaError_t ea = cudaErrorNotSupported;
          if (fused)
            ea = launch_arnoldi(g, zj, V, j, n, H, ldh, cs, sn, gv, out, w, at<double>(h, L.apart),
                                at<double>(h, L.atot), at<double>(h, L.aT), bar, flags, st);
          if (ea == cudaErrorNotSupported) {
            fused = false;
            (void)cudaGetLastError();
            CK(h, launch_matvec_dot(g, zj, V, w, partials, counter, col, st));
            // launch_matvec_dot writes (w, v0) to col[0] and ||w||^2 to col[1]; move the latter
            CK(h, cudaMemcpyAsync(wn2, col + 1, 8, cudaMemcpyDeviceToDevice, st));
            for (int i = 1; i <= j; ++i)
              CK(h, launch_mgs_pass(V + (size_t)(i - 1) * n, col + (i - 1), V + (size_t)i * n, n, w, partials, counter,
                                    col + i, 0, st));
            CK(h, launch_mgs_pass(V + (size_t)j * n, col + j, nullptr, n, w, partials, counter, col + j + 1, 1, st));
            CK(h, launch_givens(H, cs, sn, gv, j, ldh, wn2, out, st));
            // v_{j+1} = w / h_{j+1,j}; the rotation has zeroed col[j+1], out[1] keeps the value
            CK(h, launch_scale(w, out + 1, n, V + (size_t)(j + 1) * n, st));
          } else {
            CK(h, ea);
          }
        }
        mrcm_ctx::StepReadback* slot = h->rb + (j & 1);
        CK(h, cudaMemcpyAsync(slot->out, out, 24, cudaMemcpyDeviceToHost, st));
        CK(h, cudaMemcpyAsync(&slot->flags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(h, cudaEventRecord(h->rb_ev[j & 1], st));
      }
      if (pend >= 0) {
        CK(h, cudaEventSynchronize(h->rb_ev[pend & 1]));
        const mrcm_ctx::StepReadback* slot = h->rb + (pend & 1);
        const double ho[3] = {slot->out[0], slot->out[1], slot->out[2]};
        ++it;
        if (slot->flags & FLAG_TIMEOUT)
          return fail(h, MRCM_ERR_TIMEOUT, "a bounded device wait gave up (Arnoldi grid barrier or local-solve line copy)");
        if (h->cancel && *h->cancel) {
          result->iterations = it;
          return fail(h, MRCM_ERR_CANCELLED, "cancelled");
        }
        hist.push_back(ho[0]);
        k = pend + 1;
        const bool breakdown = ho[1] <= 1e-14 * ho[2];
        if (ho[0] <= tol_abs || breakdown || it >= h->prm.max_iter) break;
      }
      if (!launch) break;
      pend = j;
    }
    CK(h, launch_update(p, Z, n, H, gv, k, ldh, at<double>(h, L.atot), st));
    CK(h, launch_residual_norm(g, bb, p, V, partials, counter, beta_d, st));
    CK(h, cudaMemcpyAsync(&beta, beta_d, 8, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    hist.push_back(beta);
    if (beta <= tol_abs) break;
    if (it >= h->prm.max_iter) {
      status = MRCM_ERR_NOT_CONVERGED;
      break;
    }
    result->restarts++;
  }
  if (ux || uy) {
    const double* bcp[4];
    bc_ptrs(h, bcp);
    CK(h, launch_fluxes(g, h->bc_kind, bcp, p, ux, uy, st));
    CK(h, cudaStreamSynchronize(st));
  }
  result->iterations = it;
  result->status = status;
  result->abs_res = beta;
  result->rel_res = bnorm > 0 ? beta / bnorm : 0.0;
  const int cap = result->history ? result->history_cap : 0;
  const int nh = (int)hist.size();
  for (int i = 0; i < nh && i < cap; ++i) result->history[i] = hist[i];
  result->history_len = nh < cap ? nh : cap;
  if (status != MRCM_OK) fail(h, status, "max_iter reached before the tolerance");
  return status;
}

mrcm_status mrcm_solve_host(mrcm_handle h, const double* K_host, double* p_host, mrcm_result* result, void* stream) {
  if (!h || !p_host || !result) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = ncell(h);
  if (K_host) {
    CK(h, cudaMemcpyAsync(at<double>(h, h->lay.K), K_host, 8 * n, cudaMemcpyHostToDevice, st));
    if (h->iso) CK(h, cudaMemcpyAsync(at<double>(h, h->lay.Ky), K_host, 8 * n, cudaMemcpyHostToDevice, st));
  }
  mrcm_status rc = mrcm_factor_local(h, stream);
  if (rc != MRCM_OK) return rc;
  double* p = at<double>(h, h->lay.tmpv);
  CK(h, cudaMemsetAsync(p, 0, 8 * n, st));
  rc = mrcm_gmres_solve(h, nullptr, p, nullptr, nullptr, nullptr, result, stream);
  if (rc != MRCM_OK && rc != MRCM_ERR_NOT_CONVERGED) return rc;
  CK(h, cudaMemcpyAsync(p_host, p, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return rc;
}

void mrcm_destroy(mrcm_handle h) { delete h; }

int64_t mrcm_launch_count(void) { return g_launches.load(); }

mrcm_status mrcm_coarse_method(mrcm_handle h, int32_t* method) {
  if (!h || !method) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  if (!h->factored) return fail(h, MRCM_ERR_INVALID_ARG, "the handle is not factored");
  if (h->coarse_mf) *method = MRCM_COARSE_MULTIFRONTAL;
  else if (h->plan.NC <= COARSE_DENSE_MAX) *method = MRCM_COARSE_INVERSE;
  else *method = h->coarse_pivoted ? MRCM_COARSE_BAND_PIVOTED : MRCM_COARSE_BAND;
  return MRCM_OK;
}

mrcm_status mrcm_measure_fp64_peak(double* tflops_out, void* stream) {
  if (!tflops_out) return fail(nullptr, MRCM_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(nullptr, MRCM_ERR_CUDA, "no CUDA device");
  const int blocks = 4 * sms, threads = 256, iters = 1024;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.0f;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  // the sink is never written for these operands; a null pointer is never dereferenced
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) err = mrcm::launch_dfma_probe(nullptr, blocks, threads, iters, st);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(nullptr, MRCM_ERR_CUDA, cudaGetErrorString(err));
  const double fma = (double)blocks * threads * iters * 32.0;
  *tflops_out = 2.0 * fma / (best * 1e-3) / 1e12;
  return MRCM_OK;
}

mrcm_status mrcm_profile_enable(mrcm_handle h, int32_t enable) {
  if (!h) return fail(h, MRCM_ERR_INVALID_ARG, "null handle");
  h->prof = enable != 0;
  return MRCM_OK;
}

mrcm_status mrcm_profile_select(mrcm_handle h, uint32_t phase_mask, int32_t every) {
  if (!h) return fail(h, MRCM_ERR_INVALID_ARG, "null handle");
  if (every < 1) return fail(h, MRCM_ERR_INVALID_ARG, "every must be >= 1");
  h->prof_mask = phase_mask;
  h->prof_every = every;
  for (long long& c : h->ph_seen) c = 0;
  return MRCM_OK;
}

mrcm_status mrcm_profile_read(mrcm_handle h, double* ms, int64_t* launches, int32_t cap, int32_t reset, void* stream) {
  if (!h) return fail(h, MRCM_ERR_INVALID_ARG, "null handle");
  CK(h, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  for (size_t i = 0; i < h->ev_used; ++i) {
    float t = 0.f;
    CK(h, cudaEventElapsedTime(&t, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
    h->ph_ms[h->ev_phase[i]] += t;
  }
  h->ev_used = 0;
  const int nc = cap < MRCM_PHASES ? cap : MRCM_PHASES;
  for (int i = 0; i < nc; ++i) {
    if (ms) ms[i] = h->ph_ms[i];
    if (launches) launches[i] = h->ph_launch[i];
  }
  if (reset)
    for (int i = 0; i < MRCM_PHASES; ++i) {
      h->ph_ms[i] = 0.0;
      h->ph_launch[i] = 0;
    }
  return MRCM_OK;
}

mrcm_status mrcm_debug_get(mrcm_handle h, int32_t what, double* host_out, size_t cap, size_t* len, void* stream) {
  if (!h || !len) return fail(h, MRCM_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout& L = h->lay;
  const Plan& P = h->plan;
  const size_t n = ncell(h);
  size_t off = 0, cnt = 0;
  switch (what) {
    case MRCM_DBG_TRANS: {
      const size_t nx = h->n[0], ny = h->n[1];
      *len = (nx + 1) * ny + nx * (ny + 1);
      if (!host_out) return MRCM_OK;
      const size_t c1 = std::min(cap, (nx + 1) * ny);
      CK(h, cudaMemcpyAsync(host_out, at<double>(h, L.Tx), 8 * c1, cudaMemcpyDeviceToHost, st));
      if (cap > c1)
        CK(h, cudaMemcpyAsync(host_out + c1, at<double>(h, L.Ty), 8 * std::min(cap - c1, nx * (ny + 1)), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      return MRCM_OK;
    }
    case MRCM_DBG_PHI: off = L.phi; cnt = (size_t)P.S * 16 * P.nq * L.smax; break;
    case MRCM_DBG_PSI: off = L.psi; cnt = 4 * P.nq * n; break;
    case MRCM_DBG_MOMENTS: off = L.mom; cnt = (size_t)P.S * 32 * P.nq * P.nq; break;
    case MRCM_DBG_COARSE: off = L.gc; cnt = P.NC; break;
    case MRCM_DBG_ZMRCM:
      if (!host_out) {
        h->keep_z0 = true;  // capture the multiscale solution from now on
        *len = n;
        return MRCM_OK;
      }
      off = L.z0;
      cnt = n;
      break;
    case MRCM_DBG_G: {
      const size_t NC = P.NC;
      const int nq = P.nq, nf = 4 * nq;
      *len = NC * NC;
      if (!host_out) return MRCM_OK;
      std::vector<double> mom((size_t)P.S * 32 * nq * nq);
      CK(h, cudaMemcpyAsync(mom.data(), at<double>(h, L.mom), 8 * mom.size(), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      // moment of function fn of subdomain t on side k against test qt: [F, |f|P]
      auto M = [&](int t, int k, int fn, int qt, int which) {
        return mom[((((size_t)t * 4 + k) * nf + fn) * nq + qt) * 2 + which];
      };
      std::vector<double> G(NC * NC, 0.0);
      for (int e = 0; e < P.E; ++e) {
        const int a = P.iface[3 * e], s = P.iface[3 * e + 1], s2 = P.iface[3 * e + 2];
        for (int qt = 0; qt < nq; ++qt) {
          const size_t rf = (size_t)2 * nq * e + qt, rp = rf + nq;
          for (int r = 0; r < 4; ++r)
            for (int q = 0; q < nq; ++q) {
              if (P.rank[6 * s + r] >= 0) {
                const size_t col = (size_t)(P.off[s] + P.rank[6 * s + r]) * nq + q;
                G[rf * NC + col] += M(s, 2 * a + 1, r * nq + q, qt, 0);
                G[rp * NC + col] += M(s, 2 * a + 1, r * nq + q, qt, 1);
              }
              if (P.rank[6 * s2 + r] >= 0) {
                const size_t col = (size_t)(P.off[s2] + P.rank[6 * s2 + r]) * nq + q;
                G[rf * NC + col] += M(s2, 2 * a, r * nq + q, qt, 0);
                G[rp * NC + col] -= M(s2, 2 * a, r * nq + q, qt, 1);
              }
            }
        }
      }
      std::memcpy(host_out, G.data(), 8 * std::min(cap, G.size()));
      return MRCM_OK;
    }
    default: return fail(h, MRCM_ERR_INVALID_ARG, "unknown debug array");
  }
  *len = cnt;
  if (!host_out) return MRCM_OK;
  CK(h, cudaMemcpyAsync(host_out, h->ws + off, 8 * std::min(cap, cnt), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  return MRCM_OK;
}

}  // extern "C"
