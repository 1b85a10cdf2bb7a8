// Host planner: validation, partition and coupling numbering (MRCM-OS step 1, Sec. 2.1), workspace
// layout.  Integer work only; the tables it exports match the oracle's bit for bit.
#include <algorithm>
#include <climits>
#include <cmath>
#include <functional>
#include <sstream>

#include "internal.h"

namespace mrcm {

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static bool plan_mf(Plan& P);

std::string make_plan(const mrcm_problem& p, const mrcm_params& q, Plan& P) {
  std::ostringstream why;
  if (p.dim != 2 && p.dim != 3) return "dim must be 2 or 3";
  for (int a = 0; a < 3; ++a) {
    if (p.n[a] < 1) return "grid sizes must be >= 1";
    if (!finite_pos(p.h[a])) return "cell sizes must be positive and finite";
    if (q.sub[a] < 1) return "subdomain sizes must be >= 1";
  }
  if (p.dim == 2 && (p.n[2] != 1 || q.sub[2] != 1)) return "2-D problems need n[2] == 1 and sub[2] == 1";
  if ((long long)p.n[0] * p.n[1] * p.n[2] > (1LL << 31) - 1) return "grid too large";
  // the last subdomain along an axis takes the remainder when sub does not divide the grid; the
  // oversampling stays below the size of every subdomain so hat-Omega keeps the Robin sides of Omega
  for (int a = 0; a < p.dim; ++a) {
    const int m = (p.n[a] + q.sub[a] - 1) / q.sub[a], last = p.n[a] - (m - 1) * q.sub[a];
    if (q.oversample < 0 || q.oversample >= q.sub[a] || (m > 1 && q.oversample >= last))
      return "oversampling must satisfy 0 <= l < the size of every subdomain on every axis";
  }
  if (q.oversample < 0) return "oversampling must be >= 0";
  if (q.smooth_steps < 0) return "smooth_steps must be >= 0";
  if (!finite_pos(q.alpha)) return "alpha must be positive and finite";
  if (!finite_pos(q.tol)) return "tol must be positive and finite";
  if (q.restart < 1 || q.restart > 256) return "restart must be in 1..256";
  if (q.max_iter < 1) return "max_iter must be >= 1";
  if (q.local_prec != MRCM_PREC_FP64 && q.local_prec != MRCM_PREC_FP32) return "local_prec must be FP64 or FP32";
  if (q.smooth_kind != MRCM_SMOOTH_ADDITIVE && q.smooth_kind != MRCM_SMOOTH_MULTIPLICATIVE)
    return "smooth_kind must be MRCM_SMOOTH_ADDITIVE or MRCM_SMOOTH_MULTIPLICATIVE";
  if (q.iface_degree != 0 && q.iface_degree != 1) return "iface_degree must be 0 or 1";
  if (q.coarse_pivoting != 0 && q.coarse_pivoting != 1) return "coarse_pivoting must be 0 or 1";
  if (q.refine_setup < 0 || q.refine_setup > 2) return "refine_setup must be 0, 1 or 2";
  if (q.coarse_solver != 0 && q.coarse_solver != 1) return "coarse_solver must be 0 or 1";
  bool any_dirichlet = false;
  for (int s = 0; s < 6; ++s) {
    if (p.bc_kind[s] != MRCM_BC_DIRICHLET && p.bc_kind[s] != MRCM_BC_NEUMANN) return "bc_kind must be 0 or 1";
    if (s / 2 < p.dim && p.bc_kind[s] == MRCM_BC_DIRICHLET) any_dirichlet = true;
  }
  if (!any_dirichlet) return "at least one Dirichlet side is required (pure Neumann is singular)";

  P = Plan();
  P.dim = p.dim;
  for (int a = 0; a < 3; ++a) {
    P.n[a] = p.n[a];
    P.sub[a] = q.sub[a];
    P.m[a] = (p.n[a] + q.sub[a] - 1) / q.sub[a];
  }
  P.l = q.oversample;
  P.nq = 1 + q.iface_degree * (p.dim - 1);
  P.S = P.m[0] * P.m[1] * P.m[2];
  const int S = P.S;
  P.box.assign(6 * S, 0);
  P.obox.assign(6 * S, 0);
  P.mask.assign(S, 0);
  P.N.assign(S, 0);
  P.off.assign(S, 0);
  P.rank.assign(6 * S, -1);
  std::vector<int> coord(3 * S);
  for (int s = 0; s < S; ++s) {
    const int idx[3] = {s % P.m[0], (s / P.m[0]) % P.m[1], s / (P.m[0] * P.m[1])};
    for (int a = 0; a < 3; ++a) {
      coord[3 * s + a] = idx[a];
      const int lo = idx[a] * P.sub[a], hi = std::min(lo + P.sub[a], P.n[a]);
      P.box[6 * s + a] = lo;
      P.box[6 * s + 3 + a] = hi;
      if (a < P.dim) {
        P.obox[6 * s + a] = std::max(lo - P.l, 0);
        P.obox[6 * s + 3 + a] = std::min(hi + P.l, P.n[a]);
        if (idx[a] > 0) P.mask[s] |= 1 << (2 * a);
        if (idx[a] < P.m[a] - 1) P.mask[s] |= 1 << (2 * a + 1);
      } else {
        P.obox[6 * s + a] = lo;
        P.obox[6 * s + 3 + a] = hi;
      }
    }
    int r = 0;
    for (int k = 0; k < 6; ++k)
      if (P.mask[s] >> k & 1) P.rank[6 * s + k] = r++;
    P.N[s] = r;
  }
  int acc = 0;
  for (int s = 0; s < S; ++s) {
    P.off[s] = acc;
    acc += P.N[s];
  }
  P.E2 = acc;
  const int stride[3] = {1, P.m[0], P.m[0] * P.m[1]};
  for (int a = 0; a < P.dim; ++a)
    for (int s = 0; s < S; ++s)
      if (coord[3 * s + a] < P.m[a] - 1) {
        P.iface.push_back(a);
        P.iface.push_back(s);
        P.iface.push_back(s + stride[a]);
      }
  P.E = (int)P.iface.size() / 3;
  if (2 * P.E != P.E2) return "internal: coupling system is not square";
  // a linear side function needs two faces on its side, else it vanishes there and G is singular
  if (P.nq > 1)
    for (int s = 0; s < S; ++s)
      for (int k = 0; k < 2 * P.dim; ++k)
        if (P.mask[s] >> k & 1)
          for (int b = 0; b < P.dim; ++b)
            if (b != k / 2 && P.box[6 * s + 3 + b] - P.box[6 * s + b] < 2)
              return "iface_degree 1 needs at least two faces on every Robin side";
  P.NC = P.E2 * P.nq;
  // banded home order and band widths of G: row q of the flux (pressure) rows of interface e sits
  // at unknown q of the side it is homed at, i.e. at row_home * nq + q
  P.row_home.assign(P.E2, 0);
  P.kl = P.ku = 0;
  const int nq = P.nq;
  for (int e = 0; e < P.E; ++e) {
    const int a = P.iface[3 * e], s = P.iface[3 * e + 1], s2 = P.iface[3 * e + 2];
    const int rf = P.off[s] + P.rank[6 * s + 2 * a + 1];
    const int rp = P.off[s2] + P.rank[6 * s2 + 2 * a];
    P.row_home[2 * e] = rf;
    P.row_home[2 * e + 1] = rp;
    for (int row0 : {rf, rp}) {
      for (int t : {s, s2}) {
        const int c0 = P.off[t] * nq, c1 = (P.off[t] + P.N[t]) * nq - 1;
        P.kl = std::max(P.kl, row0 * nq + nq - 1 - c0);
        P.ku = std::max(P.ku, c1 - row0 * nq);
      }
    }
  }
  P.mf = false;
  if (p.dim == 2 && P.NC > 0 && q.coarse_solver == 0 && q.coarse_pivoting == 0) P.mf = plan_mf(P);
  if (!P.mf) {
    P.mf_front.clear();
    P.mf_idx.clear();
    P.mf_asm.clear();
    P.mf_map.clear();
    P.mf_task.clear();
    P.mf_fbuf = P.mf_vbuf = 0;
  }
  return std::string();
}

// Nested dissection of the subdomain grid into fronts for the multifrontal factorisation of G.
// Interface unknowns (a flux row and a pressure row homed at each, so rows and columns share the
// index) are grouped per interface; a rectangle of subdomains eliminates the interfaces of its
// separator (the cut between its halves) after its halves, or all its interior interfaces when it
// is a leaf.  The structural nonzeros of G couple the interfaces of one or two neighbouring
// subdomains, so a rectangle's remaining couplings after elimination are its boundary interfaces.
// Returns false (multifrontal path not used) when a front exceeds the kernels' limits.
static bool plan_mf(Plan& P) {
  const int mx = P.m[0], my = P.m[1], nq = P.nq;
  const int kv = P.kl + P.ku, ldab = 2 * P.kl + P.ku + 1;
  // interface ids by (axis, lower subdomain)
  std::vector<int> vid(2 * (size_t)mx * my, -1);
  for (int e = 0; e < P.E; ++e) vid[(size_t)P.iface[3 * e] * mx * my + P.iface[3 * e + 1]] = e;
  auto X = [&](int I, int J) { return vid[(size_t)J * mx + I]; };                      // (I,J)-(I+1,J)
  auto Y = [&](int I, int J) { return vid[(size_t)mx * my + (size_t)J * mx + I]; };    // (I,J)-(I,J+1)
  auto add_unknowns = [&](int e, std::vector<int>& out) {
    for (int q = 0; q < nq; ++q) out.push_back(P.row_home[2 * e] * nq + q);
    for (int q = 0; q < nq; ++q) out.push_back(P.row_home[2 * e + 1] * nq + q);
  };
  P.mf_front.clear();
  P.mf_idx.clear();
  std::vector<int> level;
  bool ok = true;
  std::function<int(int, int, int, int)> build = [&](int x0, int x1, int y0, int y1) -> int {
    std::vector<int> piv, ch;
    if ((x1 - x0) * (y1 - y0) <= MF_LEAF) {
      for (int J = y0; J < y1; ++J)
        for (int I = x0; I + 1 < x1; ++I) piv.push_back(X(I, J));
      for (int J = y0; J + 1 < y1; ++J)
        for (int I = x0; I < x1; ++I) piv.push_back(Y(I, J));
    } else if (x1 - x0 >= y1 - y0) {
      const int xm = (x0 + x1) / 2;
      ch = {build(x0, xm, y0, y1), build(xm, x1, y0, y1)};
      for (int J = y0; J < y1; ++J) piv.push_back(X(xm - 1, J));
    } else {
      const int ym = (y0 + y1) / 2;
      ch = {build(x0, x1, y0, ym), build(x0, x1, ym, y1)};
      for (int I = x0; I < x1; ++I) piv.push_back(Y(I, ym - 1));
    }
    ch.erase(std::remove(ch.begin(), ch.end(), -1), ch.end());
    if (piv.empty() && ch.empty()) return -1;
    std::vector<int> bnd;
    for (int J = y0; J < y1; ++J) {
      if (x0 > 0) bnd.push_back(X(x0 - 1, J));
      if (x1 < mx) bnd.push_back(X(x1 - 1, J));
    }
    for (int I = x0; I < x1; ++I) {
      if (y0 > 0) bnd.push_back(Y(I, y0 - 1));
      if (y1 < my) bnd.push_back(Y(I, y1 - 1));
    }
    MfFront fr{};
    fr.io = (int)P.mf_idx.size();
    for (int e : piv) add_unknowns(e, P.mf_idx);
    fr.np = (int)P.mf_idx.size() - fr.io;
    for (int e : bnd) add_unknowns(e, P.mf_idx);
    fr.nu = (int)P.mf_idx.size() - fr.io - fr.np;
    fr.nch = (int)ch.size();
    int lv = 0;
    for (int c = 0; c < fr.nch; ++c) {
      fr.ch[c] = ch[c];
      lv = std::max(lv, level[ch[c]] + 1);
    }
    if (fr.np > MF_MAX_NP || fr.np == 0) ok = false;
    P.mf_front.push_back(fr);
    level.push_back(lv);
    return (int)P.mf_front.size() - 1;
  };
  const int root = build(0, mx, 0, my);
  const int nf = (int)P.mf_front.size();
  if (!ok || root != nf - 1 || nf == 0) return false;
  for (int f = 0; f < nf; ++f) P.mf_front[f].par = -1;
  for (int f = 0; f < nf; ++f)
    for (int c = 0; c < P.mf_front[f].nch; ++c) P.mf_front[P.mf_front[f].ch[c]].par = f;
  // the front that eliminates each unknown
  std::vector<int> efront(P.NC, -1);
  for (int f = 0; f < nf; ++f) {
    const MfFront& fr = P.mf_front[f];
    for (int t = 0; t < fr.np; ++t) {
      int& ef = efront[P.mf_idx[fr.io + t]];
      if (ef >= 0) return false;
      ef = f;
    }
  }
  for (int u = 0; u < P.NC; ++u)
    if (efront[u] < 0) return false;
  // structural nonzeros of G, each assembled by the first front that eliminates its row or column
  std::vector<std::vector<std::pair<int, int>>> nz(nf);
  for (int e = 0; e < P.E; ++e) {
    const int s = P.iface[3 * e + 1], s2 = P.iface[3 * e + 2];
    for (int qt = 0; qt < nq; ++qt)
      for (int row : {P.row_home[2 * e] * nq + qt, P.row_home[2 * e + 1] * nq + qt})
        for (int t : {s, s2})
          for (int col = P.off[t] * nq; col < (P.off[t] + P.N[t]) * nq; ++col)
            nz[std::min(efront[row], efront[col])].push_back({row, col});
  }
  std::vector<int> pos(P.NC, -1);
  P.mf_asm.clear();
  P.mf_map.clear();
  size_t fo = 0, vo = 0;
  P.mf_max_np = P.mf_max_f = P.mf_mcap = 0;
  for (int f = 0; f < nf; ++f) {
    MfFront& fr = P.mf_front[f];
    const int fs = fr.np + fr.nu;
    for (int t = 0; t < fs; ++t) pos[P.mf_idx[fr.io + t]] = t;
    fr.ao = (int)P.mf_asm.size() / 2;
    for (auto [row, col] : nz[f]) {
      if (pos[row] < 0 || pos[col] < 0) return false;
      const long long src = (long long)kv + row - col + (long long)col * ldab;
      if (src > INT32_MAX) return false;
      P.mf_asm.push_back(pos[row] * fs + pos[col]);
      P.mf_asm.push_back((int)src);
    }
    fr.na = (int)P.mf_asm.size() / 2 - fr.ao;
    for (int c = 0; c < fr.nch; ++c) {
      const MfFront& cf = P.mf_front[fr.ch[c]];
      fr.mo[c] = (int)P.mf_map.size();
      for (int t = 0; t < cf.nu; ++t) {
        const int p = pos[P.mf_idx[cf.io + cf.np + t]];
        if (p < 0) return false;
        P.mf_map.push_back(p);
      }
    }
    for (int t = 0; t < fs; ++t) pos[P.mf_idx[fr.io + t]] = -1;
    fr.fo = (long long)fo;
    fo += (size_t)fs * fs + (size_t)fr.nu * fr.np;
    fr.vo = (int)vo;
    vo += fs;
    P.mf_max_np = std::max(P.mf_max_np, fr.np);
    P.mf_max_f = std::max(P.mf_max_f, fs);
    P.mf_mcap = std::max(P.mf_mcap, std::min(24576, std::max(fr.np * (fs + 1), fr.nu * (fr.np + 1))));
  }
  if (vo > (size_t)INT32_MAX) return false;
  P.mf_fbuf = fo;
  P.mf_vbuf = vo;
  // levels and the tile tasks of each level
  const int nl = *std::max_element(level.begin(), level.end()) + 1;
  P.mf_level.assign(nl + 1, 0);
  P.mf_order.clear();
  P.mf_task.clear();
  P.mf_task_b.assign(nl + 1, 0);
  P.mf_task_c.assign(nl + 1, 0);
  std::vector<int> tc;
  for (int L = 0; L < nl; ++L) {
    P.mf_level[L] = (int)P.mf_order.size();
    P.mf_task_b[L] = (int)P.mf_task.size() / 4;
    for (int f = 0; f < nf; ++f)
      if (level[f] == L) P.mf_order.push_back(f);
    for (int i = P.mf_level[L]; i < (int)P.mf_order.size(); ++i) {
      const int f = P.mf_order[i];
      const MfFront& fr = P.mf_front[f];
      for (int t = 0; t < fr.nu; t += MF_TILE) {
        P.mf_task.insert(P.mf_task.end(), {f, 0, 0, t});   // D columns t ..
        P.mf_task.insert(P.mf_task.end(), {f, 1, t, 0});   // B rows t ..
      }
    }
    P.mf_task_c[L] = (int)P.mf_task.size() / 4;
    for (int i = P.mf_level[L]; i < (int)P.mf_order.size(); ++i) {
      const int f = P.mf_order[i];
      const MfFront& fr = P.mf_front[f];
      for (int r = 0; r < fr.nu; r += MF_TILE)
        for (int c = 0; c < fr.nu; c += MF_TILE) P.mf_task.insert(P.mf_task.end(), {f, 2, r, c});
    }
  }
  P.mf_level[nl] = (int)P.mf_order.size();
  P.mf_task_b[nl] = P.mf_task_c[nl] = (int)P.mf_task.size() / 4;
  // B and C task starts: a level's S tasks follow its D / B tasks, so the B range of level L is
  // [task_b[L], task_c[L]) and the C range [task_c[L], task_b[L + 1])
  return true;
}

std::vector<int32_t> export_plan(const Plan& P) {
  std::vector<int32_t> out = {P.dim, P.n[0], P.n[1], P.n[2], P.sub[0], P.sub[1], P.sub[2], P.l, P.S, P.E2, P.E};
  for (int s = 0; s < P.S; ++s) {
    for (int t = 0; t < 6; ++t) out.push_back(P.box[6 * s + t]);
    for (int t = 0; t < 6; ++t) out.push_back(P.obox[6 * s + t]);
    out.push_back(P.mask[s]);
    out.push_back(P.N[s]);
    out.push_back(P.off[s]);
  }
  for (int e = 0; e < P.E; ++e)
    for (int t = 0; t < 3; ++t) out.push_back(P.iface[3 * e + t]);
  // face arrays: axis a has n[a] + 1 entries along a
  long long ext[3][3], size[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) ext[a][b] = P.n[b] + (a == b ? 1 : 0);
    size[a] = ext[a][0] * ext[a][1] * ext[a][2];
  }
  const long long aoff[3] = {0, size[0], size[0] + size[1]};
  for (int s = 0; s < P.S; ++s) {
    const int* lo = &P.box[6 * s];
    const int* hi = &P.box[6 * s + 3];
    for (int k = 0; k < 6; ++k) {
      if (!(P.mask[s] >> k & 1)) continue;
      const int a = k / 2, d = k % 2;
      int others[2], t = 0;
      for (int b = 0; b < 3; ++b)
        if (b != a) others[t++] = b;
      const int b1 = others[0], b2 = others[1];
      const int plane = d == 0 ? lo[a] : hi[a];
      out.push_back((hi[b1] - lo[b1]) * (hi[b2] - lo[b2]));
      for (int t2 = lo[b2]; t2 < hi[b2]; ++t2)
        for (int t1 = lo[b1]; t1 < hi[b1]; ++t1) {
          long long pos[3];
          pos[a] = plane;
          pos[b1] = t1;
          pos[b2] = t2;
          out.push_back((int32_t)(aoff[a] + pos[0] + ext[a][0] * (pos[1] + ext[a][1] * pos[2])));
        }
    }
  }
  return out;
}

static size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(const Plan& P, const mrcm_params& q) {
  Layout L{};
  const size_t nx = P.n[0], ny = P.n[1];
  const size_t n = nx * ny * P.n[2];
  const size_t S = P.S;
  L.elt = q.local_prec == MRCM_PREC_FP32 ? 4 : 8;
  L.wl = P.sub[0];
  L.hl = P.sub[1];
  L.wo = P.sub[0] + 2 * P.l;
  L.ho = P.sub[1] + 2 * P.l;
  auto packed = [](int w) { return ((w * (w + 1) / 2) + 3) / 4 * 4; };
  L.LSl = packed(L.wl);
  L.LSo = packed(L.wo);
  L.ldab = 2 * P.kl + P.ku + 1;
  L.smax = std::max(P.sub[0], P.sub[1]);
  L.m = q.restart;
  L.nred = RED_BLOCKS;
  const size_t E2 = P.E2, NC = P.NC, nq = P.nq;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = al(o + std::max<size_t>(bytes, 1));
    return at;
  };
  L.K = take(8 * n);
  L.Ky = take(8 * n);
  L.Tx = take(8 * (nx + 1) * ny);
  L.Ty = take(8 * nx * (ny + 1));
  L.b = take(8 * n);
  L.f = take(8 * n);
  L.bcv = take(8 * 4 * std::max(nx, ny));
  L.Linv_loc = take(L.elt * S * box_stride(L.wl, L.hl, L.LSl));
  L.Linv_ohat_r = take(P.l > 0 ? L.elt * S * box_stride(L.wo, L.ho, L.LSo) : 0);
  L.Linv_ohat_d = take(q.smooth_steps > 0 ? L.elt * S * box_stride(L.wo, L.ho, L.LSo) : 0);
  // the FP32 informed and basis solves refine once against the FP64 box operator, whose line
  // coefficients the factorisation keeps here
  const bool refine = q.local_prec == MRCM_PREC_FP32 && q.refine_setup;
  L.coef_o = take(refine && q.refine_setup == 1 && P.l > 0 ? 8 * 3 * S * (size_t)L.wo * L.ho : 0);
  L.coef_l = take(refine ? 8 * 3 * S * (size_t)L.wl * L.hl : 0);
  L.phi = take(8 * S * 16 * nq * L.smax);
  L.psi = take(8 * 4 * nq * n);
  L.mom = take(8 * S * 32 * nq * nq);
  L.psi0 = take(8 * n);
  L.z0 = take(8 * n);
  L.mom0 = take(8 * S * 8 * nq);
  L.gtr = take(8 * S * 4 * L.smax * 4);
  L.rto = take(P.l > 0 ? 8 * S * 4 * std::max(L.wo, L.ho) : 0);
  L.rtl = take(8 * S * 4 * std::max(L.wl, L.hl));
  L.G = take(8 * (size_t)L.ldab * NC);
  L.ipiv = take(4 * NC);
  L.gc = take(8 * NC);
  L.rdiag = take(8 * NC);
  L.Ginv = take(NC <= (size_t)COARSE_DENSE_MAX ? 8 * NC * NC : 0);
  {
    const bool blocked = NC > (size_t)COARSE_DENSE_MAX;
    const size_t kv = (size_t)P.kl + P.ku, nbk = blocked ? (NC + GBB_NB - 1) / GBB_NB : 0;
    const size_t WL = GBB_NB + P.kl, WU = GBB_NB + kv, nvec = kv + nbk * GBB_NB + P.kl;
    L.gbML = take(8 * nbk * WL * WL);
    L.gbMU = take(8 * nbk * WU * WU);
    L.gbX = take(blocked ? 8 * nvec : 0);
    L.gbY = take(blocked ? 8 * nvec : 0);
    L.gbF = take(8 * nbk * WU);
    L.gbC = take(8 * nbk * kv);
  }
  // multifrontal factorisation of G (k_mf.cu): tables, fronts, solve vectors, scratch words
  L.mf_fr = take(sizeof(MfFront) * P.mf_front.size());
  L.mf_ord = take(4 * P.mf_order.size());
  L.mf_lvl = take(4 * P.mf_level.size());
  L.mf_idx = take(4 * P.mf_idx.size());
  L.mf_asm = take(4 * P.mf_asm.size());
  L.mf_map = take(4 * P.mf_map.size());
  L.mf_task = take(4 * P.mf_task.size());
  L.mf_F = take(8 * P.mf_fbuf);
  L.mf_V = take(8 * P.mf_vbuf);
  L.mf_scr = take(64);
  L.mf_done = take(8 * P.mf_front.size());
  L.rho = take(8 * n);                     // FP32 right-hand sides staged on the grid (k_stage32)
  L.zt = take(8 * n);
  L.V = take(8 * (size_t)(L.m + 1) * n);
  L.Z = take(8 * (size_t)L.m * n);
  L.w = take(8 * n);
  L.Hs = take(8 * ((size_t)(L.m + 1) * L.m + 4 * (L.m + 1) + 64));
  L.red = take(8 * RED_DOUBLES + 64);
  L.flags = take(4 * 64);
  L.tmpv = take(8 * n);
  const size_t ldh = (size_t)L.m + 1;
  L.apart = take(8 * (2 * ldh + 3) * ARNOLDI_MAX_BLOCKS);
  L.atot = take(8 * (2 * ldh + 3));
  L.aT = take(8 * ldh * ldh);
  // device copies of the plan tables: iface[3E], home[2E], off[S], rank[6S], coff[S]
  L.tab = take(4 * (3 * P.E + E2 + S + 6 * S + S + 16));
  L.total = o;
  return L;
}

}  // namespace mrcm
