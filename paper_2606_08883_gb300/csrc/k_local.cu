// Local Robin / Dirichlet problems on subdomain boxes (Eq. 5-6, Eq. 11-12, Eq. 15) and the
// overlapping-Schwarz local solves.  One CTA per subdomain.
//
// A box of width w (x) and height h (lines along x, x fastest) has a block-tridiagonal operator:
// tridiagonal line blocks D_J and diagonal couplings -E_J between lines J-1 and J.  It is
// factored from both ends towards the middle line m = h/2 (a twisted block LDL^T):
//   top     S_0 = D_0,          S_J = D_J - E_J S_{J-1}^-1 E_J            J = 1 .. m-1
//   bottom  S_{h-1} = D_{h-1},  S_J = D_J - E_{J+1} S_{J+1}^-1 E_{J+1}    J = h-2 .. m+1
//   middle  S_m = D_m - E_m S_{m-1}^-1 E_m - E_{m+1} S_{m+1}^-1 E_{m+1}
// and only the inverses S_J^-1 are stored (symmetric, packed lower triangle, one line block per
// line; each by Cholesky S_J = L L^T, L^-1, S_J^-1 = L^-T L^-1), followed by the couplings E_J.  A solve eliminates from both ends
//   u_J = b_J + E_J S_{J-1}^-1 u_{J-1} (top),  u_J = b_J + E_{J+1} S_{J+1}^-1 u_{J+1} (bottom),
//   x_m = S_m^-1 u_m with u_m = b_m + E_m S_{m-1}^-1 u_{m-1} + E_{m+1} S_{m+1}^-1 u_{m+1},
// and substitutes back outwards: x_J = S_J^-1 (u_J + E_{J+1} x_{J+1}) above the middle,
// x_J = S_J^-1 (u_J + E_J x_{J-1}) below it.  The two ends run in the same step, so a solve is
// about h/2 + 1 + h/2 steps deep instead of 2h - 1, and a restricted Schwarz solve stops its back
// substitution at the first and last lines it keeps (the oversampling lines are never formed).
// Every step streams its (up to two) line blocks through a cp.async pipeline and is one or two
// symmetric matrix-vector products whose epilogue forms the next step's input, so a step costs
// one barrier.
//
// Oversampled boxes are padded to the full (sub + 2l)^2 size; cells outside the grid get identity
// rows with zero couplings and zero data, which leaves the clipped region's solution unchanged.
#include <cstdint>

#include "common.cuh"

namespace mrcm {

struct Box {
  int ox, oy, w, h;
};

__device__ __forceinline__ Box box_of(const Geo& g, int s, bool ohat) {
  const int I = s % g.mx, J = s / g.mx;
  Box b;
  const int l = ohat ? g.l : 0;
  b.ox = I * g.sx - l;
  b.oy = J * g.sy - l;
  b.w = g.sx + 2 * l;
  b.h = g.sy + 2 * l;
  return b;
}

__device__ __forceinline__ bool active(const Geo& g, int gx, int gy) {
  return gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
}

// Cells of subdomain s along x and along y: the subdomain size, except for the last subdomain of a
// row or column of a grid that the size does not divide, which takes the remainder.  Its box keeps
// the full padded shape; the cells past the grid are identity rows.
__device__ __forceinline__ int sub_w(const Geo& g, int s) { return min(g.sx, g.nx - (s % g.mx) * g.sx); }
__device__ __forceinline__ int sub_h(const Geo& g, int s) { return min(g.sy, g.ny - (s / g.mx) * g.sy); }
// faces on side k (-x, +x, -y, +y) of Omega_s
__device__ __forceinline__ int side_len(const Geo& g, int s, int k) { return k < 2 ? sub_h(g, s) : sub_w(g, s); }

// permeability across faces normal to axis a (the tensor component along a)
__device__ __forceinline__ double Kc(const Geo& g, int a, int gx, int gy) {
  return (a == 0 ? g.K : g.Ky)[(size_t)gy * g.nx + gx];
}

// Robin coefficient t_R of the face between (gx, gy) inside and its neighbour along axis a / dir.
__device__ __forceinline__ double face_tr(const Geo& g, int gx, int gy, int a, int dir, double* beta, double* tau) {
  const int nx2 = gx + (a == 0 ? dir : 0), ny2 = gy + (a == 1 ? dir : 0);
  const double area = a == 0 ? g.hy * g.hz : g.hx * g.hz;
  const double ha = a == 0 ? g.hx : g.hy;
  const double Hs = a == 0 ? g.sx * g.hx : g.sy * g.hy;
  return robin_tr(Kc(g, a, gx, gy), Kc(g, a, nx2, ny2), area, ha, Hs, g.alpha, beta, tau);
}

// t_R table of box s's Robin faces ([4 sides][rl], k_robin_tab), or null before it exists
__device__ __forceinline__ const double* robin_tab(const Geo& g, int s, bool ohat, int& rl) {
  rl = ohat ? g.rlo : g.rll;
  const double* t = ohat ? g.rto : g.rtl;
  return t ? t + (size_t)s * 4 * rl : nullptr;
}

// Line-block coefficients at local (x, J): diagonal, coupling to x+1 (value T, entry -T),
// coupling to line J-1 (value T, entry -T).  The Robin faces' t_R come from the box's table rt
// when given (the same values, formed once per set-up) instead of per call.
// TAB_ONLY: rt is known to be present for Robin boxes (the sweep factorisation), so the per-call
// form is left out.
template <bool TAB_ONLY = false>
__device__ __forceinline__ void line_coeffs(const Geo& g, const Box& b, bool robin, int J, int x, double& diag,
                                            double& offr, double& eup, const double* rt = nullptr, int rl = 0) {
  const int gx = b.ox + x, gy = b.oy + J;
  if (!active(g, gx, gy)) {
    diag = 1.0;
    offr = 0.0;
    eup = 0.0;
    return;
  }
  const double* Tx = g.Tx + (size_t)gy * (g.nx + 1);
  const double tw = Tx[gx], te = Tx[gx + 1];
  const double ts = g.Ty[(size_t)gy * g.nx + gx], tn = g.Ty[(size_t)(gy + 1) * g.nx + gx];
  double d = (tw + te) + (ts + tn);
  if (robin && rt) {
    if (x == 0 && gx - 1 >= 0) d += rt[J] - tw;
    if (x == b.w - 1 && gx + 1 < g.nx) d += rt[rl + J] - te;
    if (J == 0 && gy - 1 >= 0) d += rt[2 * rl + x] - ts;
    if (J == b.h - 1 && gy + 1 < g.ny) d += rt[3 * rl + x] - tn;
  } else if (!TAB_ONLY && robin) {
    if (x == 0 && gx - 1 >= 0) d += face_tr(g, gx, gy, 0, -1, nullptr, nullptr) - tw;
    if (x == b.w - 1 && gx + 1 < g.nx) d += face_tr(g, gx, gy, 0, +1, nullptr, nullptr) - te;
    if (J == 0 && gy - 1 >= 0) d += face_tr(g, gx, gy, 1, -1, nullptr, nullptr) - ts;
    if (J == b.h - 1 && gy + 1 < g.ny) d += face_tr(g, gx, gy, 1, +1, nullptr, nullptr) - tn;
  }
  diag = d;
  offr = (x + 1 < b.w && active(g, gx + 1, gy)) ? te : 0.0;
  eup = (J > 0 && active(g, gx, gy - 1)) ? ts : 0.0;
}

// packed lower-triangle row index of linear position k (row i holds i+1 entries)
__device__ __forceinline__ int tri_row(int k) {
  int i = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > k) --i;
  while ((i + 1) * (i + 2) / 2 <= k) ++i;
  return i;
}

// ============================================================================================
// Factor: one CTA per subdomain box; dense w x w working arrays in shared memory.
// ============================================================================================
// packed-triangle position t -> (row i, column j <= i), and advancing it by `step` positions
__device__ __forceinline__ void tri_at(int t, int& i, int& j) {
  i = tri_row(t);
  j = t - i * (i + 1) / 2;
}
__device__ __forceinline__ void tri_advance(int& i, int& j, int step) {
  j += step;
  while (j > i) {
    j -= i + 1;
    ++i;
  }
}

// nch = 2: the top and the bottom recursion of the twisted order advance together, one line each
// per iteration on one half of the CTA (each half with its own working arrays), and the middle line
// follows; nch = 1: the lines one after the other (boxes too wide for two sets of working arrays).
// Each line: Schur complement, right-looking Cholesky (the next diagonal's square root is taken by
// the thread that updates it), L^-1 by elimination on the identity, and S^-1 = L^-T L^-1.  The
// scaled column of L (Cholesky) and the scaled row of L^-1 are written before the updates that
// read them (two barriers per column), so every update entry is one FMA: the FP64 pipe, which
// bounds the FP64 factorisation, does half the work of scaling inside the update.
template <typename T>
__global__ void __launch_bounds__(256) k_factor(Geo g, int kind, int LS, T* __restrict__ Linv, int* flags, int nch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const bool ohat = kind != BOX_OMEGA_ROBIN;
  const bool robin = kind != BOX_OHAT_DIRICHLET;
  const Box b = box_of(g, s, ohat);
  int rl;
  const double* rt = robin_tab(g, s, ohat, rl);
  const int w = b.w, h = b.h, m = h / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nth = nt / nch, half = tid / nth, tidh = tid - half * nth;
  const size_t per = 4 * (size_t)w * w + 4 * (size_t)w;   // one recursion's working arrays
  T* Sm = reinterpret_cast<T*>(smem_raw) + half * per;   // Schur complement, then inverse work rows
  T* Lm = Sm + w * w;                      // Cholesky factor of the line block
  T* Lc = Lm + w * w;                      // L_JJ^-1 of the current line
  T* Sp = Lc + w * w;                      // S^-1 of the previous (then current) line, lower part
  T* ev = Sp + w * w;                      // couplings to the previous line
  T* rinv = ev + w;                        // reciprocal diagonal of Lm
  T* ev2 = rinv + w;                       // second coupling vector (middle line)
  // the bottom recursion's last S^-1, read by the middle line when nch = 2
  const T* Sp_bot = reinterpret_cast<T*>(smem_raw) + (nch == 2 ? per : 0) + 3 * (size_t)w * w;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  T* out = Linv + (size_t)s * box_stride(w, h, LS);
  T* ec_out = out + (size_t)h * LS;        // line couplings E_J[x], read by every solve
  const int npk = w * (w + 1) / 2;
  const int iters = nch == 2 ? (m > h - 1 - m ? m : h - 1 - m) + 1 : h;
  for (int it = 0; it < iters; ++it) {
    // this half's line: top lines 0..m-1, bottom lines h-1..m+1, then the middle line m
    bool top, bottom, mid, active;
    int J;
    if (nch == 2) {
      const bool last = it == iters - 1;
      top = !last && half == 0 && it < m;
      bottom = !last && half == 1 && h - 1 - it >= m + 1;
      mid = last && half == 0;
      J = last ? m : (half == 0 ? it : h - 1 - it);
      active = top || bottom || mid;
    } else {
      top = it < m;
      bottom = !top && it < h - 1;
      mid = !top && !bottom;
      J = top ? it : (bottom ? h - 1 - (it - m) : m);
      active = true;
    }
    // previous line of the same recursion and its coupling vector: top uses E_J = eup(J),
    // bottom uses E_{J+1} = eup(J+1)
    const bool has_prev = top ? J > 0 : (bottom ? J < h - 1 : false);
    // (1) S_J = D_J - E S_prev^-1 E (middle: minus both sides), lower triangle
    if (active)
      for (int i = tidh; i < w; i += nth) {
        double d, o, e;
        line_coeffs(g, b, robin, J, i, d, o, e, rt, rl);
        ec_out[(size_t)J * w + i] = (T)e;
        Sm[i * w + i] = (T)d;
        if (i + 1 < w) Sm[(i + 1) * w + i] = (T)(-o);
        if (top) {
          ev[i] = (T)e;
        } else if (bottom) {
          double d2, o2, e2;
          line_coeffs(g, b, robin, J + 1, i, d2, o2, e2, rt, rl);
          ev[i] = (T)e2;
        } else {
          ev[i] = (T)e;                      // E_m (towards line m-1)
          double d2, o2, e2 = 0.0;
          if (J + 1 < h) line_coeffs(g, b, robin, J + 1, i, d2, o2, e2, rt, rl);
          ev2[i] = (T)e2;                    // E_{m+1} (towards line m+1)
        }
      }
    __syncthreads();
    if (active) {
      const bool mid_up = mid && m > 0;          // S_{m-1}^-1: own Sp (nch = 2) or the stored top line
      const bool mid_dn = mid && m + 1 < h;      // S_{m+1}^-1: the bottom recursion's Sp
      const T* Sup = out + (size_t)(m > 0 ? m - 1 : 0) * LS;
      int i, j;
      tri_at(tidh, i, j);
      for (int k = tidh; k < npk; k += nth, tri_advance(i, j, nth)) {
        T v = (i == j || i == j + 1) ? Sm[i * w + j] : (T)0;
        if (has_prev) v -= ev[i] * ev[j] * Sp[i * w + j];
        if (mid_up) v -= ev[i] * ev[j] * (nch == 2 ? Sp[i * w + j] : Sup[k]);
        if (mid_dn) v -= ev2[i] * ev2[j] * (nch == 2 ? Sp_bot[i * w + j] : Sp[i * w + j]);
        Sm[i * w + j] = v;
      }
    }
    __syncthreads();
    // (2) Cholesky of S_J: right-looking, column k of L written to Lm, trailing update in Sm
    if (active && tidh == 0) {
      T p = Sm[0];
      if (!(p > (T)0) || !isfinite((double)p)) {
        bad = 1;
        p = (T)1;
      }
      const T d = sqrt(p);
      Lm[0] = d;
      rinv[0] = (T)1 / d;
    }
    __syncthreads();
    for (int k = 0; k < w; ++k) {
      // column k of L first (one barrier), then the trailing update with one FMA per entry
      const int mm = w - k - 1;
      if (active) {
        const T rd = rinv[k];
        for (int i = tidh; i < mm; i += nth) Lm[(k + 1 + i) * w + k] = Sm[(k + 1 + i) * w + k] * rd;
      }
      __syncthreads();
      if (active) {
        const int nup = mm * (mm + 1) / 2;
        int ii, jj;
        tri_at(tidh, ii, jj);
        for (int t = tidh; t < nup; t += nth, tri_advance(ii, jj, nth)) {
          const int i = k + 1 + ii, j = k + 1 + jj;
          const T v = Sm[i * w + j] - Lm[i * w + k] * Lm[j * w + k];
          Sm[i * w + j] = v;
          if (t == 0) {  // the next diagonal: its square root for column k + 1
            T p = v;
            if (!(p > (T)0) || !isfinite((double)p)) {
              bad = 1;
              p = (T)1;
            }
            const T d = sqrt(p);
            Lm[(k + 1) * w + k + 1] = d;
            rinv[k + 1] = (T)1 / d;
          }
        }
      }
      __syncthreads();
    }
    // (3) Lc = Lm^-1 by right-looking elimination on the identity (work rows in Sm)
    if (active)
      for (int k = tidh; k < w * w; k += nth) {
        const int i = k / w, j = k - i * w;
        Sm[k] = (i == j) ? (T)1 : (T)0;
      }
    __syncthreads();
    for (int k = 0; k < w; ++k) {
      // row k of L^-1 first (one barrier), then the rows below with one FMA per entry
      if (active) {
        const T rk = rinv[k];
        for (int c = tidh; c <= k; c += nth) Lc[k * w + c] = Sm[k * w + c] * rk;
      }
      __syncthreads();
      if (active) {
        const int rows = w - k - 1, cols = k + 1;
        for (int t = tidh; t < rows * cols; t += nth) {
          const int i = k + 1 + t / cols, c = t % cols;
          Sm[i * w + c] -= Lm[i * w + k] * Lc[k * w + c];
        }
      }
      __syncthreads();
    }
    // (4) S_J^-1 = Lc^T Lc (lower part), store packed, keep for the next line's Schur complement;
    //     two entries per pass for two independent sums
    if (active) {
      int i0, j0, i1, j1;
      tri_at(tidh, i0, j0);
      i1 = i0;
      j1 = j0;
      tri_advance(i1, j1, nth);
      for (int k = tidh; k < npk; k += 2 * nth) {
        const bool two = k + nth < npk;
        T a0 = 0, a1 = 0;
        if (two) {
          // the second entry follows the first in packed order, so i1 >= i0: the first entry's
          // head, then both together (each summed in increasing q, as a single sum would be)
          for (int q = i0; q < i1; ++q) a0 += Lc[q * w + i0] * Lc[q * w + j0];
          for (int q = i1; q < w; ++q) {
            a0 += Lc[q * w + i0] * Lc[q * w + j0];
            a1 += Lc[q * w + i1] * Lc[q * w + j1];
          }
        } else {
          for (int q = i0; q < w; ++q) a0 += Lc[q * w + i0] * Lc[q * w + j0];
        }
        Sp[i0 * w + j0] = a0;
        out[(size_t)J * LS + k] = a0;
        if (two) {
          Sp[i1 * w + j1] = a1;
          out[(size_t)J * LS + k + nth] = a1;
        }
        tri_advance(i0, j0, 2 * nth);
        tri_advance(i1, j1, 2 * nth);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicOr(flags, FLAG_SINGULAR_LOCAL);
}

// --------------------------------------------------------------------------------------------
// FP32 factorisation for boxes up to 36 cells wide, register-resident: one warp per recursion of
// the twisted order (two warps per box), lane i holding row i of the line block; a width W above
// 32 keeps the (W-32) x (W-32) corner of the last rows in every lane (the rest of those rows is
// columns 32.. of the lanes' rows, by symmetry).  Each line: the Schur complement from the
// previous line's inverse (still in registers), Jacobi scaling to a unit diagonal, and S^-1 by the
// symmetric Gauss-Jordan sweep (pivot k: a_ij -= a_ik a_kj / a_kk for i, j != k, row and column k
// divided by the pivot, a_kk = -1 / a_kk; after every pivot the array holds -S^-1).  The pivots of
// the scaled SPD block lie in (0, 1], so the pivot row takes the same one-FMA update as the others
// (a_kj - (1 - 1/d) a_kj, rounding error at most |d - 1| eps).  The pivot row is published through
// shared memory (double-buffered, one warp barrier per pivot).  S_J^-1 = -R a R is written in the
// packed lower layout of k_factor, E_J after the blocks.
// --------------------------------------------------------------------------------------------
template <int W>
struct SweepSmem {
  static constexpr int STG = (W * (W + 1) / 2 + 3) & ~3;
  float bc[2][W];                  // pivot row
  float dv[W], ov[W], uv[W], rv[W], vv[W];
  float stage[STG];                // S_J^-1, packed lower
};

// coefficients of cell x of line J as floats (identity rows past the box width); with cf, also
// stored there in FP64 [d, o, e] (the refinement of the FP32 set-up solves reads them)
__device__ __forceinline__ void line_coeffs_f(const Geo& g, const Box& b, bool robin, int J, int x, float& d, float& o,
                                              float& e, double* cf, const double* rt, int rl) {
  if (x >= b.w) {
    d = 1.f;
    o = 0.f;
    e = 0.f;
    return;
  }
  double dd, oo, ee;
  line_coeffs<true>(g, b, robin, J, x, dd, oo, ee, rt, rl);
  d = (float)dd;
  o = (float)oo;
  e = (float)ee;
  if (cf) {
    cf[0] = dd;
    cf[1] = oo;
    cf[2] = ee;
  }
}

template <int W>
__global__ void __launch_bounds__(64) k_factor_sweep(Geo g, int kind, int LS, float* __restrict__ Linv,
                                                     int* flags, double* __restrict__ coef) {
  static_assert(W % 4 == 0 && W <= 36, "sweep widths: multiples of 4 up to 36");
  constexpr int C = W > 32 ? W - 32 : 0;   // corner size
  constexpr int C1 = C > 0 ? C : 1;
  constexpr int R0 = W < 32 ? W : 32;      // rows held one per lane
  __shared__ __align__(16) SweepSmem<W> sm_all[2];
  const int s = blockIdx.x;
  const bool ohat = kind != BOX_OMEGA_ROBIN;
  const bool robin = kind != BOX_OHAT_DIRICHLET;
  const Box b = box_of(g, s, ohat);
  int rl;
  const double* rt = robin_tab(g, s, ohat, rl);
  const int w = b.w, h = b.h, m = h / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  SweepSmem<W>& sm = sm_all[wid];
  float* out = Linv + (size_t)s * box_stride(w, h, LS);
  float* ec_out = out + (size_t)h * LS;
  bool bad = false;

  float a[W];          // row `lane` of the working array
  // the corner block (rows and columns 32.., W > 32): entry (cp, cq) held by lane cp C + cq only;
  // the corner rows' Jacobi scales are shared through sm.rv[32..]
  const bool cown_on = C > 0 && lane < C * C;
  const int cp = cown_on ? lane / C1 : 0, cq = cown_on ? lane - (lane / C1) * C1 : 0;
  float cown = 0.f;
  float r_own = 1.f;   // Jacobi scale of row `lane` of the previous line
  float ep0 = 0.f, ep1 = 0.f;   // bottom recursion: E_{J+1} of cells lane and 32 + lane
#pragma unroll
  for (int j = 0; j < W; ++j) a[j] = 0.f;

  // top lines 0..m-1 (warp 0) and bottom lines h-1..m+1 (warp 1) side by side, then the middle
  // line m on warp 0 once both recursions are done
  const int nsteps = wid == 0 ? m : h - 1 - m;
  const int iters = m > h - 1 - m ? m : h - 1 - m;
  for (int it = 0; it <= iters; ++it) {
    const bool mid = it == iters;
    if (mid) __syncthreads();
    if (mid ? wid != 0 : it >= nsteps) continue;
    const bool top = !mid && wid == 0;
    const int J = mid ? m : (top ? it : h - 1 - it);
    const bool has_prev = mid ? m > 0 : it > 0;
    const bool dn = mid && m + 1 < h;      // the middle line's second neighbour S_{m+1}^-1
    // (1) line data: diagonal, right coupling, u_x = E_x r_x towards the previous line
    float d0, o0, e0, d1 = 1.f, o1 = 0.f, e1 = 0.f;
    double* cfl = coef ? coef + (((size_t)s * h + J) * w) * 3 : nullptr;   // this line's FP64 coefficients
    line_coeffs_f(g, b, robin, J, lane, d0, o0, e0, cfl ? cfl + 3 * lane : nullptr, rt, rl);
    if (lane < C) line_coeffs_f(g, b, robin, J, 32 + lane, d1, o1, e1, cfl ? cfl + 3 * (32 + lane) : nullptr, rt, rl);
    if (lane < w) ec_out[(size_t)J * w + lane] = e0;
    if (lane < C && 32 + lane < w) ec_out[(size_t)J * w + 32 + lane] = e1;
    const float eu0 = (top || mid) ? e0 : ep0, eu1 = (top || mid) ? e1 : ep1;
    ep0 = e0;
    ep1 = e1;
    float f0 = 0.f, f1 = 0.f;
    if (dn) {
      float d_, o_;
      line_coeffs_f(g, b, robin, m + 1, lane, d_, o_, f0, nullptr, rt, rl);
      if (lane < C) line_coeffs_f(g, b, robin, m + 1, 32 + lane, d_, o_, f1, nullptr, rt, rl);
    }
    if (lane < W) {
      sm.dv[lane] = d0;
      sm.ov[lane] = o0;
      sm.uv[lane] = has_prev ? eu0 * r_own : 0.f;
      sm.vv[lane] = f0;
    }
    if (lane < C) {
      sm.dv[32 + lane] = d1;
      sm.ov[32 + lane] = o1;
      sm.uv[32 + lane] = has_prev ? eu1 * sm.rv[32 + lane] : 0.f;   // the previous line's corner scale
      sm.vv[32 + lane] = f1;
    }
    __syncwarp();
    // (2) Schur complement: row `lane` and the corner
    {
      const float ui = lane < W ? sm.uv[lane] : 0.f;
      const float di = lane < W ? sm.dv[lane] : 1.f;
      const float oi = lane < W ? sm.ov[lane] : 0.f;
      const float om = (lane > 0 && lane < W) ? sm.ov[lane - 1] : 0.f;
#pragma unroll
      for (int j = 0; j < W; ++j) {
        float v = (ui * sm.uv[j]) * a[j];
        if (j == lane) v += di;
        if (j == lane + 1) v -= oi;
        if (j == lane - 1) v -= om;
        a[j] = v;
      }
      if (cown_on) {
        float v = (sm.uv[32 + cp] * sm.uv[32 + cq]) * cown;
        if (cp == cq) v += sm.dv[32 + cp];
        if (cq == cp + 1) v -= sm.ov[32 + cp];
        if (cq == cp - 1) v -= sm.ov[32 + cq];
        cown = v;
      }
      if (dn) {   // - E_{m+1} S_{m+1}^-1 E_{m+1}, from the bottom recursion's staged last block
        const float* sx = sm_all[1].stage;
        const float vi = lane < w ? sm.vv[lane] : 0.f;
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (lane < w && j < w) {
            const int hi = j > lane ? j : lane, lo = j > lane ? lane : j;
            a[j] -= (vi * sm.vv[j]) * sx[hi * (hi + 1) / 2 + lo];
          }
        if (cown_on && 32 + cp < w && 32 + cq < w) {
          const int hi = cp > cq ? cp : cq, lo = cp > cq ? cq : cp;
          cown -= (sm.vv[32 + cp] * sm.vv[32 + cq]) * sx[(32 + hi) * (33 + hi) / 2 + 32 + lo];
        }
      }
    }
    // (3) Jacobi scaling to a unit diagonal
    {
      float dg = 1.f;
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j == lane) dg = a[j];
      if (lane < W && !(dg > 0.f && isfinite(dg))) {
        bad = true;
        dg = 1.f;
      }
      r_own = lane < W ? rsqrtf(dg) : 1.f;
      if (lane < W) sm.rv[lane] = r_own;
      if (cown_on && cp == cq) {
        float cd = cown;
        if (!(cd > 0.f && isfinite(cd))) {
          bad = true;
          cd = 1.f;
        }
        sm.rv[32 + cp] = rsqrtf(cd);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < W; ++j) a[j] *= r_own * sm.rv[j];
      if (cown_on) cown *= sm.rv[32 + cp] * sm.rv[32 + cq];
    }
    // (4) symmetric Gauss-Jordan sweep over the W pivots
#pragma unroll
    for (int k = 0; k < W; ++k) {
      float* bk = sm.bc[k & 1];
      // the pivot row, published as column k (symmetric up to rounding): one entry per lane, and
      // for k < 32 the corner columns of row k from lane k
      if (lane < W) bk[lane] = a[k];
      if (C > 0 && k < 32 && lane == k) {
#pragma unroll
        for (int q = 0; q < C; q += 4)
          *reinterpret_cast<float4*>(bk + 32 + q) = make_float4(a[32 + q], a[33 + q], a[34 + q], a[35 + q]);
      }
      if (C > 0 && k >= 32 && cown_on && cp == k - 32) bk[32 + cq] = cown;   // corner part of row k
      __syncwarp();
      float rowk[W];
#pragma unroll
      for (int j = 0; j < W; j += 4) {
        const float4 t = *reinterpret_cast<const float4*>(bk + j);
        rowk[j] = t.x;
        rowk[j + 1] = t.y;
        rowk[j + 2] = t.z;
        rowk[j + 3] = t.w;
      }
      float dk = rowk[k];
      if (!(dk > 0.f && isfinite(dk))) {
        bad = true;
        dk = 1.f;
      }
      const float rinv = __fdividef(1.f, dk);   // dk is near 1 after the Jacobi scaling
      const bool me = k < 32 && lane == k;
      const float gsc = me ? 1.f - rinv : a[k] * rinv;
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j != k) a[j] = fmaf(-gsc, rowk[j], a[j]);
      a[k] = me ? -rinv : gsc;
      if (C > 0 && cown_on) {   // this lane's corner entry, from row k's corner part in shared memory
        const float rp = bk[32 + cp], rq = bk[32 + cq];
        if (k < 32) {
          cown = fmaf(-(rp * rinv), rq, cown);
        } else {
          const bool pk = 32 + cp == k, qk = 32 + cq == k;
          cown = pk && qk ? -rinv : pk ? rq * rinv : qk ? rp * rinv : fmaf(-(rp * rinv), rq, cown);
        }
      }
    }
    // (5) S^-1 = -R a R, packed lower, through the staging array
    __syncwarp();
    if (lane < w) {
      const int base = lane * (lane + 1) / 2;
#pragma unroll
      for (int j = 0; j < R0; ++j)
        if (j <= lane) sm.stage[base + j] = -(r_own * sm.rv[j]) * a[j];
#pragma unroll
      for (int p = 0; p < C; ++p)   // rows 32 + p, columns lane < 32
        if (32 + p < w) sm.stage[(32 + p) * (33 + p) / 2 + lane] = -(r_own * sm.rv[32 + p]) * a[32 + p];
    }
    if (cown_on && cq <= cp && 32 + cp < w)
      sm.stage[(32 + cp) * (33 + cp) / 2 + 32 + cq] = -(sm.rv[32 + cp] * sm.rv[32 + cq]) * cown;
    __syncwarp();
    const int npk = w * (w + 1) / 2;
    for (int t = lane; t < npk; t += 32) out[(size_t)J * LS + t] = sm.stage[t];
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_SINGULAR_LOCAL);
}

template <int W>
static cudaError_t launch_factor_sweep(const Geo& g, int kind, int LS, float* Linv, int* flags, double* coef,
                                       cudaStream_t st) {
  k_factor_sweep<W><<<g.mx * g.my, 64, 0, st>>>(g, kind, LS, Linv, flags, coef);
  count_launch(1);
  return cudaGetLastError();
}

// FP64 line coefficients [diagonal, x coupling to the right, y coupling to the line above] of every
// cell of every box of one kind, for the refinement step of the FP32 set-up solves
__global__ void k_line_coef(Geo g, int kind, double* __restrict__ coef) {
  const int s = blockIdx.x;
  const bool ohat = kind != BOX_OMEGA_ROBIN;
  const bool robin = kind != BOX_OHAT_DIRICHLET;
  const Box b = box_of(g, s, ohat);
  int rl;
  const double* rt = robin_tab(g, s, ohat, rl);
  for (int c = threadIdx.x; c < b.w * b.h; c += blockDim.x) {
    const int J = c / b.w, x = c - J * b.w;
    double d, o, e;
    line_coeffs(g, b, robin, J, x, d, o, e, rt, rl);
    double* cf = coef + ((size_t)s * b.w * b.h + c) * 3;
    cf[0] = d;
    cf[1] = o;
    cf[2] = e;
  }
}

cudaError_t launch_line_coef(const Geo& g, int kind, double* coef, cudaStream_t st) {
  k_line_coef<<<g.mx * g.my, 256, 0, st>>>(g, kind, coef);
  count_launch(1);
  return cudaGetLastError();
}

size_t factor_smem_bytes(int w, bool fp32, int nch) {
  const size_t e = fp32 ? 4 : 8;
  return e * nch * (4 * (size_t)w * w + 4 * (size_t)w) + 16;
}

cudaError_t launch_factor(const Geo& g, int kind, int w, int hgt, int LS, void* Linv, bool fp32, int* flags,
                          cudaStream_t st, double* coef) {
  (void)hgt;
  const int S = g.mx * g.my;
  // both recursions at once when two sets of working arrays still leave room for two CTAs per SM
  const int nch = factor_smem_bytes(w, fp32, 2) <= 112 * 1024 ? 2 : 1;
  const size_t sm = factor_smem_bytes(w, fp32, nch);
  if (fp32 && w <= 36) {   // register-resident sweep, box width padded to a multiple of 4
    // it reads the Robin faces' t_R from the box tables only (k_robin_tab, formed with the assembly)
    if ((kind == BOX_OHAT_ROBIN && !g.rto) || (kind == BOX_OMEGA_ROBIN && !g.rtl)) return cudaErrorInvalidValue;
    float* L = (float*)Linv;
    if (w <= 16) return launch_factor_sweep<16>(g, kind, LS, L, flags, coef, st);
    if (w <= 20) return launch_factor_sweep<20>(g, kind, LS, L, flags, coef, st);
    if (w <= 24) return launch_factor_sweep<24>(g, kind, LS, L, flags, coef, st);
    if (w <= 28) return launch_factor_sweep<28>(g, kind, LS, L, flags, coef, st);
    if (w <= 32) return launch_factor_sweep<32>(g, kind, LS, L, flags, coef, st);
    return launch_factor_sweep<36>(g, kind, LS, L, flags, coef, st);
  }
  if (coef) {   // the other factorisations leave the coefficients to their own kernel
    const cudaError_t e = launch_line_coef(g, kind, coef, st);
    if (e != cudaSuccess) return e;
  }
  if (fp32) {
    const cudaError_t e = raise_smem_limit<k_factor<float>>();
    if (e != cudaSuccess) return e;
    k_factor<float><<<S, 256, sm, st>>>(g, kind, LS, (float*)Linv, flags, nch);
    count_launch(1);
  } else {
    const cudaError_t e = raise_smem_limit<k_factor<double>>();
    if (e != cudaSuccess) return e;
    k_factor<double><<<S, 256, sm, st>>>(g, kind, LS, (double*)Linv, flags, nch);
    count_launch(1);
  }
  return cudaGetLastError();
}

// ============================================================================================
// Solve: forward / backward sweeps over the line blocks, with mode-specific data in and out.
// ============================================================================================
enum SolveMode : int { MODE_INFORMED = 0, MODE_BASIS = 1, MODE_PARTICULAR = 2, MODE_SCHWARZ = 3 };

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// mbarrier-completed bulk copies (one per line block) for box-resident solves
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Waits for phase 0 of bar to complete; gives up (returns false) after a bounded number of polls.
__device__ __forceinline__ bool mbar_wait0(unsigned long long* bar) {
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar))
        : "memory");
    if (done) return true;
  }
  return false;
}

struct SolveArgs {
  const void* Linv;
  int LS;
  const double* in;    // particular, schwarz: r; basis: phi
  double* out;         // particular: psi0; schwarz: z after the sweep; basis: psi; informed: phi
  double* mom;         // particular: mom0 [S][4 sides][nq tests][2]; basis: mom [S][4 sides][4 nq][nq tests][2]
  const double* zin;   // schwarz: z before the sweep (read only)
  int* flags;          // device status word (FLAG_TIMEOUT if a bounded wait gives up)
  int colour;          // schwarz: -1 all boxes, else only the boxes of this colour (see colour_box)
  int q;               // informed, basis: the degree of the side functions this launch handles
  const double* coef;  // FP32 informed, basis: the box's FP64 line coefficients [S][h][w][d, o, e]
  const float* in32;   // FP32 particular, additive Schwarz: the right-hand side already formed on the grid
                       // in FP32 (r, or the sweep's residual r - A z), fetched by asynchronous copies
};

// Degree-q function of a box side at its face t of len: 1, or the linear function of the position
// along the side scaled to [-1, 1] over the side (the multiplier and test functions of Sec. 2.1)
__device__ __forceinline__ double side_fn(int q, int t, int len) {
  return q == 0 ? 1.0 : 2.0 * (t + 0.5) / len - 1.0;
}

// Subdomain of the b-th box of a colour: colour bit 0 = parity of the x index, bit 1 = of the y
// index; boxes of a colour in row-major order of their subdomains.
__device__ __forceinline__ int colour_box(const Geo& g, int colour, int b) {
  const int cx = colour & 1, cy = (colour >> 1) & 1;
  const int nxc = (g.mx - cx + 1) / 2;
  const int I = cx + 2 * (b % nxc), J = cy + 2 * (b / nxc);
  return J * g.mx + I;
}

// Gamma face t of side k of Omega_s: inside cell (global) and face transmissibility T_f.  A +x or
// +y side is a Robin side only when the subdomain is not the last along that axis, so it has the
// full subdomain size there.
__device__ __forceinline__ void gamma_face(const Geo& g, int s, int k, int t, int& gx, int& gy, int& ox2, int& oy2,
                                           double& Tf) {
  const int I = s % g.mx, J = s / g.mx;
  const int x0 = I * g.sx, y0 = J * g.sy;
  switch (k) {
    case 0: gx = x0; gy = y0 + t; ox2 = gx - 1; oy2 = gy; Tf = g.Tx[(size_t)gy * (g.nx + 1) + x0]; break;
    case 1: gx = x0 + g.sx - 1; gy = y0 + t; ox2 = gx + 1; oy2 = gy; Tf = g.Tx[(size_t)gy * (g.nx + 1) + x0 + g.sx]; break;
    case 2: gx = x0 + t; gy = y0; ox2 = gx; oy2 = gy - 1; Tf = g.Ty[(size_t)y0 * g.nx + gx]; break;
    default: gx = x0 + t; gy = y0 + g.sy - 1; ox2 = gx; oy2 = gy + 1; Tf = g.Ty[(size_t)(y0 + g.sy) * g.nx + gx]; break;
  }
}

__device__ __forceinline__ bool robin_side(const Geo& g, int s, int k) {
  const int I = s % g.mx, J = s / g.mx;
  switch (k) {
    case 0: return I > 0;
    case 1: return I < g.mx - 1;
    case 2: return J > 0;
    default: return J < g.my - 1;
  }
}


// Threads per row of a line product: FP64 runs against the DFMA pipe, so two threads per row keep
// the shuffle adds to one per output; FP32 runs against latency, so four threads shorten the chain.
template <typename T>
struct LineTPR {
  static constexpr int value = sizeof(T) == 8 ? 2 : 4;
};

// Up to two symmetric products per step, S_A x_A (threads [0, w TPR)) and S_B x_B (threads
// [w TPR, 2 w TPR)), S in packed lower storage.  Every thread of the block reaches the shuffles (a
// product that is off this step, or a thread past the rows, contributes zeros); epi(half, i, r, v)
// is called once per output by the first thread of row i, so a step can produce the next step's
// input directly.
template <typename T, int NR, class Epi>
__device__ __forceinline__ void gemv_pair(const T* PA, const T* inA, bool onA, const T* PB, const T* inB, bool onB,
                                          int w, Epi epi) {
  constexpr int TPR = LineTPR<T>::value;
  const int r0 = threadIdx.x / TPR, q = threadIdx.x % TPR;
  const int half = r0 >= w ? 1 : 0;
  const int i = r0 - half * w;
  const bool on = (half == 0 ? onA : onB) && r0 < 2 * w;
  const T* P = half == 0 ? PA : PB;
  const T* in = half == 0 ? inA : inB;
  T acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0;
  if (on) {
    const T* row = P + i * (i + 1) / 2;
    for (int c = q; c < w; c += TPR) {
      const T sv = c <= i ? row[c] : P[c * (c + 1) / 2 + i];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] += sv * in[c * NR + r];
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  if (on && q == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) epi(half, i, r, acc[r]);
  }
}

template <typename T>
__device__ __forceinline__ void issue_line(T* buf, const T* src, int LS, bool valid) {
  if (valid) {
    const int nch = LS * (int)sizeof(T) / 16;
    for (int c = threadIdx.x; c < nch; c += blockDim.x)
      cp_async16(reinterpret_cast<unsigned char*>(buf) + 16 * c, reinterpret_cast<const unsigned char*>(src) + 16 * c);
  }
}

// Line blocks used by step st of a twisted solve (-1: none).  Steps 0..nf-1 eliminate (top line t,
// bottom line h-1-t), step nf is the middle line, the rest substitute back (m-1-t, m+1+t) down to
// line lo_keep and up to line hi_keep.
struct Twist {
  int h, m, nf, nb, lo_keep, hi_keep;
  __device__ __forceinline__ void lines(int st, int& A, int& B) const {
    if (st < nf) {
      A = st < m ? st : -1;
      B = h - 1 - st >= m + 1 ? h - 1 - st : -1;
    } else if (st == nf) {
      A = m;
      B = -1;
    } else {
      const int t = st - nf - 1;
      A = m - 1 - t >= lo_keep ? m - 1 - t : -1;
      B = m + 1 + t <= hi_keep ? m + 1 + t : -1;
    }
  }
};

// ---------------------------------------------------------------------------------------------
// FP32 twisted solve of a resident box of width w <= W (W = 32 or 36) on two warps: warp 0 runs
// the top recursion and the middle line, warp 1 the bottom recursion, each lane one row of the
// line blocks (the W - 32 last rows of a 36-wide box from the lanes' columns, by symmetry, with a
// shared-memory transpose sum).  Row i of the packed block is read at T(i) + j for j <= i and at
// T(j) + i above (T(k) = k (k + 1) / 2): both conflict-free across a warp.  The warps hand steps
// over through warp barriers only and meet at the middle line; the bottom recursion's contribution
// to the middle goes to cb, added before the middle step.  Same arithmetic per output as the block
// kernel's line products up to the order of the sums.  Returns false when a line block never
// arrived (the caller reports the timeout).
template <int W, int NR, bool EXACT>
__device__ __forceinline__ void warp_line_product(const float* __restrict__ S, const float* __restrict__ in, int w_rt,
                                                  int lane, float (&y)[NR], float& yc, float* part) {
  constexpr int C = W > 32 ? W - 32 : 0;
  const int w = EXACT ? W : w_rt;   // the box width (a compile-time constant when it equals W)
  const int i = lane < w ? lane : 0;
  const int Ti = i * (i + 1) / 2;
  // the lane's row of S first, all loads issued before any product: the row-form entries
  // (T(i) + j) and the column-form ones (T(j) + i) as separate loads, each conflict-free
  float sr[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    if (j < w) {
      if (j == 0) {
        sr[j] = S[Ti];
      } else if (j >= 32) {
        sr[j] = S[j * (j + 1) / 2 + i];
      } else {
        const float lo = S[Ti + j], up = S[j * (j + 1) / 2 + i];
        sr[j] = j <= i ? lo : up;
      }
    } else {
      sr[j] = 0.f;
    }
  }
  float a0[NR], a1[NR], own[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    a0[r] = 0.f;
    a1[r] = 0.f;
    own[r] = in[i * NR + r];
  }
  float pc[C > 0 ? C : 1][NR];
  if constexpr (NR == 1) {
    float u[W];   // broadcast reads: four at a time when the line starts on 16 bytes (w % 4 == 0)
    if ((w & 3) == 0) {
#pragma unroll
      for (int j = 0; j < W; j += 4) {
        if (j < w) {
          const float4 t = *reinterpret_cast<const float4*>(in + j);
          u[j] = t.x;
          u[j + 1] = t.y;
          u[j + 2] = t.z;
          u[j + 3] = t.w;
        } else {
          u[j] = u[j + 1] = u[j + 2] = u[j + 3] = 0.f;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < W; ++j) u[j] = j < w ? in[j] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
      if (j & 1) a1[0] = fmaf(sr[j], u[j], a1[0]);
      else a0[0] = fmaf(sr[j], u[j], a0[0]);
      if (j >= 32) pc[(j - 32) % (C > 0 ? C : 1)][0] = sr[j] * own[0];
    }
  } else {
#pragma unroll
    for (int j = 0; j < W; ++j) {
      float4 t = *reinterpret_cast<const float4*>(in + j * NR);
      if (j >= w) t = make_float4(0.f, 0.f, 0.f, 0.f);
      const float v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int r = 0; r < NR; ++r) a0[r] = fmaf(sr[j], v[r], a0[r]);
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < NR; ++r) pc[(j - 32) % (C > 0 ? C : 1)][r] = sr[j] * own[r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) y[r] = a0[r] + a1[r];
  yc = 0.f;
  if (C > 0) {
    // rows 32 + p: sum over the lanes (columns j < 32) by a transpose through shared memory, then
    // the corner block
#pragma unroll
    for (int p = 0; p < (C > 0 ? C : 1); ++p)
#pragma unroll
      for (int r = 0; r < NR; ++r) part[(p * NR + r) * 32 + lane] = lane < w ? pc[p][r] : 0.f;
    __syncwarp();
    if (lane < C * NR) {
      const int p = lane / NR, r = lane - p * NR;
      if (32 + p < w) {
        const float4* pp = reinterpret_cast<const float4*>(part + lane * 32);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          const float4 u = pp[k], v = pp[k + 1];
          s0 += (u.x + u.y) + (u.z + u.w);
          s1 += (v.x + v.y) + (v.z + v.w);
        }
        float cs = s0 + s1;
        for (int q = 0; q < C; ++q) {
          if (32 + q >= w) break;
          const int hi = p > q ? p : q, lo = p > q ? q : p;
          cs = fmaf(S[(32 + hi) * (33 + hi) / 2 + 32 + lo], in[(32 + q) * NR + r], cs);
        }
        yc = cs;
      }
    }
    __syncwarp();
  }
}

// Waits for the phase of the given parity of bar; gives up (false) after a bounded number of polls.
__device__ __forceinline__ bool mbar_wait_parity(unsigned long long* bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr int ENG_NBUF = 16;   // k_solve depth code of the two-warp steps with a ring per warp
constexpr int ENG_D = 3;       // line blocks in flight per warp

// Line blocks of the two-warp steps: either resident (every block of the box in shared memory,
// one mbarrier each, copied at the start) or streamed, each warp through its own ring of ENG_D
// slots refilled by a bulk copy as soon as the warp has used a slot.  A warp takes its blocks in
// a fixed order, numbered across the refinement passes (seq): warp 0 lines 0..m-1, m, then m-1
// down to lo_keep; warp 1 lines h-1 down to m+1, then m+1 up to hi_keep.
struct LineSrc {
  bool ring;
  const float* Lb;             // resident blocks
  unsigned long long* bars;    // resident: one per line; ring: [2][ENG_D]
  const float* Lg;             // ring: the box's blocks in global memory
  float* slots;                // ring: [2][ENG_D][LS]
  int LS;
};

__device__ __forceinline__ int eng_line(const Twist& tw, int wid, int k) {
  if (wid == 0) return k <= tw.m ? k : 2 * tw.m - k;
  const int ne = tw.h - 1 - tw.m;
  return k < ne ? tw.h - 1 - k : tw.m + 1 + (k - ne);
}
__device__ __forceinline__ int eng_count(const Twist& tw, int wid) {
  return wid == 0 ? tw.m + 1 + (tw.m - tw.lo_keep) : (tw.h - 1 - tw.m) + (tw.hi_keep - tw.m);
}

template <int W, int NR, bool EXACT>
__device__ bool twisted_engine(const Twist& tw, int w_rt, const LineSrc& src, int& base, float* Y, const float* Ec,
                               float* cb, float* xm, float* tv, float* part_all) {
  const int w = EXACT ? W : w_rt;
  constexpr int C = W > 32 ? W - 32 : 0;
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int h = tw.h, m = tw.m, LS = src.LS;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  float* part = part_all + (wid & 1) * (C > 0 ? C : 1) * NR * 32;
  const int xr = lane < w ? lane : -1;                       // this lane's row
  const int xc = (C > 0 && lane < C * NR) ? 32 + lane / NR : -1;   // its corner row (one rhs)
  const int rc = (C > 0 && lane < C * NR) ? lane % NR : 0;
  const bool xc_on = xc >= 0 && xc < w;
  float y[NR], yc;
  const int nseq = wid < 2 ? eng_count(tw, wid) : 0;
  // ring: lane 0 of the warp issues the copy of block k of this pass into slot (base + k) % ENG_D
  auto issue = [&](int k) {
    if (!src.ring || wid >= 2 || lane != 0 || k >= nseq) return;
    const int gk = base + k, slot = gk % ENG_D;
    float* dst = src.slots + ((size_t)wid * ENG_D + slot) * LS;
    bulk_load(dst, src.Lg + (size_t)eng_line(tw, wid, k) * LS, (unsigned)(LS * sizeof(float)),
              &src.bars[wid * ENG_D + slot]);
  };
  // block k of this pass: refill the slot freed by block k - 1, then wait for block k
  auto fetch = [&](int k) -> const float* {
    const float* S;
    bool ok;
    if (src.ring) {
      issue(k + ENG_D - 1);
      const int gk = base + k, slot = gk % ENG_D;
      ok = mbar_wait_parity(&src.bars[wid * ENG_D + slot], (unsigned)(gk / ENG_D) & 1u);
      S = src.slots + ((size_t)wid * ENG_D + slot) * LS;
    } else {
      const int L = eng_line(tw, wid, k);
      ok = mbar_wait0(&src.bars[L]);
      S = src.Lb + (size_t)L * LS;
    }
    if (!ok && lane == 0) s_fail = 1;
    __syncwarp();
    return S;
  };
  for (int k = 0; k < ENG_D - 1; ++k) issue(k);
  int k = 0;
  // ---- elimination: warp 0 from the top (u_{A+1} += E_{A+1} S_A^-1 u_A), warp 1 from the bottom
  //      (u_{B-1} += E_B S_B^-1 u_B, into cb at the middle line)
  // the couplings of a step's outputs are loaded before its product (they may come from global memory)
  auto ecpl = [&](int line, int x) -> float { return x >= 0 ? Ec[(size_t)line * w + x] : 0.f; };
  const int xr32 = (xr >= 0 && xr < 32) ? xr : -1, xcv = xc_on ? xc : -1;
  if (wid == 0) {
    for (int A = 0; A < m; ++A, ++k) {
      const float er = ecpl(A + 1, xr32), ec = ecpl(A + 1, xcv);
      const float* S = fetch(k);
      warp_line_product<W, NR, EXACT>(S, Y + (size_t)A * w * NR, w, lane, y, yc, part);
      float* dst = Y + (size_t)(A + 1) * w * NR;
      if (xr32 >= 0)
#pragma unroll
        for (int r = 0; r < NR; ++r) dst[xr32 * NR + r] += er * y[r];
      if (xc_on) dst[xc * NR + rc] += ec * yc;
      __syncwarp();
    }
  } else if (wid == 1) {
    for (int B = h - 1; B >= m + 1; --B, ++k) {
      const float er = ecpl(B, xr32), ec = ecpl(B, xcv);
      const float* S = fetch(k);
      warp_line_product<W, NR, EXACT>(S, Y + (size_t)B * w * NR, w, lane, y, yc, part);
      float* dst = B - 1 == m ? cb : Y + (size_t)(B - 1) * w * NR;
      if (xr32 >= 0)
#pragma unroll
        for (int r = 0; r < NR; ++r) dst[xr32 * NR + r] += er * y[r];
      if (xc_on) dst[xc * NR + rc] += ec * yc;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int t = tid; t < w * NR; t += blockDim.x) Y[(size_t)m * w * NR + t] += cb[t];
  __syncthreads();
  float* tA0 = tv;
  float* tA1 = tv + w * NR;
  float* tB0 = tv + 2 * w * NR;
  float* tB1 = tv + 3 * w * NR;
  // ---- middle line: x_m = S_m^-1 u_m; the first back inputs u_{m-1} + E_m x_m, u_{m+1} + E_{m+1} x_m
  if (wid == 0) {
    const float eu_r = ecpl(m, xr32), eu_c = ecpl(m, xcv);
    const float ed_r = m + 1 < h ? ecpl(m + 1, xr32) : 0.f, ed_c = m + 1 < h ? ecpl(m + 1, xcv) : 0.f;
    const float* S = fetch(k++);
    warp_line_product<W, NR, EXACT>(S, Y + (size_t)m * w * NR, w, lane, y, yc, part);
    const bool up = m - 1 >= tw.lo_keep, dn = m + 1 <= tw.hi_keep;
    auto emit = [&](int x, int r, float v, float eu, float ed) {
      xm[x * NR + r] = v;
      if (up) tA0[x * NR + r] = Y[((size_t)(m - 1) * w + x) * NR + r] + eu * v;
      if (dn) tB0[x * NR + r] = Y[((size_t)(m + 1) * w + x) * NR + r] + ed * v;
    };
    if (xr32 >= 0)
#pragma unroll
      for (int r = 0; r < NR; ++r) emit(xr32, r, y[r], eu_r, ed_r);
    if (xc_on) emit(xc, rc, yc, eu_c, ed_c);
    __syncwarp();
  }
  __syncthreads();
  // ---- back substitution: x_A = S_A^-1 (u_A + E_{A+1} x_{A+1}) upwards from m - 1 (warp 0),
  //      x_B = S_B^-1 (u_B + E_B x_{B-1}) downwards from m + 1 (warp 1)
  if (wid == 0) {
    int t = 0;
    for (int A = m - 1; A >= tw.lo_keep; --A, ++t, ++k) {
      const float* in = (t & 1) ? tA1 : tA0;
      float* nx = (t & 1) ? tA0 : tA1;
      const float er = ecpl(A, xr32), ec = ecpl(A, xcv);
      const float* S = fetch(k);
      warp_line_product<W, NR, EXACT>(S, in, w, lane, y, yc, part);
      const bool more = A - 1 >= tw.lo_keep;
      auto emit = [&](int x, int r, float v, float e) {
        Y[((size_t)A * w + x) * NR + r] = v;
        if (more) nx[x * NR + r] = Y[((size_t)(A - 1) * w + x) * NR + r] + e * v;
      };
      if (xr32 >= 0)
#pragma unroll
        for (int r = 0; r < NR; ++r) emit(xr32, r, y[r], er);
      if (xc_on) emit(xc, rc, yc, ec);
      __syncwarp();
    }
  } else if (wid == 1) {
    int t = 0;
    for (int B = m + 1; B <= tw.hi_keep; ++B, ++t, ++k) {
      const float* in = (t & 1) ? tB1 : tB0;
      float* nx = (t & 1) ? tB0 : tB1;
      const float er = B + 1 < h ? ecpl(B + 1, xr32) : 0.f, ec = B + 1 < h ? ecpl(B + 1, xcv) : 0.f;
      const float* S = fetch(k);
      warp_line_product<W, NR, EXACT>(S, in, w, lane, y, yc, part);
      const bool more = B + 1 <= tw.hi_keep;
      auto emit = [&](int x, int r, float v, float e) {
        Y[((size_t)B * w + x) * NR + r] = v;
        if (more) nx[x * NR + r] = Y[((size_t)(B + 1) * w + x) * NR + r] + e * v;
      };
      if (xr32 >= 0)
#pragma unroll
        for (int r = 0; r < NR; ++r) emit(xr32, r, y[r], er);
      if (xc_on) emit(xc, rc, yc, ec);
      __syncwarp();
    }
  }
  base += nseq;
  __syncthreads();
  if (s_fail && src.ring && wid < 2 && lane == 0) {
    // a copy never arrived: let this warp's copies in flight land (bounded) before returning
    for (int kk = 0; kk < ENG_D; ++kk) {
      const int gk = base - 1 - kk;
      if (gk >= 0) (void)mbar_wait_parity(&src.bars[wid * ENG_D + gk % ENG_D], (unsigned)(gk / ENG_D) & 1u);
    }
  }
  __syncthreads();
  return s_fail == 0;
}

// Position of cell (x, J) on the perimeter of a w x h box (-1 inside): the first line, the last
// line, then the first and the last column between them.
__device__ __forceinline__ int perim_index(int x, int J, int w, int h) {
  if (J == 0) return x;
  if (J == h - 1) return w + x;
  if (x == 0) return 2 * w + J - 1;
  if (x == w - 1) return 2 * w + (h - 2) + J - 1;
  return -1;
}

// NBUF steps of line blocks in flight (two blocks per step; prefetch distance NBUF - 1), or, for
// NBUF = 0, the whole box resident: every line block is copied once at the start (one bulk copy and
// one mbarrier per line, issued in the order the elimination uses them) and serves both the
// elimination and the back substitution.
template <typename T, int MODE, int NR, int NBUF>
__global__ void __launch_bounds__(NBUF == ENG_NBUF ? 64 : 512, 1) k_solve(Geo g, SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool RES = NBUF == 0;
  constexpr bool ENG = NBUF == ENG_NBUF;   // FP32 two-warp steps, a line ring per warp (64 threads)
  const int s = (MODE == MODE_SCHWARZ && a.colour >= 0) ? colour_box(g, a.colour, blockIdx.x) : (int)blockIdx.x;
  // the particular solve runs on the extended region when there is one (the source term's basis
  // function is built there like the others; its restriction to Omega_s is psi_s0)
  const bool ohat = (MODE == MODE_INFORMED || MODE == MODE_SCHWARZ || (MODE == MODE_PARTICULAR && g.l > 0));
  const Box b = box_of(g, s, ohat);
  const int w = b.w, hgt = b.h, LS = a.LS;
  T* Lb = reinterpret_cast<T*>(smem_raw);    // [NBUF][2][LS] line blocks, or [hgt][LS] (resident)
  T* Y = Lb + (RES ? (size_t)hgt * LS : ENG ? (size_t)2 * ENG_D * LS : (size_t)2 * NBUF * LS);  // [hgt][w][NR]: b, u, then x
  T* tv = Y + (size_t)hgt * w * NR;          // [4][w][NR] ping-pong inputs of the back steps (top, bottom)
  T* xm = tv + 4 * w * NR;                   // [w][NR] x of the middle line
  T* cb = xm + w * NR;                       // [w][NR] bottom contribution to the middle (odd h)
  T* Ec = reinterpret_cast<T*>(              // [hgt][w] line couplings (16-byte aligned, padded copy)
      smem_raw + ((reinterpret_cast<unsigned char*>(cb + w * NR) - smem_raw + 15) & ~(size_t)15));
  const int ecn = ENG ? 0 : (hgt * w + 3) & ~3;   // the ring variant reads the couplings from global memory
  unsigned long long* bars =                 // [hgt] line-block barriers (resident), [2][ENG_D] (ring)
      reinterpret_cast<unsigned long long*>(smem_raw + ((reinterpret_cast<unsigned char*>(Ec + ecn) - smem_raw + 7) & ~(size_t)7));
  // FP32 set-up solves (informed spaces, basis) may take one step of iterative refinement (when
  // given the box's FP64 line coefficients): the first solution x0 is kept in X0, the residual
  // b - A x0 is formed in FP64 and solved again, and the outputs use x0 + delta in FP64
  const bool REF = sizeof(T) == 4 && (MODE == MODE_INFORMED || MODE == MODE_BASIS) && a.coef != nullptr;
  T* X0 = reinterpret_cast<T*>(                // [hgt][w][NR] first solution (REF only)
      smem_raw + ((reinterpret_cast<unsigned char*>(bars + (ENG ? 2 * ENG_D : hgt)) - smem_raw + 15) & ~(size_t)15));
  float* part_all = reinterpret_cast<float*>(  // [2 warps][4][NR][32] corner-row sums (FP32 two-warp steps)
      smem_raw + ((reinterpret_cast<unsigned char*>(X0 + (REF ? (size_t)hgt * w * NR : 0)) - smem_raw + 15) &
                  ~(size_t)15));
  // REF: the right-hand side on the box perimeter in FP64 [2w + 2h - 4][NR] (it is zero inside), kept
  // from the prologue for the refinement residual
  double* bE = reinterpret_cast<double*>(
      smem_raw + ((reinterpret_cast<unsigned char*>(part_all + 2 * 4 * NR * 32) - smem_raw + 15) & ~(size_t)15));
  const int tid = threadIdx.x, nt = blockDim.x;
  const T* Lg = reinterpret_cast<const T*>(a.Linv) + (size_t)s * box_stride(w, hgt, LS);
  // the couplings join the first copy group (ring) or their own group (resident)
  for (int c = tid; c < ecn * (int)sizeof(T) / 16; c += nt)
    cp_async16(reinterpret_cast<unsigned char*>(Ec) + 16 * c, reinterpret_cast<const unsigned char*>(Lg + (size_t)hgt * LS) + 16 * c);
  if (RES || ENG) cp_async_commit();
  Twist tw;
  tw.h = hgt;
  tw.m = hgt / 2;
  tw.nf = tw.m > hgt - 1 - tw.m ? tw.m : hgt - 1 - tw.m;
  // a restricted Schwarz solve keeps only the lines of its subdomain; an extended particular solve
  // also keeps the line beyond each y side, which holds the outside cells of that side's faces
  tw.lo_keep = MODE == MODE_SCHWARZ ? g.l : (ohat ? g.l - 1 : 0);
  tw.hi_keep = MODE == MODE_SCHWARZ ? hgt - 1 - g.l : (ohat ? hgt - g.l : hgt - 1);
  {
    const int nt_ = tw.m - tw.lo_keep, nb_ = tw.hi_keep - tw.m;
    tw.nb = nt_ > nb_ ? nt_ : nb_;
    if (tw.nb < 0) tw.nb = 0;
  }
  const int nsteps = tw.nf + 1 + tw.nb;
  auto issue_step = [&](int st) {
    if (RES || ENG) return;
    if (st < nsteps) {
      int A, B;
      tw.lines(st, A, B);
      T* slot = Lb + (size_t)(st % (NBUF > 0 ? NBUF : 1)) * 2 * LS;
      issue_line(slot, Lg + (size_t)(A > 0 ? A : 0) * LS, LS, A >= 0);
      issue_line(slot + LS, Lg + (size_t)(B > 0 ? B : 0) * LS, LS, B >= 0);
    }
    cp_async_commit();  // one group per step, empty past the last, so the wait count stays uniform
  };
  if constexpr (RES) {
    if (tid == 0) {
      for (int L = 0; L < hgt; ++L) mbar_init(&bars[L], 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
      const unsigned bytes = (unsigned)(LS * sizeof(T));
      for (int t = 0; t < tw.nf; ++t) {
        if (t < tw.m) bulk_load(Lb + (size_t)t * LS, Lg + (size_t)t * LS, bytes, &bars[t]);
        const int B = hgt - 1 - t;
        if (B >= tw.m + 1) bulk_load(Lb + (size_t)B * LS, Lg + (size_t)B * LS, bytes, &bars[B]);
      }
      bulk_load(Lb + (size_t)tw.m * LS, Lg + (size_t)tw.m * LS, bytes, &bars[tw.m]);
    }
  } else if constexpr (ENG) {
    if (tid == 0) {
      for (int k = 0; k < 2 * ENG_D; ++k) mbar_init(&bars[k], 1);
      mbar_init_fence();
    }
    __syncthreads();
  } else {
    for (int p = 0; p < NBUF - 1; ++p) issue_step(p);  // NBUF = 1: no prefetch, each step loads its own lines
  }

  // ---------------- right-hand sides into Y
  for (int k = tid; k < hgt * w * NR; k += nt) Y[k] = (T)0;
  for (int k = tid; k < w * NR; k += nt) cb[k] = (T)0;
  if (REF)
    for (int k = tid; k < (2 * w + 2 * hgt - 4) * NR; k += nt) bE[k] = 0.0;
  __syncthreads();
  bool staged = false;
  if constexpr (sizeof(T) == 4 && NR == 1 && (MODE == MODE_PARTICULAR || MODE == MODE_SCHWARZ)) {
    if (a.in32 != nullptr) {
      // one round of 4-byte asynchronous copies of the box's cells (cells off the grid stay 0)
      for (int k = tid; k < hgt * w; k += nt) {
        const int J = k / w, x = k - J * w;
        const int gx = b.ox + x, gy = b.oy + J;
        if (active(g, gx, gy)) {
          const unsigned sa = (unsigned)__cvta_generic_to_shared(Y + k);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(a.in32 + (size_t)gy * g.nx + gx)
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
      staged = true;
    }
  }
  if (staged) {
  } else if (MODE == MODE_PARTICULAR) {
    // four cells per thread per pass, all loads before the stores
    const double* __restrict__ rin = a.in;
    for (int k0 = tid; k0 < hgt * w; k0 += 4 * nt) {
      double v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = k0 + e * nt, J = k / w, x = k % w;
        const int gx = b.ox + x, gy = b.oy + J;
        v[e] = (k < hgt * w && active(g, gx, gy)) ? rin[(size_t)gy * g.nx + gx] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k0 + e * nt < hgt * w) Y[(k0 + e * nt) * NR] = (T)v[e];
    }
  } else if (MODE == MODE_SCHWARZ) {
    // rho = r - A z on the box, from the sweep's input z (read only; the output goes elsewhere),
    // in the precision of the local solve; four cells per thread per pass, all loads first
    const double* __restrict__ z = a.zin;
    const double* __restrict__ rin = a.in;
    const double* __restrict__ Txg = g.Tx;
    const double* __restrict__ Tyg = g.Ty;
    for (int k0 = tid; k0 < hgt * w; k0 += 4 * nt) {
      double zc[4], zw[4], ze[4], zs[4], zn[4], t0[4], t1[4], t2[4], t3[4], rv[4];
      bool on[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = k0 + e * nt, J = k / w, x = k % w;
        const int gx = b.ox + x, gy = b.oy + J;
        on[e] = k < hgt * w && active(g, gx, gy);
        zc[e] = zw[e] = ze[e] = zs[e] = zn[e] = t0[e] = t1[e] = t2[e] = t3[e] = rv[e] = 0.0;
        if (on[e]) {
          const size_t c = (size_t)gy * g.nx + gx;
          zc[e] = z[c];
          if (gx > 0) zw[e] = z[c - 1];
          if (gx < g.nx - 1) ze[e] = z[c + 1];
          if (gy > 0) zs[e] = z[c - g.nx];
          if (gy < g.ny - 1) zn[e] = z[c + g.nx];
          const size_t cx = (size_t)gy * (g.nx + 1) + gx;
          t0[e] = Txg[cx];
          t1[e] = Txg[cx + 1];
          t2[e] = Tyg[c];
          t3[e] = Tyg[c + g.nx];
          rv[e] = rin[c];
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (!on[e]) continue;
        const T c0 = (T)zc[e];
        const T wx = (T)t1[e] * (c0 - (T)ze[e]) - (T)t0[e] * ((T)zw[e] - c0);
        const T wy = (T)t3[e] * (c0 - (T)zn[e]) - (T)t2[e] * ((T)zs[e] - c0);
        Y[(k0 + e * nt) * NR] = (T)rv[e] - (wx + wy);
      }
    }
  } else if (MODE == MODE_INFORMED) {
    // lambda^r = 1 on the faces of Robin side r of the oversampled box
    int rl_inf;
    const double* rt_inf = robin_tab(g, s, true, rl_inf);
    for (int r = 0; r < 4; ++r) {
      if (!robin_side(g, s, r)) continue;
      const int len = (r < 2) ? hgt : w;
      for (int t = tid; t < len; t += nt) {
        int x, J, ax, dir;
        switch (r) {
          case 0: x = 0; J = t; ax = 0; dir = -1; break;
          case 1: x = w - 1; J = t; ax = 0; dir = +1; break;
          case 2: x = t; J = 0; ax = 1; dir = -1; break;
          default: x = t; J = hgt - 1; ax = 1; dir = +1; break;
        }
        const int gx = b.ox + x, gy = b.oy + J;
        if (!active(g, gx, gy)) continue;
        double lam = 1.0;
        if (a.q) {  // position along the side of the oversampled region (clipped to the grid)
          const int lo = ax == 0 ? max(b.oy, 0) : max(b.ox, 0);
          const int hi = ax == 0 ? min(b.oy + hgt, g.ny) : min(b.ox + w, g.nx);
          lam = side_fn(a.q, (ax == 0 ? gy : gx) - lo, hi - lo);
        }
        const double bv = (rt_inf ? rt_inf[r * rl_inf + t] : face_tr(g, gx, gy, ax, dir, nullptr, nullptr)) * lam;
        Y[(J * w + x) * NR + r] += (T)bv;
        if (REF) bE[perim_index(x, J, w, hgt) * NR + r] += bv;
      }
      __syncthreads();
    }
  } else {  // MODE_BASIS: t_R phi^r on the Gamma faces of each Robin side
    for (int k = 0; k < 4; ++k) {
      if (!robin_side(g, s, k)) continue;
      const int len = side_len(g, s, k);
      for (int t = tid; t < len; t += nt) {
        int gx, gy, ox2, oy2;
        double Tf;
        gamma_face(g, s, k, t, gx, gy, ox2, oy2, Tf);
        const double tr = g.gtr[(((size_t)s * 4 + k) * g.smax + t) * 4];
        const int x = gx - b.ox, J = gy - b.oy;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const double ph = a.in[((((size_t)s * 4 + r) * g.nq + a.q) * 4 + k) * g.smax + t];
          Y[(J * w + x) * NR + r] += (T)(tr * ph);
          if (REF) bE[perim_index(x, J, w, hgt) * NR + r] += tr * ph;
        }
      }
      __syncthreads();
    }
  }
  if constexpr (RES || ENG) cp_async_wait<0>();  // couplings (each thread waits for its own copies)

  const int m = tw.m;
  T* tA0 = tv;                   // top back inputs (ping-pong)
  T* tA1 = tv + w * NR;
  T* tB0 = tv + 2 * w * NR;      // bottom back inputs (ping-pong)
  T* tB1 = tv + 3 * w * NR;
  int eng_base = 0;   // line blocks the two-warp steps have taken so far (ring slots and phases)
  for (int pass = 0; pass < (REF ? 2 : 1); ++pass) {
  if (REF && pass == 1) {
    // x0 aside; r = b - A x0 in FP64 per cell (A from the box's FP64 line coefficients: diagonal d,
    // x coupling o to the right, y coupling e to the line above), rounded into Y for the second solve
    for (int k = tid; k < hgt * w * NR; k += nt) X0[k] = Y[k];
    for (int k = tid; k < w * NR; k += nt) cb[k] = (T)0;
    __syncthreads();
    for (int c = tid; c < hgt * w; c += nt) {
      const int J = c / w, x = c - J * w;
      const double* cf = a.coef + (((size_t)s * hgt + J) * w + x) * 3;
      const double d = cf[0], o = cf[1], e = cf[2];
      const double oL = x > 0 ? cf[-3 + 1] : 0.0, eD = J + 1 < hgt ? cf[3 * (size_t)w + 2] : 0.0;
      const int gx = b.ox + x, gy = b.oy + J;
      const bool on = active(g, gx, gy);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double ax = d * (double)X0[c * NR + r];
        if (x + 1 < w) ax -= o * (double)X0[(c + 1) * NR + r];
        if (x > 0) ax -= oL * (double)X0[(c - 1) * NR + r];
        if (J > 0) ax -= e * (double)X0[(c - w) * NR + r];
        if (J + 1 < hgt) ax -= eD * (double)X0[(c + w) * NR + r];
        // the right-hand side, kept in FP64 on the perimeter by the prologue
        const int pe = perim_index(x, J, w, hgt);
        const double bv = (on && pe >= 0) ? bE[pe * NR + r] : 0.0;
        Y[c * NR + r] = (T)(bv - ax);
      }
    }
    __syncthreads();
    if constexpr (!RES && !ENG)
      for (int p = 0; p < NBUF - 1; ++p) issue_step(p);
  }
  bool two_warp = false;
  if constexpr ((RES || ENG) && sizeof(T) == 4) {
    // FP32 boxes up to 36 wide: the two-warp steps (no block barrier per step), on the resident
    // blocks or on a ring per warp (the launcher takes ENG only for such boxes)
    if (ENG || (w <= 36 && hgt >= 2)) {
      LineSrc src;
      src.ring = ENG;
      src.Lb = reinterpret_cast<const float*>(Lb);
      src.bars = bars;
      src.Lg = reinterpret_cast<const float*>(Lg);
      src.slots = reinterpret_cast<float*>(Lb);
      src.LS = LS;
      float* Yf = reinterpret_cast<float*>(Y);
      const float* Ef = reinterpret_cast<const float*>(ENG ? Lg + (size_t)hgt * LS : Ec);
      float* cf = reinterpret_cast<float*>(cb);
      float* xf = reinterpret_cast<float*>(xm);
      float* tf = reinterpret_cast<float*>(tv);
      // exact-width instantiations for boxes 32 and 36 wide (no per-column width tests)
      const bool ok = w == 32   ? twisted_engine<32, NR, true>(tw, w, src, eng_base, Yf, Ef, cf, xf, tf, part_all)
                      : w == 36 ? twisted_engine<36, NR, true>(tw, w, src, eng_base, Yf, Ef, cf, xf, tf, part_all)
                      : w <= 32 ? twisted_engine<32, NR, false>(tw, w, src, eng_base, Yf, Ef, cf, xf, tf, part_all)
                                : twisted_engine<36, NR, false>(tw, w, src, eng_base, Yf, Ef, cf, xf, tf, part_all);
      if (!ok) {
        if (tid == 0) {
          atomicOr(a.flags, FLAG_TIMEOUT);
          if (RES)
            for (int L = 0; L < hgt; ++L) (void)mbar_wait0(&bars[L]);
        }
        __syncthreads();
        return;
      }
      two_warp = true;
    }
  }
  for (int st = 0; st < (two_warp ? 0 : nsteps); ++st) {
    int A, B;
    tw.lines(st, A, B);
    const T* LA;
    const T* LBk;
    if constexpr (RES) {
      bool ok = true;
      if (A >= 0) ok = mbar_wait0(&bars[A]);
      if (B >= 0) ok = mbar_wait0(&bars[B]) && ok;
      if (__syncthreads_or(!ok)) {
        // a line block never arrived: report, let every copy of this CTA land (bounded), stop
        if (tid == 0) {
          atomicOr(a.flags, FLAG_TIMEOUT);
          for (int L = 0; L < hgt; ++L) (void)mbar_wait0(&bars[L]);
        }
        __syncthreads();
        return;
      }
      LA = Lb + (size_t)(A > 0 ? A : 0) * LS;
      LBk = Lb + (size_t)(B > 0 ? B : 0) * LS;
    } else {
      if constexpr (NBUF == 1) {
        __syncthreads();  // the previous step is done with the single slot
        issue_step(st);
        cp_async_wait<0>();
        __syncthreads();
      } else {
        cp_async_wait<NBUF - 2>();
        __syncthreads();
        issue_step(st + NBUF - 1);
      }
      LA = Lb + (size_t)(st % (NBUF > 0 ? NBUF : 1)) * 2 * LS;
      LBk = LA + LS;
    }
    if (st < tw.nf) {
      // ---- elimination: top line A (u_{A+1} += E_{A+1} S_A^-1 u_A), bottom line B
      //      (u_{B-1} += E_B S_B^-1 u_B); the bottom's last contribution to the middle goes to cb
      //      when the two ends reach the middle in the same step (odd h)
      const bool to_cb = B == m + 1 && A == m - 1;
      gemv_pair<T, NR>(LA, Y + (size_t)(A > 0 ? A : 0) * w * NR, A >= 0, LBk, Y + (size_t)(B > 0 ? B : 0) * w * NR,
                       B >= 0, w, [&](int half, int i, int r, T v) {
                         if (half == 0) {
                           Y[((size_t)(A + 1) * w + i) * NR + r] += Ec[(A + 1) * w + i] * v;
                         } else {
                           T* dst = to_cb ? cb : Y + (size_t)(B - 1) * w * NR;
                           dst[i * NR + r] += Ec[B * w + i] * v;
                         }
                       });
    } else if (st == tw.nf) {
      // ---- middle line: x_m = S_m^-1 u_m; first back inputs u_{m-1} + E_m x_m, u_{m+1} + E_{m+1} x_m
      if (hgt & 1) {
        for (int k = tid; k < w * NR; k += nt) Y[(size_t)m * w * NR + k] += cb[k];
        __syncthreads();
      }
      const bool up = m - 1 >= tw.lo_keep, dn = m + 1 <= tw.hi_keep;
      gemv_pair<T, NR>(LA, Y + (size_t)m * w * NR, true, LA, Y, false, w, [&](int, int i, int r, T v) {
        xm[i * NR + r] = v;
        if (up) tA0[i * NR + r] = Y[((size_t)(m - 1) * w + i) * NR + r] + Ec[m * w + i] * v;
        if (dn) tB0[i * NR + r] = Y[((size_t)(m + 1) * w + i) * NR + r] + Ec[(m + 1) * w + i] * v;
      });
    } else {
      // ---- back substitution: x_A = S_A^-1 (u_A + E_{A+1} x_{A+1}), x_B = S_B^-1 (u_B + E_B x_{B-1})
      const int t = st - tw.nf - 1;
      const T* inA = (t & 1) ? tA1 : tA0;
      T* nxA = (t & 1) ? tA0 : tA1;
      const T* inB = (t & 1) ? tB1 : tB0;
      T* nxB = (t & 1) ? tB0 : tB1;
      const bool moreA = A - 1 >= tw.lo_keep, moreB = B + 1 <= tw.hi_keep;
      gemv_pair<T, NR>(LA, inA, A >= 0, LBk, inB, B >= 0, w, [&](int half, int i, int r, T v) {
        if (half == 0) {
          Y[((size_t)A * w + i) * NR + r] = v;
          if (moreA) nxA[i * NR + r] = Y[((size_t)(A - 1) * w + i) * NR + r] + Ec[A * w + i] * v;
        } else {
          Y[((size_t)B * w + i) * NR + r] = v;
          if (moreB) nxB[i * NR + r] = Y[((size_t)(B + 1) * w + i) * NR + r] + Ec[(B + 1) * w + i] * v;
        }
      });
    }
  }
  if constexpr (!RES) cp_async_wait<0>();
  __syncthreads();
  for (int k = tid; k < w * NR; k += nt) Y[(size_t)m * w * NR + k] = xm[k];
  __syncthreads();
  }  // passes
  // the solution entry idx: x0 + delta after a refinement step, else the solve's result
  auto xv = [&](size_t idx) -> double { return REF ? (double)X0[idx] + (double)Y[idx] : (double)Y[idx]; };

  // ---------------- outputs
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (MODE == MODE_PARTICULAR) {
    // psi_s0 on Omega_s, and its side moments against the test functions of degree 0, 1.  The
    // Gamma-face coefficients [t_R, beta, T_f, |f| / tau] were stored by the basis solves.
    //   l = 0: the Robin traces with zero data, F = t_R x_c, |f| P = beta F;
    //   l > 0: the traces of the extended solution q, F = T_f (q_c - q_c'), |f| P = |f| q_c - (|f| / tau) F
    //          (equal to the Robin traces of the local solve with the informed particular data).
    const int lo = ohat ? g.l : 0;
    const int ws = sub_w(g, s), hs = sub_h(g, s);
    for (int k = tid; k < ws * hs; k += nt) {
      const int y = k / ws, x = k % ws;
      a.out[(size_t)(b.oy + lo + y) * g.nx + b.ox + lo + x] = (double)Y[(lo + y) * w + lo + x];
    }
    for (int kside = wid; kside < 4; kside += nw) {
      double F[2] = {0.0, 0.0}, Pw[2] = {0.0, 0.0};  // against the test functions of degree 0, 1
      if (robin_side(g, s, kside)) {
        const int len = side_len(g, s, kside);
        const double area = kside < 2 ? g.hy * g.hz : g.hx * g.hz;
        // inside cell of face t in box coordinates, and the step to its outside cell
        const int dx = kside == 0 ? -1 : (kside == 1 ? 1 : 0), dy = kside == 2 ? -1 : (kside == 3 ? 1 : 0);
        for (int t = lane; t < len; t += 32) {
          const int x = lo + (kside < 2 ? (kside == 0 ? 0 : g.sx - 1) : t);
          const int y = lo + (kside < 2 ? t : (kside == 2 ? 0 : g.sy - 1));
          const double* cf = g.gtr + (((size_t)s * 4 + kside) * g.smax + t) * 4;
          const double qc = (double)Y[y * w + x];
          double fl, pw;
          if (ohat) {
            fl = cf[2] * (qc - (double)Y[(y + dy) * w + x + dx]);
            pw = area * qc - cf[3] * fl;
          } else {
            fl = cf[0] * qc;
            pw = cf[1] * fl;
          }
#pragma unroll
          for (int qt = 0; qt < 2; ++qt)
            if (qt < g.nq) {
              const double wt = side_fn(qt, t, len);
              F[qt] += wt * fl;
              Pw[qt] += wt * pw;
            }
        }
      }
#pragma unroll
      for (int qt = 0; qt < 2; ++qt) {
        if (qt >= g.nq) break;
        const double Fs = warp_sum(F[qt]), Ps = warp_sum(Pw[qt]);
        if (lane == 0) {
          a.mom[(((size_t)s * 4 + kside) * g.nq + qt) * 2] = Fs;
          a.mom[(((size_t)s * 4 + kside) * g.nq + qt) * 2 + 1] = Ps;
        }
      }
    }
  } else if (MODE == MODE_SCHWARZ) {
    const int ws = sub_w(g, s), hs = sub_h(g, s);
    for (int k = tid; k < ws * hs; k += nt) {
      const int y = k / ws, x = k % ws;
      const int gx = b.ox + g.l + x, gy = b.oy + g.l + y;
      const size_t c = (size_t)gy * g.nx + gx;
      a.out[c] = a.zin[c] + (double)Y[(g.l + y) * w + g.l + x];
    }
  } else if (MODE == MODE_BASIS) {
    for (int k = tid; k < hgt * w * NR; k += nt) {
      const int r = k % NR, c = k / NR, J = c / w, x = c % w;
      if (active(g, b.ox + x, b.oy + J))
        a.out[((size_t)r * g.nq + a.q) * g.nx * g.ny + (size_t)(b.oy + J) * g.nx + b.ox + x] = xv(k);
    }
    // moments: 16 (side, function) pairs, one warp each
    for (int pr = wid; pr < 16; pr += nw) {
      const int kside = pr / 4, r = pr % 4;
      double F[2] = {0.0, 0.0}, Pw[2] = {0.0, 0.0};  // against the test functions of degree 0, 1
      if (robin_side(g, s, kside)) {
        const int len = side_len(g, s, kside);
        for (int t = lane; t < len; t += 32) {
          int gx, gy, ox2, oy2;
          double Tf;
          gamma_face(g, s, kside, t, gx, gy, ox2, oy2, Tf);
          const double* cf = g.gtr + (((size_t)s * 4 + kside) * g.smax + t) * 4;   // [t_R, beta, T_f, |f|/tau]
          const double tr = cf[0], beta = cf[1];
          const double area = kside < 2 ? g.hy * g.hz : g.hx * g.hz;
          const double ph = a.in[((((size_t)s * 4 + r) * g.nq + a.q) * 4 + kside) * g.smax + t];
          const double fl = tr * (xv(((size_t)(gy - b.oy) * w + (gx - b.ox)) * NR + r) - ph);
          const double pw = area * ph + beta * fl;
#pragma unroll
          for (int qt = 0; qt < 2; ++qt)
            if (qt < g.nq) {
              const double wt = side_fn(qt, t, len);
              F[qt] += wt * fl;
              Pw[qt] += wt * pw;
            }
        }
      }
      const int fn = r * g.nq + a.q;
#pragma unroll
      for (int qt = 0; qt < 2; ++qt) {
        if (qt >= g.nq) break;
        const double Fs = warp_sum(F[qt]), Ps = warp_sum(Pw[qt]);
        if (lane == 0) {
          a.mom[((((size_t)s * 4 + kside) * 4 * g.nq + fn) * g.nq + qt) * 2] = Fs;
          a.mom[((((size_t)s * 4 + kside) * 4 * g.nq + fn) * g.nq + qt) * 2 + 1] = Ps;
        }
      }
    }
  } else {  // MODE_INFORMED: phi_s^r on every Gamma face
    for (int k = 0; k < 4; ++k) {
      const int len = side_len(g, s, k);
      const bool rs = robin_side(g, s, k);
      for (int t = tid; t < len * NR; t += nt) {
        const int r = t % NR, f = t / NR;
        double ph = 0.0;
        if (rs && robin_side(g, s, r)) {
          int gx, gy, ox2, oy2;
          double Tf;
          gamma_face(g, s, k, f, gx, gy, ox2, oy2, Tf);
          const double* cf = g.gtr + (((size_t)s * 4 + k) * g.smax + f) * 4;   // [t_R, beta, T_f, |f|/tau]
          const double qc = xv(((size_t)(gy - b.oy) * w + (gx - b.ox)) * NR + r);
          const double qo = xv(((size_t)(oy2 - b.oy) * w + (ox2 - b.ox)) * NR + r);
          const double F = Tf * (qc - qo);
          const double area = k < 2 ? g.hy * g.hz : g.hx * g.hz;
          const double pi = qc - F * cf[3] / area;
          ph = -cf[1] * F / area + pi;
        }
        a.out[((((size_t)s * 4 + r) * g.nq + a.q) * 4 + k) * g.smax + f] = ph;
      }
    }
  }
}

template <typename T, int MODE, int NR, int NBUF>
static size_t solve_smem(const Geo& g, const SolveArgs& a, bool ohat) {
  const int w = g.sx + (ohat ? 2 * g.l : 0), h = g.sy + (ohat ? 2 * g.l : 0);
  const size_t lines = NBUF == 0 ? (size_t)h * a.LS : NBUF == ENG_NBUF ? 2 * ENG_D * (size_t)a.LS : 2 * NBUF * (size_t)a.LS;
  const size_t ecn = NBUF == ENG_NBUF ? 0 : ((size_t)h * w + 3) & ~(size_t)3;
  const bool REF = sizeof(T) == 4 && (MODE == MODE_INFORMED || MODE == MODE_BASIS) && a.coef != nullptr;
  return sizeof(T) * (lines + (size_t)h * w * NR + 6 * (size_t)w * NR + ecn) + 8 * (size_t)(NBUF == ENG_NBUF ? 2 * ENG_D : h) + 32 +
         (REF ? sizeof(T) * (size_t)h * w * NR + 16 : 0) +
         (sizeof(T) == 4 && (NBUF == 0 || NBUF == ENG_NBUF) ? 4 * (2 * 4 * NR * 32) + 16 : 0) +
         (REF ? 4 * (2 * 4 * NR * 32) + 8 * (size_t)(2 * w + 2 * h) * NR + 32 : 0);
}

template <typename T, int MODE, int NR, int NBUF>
static cudaError_t launch_solve_nb(const Geo& g, const SolveArgs& a, size_t sm, bool ohat, cudaStream_t st) {
  const cudaError_t e = raise_smem_limit<k_solve<T, MODE, NR, NBUF>>();
  if (e != cudaSuccess) return e;
  // two line products per step, LineTPR threads per row; at least four warps for the moment sums
  const int w = g.sx + (ohat ? 2 * g.l : 0);
  int threads = (2 * w * LineTPR<T>::value + 31) / 32 * 32;
  if (threads < 128) threads = 128;
  if (NBUF == ENG_NBUF) threads = 64;   // the two warps of the two-warp steps
  int grid = g.mx * g.my;
  if (MODE == MODE_SCHWARZ && a.colour >= 0)
    grid = ((g.mx - (a.colour & 1) + 1) / 2) * ((g.my - ((a.colour >> 1) & 1) + 1) / 2);
  if (grid == 0) return cudaSuccess;
  k_solve<T, MODE, NR, NBUF><<<grid, threads, sm, st>>>(g, a);
  count_launch(1);
  return cudaGetLastError();
}

// Line blocks: the built-in choice keeps the whole box resident for FP32 solves when two CTAs still
// fit on an SM (their steps are short, so a prefetch ring cannot run far enough ahead of memory
// latency), else eight steps in flight; FP64 solves keep four steps in flight; fewer when they would
// not fit next to the right-hand sides, down to one (no prefetch) for the widest boxes with four
// right-hand sides.  The depth changes no arithmetic, so the autotuner may replace that choice by
// the fastest depth that fits, timed on the first launch of the shape; a sweep that updates in
// place (one colour of a multiplicative sweep) is not repeatable and keeps the built-in choice.
template <typename T, int MODE, int NR>
static cudaError_t launch_solve_depth(const Geo& g, const SolveArgs& a, bool ohat, int nbuf, cudaStream_t st) {
  switch (nbuf) {
    case 0: return launch_solve_nb<T, MODE, NR, 0>(g, a, solve_smem<T, MODE, NR, 0>(g, a, ohat), ohat, st);
    case ENG_NBUF:
      if constexpr (sizeof(T) == 4)
        return launch_solve_nb<T, MODE, NR, ENG_NBUF>(g, a, solve_smem<T, MODE, NR, ENG_NBUF>(g, a, ohat), ohat, st);
      return cudaErrorInvalidValue;
    case 8: return launch_solve_nb<T, MODE, NR, 8>(g, a, solve_smem<T, MODE, NR, 8>(g, a, ohat), ohat, st);
    case 4: return launch_solve_nb<T, MODE, NR, 4>(g, a, solve_smem<T, MODE, NR, 4>(g, a, ohat), ohat, st);
    case 2: return launch_solve_nb<T, MODE, NR, 2>(g, a, solve_smem<T, MODE, NR, 2>(g, a, ohat), ohat, st);
    default: return launch_solve_nb<T, MODE, NR, 1>(g, a, solve_smem<T, MODE, NR, 1>(g, a, ohat), ohat, st);
  }
}

template <typename T, int MODE, int NR>
static cudaError_t launch_solve_t(const Geo& g, const SolveArgs& a, bool ohat, cudaStream_t st) {
  constexpr size_t kMaxSmem = 227 * 1024;
  constexpr size_t kBudget = 100 * 1024;  // keep two CTAs per SM when possible
  const size_t sm[6] = {solve_smem<T, MODE, NR, 0>(g, a, ohat), solve_smem<T, MODE, NR, 8>(g, a, ohat),
                        solve_smem<T, MODE, NR, 4>(g, a, ohat), solve_smem<T, MODE, NR, 2>(g, a, ohat),
                        solve_smem<T, MODE, NR, 1>(g, a, ohat), solve_smem<T, MODE, NR, ENG_NBUF>(g, a, ohat)};
  const int depth[6] = {0, 8, 4, 2, 1, ENG_NBUF};
  // FP32 boxes up to 36 wide (at least 2 ENG_D lines high) take the two-warp steps with a line
  // ring per warp by default
  const int bw = g.sx + (ohat ? 2 * g.l : 0), bh = g.sy + (ohat ? 2 * g.l : 0);
  const bool eng = sizeof(T) == 4 && bw <= 36 && bh >= 2 * ENG_D && sm[5] <= kMaxSmem;
  int builtin = 1;
  if (eng) builtin = ENG_NBUF;
  else if (sizeof(T) == 4 && sm[0] <= kBudget + 14 * 1024) builtin = 0;
  else if (sizeof(T) == 4 && sm[1] <= kBudget) builtin = 8;
  else if (sm[2] <= kMaxSmem) builtin = 4;
  else if (sm[3] <= kMaxSmem) builtin = 2;
  int cand[6], nc = 0;
  for (int i = 0; i < 6; ++i)
    if (sm[i] <= kMaxSmem && (i < 5 || eng)) cand[nc++] = depth[i];
  const bool repeatable = !(MODE == MODE_SCHWARZ && a.zin == a.out);
  if (repeatable && nc > 1) {
    const int w = g.sx + (ohat ? 2 * g.l : 0), h = g.sy + (ohat ? 2 * g.l : 0);
    const int key[6] = {(int)sizeof(T), MODE, NR, w, h, a.colour >= 0 ? -1 - a.colour : g.mx * g.my};
    cudaError_t err = cudaSuccess;
    const int pick = autotune(TUNE_LOCAL_SOLVE, key, nc, st,
                              [&](int i) { return launch_solve_depth<T, MODE, NR>(g, a, ohat, cand[i], st); }, &err);
    if (err != cudaSuccess) return err;
    if (pick >= 0) return launch_solve_depth<T, MODE, NR>(g, a, ohat, cand[pick], st);
  }
  return launch_solve_depth<T, MODE, NR>(g, a, ohat, builtin, st);
}

template <int MODE, int NR>
static cudaError_t launch_solve(const Geo& g, const SolveArgs& a, bool ohat, bool fp32, cudaStream_t st) {
  return fp32 ? launch_solve_t<float, MODE, NR>(g, a, ohat, st) : launch_solve_t<double, MODE, NR>(g, a, ohat, st);
}

// l = 0: the informed space is the side functions themselves, phi_s^{k,q} = degree-q function on side k
__global__ void k_phi_indicator(Geo g, double* phi) {
  const int s = blockIdx.x;
  const int per = 16 * g.nq * g.smax;
  for (int t = threadIdx.x; t < per; t += blockDim.x) {
    const int fn = t / (4 * g.smax), k = (t / g.smax) % 4, f = t % g.smax;
    const int r = fn / g.nq, q = fn % g.nq;
    const int len = side_len(g, s, k);
    double v = 0.0;
    if (r == k && f < len && robin_side(g, s, k)) v = side_fn(q, f, len);
    phi[(size_t)s * per + t] = v;
  }
}

cudaError_t launch_informed(const Geo& g, const void* Linv, int LS, bool fp32, double* phi, int q, int* flags,
                            cudaStream_t st, const double* coef) {
  if (g.l == 0) {
    if (q > 0) return cudaSuccess;  // one launch writes the functions of every degree
    k_phi_indicator<<<g.mx * g.my, 128, 0, st>>>(g, phi);
    count_launch(1);
    return cudaGetLastError();
  }
  SolveArgs a{Linv, LS, nullptr, phi, nullptr, nullptr, flags, -1, q, coef};
  return launch_solve<MODE_INFORMED, 4>(g, a, true, fp32, st);
}

cudaError_t launch_basis(const Geo& g, const void* Linv, int LS, bool fp32, const double* phi, int q, double* psi,
                         double* mom, int* flags, cudaStream_t st, const double* coef) {
  SolveArgs a{Linv, LS, phi, psi, mom, nullptr, flags, -1, q, coef};
  return launch_solve<MODE_BASIS, 4>(g, a, false, fp32, st);
}

// FP32 right-hand sides of the FP32 particular solves and additive sweeps, formed once on the grid
// (z == nullptr: r; else the sweep's residual r - A z in FP64, rounded once), so that each box
// fetches its cells with one round of asynchronous copies instead of forming them
__global__ void k_stage32(Geo g, const double* __restrict__ r, const double* __restrict__ z, float* __restrict__ out) {
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
  if (gx >= g.nx) return;
  const size_t c = (size_t)gy * g.nx + gx;
  double v = r[c];
  if (z) {
    const double zc = z[c];
    const double zw = gx > 0 ? z[c - 1] : 0.0, ze = gx < g.nx - 1 ? z[c + 1] : 0.0;
    const double zs = gy > 0 ? z[c - g.nx] : 0.0, zn = gy < g.ny - 1 ? z[c + g.nx] : 0.0;
    const size_t cx = (size_t)gy * (g.nx + 1) + gx;
    // r minus the four face fluxes, each from its difference: four subtractions and four FMAs
    v = fma(-g.Tx[cx + 1], zc - ze, v);
    v = fma(-g.Tx[cx], zc - zw, v);
    v = fma(-g.Ty[c + g.nx], zc - zn, v);
    v = fma(-g.Ty[c], zc - zs, v);
  }
  out[c] = (float)v;
}

cudaError_t launch_stage32(const Geo& g, const double* r, const double* z, float* out, cudaStream_t st) {
  dim3 grid((g.nx + 255) / 256, g.ny);
  k_stage32<<<grid, 256, 0, st>>>(g, r, z, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_particular(const Geo& g, const void* Linv, int LS, bool fp32, const double* r, double* psi0,
                              double* mom0, int* flags, cudaStream_t st, const float* in32) {
  SolveArgs a{Linv, LS, r, psi0, mom0, nullptr, flags, -1};
  if (fp32 && in32) a.in32 = in32;
  return launch_solve<MODE_PARTICULAR, 1>(g, a, g.l > 0, fp32, st);
}

// colour -1: every box (additive sweep, zin and zout distinct); colour c: the boxes of colour c only,
// in place allowed (zin == zout): boxes of one colour are two subdomains apart and the oversampling
// is narrower than a subdomain, so no box reads (region plus the stencil's one-cell rim) a cell
// that another box of its colour writes.
cudaError_t launch_schwarz(const Geo& g, const void* Linv, int LS, bool fp32, const double* r, const double* zin,
                           double* zout, int* flags, int colour, cudaStream_t st, const float* in32) {
  SolveArgs a{Linv, LS, r, zout, nullptr, zin, flags, colour};
  if (fp32 && in32 && colour < 0) a.in32 = in32;   // additive: every box from the same staged residual
  return launch_solve<MODE_SCHWARZ, 1>(g, a, true, fp32, st);
}

// Robin coefficients of every Gamma face of every subdomain, [S][4 sides][smax][t_R, beta, T_f,
// |f| / tau] (Eq. 6), formed once per set-up: the basis and informed solves and the particular
// solves' moments read them instead of evaluating the harmonic means and divisions per use
__global__ void k_gamma_coef(Geo g) {
  const int s = blockIdx.x;
  for (int u = threadIdx.x; u < 4 * g.smax; u += blockDim.x) {
    const int k = u / g.smax, t = u - k * g.smax;
    if (!robin_side(g, s, k) || t >= side_len(g, s, k)) continue;
    int gx, gy, ox2, oy2;
    double Tf, beta, tau;
    gamma_face(g, s, k, t, gx, gy, ox2, oy2, Tf);
    const double tr = face_tr(g, gx, gy, k / 2, (k & 1) ? 1 : -1, &beta, &tau);
    const double area = k < 2 ? g.hy * g.hz : g.hx * g.hz;
    double* cf = g.gtr + (((size_t)s * 4 + k) * g.smax + t) * 4;
    cf[0] = tr;
    cf[1] = beta;
    cf[2] = Tf;
    cf[3] = area / tau;
  }
}

cudaError_t launch_gamma_coef(const Geo& g, cudaStream_t st) {
  k_gamma_coef<<<g.mx * g.my, 128, 0, st>>>(g);
  count_launch(1);
  return cudaGetLastError();
}

// t_R (Eq. 6) of the Robin faces of each box, [S][4 sides][len] by the box's local position along
// the side (y for the x sides, x for the y sides): the faces from an in-grid cell on the box's
// outer row or column to an in-grid neighbour outside the box; 0 elsewhere.  Formed once per
// set-up, so the factorisations (a line per step, the Robin faces on its critical path) and the
// informed solves read the harmonic means and divisions instead of evaluating them.
__global__ void k_robin_tab(Geo g, int ohat, double* __restrict__ out, int len) {
  const int s = blockIdx.x;
  const Box b = box_of(g, s, ohat != 0);
  for (int u = threadIdx.x; u < 4 * len; u += blockDim.x) {
    const int k = u / len, t = u - k * len;
    const int x = k == 0 ? 0 : k == 1 ? b.w - 1 : t;
    const int J = k < 2 ? t : k == 2 ? 0 : b.h - 1;
    const bool on_side = k < 2 ? t < b.h : t < b.w;
    const int gx = b.ox + x, gy = b.oy + J;
    const int nx2 = gx + (k == 0 ? -1 : k == 1 ? 1 : 0), ny2 = gy + (k == 2 ? -1 : k == 3 ? 1 : 0);
    double v = 0.0;
    if (on_side && active(g, gx, gy) && active(g, nx2, ny2))
      v = face_tr(g, gx, gy, k / 2, (k & 1) ? 1 : -1, nullptr, nullptr);
    out[((size_t)s * 4 + k) * len + t] = v;
  }
}

cudaError_t launch_robin_tab(const Geo& g, bool ohat, double* out, cudaStream_t st) {
  k_robin_tab<<<g.mx * g.my, 128, 0, st>>>(g, ohat ? 1 : 0, out, ohat ? g.rlo : g.rll);
  count_launch(1);
  return cudaGetLastError();
}

// z = psi0 + sum over Robin sides k and degrees q of c_{s,k,q} psi_{k,q}   (reconstruction, per cell)
__global__ void k_reconstruct(Geo g, const double* __restrict__ psi0, const double* __restrict__ psi,
                              const int* __restrict__ cidx, const double* __restrict__ c, double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= g.nx) return;
  const int s = (j / g.sy) * g.mx + i / g.sx;
  const size_t cell = (size_t)j * g.nx + i;
  const size_t n = (size_t)g.nx * g.ny;
  double v = psi0[cell];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int ci = cidx[s * 4 + k];
    if (ci >= 0)
      for (int q = 0; q < g.nq; ++q) v += c[(size_t)ci * g.nq + q] * psi[(size_t)(k * g.nq + q) * n + cell];
  }
  z[cell] = v;
}

cudaError_t launch_reconstruct(const Geo& g, const double* psi0, const double* psi, const int* cidx, const double* c,
                               double* z, cudaStream_t st) {
  k_reconstruct<<<dim3((g.nx + 127) / 128, g.ny), 128, 0, st>>>(g, psi0, psi, cidx, c, z);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace mrcm
