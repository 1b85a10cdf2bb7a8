// Coupling system of MRCM-O (Eq. 13-14) with piecewise-constant M_H, V_H on each interface.
//
// Unknowns c_{s,k}: one per Robin side of each subdomain (canonical order: subdomain, then side).
// Rows: per interface e = (axis a, lower s, upper s'), the flux row
//   sum_f F_s(f) + F_s'(f) = 0  and the pressure row  sum_f |f| (P_s(f) - P_s'(f)) = 0,
// with the side moments of the basis traces (from the basis solves) as coefficients and the
// particular traces as right-hand side.  Rows are placed at a "home" position next to the unknowns
// they mostly depend on (flux row at (s, +a), pressure row at (s', -a)), which makes G banded with
// half-bandwidth about 4 m_x; it is factored by band LU with partial pivoting (row interchanges
// only) in LAPACK band layout: A(i, j) at ab[kv + i - j + j * ldab], kv = kl + ku, ldab = 2 kl + ku + 1.
#include <cooperative_groups.h>

#include "common.cuh"

namespace mrcm {

// G entries from the side moments mom[s][side][function r nq + q][test qt][F, |f|P]; ab must be
// zeroed.  Interface e has nq flux rows and nq pressure rows (one per test function qt), homed at
// row_home * nq + qt; unknown (t, side r, degree q) is column (off_t + rank_t(r)) nq + q.
__global__ void k_coarse_assemble(CoarseDev c, const double* __restrict__ mom, int E) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int kv = c.kl + c.ku, nq = c.nq, nf = 4 * nq;
  const int a = c.iface[3 * e], s = c.iface[3 * e + 1], s2 = c.iface[3 * e + 2];
  const int ks = 2 * a + 1, ks2 = 2 * a;  // +a side of s, -a side of s'
  for (int qt = 0; qt < nq; ++qt) {
    const int rf = c.home[2 * e] * nq + qt, rp = c.home[2 * e + 1] * nq + qt;
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < nq; ++q) {
        const int k1 = c.rank[6 * s + r];
        if (k1 >= 0) {
          const int col = (c.off[s] + k1) * nq + q;
          const double* m = mom + ((((size_t)s * 4 + ks) * nf + r * nq + q) * nq + qt) * 2;
          c.ab[(size_t)(kv + rf - col) + (size_t)col * c.ldab] = m[0];
          c.ab[(size_t)(kv + rp - col) + (size_t)col * c.ldab] = m[1];
        }
        const int k2 = c.rank[6 * s2 + r];
        if (k2 >= 0) {
          const int col = (c.off[s2] + k2) * nq + q;
          const double* m = mom + ((((size_t)s2 * 4 + ks2) * nf + r * nq + q) * nq + qt) * 2;
          c.ab[(size_t)(kv + rf - col) + (size_t)col * c.ldab] = m[0];
          c.ab[(size_t)(kv + rp - col) + (size_t)col * c.ldab] = -m[1];
        }
      }
  }
}

// Rows of test function qt of interface e (banded order) and their right-hand sides -(F_s + F_s'),
// -(P_s - P_s') from the particular side moments mom0[S][4 sides][nq tests][F, |f|P].
__device__ __forceinline__ void coarse_rhs_rows(const CoarseDev& c, const double* __restrict__ mom0, int e, int qt,
                                                int& rf, double& gf, int& rp, double& gp) {
  const int a = c.iface[3 * e], s = c.iface[3 * e + 1], s2 = c.iface[3 * e + 2];
  const int nq = c.nq;
  const double* m1 = mom0 + (((size_t)s * 4 + 2 * a + 1) * nq + qt) * 2;
  const double* m2 = mom0 + (((size_t)s2 * 4 + 2 * a) * nq + qt) * 2;
  rf = c.home[2 * e] * nq + qt;
  rp = c.home[2 * e + 1] * nq + qt;
  gf = -(m1[0] + m2[0]);
  gp = -(m1[1] - m2[1]);
}

__global__ void k_coarse_rhs(CoarseDev c, const double* __restrict__ mom0, int E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * c.nq) return;
  int rf, rp;
  double gf, gp;
  coarse_rhs_rows(c, mom0, t / c.nq, t % c.nq, rf, gf, rp, gp);
  c.g[rf] = gf;
  c.g[rp] = gp;
}

// Unblocked band LU with partial pivoting, one CTA.
__global__ void __launch_bounds__(512) k_gbtf2(CoarseDev c, int* flags) {
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  double* ab = c.ab;
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_jp, s_ju, s_ok;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  int ju = 0;
  for (int j = 0; j < n; ++j) {
    const int km = min(kl, n - 1 - j);
    // pivot: first index of the largest magnitude in column j, rows j..j+km
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = tid; i <= km; i += nt) {
      const double v = fabs(ab[(size_t)(kv + i) + (size_t)j * ld]);
      if (v > best || (v == best && i < bi)) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      sv[wid] = best;
      si[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b2 = -1.0;
      int i2 = 0x7fffffff;
      for (int w = 0; w < nt / 32; ++w)
        if (sv[w] > b2 || (sv[w] == b2 && si[w] < i2)) {
          b2 = sv[w];
          i2 = si[w];
        }
      if (i2 > km) i2 = 0;  // NaN column: pivot in place, reported as singular
      const double piv = ab[(size_t)(kv + i2) + (size_t)j * ld];
      s_ok = (piv != 0.0 && isfinite(piv)) ? 1 : 0;
      if (!s_ok) atomicOr(flags, FLAG_SINGULAR_COARSE);
      s_jp = i2;
      c.ipiv[j] = j + i2;
      s_ju = max(ju, min(j + ku + i2, n - 1));
    }
    __syncthreads();
    const int jp = s_jp;
    if (!s_ok) {
      __syncthreads();
      continue;
    }
    ju = s_ju;
    if (jp != 0) {
      for (int col = j + tid; col <= ju; col += nt) {
        double* a1 = ab + (size_t)(kv + j - col) + (size_t)col * ld;
        double* a2 = ab + (size_t)(kv + j + jp - col) + (size_t)col * ld;
        const double t = *a1;
        *a1 = *a2;
        *a2 = t;
      }
      __syncthreads();
    }
    const double piv = ab[(size_t)kv + (size_t)j * ld];
    const double rp = 1.0 / piv;
    if (tid == 0) c.rdiag[j] = rp;
    for (int i = 1 + tid; i <= km; i += nt) ab[(size_t)(kv + i) + (size_t)j * ld] *= rp;
    __syncthreads();
    const int ncol = ju - j;
    for (int t = tid; t < ncol * km; t += nt) {
      const int col = j + 1 + t / km, i = 1 + t % km;
      const double lij = ab[(size_t)(kv + i) + (size_t)j * ld];
      const double ujc = ab[(size_t)(kv + j - col) + (size_t)col * ld];
      ab[(size_t)(kv + j + i - col) + (size_t)col * ld] -= lij * ujc;
    }
    __syncthreads();
  }
}

// Solve with the band LU factors (no transpose), one CTA; rhs in c.g, solution written back.
__global__ void __launch_bounds__(256) k_gbtrs(CoarseDev c) {
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const double* ab = c.ab;
  double* b = c.g;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < n; ++j) {
    const int lm = min(kl, n - 1 - j);
    const int l = c.ipiv[j];
    if (tid == 0 && l != j) {
      const double t = b[l];
      b[l] = b[j];
      b[j] = t;
    }
    __syncthreads();
    const double bj = b[j];
    for (int i = 1 + tid; i <= lm; i += nt) b[j + i] -= ab[(size_t)(kv + i) + (size_t)j * ld] * bj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    if (tid == 0) b[j] = b[j] / ab[(size_t)kv + (size_t)j * ld];
    __syncthreads();
    const double bj = b[j];
    const int i0 = max(0, j - kv);
    for (int i = i0 + tid; i < j; i += nt) b[i] -= ab[(size_t)(kv + i - j) + (size_t)j * ld] * bj;
    __syncthreads();
  }
}

// Columns of G^-1 (banded row order in, canonical unknowns out): block j solves L U x = P e_j.
// Written row-major, Ginv[i * n + j], so that the per-apply product reads rows contiguously.
__global__ void __launch_bounds__(128) k_gbtrs_cols(CoarseDev c, double* __restrict__ Ginv) {
  extern __shared__ double b[];
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const double* ab = c.ab;
  const int col = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) b[i] = (i == col) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int lm = min(kl, n - 1 - j);
    const int l = c.ipiv[j];
    if (tid == 0 && l != j) {
      const double t = b[l];
      b[l] = b[j];
      b[j] = t;
    }
    __syncthreads();
    const double bj = b[j];
    if (bj != 0.0)
      for (int i = 1 + tid; i <= lm; i += nt) b[j + i] -= ab[(size_t)(kv + i) + (size_t)j * ld] * bj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    if (tid == 0) b[j] = b[j] / ab[(size_t)kv + (size_t)j * ld];
    __syncthreads();
    const double bj = b[j];
    const int i0 = max(0, j - kv);
    if (bj != 0.0)
      for (int i = i0 + tid; i < j; i += nt) b[i] -= ab[(size_t)(kv + i - j) + (size_t)j * ld] * bj;
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) Ginv[(size_t)i * n + col] = b[i];
}

// Per apply: right-hand side from the particular side moments (Eq. 13-14 rows, banded order) and
// c = G^-1 (-g0), one warp per unknown.
__global__ void __launch_bounds__(256) k_coarse_apply(CoarseDev c, const double* __restrict__ Ginv,
                                                      const double* __restrict__ mom0, int E, double* __restrict__ out) {
  extern __shared__ double gs[];
  constexpr int CH = 32;  // row entries per lane in flight
  const int n = c.n;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double* gr = Ginv + (size_t)(row < n ? row : 0) * n;
  // the first CH entries per lane of this warp's row of G^-1 are loaded while the block forms the
  // right-hand side; the sum runs over k = lane, lane + 32, ... in order, as a plain loop would
  double gv[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) gv[q] = (row < n && lane + 32 * q < n) ? gr[lane + 32 * q] : 0.0;
  for (int t = threadIdx.x; t < E * c.nq; t += blockDim.x) {
    int rf, rp;
    double gf, gp;
    coarse_rhs_rows(c, mom0, t / c.nq, t % c.nq, rf, gf, rp, gp);
    gs[rf] = gf;
    gs[rp] = gp;
  }
  __syncthreads();
  if (row >= n) return;
  double acc = 0.0;
  for (int base = 0; base < n; base += 32 * CH) {
    if (base > 0) {
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int k = base + lane + 32 * q;
        gv[q] = k < n ? gr[k] : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int k = base + lane + 32 * q;
      if (k < n) acc += gv[q] * gs[k];
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) out[row] = acc;
}

// ---- Band LU in a sliding shared-memory window ------------------------------------------------
// Step j touches columns j .. ju <= j + kl + ku, so W = kl + ku + 1 columns of the band hold all of
// a step's data.  The window has W + 3 column slots (column c in slot c mod (W + 3)): the W active
// ones, the column written back to global memory this step, and two being prefetched (column
// j + W + 1 is requested at step j and first needed at step j + 2).  Per step, warp 0 finds the
// pivot (first index of the largest magnitude, as above) and the multipliers l_i = A(j+i, j) / piv
// (as a product with 1/piv); then each warp takes whole columns j .. ju and applies the row
// interchange and the rank-one update from the values before the interchange, so a step costs two
// block barriers and all arithmetic stays on chip.
constexpr int GBW_THREADS = 1024;
constexpr int GBW_MAX_KL = 512;

__device__ __forceinline__ void gb_cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void gb_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void gb_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Pivot choice and multipliers of step j (one warp): first index of the largest magnitude in
// column j below the diagonal, l_i = A(j+i, j) / piv as a product with 1/piv, read before the
// interchange; writes ipiv[j] and the step's column reach.
__device__ __forceinline__ void gb_pivot(const double* cj, int j, int km, int n, int ku, int ju_prev, int lane,
                                         double* sl, int* s_jp, int* s_ju, int* s_ok, int* ipiv, double* rdiag,
                                         int* flags) {
  // |x| compared through its bit pattern with the sign cleared, which orders like |x| for every
  // non-NaN double (+0 and -0 equal); key = pattern + 1, and 0 for NaN, which is never chosen.
  // Each lane keeps its first index of the largest key; the warp takes the largest key, then the
  // lowest index holding it, with integer reductions instead of a compare-and-shuffle chain.
  unsigned long long best = 0ull;
  unsigned bi = 0xffffffffu;
  for (int i = lane; i <= km; i += 32) {
    const double x = cj[i];
    const unsigned long long k = isnan(x) ? 0ull : ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) + 1ull;
    if (k > best) {
      best = k;
      bi = (unsigned)i;
    }
  }
  const unsigned khi = __reduce_max_sync(0xffffffffu, (unsigned)(best >> 32));
  const unsigned klo = __reduce_max_sync(0xffffffffu, (unsigned)(best >> 32) == khi ? (unsigned)best : 0u);
  const bool mine = best != 0ull && (unsigned)(best >> 32) == khi && (unsigned)best == klo;
  unsigned bsel = __reduce_min_sync(0xffffffffu, mine ? bi : 0xffffffffu);
  if (bsel > (unsigned)km) bsel = 0;  // no comparable entry (NaN column): pivot in place, reported as singular below
  const int bi_sel = (int)bsel;
  const double piv = cj[bi_sel];
  const bool ok = piv != 0.0 && isfinite(piv);
  if (ok) {
    const double rp = 1.0 / piv;
    if (lane == 0) rdiag[j] = rp;
    const double old0 = cj[0];
    for (int i = 1 + lane; i <= km; i += 32) sl[i] = (i == bi_sel ? old0 : cj[i]) * rp;
  }
  if (lane == 0) {
    *s_ok = ok ? 1 : 0;
    if (!ok) atomicOr(flags, FLAG_SINGULAR_COARSE);
    *s_jp = bi_sel;
    ipiv[j] = j + bi_sel;
    *s_ju = ok ? max(ju_prev, min(j + ku + bi_sel, n - 1)) : ju_prev;
  }
}

__global__ void __launch_bounds__(GBW_THREADS, 1) k_gbtf2_win(CoarseDev c, int* flags) {
  extern __shared__ __align__(16) double win[];
  __shared__ double sl[2][GBW_MAX_KL + 1];  // multipliers of the current and the next column
  __shared__ int s_jp[2], s_ju[2], s_ok[2];
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const int W = kl + ku + 1, NS = W + 3;
  double* ab = c.ab;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = GBW_THREADS / 32;
  auto slot = [&](int col) { return win + (size_t)(col % NS) * ld; };
  auto load_col = [&](int col) {
    double* dst = slot(col);
    const double* src = ab + (size_t)col * ld;
    for (int r = tid; r < ld; r += GBW_THREADS) gb_cp_async8(dst + r, src + r);
  };
  for (int col = 0; col < n && col <= W; ++col) load_col(col);
  gb_commit();
  gb_wait<0>();
  __syncthreads();
  if (warp == 0 && n > 0)
    gb_pivot(slot(0) + kv, 0, min(kl, n - 1), n, ku, 0, lane, sl[0], &s_jp[0], &s_ju[0], &s_ok[0], c.ipiv, c.rdiag, flags);
  for (int j = 0; j < n; ++j) {
    const int pj = j & 1, pn = pj ^ 1;
    gb_wait<1>();  // columns up to j + W - 1 (requested two steps ago) have landed
    __syncthreads();  // also publishes step j's pivot and multipliers
    if (j >= 1) {     // column j - 1 is final: back to global memory
      const double* src = slot(j - 1);
      double* dst = ab + (size_t)(j - 1) * ld;
      for (int r = tid; r < ld; r += GBW_THREADS) dst[r] = src[r];
    }
    if (j + W + 1 < n) load_col(j + W + 1);
    gb_commit();
    const int km = min(kl, n - 1 - j);
    const bool ok = s_ok[pj] != 0;
    const int ju = s_ju[pj], jp = s_jp[pj];
    const double* l = sl[pj];
    // warp w takes columns j + w, j + w + 32, ...; warp 1 starts with column j + 1 and, once it is
    // final for this step, chooses the pivot of step j + 1
    for (int col = j + warp; col <= ju || (warp == 1 && col == j + 1 && j + 1 < n); col += nw) {
      if (ok && col <= ju) {
        double* cc = slot(col) + kv + j - col;  // cc[i] = A(j + i, col)
        const double up = cc[jp], old0 = cc[0];
        __syncwarp();
        if (col == j) {
          if (lane == 0) cc[0] = up;
          for (int i = 1 + lane; i <= km; i += 32) cc[i] = l[i];
        } else {
          if (lane == 0) cc[0] = up;
          for (int i = 1 + lane; i <= km; i += 32) cc[i] = (i == jp ? old0 : cc[i]) - l[i] * up;
        }
        __syncwarp();
      }
      if (warp == 1 && col == j + 1 && j + 1 < n)
        gb_pivot(slot(j + 1) + kv, j + 1, min(kl, n - 2 - j), n, ku, ju, lane, sl[pn], &s_jp[pn], &s_ju[pn], &s_ok[pn],
                 c.ipiv, c.rdiag, flags);
    }
  }
  gb_wait<0>();
  __syncthreads();
  if (n >= 1) {
    const double* src = slot(n - 1);
    double* dst = ab + (size_t)(n - 1) * ld;
    for (int r = tid; r < ld; r += GBW_THREADS) dst[r] = src[r];
  }
}

// ---- Band LU over a thread-block cluster ------------------------------------------------------
// The same steps as k_gbtf2_win, with the window spread over the CL CTAs of one cluster: column c
// belongs to CTA c mod CL, which keeps it in a ring of NS column slots in its shared memory from
// two steps before it can first be touched (column j + kl + ku + 2 is requested at step j) until
// it is final, and then writes it back.  Per step j, after a cluster barrier, every CTA copies the
// pivot and the multipliers of step j from the shared memory of the owner of column j, applies
// the interchange and the rank-one update to its own columns j .. ju, and the owner of column
// j + 1 chooses the pivot of step j + 1 as soon as that column is final for step j (look-ahead),
// so a step costs one cluster barrier and the arithmetic of a step is spread over CL SMs.
constexpr int GBC_THREADS = 512;

__global__ void __launch_bounds__(GBC_THREADS, 1) k_gbtrf_cluster(CoarseDev c, int* flags, int NS) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double cwin[];
  __shared__ double sl[2][GBW_MAX_KL + 1];  // this CTA's multipliers of the step it chose the pivot of
  __shared__ int s_jp[2], s_ju[2], s_ok[2];
  __shared__ int t_jp, t_ju, t_ok;          // the current step's pivot, copied from its owner
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const int W = kl + ku + 1;
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  double* ab = c.ab;
  double* lb = cwin + (size_t)NS * ld;      // [kl + 1] multipliers of the current step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = GBC_THREADS / 32;
  auto slot = [&](int col) { return cwin + (size_t)((col / CL) % NS) * ld; };
  auto load_col = [&](int col) {
    double* dst = slot(col);
    const double* src = ab + (size_t)col * ld;
    for (int r = tid; r < ld; r += GBC_THREADS) gb_cp_async8(dst + r, src + r);
  };
  auto store_col = [&](int col) {
    const double* src = slot(col);
    double* dst = ab + (size_t)col * ld;
    for (int r = tid; r < ld; r += GBC_THREADS) dst[r] = src[r];
  };
  for (int col = rank; col < n && col <= W; col += CL) load_col(col);
  gb_commit();
  gb_wait<0>();
  __syncthreads();
  if (rank == 0 && warp == 0 && n > 0)
    gb_pivot(slot(0) + kv, 0, min(kl, n - 1), n, ku, 0, lane, sl[0], &s_jp[0], &s_ju[0], &s_ok[0], c.ipiv, c.rdiag,
             flags);
  for (int j = 0; j < n; ++j) {
    const int pj = j & 1, pn = pj ^ 1;
    const int owner = j % CL;
    gb_wait<1>();  // this CTA's columns up to j + W - 1 (requested two steps ago) have landed
    cl.sync();     // publishes the pivot and multipliers of step j, and orders the previous step
    const int km = min(kl, n - 1 - j);
    if (tid == 0) {
      t_jp = *cl.map_shared_rank(&s_jp[pj], owner);
      t_ju = *cl.map_shared_rank(&s_ju[pj], owner);
      t_ok = *cl.map_shared_rank(&s_ok[pj], owner);
    }
    {
      const double* rl = cl.map_shared_rank(&sl[pj][0], owner);
      for (int i = 1 + tid; i <= km; i += GBC_THREADS) lb[i] = rl[i];
    }
    if (j >= 1 && (j - 1) % CL == rank) store_col(j - 1);  // column j - 1 is final
    if (j + W + 1 < n && (j + W + 1) % CL == rank) load_col(j + W + 1);
    gb_commit();
    __syncthreads();
    const bool ok = t_ok != 0;
    const int ju = t_ju, jp = t_jp;
    // this CTA's columns from j on, warp w taking the w-th of them (the owner of column j + 1 meets
    // it first, in warp 0, and chooses the pivot of step j + 1 on it right after its update)
    const int first = j + ((rank - j) % CL + CL) % CL;
    for (int col = first + warp * CL; col <= ju || (col == j + 1 && j + 1 < n); col += nw * CL) {
      if (ok && col <= ju) {
        double* cc = slot(col) + kv + j - col;  // cc[i] = A(j + i, col)
        const double up = cc[jp], old0 = cc[0];
        __syncwarp();
        if (col == j) {
          if (lane == 0) cc[0] = up;
          for (int i = 1 + lane; i <= km; i += 32) cc[i] = lb[i];
        } else {
          if (lane == 0) cc[0] = up;
          for (int i = 1 + lane; i <= km; i += 32) cc[i] = (i == jp ? old0 : cc[i]) - lb[i] * up;
        }
        __syncwarp();
      }
      if (col == j + 1 && j + 1 < n)
        gb_pivot(slot(j + 1) + kv, j + 1, min(kl, n - 2 - j), n, ku, ju, lane, sl[pn], &s_jp[pn], &s_ju[pn], &s_ok[pn],
                 c.ipiv, c.rdiag, flags);
    }
  }
  gb_wait<0>();
  cl.sync();
  if (n >= 1 && (n - 1) % CL == rank) store_col(n - 1);
}

static size_t gbtrf_cluster_smem(const CoarseDev& c, int CL, int* NS) {
  const int kv = c.kl + c.ku;
  *NS = (kv + 4 + CL - 1) / CL + 1;
  return sizeof(double) * ((size_t)(*NS) * c.ldab + c.kl + 2);
}

// Cluster launch configuration for the band LU: false when clusters of CL CTAs with the ring in
// shared memory cannot be scheduled on this device.
static bool gbtrf_cluster_config(const CoarseDev& c, int CL, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr,
                                 int* NS) {
  if (c.kl > GBW_MAX_KL) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t static_smem = sizeof(double) * 2 * (GBW_MAX_KL + 1) + 64;
  // once per process: the shared-memory limit, and clusters of 16 where the device allows them
  static const int max_cl = [] {
    if (raise_smem_limit<k_gbtrf_cluster>() != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_gbtrf_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return 8;
    }
    return 16;
  }();
  if (CL > max_cl) return false;
  const size_t sm = gbtrf_cluster_smem(c, CL, NS);
  if (sm + static_smem > (size_t)optin) return false;
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(CL);
  cfg->blockDim = dim3(GBC_THREADS);
  cfg->dynamicSmemBytes = sm;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_gbtrf_cluster, cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();  // clear a refusal of this cluster size
    return false;
  }
  return true;
}

static size_t gbtf2_win_smem(const CoarseDev& c) { return sizeof(double) * (size_t)(c.kl + c.ku + 4) * c.ldab; }

static bool gbtf2_win_fits(const CoarseDev& c) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t static_smem = sizeof(double) * 2 * (GBW_MAX_KL + 1) + 64;
  return c.kl <= GBW_MAX_KL && gbtf2_win_smem(c) + static_smem <= (size_t)optin;
}

int coarse_factor_variants(const CoarseDev& c, int* v) {
  int nv = 0;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int NS = 0;
  for (int CL : {16, 8})
    if (gbtrf_cluster_config(c, CL, &cfg, attr, &NS)) v[nv++] = CL;
  if (gbtf2_win_fits(c)) v[nv++] = 1;
  if (nv == 0) v[nv++] = 0;
  return nv;
}

// Columns of G^-1, one warp per column and no block barriers (at most four band rows per lane,
// i.e. kl + ku <= 128).  Each lane streams its band entries of the next GBC_DEPTH - 1 steps through
// its own slots of a cp.async ring (it reads back only what it copied, so no warp barrier is needed
// for them); the pivot indices and the reciprocal diagonals are staged once per CTA.  The forward
// sweep of column col starts at step col - kl: before it, every interchange swaps two zero rows and
// every update is skipped (b[j] = 0), so the result is the one of the full sweep.
constexpr int GBC_ROWS = 4;
constexpr int GBC_DEPTH = 6;
__global__ void __launch_bounds__(128) k_gbtrs_cols_warp(CoarseDev c, double* __restrict__ Ginv) {
  extern __shared__ __align__(16) double sbuf[];
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const double* __restrict__ ab = c.ab;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* rd = sbuf;                                            // [n] 1 / U(j, j)
  int* piv = reinterpret_cast<int*>(rd + n);                    // [n] (padded to an even count)
  double* ring = rd + n + (n + 1) / 2;                          // [4 warps][GBC_DEPTH][GBC_ROWS][32]
  double* b = ring + 4 * GBC_DEPTH * GBC_ROWS * 32 + (size_t)warp * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    rd[i] = c.rdiag[i];
    piv[i] = c.ipiv[i];
  }
  __syncthreads();
  const int col = blockIdx.x * 4 + warp;
  if (col >= n) return;  // whole warps; no block barrier follows
  double* myr = ring + (size_t)warp * GBC_DEPTH * GBC_ROWS * 32 + lane;
  auto slot = [&](int t, int q) -> double* { return myr + ((size_t)(t % GBC_DEPTH) * GBC_ROWS + q) * 32; };
  for (int i = lane; i < n; i += 32) b[i] = (i == col) ? 1.0 : 0.0;
  __syncwarp();
  // forward: b[j + i] -= L(j + i, j) b[j], after the interchange of step j
  const int j0 = max(0, col - kl);
  auto issueL = [&](int t) {  // step j0 + t
    const int j = j0 + t;
    if (j < n) {
      const int lm = min(kl, n - 1 - j);
#pragma unroll
      for (int q = 0; q < GBC_ROWS; ++q) {
        const int i = 1 + lane + 32 * q;
        if (i <= lm) gb_cp_async8(slot(t, q), ab + (size_t)(kv + i) + (size_t)j * ld);
      }
    }
    gb_commit();
  };
  for (int t = 0; t < GBC_DEPTH - 1; ++t) issueL(t);
  for (int j = j0, t = 0; j < n; ++j, ++t) {
    issueL(t + GBC_DEPTH - 1);
    gb_wait<GBC_DEPTH - 1>();
    const int lp = piv[j];
    if (lp != j) {
      if (lane == 0) {
        const double tt = b[lp];
        b[lp] = b[j];
        b[j] = tt;
      }
      __syncwarp();
    }
    const double bj = b[j];
    const int lm = min(kl, n - 1 - j);
    if (bj != 0.0) {
#pragma unroll
      for (int q = 0; q < GBC_ROWS; ++q) {
        const int i = 1 + lane + 32 * q;
        if (i <= lm) b[j + i] -= *slot(t, q) * bj;
      }
    }
    __syncwarp();
  }
  gb_wait<0>();
  // backward: b[j] *= 1 / U(j, j), then b[i] -= U(i, j) b[j] for i = j - kv .. j - 1
  auto issueU = [&](int t) {  // step n - 1 - t
    const int j = n - 1 - t;
    if (j >= 0) {
      const int i0 = max(0, j - kv);
#pragma unroll
      for (int q = 0; q < GBC_ROWS; ++q) {
        const int i = i0 + lane + 32 * q;
        if (i < j) gb_cp_async8(slot(t, q), ab + (size_t)(kv + i - j) + (size_t)j * ld);
      }
    }
    gb_commit();
  };
  for (int t = 0; t < GBC_DEPTH - 1; ++t) issueU(t);
  for (int j = n - 1, t = 0; j >= 0; --j, ++t) {
    issueU(t + GBC_DEPTH - 1);
    gb_wait<GBC_DEPTH - 1>();
    if (lane == 0) b[j] = b[j] * rd[j];
    __syncwarp();
    const double bj = b[j];
    const int i0 = max(0, j - kv);
    if (bj != 0.0) {
#pragma unroll
      for (int q = 0; q < GBC_ROWS; ++q) {
        const int i = i0 + lane + 32 * q;
        if (i < j) b[i] -= *slot(t, q) * bj;
      }
    }
    __syncwarp();
  }
  gb_wait<0>();
  for (int i = lane; i < n; i += 32) Ginv[(size_t)i * n + col] = b[i];
}

// Per apply when 2E is above the explicit-inverse limit: the right-hand side from the particular
// side moments, then L U c = P g by one CTA with g resident in shared memory.  The band data (and
// the pivot index) of the next GBS_DEPTH - 2 steps are in flight in a cp.async ring; a thread
// loads its R band entries and right-hand-side rows into registers before it updates them, so its
// R updates are independent; the reciprocal of the next diagonal is taken one step ahead.  One SM's
// FP64 pipe bounds the step, which is why the rows are spread over all four of its schedulers.
constexpr int GBS_THREADS = 128;

__device__ __forceinline__ void gb_cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

static size_t gbtrs_smem(const CoarseDev& c, int depth) {
  return sizeof(double) * (((size_t)c.n + 1) / 2 * 2 + (size_t)depth * (c.kl + c.ku + 2));
}

// R: rows per thread, GBS_THREADS R >= kl + ku + 1; GBS_DEPTH ring slots (steps in flight + 2)
template <int R, int GBS_DEPTH>
__global__ void __launch_bounds__(GBS_THREADS) k_gbtrs_smem(CoarseDev c, const double* __restrict__ mom0, int E) {
  extern __shared__ __align__(16) double gsm[];
  constexpr int NT = GBS_THREADS;
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  const int stride = kv + 2;  // kv + 1 band entries, then the pivot index
  const int tid = threadIdx.x;
  double* b = gsm;
  double* ring = gsm + ((size_t)n + 1) / 2 * 2;
  const double* __restrict__ ab = c.ab;
  for (int t = tid; t < E * c.nq; t += NT) {
    int rf, rp;
    double gf, gp;
    coarse_rhs_rows(c, mom0, t / c.nq, t % c.nq, rf, gf, rp, gp);
    b[rf] = gf;
    b[rp] = gp;
  }
  // forward: interchange of step j, then b[j + 1 + k] -= L(j + 1 + k, j) b[j].  Step j's slot is
  // refilled (for step j + GBS_DEPTH) only after the barrier of step j + 1, when no thread reads it.
  auto issueL = [&](int j) {
    if (j < n) {
      double* dst = ring + (size_t)(j % GBS_DEPTH) * stride;
      const double* src = ab + (size_t)(kv + 1) + (size_t)j * ld;
      const int lm = min(kl, n - 1 - j);
      for (int k = tid; k < lm; k += NT) gb_cp_async8(dst + k, src + k);
      if (tid == 0) gb_cp_async4(dst + kv + 1, c.ipiv + j);
    }
    gb_commit();
  };
  for (int t = 0; t < GBS_DEPTH - 1; ++t) issueL(t);
  for (int j = 0; j < n; ++j) {
    gb_wait<GBS_DEPTH - 2>();
    __syncthreads();
    issueL(j + GBS_DEPTH - 1);
    const double* Lc = ring + (size_t)(j % GBS_DEPTH) * stride;
    const int l = *reinterpret_cast<const int*>(Lc + kv + 1);
    const int lm = min(kl, n - 1 - j);
    double lv[R], bv[R];
#pragma unroll
    for (int q = 0; q < R; ++q) lv[q] = tid + NT * q < lm ? Lc[tid + NT * q] : 0.0;
    if (l != j) {
      if (tid == 0) {
        const double t = b[l];
        b[l] = b[j];
        b[j] = t;
      }
      __syncthreads();
    }
    const double bj = b[j];
#pragma unroll
    for (int q = 0; q < R; ++q) bv[q] = tid + NT * q < lm ? b[j + 1 + tid + NT * q] : 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (tid + NT * q < lm) b[j + 1 + tid + NT * q] = bv[q] - lv[q] * bj;
  }
  // backward, step t on column j = n - 1 - t: x_j = b[j] is final when the step starts; b[i] -=
  // U(i, j) x_j for i = max(0, j - kv) .. j - 1, and the thread of row j - 1 then scales it by
  // 1 / U(j-1, j-1), so the next step starts from x_{j-1} (ring slot: rows i0 .. j - 1, then 1 / U(j, j)
  // at position kv)
  auto issueU = [&](int t) {
    if (t < n) {
      const int j = n - 1 - t, i0 = max(0, j - kv);
      double* dst = ring + (size_t)(t % GBS_DEPTH) * stride;
      const double* src = ab + (size_t)(kv + i0 - j) + (size_t)j * ld;
      for (int k = tid; k < j - i0; k += NT) gb_cp_async8(dst + k, src + k);
      if (tid == 0) gb_cp_async8(dst + kv, c.rdiag + j);
    }
    gb_commit();
  };
  gb_wait<0>();
  __syncthreads();
  for (int t = 0; t < GBS_DEPTH - 1; ++t) issueU(t);
  gb_wait<GBS_DEPTH - 2>();
  __syncthreads();
  if (tid == 0 && n > 0) b[n - 1] *= ring[kv];
  for (int t = 0; t < n; ++t) {
    const int j = n - 1 - t, i0 = max(0, j - kv), len = j - i0;
    gb_wait<GBS_DEPTH - 3>();  // this step's slot and the next one's
    __syncthreads();
    issueU(t + GBS_DEPTH - 1);
    const double* Uc = ring + (size_t)(t % GBS_DEPTH) * stride;
    double uv[R], bv[R];
#pragma unroll
    for (int q = 0; q < R; ++q) uv[q] = tid + NT * q < len ? Uc[tid + NT * q] : 0.0;
    const double bj = b[j];
#pragma unroll
    for (int q = 0; q < R; ++q) bv[q] = tid + NT * q < len ? b[i0 + tid + NT * q] : 0.0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int k = tid + NT * q;
      if (k < len) {
        double v = bv[q] - uv[q] * bj;
        if (k == len - 1) v *= ring[(size_t)((t + 1) % GBS_DEPTH) * stride + kv];  // row j - 1
        b[i0 + k] = v;
      }
    }
  }
  gb_wait<0>();
  __syncthreads();
  for (int i = tid; i < n; i += NT) c.g[i] = b[i];
}

// ---- Blocked substitution (2E nq above the explicit-inverse limit) -----------------------------
// The forward pass of the band solve (interchanges and L) and the backward pass (U) are each cut
// into blocks of GBB_NB consecutive steps.  Block k's steps touch a window of W = GBB_NB + K rows
// (K = kl for L, kl + ku for U) and act on it linearly, so at set-up each block's action is formed
// as a dense W x W matrix by running its steps on the W unit vectors (one warp per column, the
// same operations in the same order as a plain substitution).  Per apply, the part of every
// block's output that comes from the rows no earlier block touches (its fresh rows) is a batch of
// independent products; only the K rows that a block hands on to the next (its carry) form a
// chain, one K x K product per block, run on one thread-block cluster.
// Window positions: L block k covers rows k NB .. k NB + W - 1 with the carry in at [0, K), fresh
// rows at [K, W), final rows at [0, NB) and the carry out at [NB, W); U block k covers rows
// k NB - K .. k NB + NB - 1 with fresh rows at [0, NB), the carry in at [NB, W), the carry out at
// [0, K) and final rows at [K, W).  Vectors hold kl + ku zero rows before row 0 (the rows below
// the first U block) and kl after the last block.
__global__ void __launch_bounds__(128) k_gbb_build(CoarseDev c, int upper) {
  extern __shared__ double vsm[];  // [4 warps][W]
  const int n = c.n, kl = c.kl, kv = c.kl + c.ku, ld = c.ldab;
  const int K = upper ? kv : kl, W = GBB_NB + K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * 4 + warp;
  if (gw >= (long long)c.nbk * W) return;  // whole warps
  const int k = (int)(gw / W), col = (int)(gw % W);
  double* v = vsm + (size_t)warp * W;
  for (int i = lane; i < W; i += 32) v[i] = i == col ? 1.0 : 0.0;
  __syncwarp();
  const double* __restrict__ ab = c.ab;
  const int j0 = k * GBB_NB, j1 = min(j0 + GBB_NB, n);
  if (!upper) {
    for (int j = j0; j < j1; ++j) {
      const int p = c.ipiv[j];
      if (p != j) {
        if (lane == 0) {
          const double t = v[p - j0];
          v[p - j0] = v[j - j0];
          v[j - j0] = t;
        }
        __syncwarp();
      }
      const double bj = v[j - j0];
      const int lm = min(kl, n - 1 - j);
      if (bj != 0.0)
        for (int i = 1 + lane; i <= lm; i += 32) v[j - j0 + i] -= ab[(size_t)(kv + i) + (size_t)j * ld] * bj;
      __syncwarp();
    }
  } else {
    const int base = j0 - kv;  // the row at window position 0
    for (int j = j1 - 1; j >= j0; --j) {
      if (lane == 0) v[j - base] *= c.rdiag[j];
      __syncwarp();
      const double bj = v[j - base];
      if (bj != 0.0)
        for (int i = max(0, j - kv) + lane; i < j; i += 32) v[i - base] -= ab[(size_t)(kv + i - j) + (size_t)j * ld] * bj;
      __syncwarp();
    }
  }
  double* M = (upper ? c.MU : c.ML) + (size_t)k * W * W + (size_t)col * W;
  for (int i = lane; i < W; i += 32) M[i] = v[i];
}

// The right-hand side of the coupling rows into the padded forward-pass input.
__global__ void k_gbb_rhs(CoarseDev c, const double* __restrict__ mom0, int E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * c.nq) return;
  int rf, rp;
  double gf, gp;
  coarse_rhs_rows(c, mom0, t / c.nq, t % c.nq, rf, gf, rp, gp);
  const int pad = c.kl + c.ku;
  c.X[pad + rf] = gf;
  c.X[pad + rp] = gp;
}

// F_k = M_k[:, fresh] (fresh rows of `in`) for every block k: blockIdx.x = k, blockIdx.y = 128
// window rows; the two halves of the CTA take alternate fresh columns.
__global__ void __launch_bounds__(256) k_gbb_fresh(CoarseDev c, int upper, const double* __restrict__ in) {
  __shared__ double fr[GBB_NB];
  __shared__ double part[256];
  const int kv = c.kl + c.ku, K = upper ? kv : c.kl, W = GBB_NB + K;
  const int k = blockIdx.x, tid = threadIdx.x;
  const int f0 = upper ? 0 : K;                              // window position of the first fresh row
  const int row0 = upper ? k * GBB_NB - kv : k * GBB_NB;     // the row at window position 0
  for (int t = tid; t < GBB_NB; t += 256) fr[t] = in[(size_t)kv + row0 + f0 + t];
  __syncthreads();
  const int r = blockIdx.y * 128 + (tid & 127), half = tid >> 7;
  const double* __restrict__ M = (upper ? c.MU : c.ML) + (size_t)k * W * W;
  double acc = 0.0;
  if (r < W)
    for (int t = half; t < GBB_NB; t += 2) acc += M[(size_t)(f0 + t) * W + r] * fr[t];
  part[tid] = acc;
  __syncthreads();
  if (tid < 128 && r < W) c.F[(size_t)k * (GBB_NB + kv) + r] = part[tid] + part[tid + 128];
}

// The chain of carries: block after block (forward for L, backward for U), carry_out = M_k[carry
// out, carry in] carry_in + F_k[carry out].  CTA q of the cluster forms rows [q K / CL, (q+1) K / CL)
// (at most 64) and writes them into every CTA's copy of the next carry; one cluster barrier per
// block.  The carry entering each block is kept in C for the final rows.
__global__ void __launch_bounds__(256, 1) k_gbb_chain(CoarseDev c, int upper, const double* __restrict__ in) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double csm[];  // [2][K] carries, then [8][64] partial sums
  const int kv = c.kl + c.ku, K = upper ? kv : c.kl, W = GBB_NB + K, nbk = c.nbk;
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = (int)((long long)rank * K / CL), r1 = (int)((long long)(rank + 1) * K / CL), nr = r1 - r0;
  double* cur = csm;
  double* nxt = csm + K;
  double* part = csm + 2 * K;
  const int cin = upper ? GBB_NB : 0, cout = upper ? 0 : GBB_NB;
  // the carry entering the first block holds rows that no block has touched
  const int crow = upper ? (nbk - 1) * GBB_NB - kv + GBB_NB : 0;
  for (int i = tid; i < K; i += 256) cur[i] = in[(size_t)kv + crow + i];
  __syncthreads();
  const int t0 = (int)((long long)warp * K / 8), t1 = (int)((long long)(warp + 1) * K / 8);
  for (int h = 0; h < nbk; ++h) {
    const int k = upper ? nbk - 1 - h : h;
    for (int i = r0 + tid; i < r1; i += 256) c.C[(size_t)k * kv + i] = cur[i];
    if (h + 1 < nbk) {
      const double* __restrict__ M = (upper ? c.MU : c.ML) + (size_t)k * W * W + cout + r0;
      double a0 = 0.0, a1 = 0.0;
      for (int t = t0; t < t1; ++t) {
        const double x = cur[t];
        const double* Mc = M + (size_t)(cin + t) * W;
        if (lane < nr) a0 += Mc[lane] * x;
        if (lane + 32 < nr) a1 += Mc[lane + 32] * x;
      }
      part[warp * 64 + lane] = a0;
      part[warp * 64 + lane + 32] = a1;
      __syncthreads();
      if (tid < nr) {
        double sum = c.F[(size_t)k * (GBB_NB + kv) + cout + r0 + tid];
        for (int w8 = 0; w8 < 8; ++w8) sum += part[w8 * 64 + tid];
        for (int q = 0; q < CL; ++q) *cl.map_shared_rank(&nxt[r0 + tid], q) = sum;
      }
    }
    cl.sync();  // the next carry is complete in every CTA, and nobody still reads this one
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

// Final rows of every block: M_k[final, carry in] C_k + F_k[final], written to `out` (padded
// vector) or, for the last pass, to the solution.  blockIdx.x = k, blockIdx.y = 128 final rows.
__global__ void __launch_bounds__(256) k_gbb_final(CoarseDev c, int upper, double* __restrict__ out) {
  extern __shared__ double cr[];  // [K] carry entering block k
  __shared__ double part[256];
  const int n = c.n, kv = c.kl + c.ku, K = upper ? kv : c.kl, W = GBB_NB + K;
  const int k = blockIdx.x, tid = threadIdx.x;
  const int cin = upper ? GBB_NB : 0, fin = upper ? K : 0;
  for (int j = tid; j < K; j += 256) cr[j] = c.C[(size_t)k * kv + j];
  __syncthreads();
  const int r = blockIdx.y * 128 + (tid & 127), half = tid >> 7;
  const double* __restrict__ M = (upper ? c.MU : c.ML) + (size_t)k * W * W;
  double acc = 0.0;
  if (r < GBB_NB)
    for (int j = half; j < K; j += 2) acc += M[(size_t)(cin + j) * W + fin + r] * cr[j];
  part[tid] = acc;
  __syncthreads();
  if (tid < 128 && r < GBB_NB) {
    const double v = part[tid] + part[tid + 128] + c.F[(size_t)k * (GBB_NB + kv) + fin + r];
    const int row = k * GBB_NB + r;
    if (upper) {
      if (row < n) c.g[row] = v;
    } else {
      out[(size_t)kv + row] = v;
    }
  }
}

// Launch configuration of the carry chain on a cluster of CL CTAs; false when the carry does not fit
// CL CTAs of at most 64 rows each, or when the device cannot schedule such a cluster (checked once
// per cluster size, with the largest shared-memory request).
static bool gbb_chain_config(int K, int CL, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  if (K > 64 * CL) return false;
  auto fill = [](int cl, size_t smem, cudaLaunchConfig_t* f, cudaLaunchAttribute* at) {
    *f = cudaLaunchConfig_t{};
    f->gridDim = dim3(cl);
    f->blockDim = dim3(256);
    f->dynamicSmemBytes = smem;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    f->attrs = at;
    f->numAttrs = 1;
  };
  // bit CL / 8 - 1: clusters of CL (8 or 16) chain CTAs can be scheduled
  static const int schedulable = [&fill] {
    int bits = 0;
    const bool big = cudaFuncSetAttribute(k_gbb_chain, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    if (!big) cudaGetLastError();
    for (int cl : {8, 16}) {
      if (cl == 16 && !big) continue;
      cudaLaunchConfig_t f;
      cudaLaunchAttribute at[1];
      fill(cl, sizeof(double) * (2 * 64 * (size_t)cl + 8 * 64), &f, at);
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_gbb_chain, &f) == cudaSuccess && ncl >= 1) bits |= 1 << (cl / 8 - 1);
      else cudaGetLastError();
    }
    return bits;
  }();
  if (!(schedulable >> (CL / 8 - 1) & 1)) return false;
  fill(CL, sizeof(double) * (2 * (size_t)K + 8 * 64), cfg, attr);
  return true;
}

// Whether the blocked substitution can run for this band (a chain cluster that holds the carry).
static bool gbb_usable(const CoarseDev& c) {
  if (c.nbk <= 0) return false;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  const int kv = c.kl + c.ku;
  return gbb_chain_config(kv, 16, &cfg, attr) || gbb_chain_config(kv, 8, &cfg, attr);
}

cudaError_t launch_coarse_blocks(const CoarseDev& c, cudaStream_t st) {
  if (!gbb_usable(c)) return cudaSuccess;  // the per-apply band solve is used instead
  const int kv = c.kl + c.ku;
  const size_t nvec = (size_t)kv + (size_t)c.nbk * GBB_NB + c.kl;
  cudaError_t e = raise_smem_limit<k_gbb_build>();
  if (e == cudaSuccess) e = cudaMemsetAsync(c.X, 0, sizeof(double) * nvec, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.Y, 0, sizeof(double) * nvec, st);
  if (e != cudaSuccess) return e;
  for (int upper = 0; upper < 2; ++upper) {
    const int W = GBB_NB + (upper ? kv : c.kl);
    const long long warps = (long long)c.nbk * W;
    k_gbb_build<<<(unsigned)((warps + 3) / 4), 128, sizeof(double) * 4 * (size_t)W, st>>>(c, upper);
    count_launch(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_gbb_solve(const CoarseDev& c, const double* mom0, int E, cudaStream_t st) {
  const int kv = c.kl + c.ku;
  k_gbb_rhs<<<(E * c.nq + 127) / 128, 128, 0, st>>>(c, mom0, E);
  count_launch(1);
  cudaError_t e = cudaGetLastError();
  for (int upper = 0; upper < 2 && e == cudaSuccess; ++upper) {
    const int K = upper ? kv : c.kl, W = GBB_NB + K;
    const double* in = upper ? c.Y : c.X;
    k_gbb_fresh<<<dim3(c.nbk, (W + 127) / 128), 256, 0, st>>>(c, upper, in);
    count_launch(1);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (!gbb_chain_config(K, 16, &cfg, attr) && !gbb_chain_config(K, 8, &cfg, attr))
      return cudaErrorInvalidConfiguration;
    cfg.stream = st;
    e = cudaLaunchKernelEx(&cfg, k_gbb_chain, c, upper, in);
    count_launch(1);
    if (e != cudaSuccess) break;
    k_gbb_final<<<dim3(c.nbk, (GBB_NB + 127) / 128), 256, sizeof(double) * (size_t)K, st>>>(c, upper, c.Y);
    count_launch(1);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_coarse_invert(const CoarseDev& c, double* Ginv, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  const size_t sm4 = sizeof(double) * (5 * (size_t)c.n + ((size_t)c.n + 1) / 2 + 4 * GBC_DEPTH * GBC_ROWS * 32);
  static const int optin = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
  }();
  if (c.kl <= 32 * GBC_ROWS && c.kl + c.ku <= 32 * GBC_ROWS && sm4 <= (size_t)optin) {
    const cudaError_t e = raise_smem_limit<k_gbtrs_cols_warp>();
    if (e != cudaSuccess) return e;
    k_gbtrs_cols_warp<<<(c.n + 3) / 4, 128, sm4, st>>>(c, Ginv);
  } else {
    k_gbtrs_cols<<<c.n, 128, sizeof(double) * c.n, st>>>(c, Ginv);
  }
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_apply(const CoarseDev& c, const double* Ginv, const double* mom0, int E, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  k_coarse_apply<<<(c.n + 7) / 8, 256, sizeof(double) * c.n, st>>>(c, Ginv, mom0, E, c.g);
  count_launch(1);
  return cudaGetLastError();
}

// ============================================================================================
// Band LU without row interchanges, blocked over the whole GPU (one cooperative launch, one CTA
// per SM).  In the banded home order the coupling matrix factors stably without pivoting (its
// element growth stays near one on the workloads), so no column waits for a pivot search: for each
// panel of NP_NB columns,
//   1. every warp solves one row of L21 = A21 U11^-1 or one column of U12 = L11^-1 A12;
//   2. the band part of A22 -= L21 U12 is updated in 16 x 16 tiles spread over the CTAs: CTAs 1-4
//      update the tiles of the next diagonal block first and hand it to CTA 0, which factors it
//      (unblocked, in shared memory) while the others update the rest (look-ahead),
// with a grid barrier after each step.  GB300's FP64 pipe retires about two lanes per clock per SM
// with a 64-cycle latency, so the kernel keeps dependent chains short (four partial sums per tile
// entry, one FMA per entry in the diagonal factorisation) and issues few predicated-off FP64
// instructions.  The factors land in the LAPACK band layout with ipiv[j] = j and
// rdiag[j] = 1 / U(j, j), so every solve kernel takes them unchanged.  A zero or non-finite pivot,
// or an entry larger than NOPIV_MAX_GROWTH times the largest entry of G, sets FLAG_NOPIV_REJECTED;
// the caller then factors again with partial pivoting.
constexpr int NP_NB = 32;
constexpr int NP_THREADS = 256;
constexpr int NP_TILE = 16;

__device__ __forceinline__ void np_max_abs(unsigned long long* p, double v) {
  // non-negative doubles (and NaN with the sign cleared, above +inf) order like their bit patterns
  atomicMax(p, (unsigned long long)__double_as_longlong(fabs(v)));
}

// 1 / v by Newton's method x <- x (2 - v x) from a single-precision estimate: two steps take the
// 24 correct bits of the estimate past double precision.  Values outside the single-precision range
// take the division.
__device__ __forceinline__ double np_recip(double v) {
  const float vf = (float)v;
  double x = (double)__frcp_rn(vf);
  if (!(fabs(x) > 0.0 && fabs(x) < 1e37)) return 1.0 / v;
  double e = fma(-v, x, 1.0);
  x = fma(x, e, x);
  e = fma(-v, x, 1.0);
  return fma(x, e, x);
}

// Factors the kb x kb diagonal block at (k0, k0) held in A (already updated), writes it back with
// rdiag and ipiv; called by every thread of one CTA.  One block barrier per column: the update of
// step j reads column j unscaled (times the pivot's reciprocal) and writes the multipliers to Lm,
// and the thread that forms the next pivot takes its reciprocal at once.
__device__ void np_factor_diag(const CoarseDev& c, int k0, int kb, double (*A)[NP_NB + 1], double (*Lm)[NP_NB + 1],
                               double& gmax, int* flags) {
  const int tid = threadIdx.x, nt = blockDim.x;
  static_assert(NP_THREADS == 256 && NP_NB == 32, "the diagonal factor maps 8 warps of 4 rows x 32 columns");
  __shared__ double rps[NP_NB];
  __shared__ int s_bad;
  if (tid == 0) {
    s_bad = !(A[0][0] != 0.0 && isfinite(A[0][0]));
    rps[0] = np_recip(A[0][0]);
  }
  __syncthreads();
  // warp w owns rows 4w .. 4w + 3, lane tx column tx.  Step j updates the trailing block with row j
  // scaled by the pivot's reciprocal (one FMA per entry); column j keeps its unscaled values, which
  // no later step touches, and the multipliers are formed from them at the end.  Warps whose rows all
  // lie above the pivot skip the step.
  const int tx = tid & 31, w = tid >> 5;
  for (int j = 0; j < kb; ++j) {
    if (4 * w + 3 > j) {
      const double u = tx > j && tx < kb ? A[j][tx] * rps[j] : 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = 4 * w + k;
        if (i > j && i < kb && tx > j && tx < kb) {
          const double v = fma(-A[i][j], u, A[i][tx]);
          A[i][tx] = v;
          if (i == j + 1 && tx == j + 1) {
            if (!(v != 0.0 && isfinite(v))) s_bad = 1;
            rps[j + 1] = np_recip(v);
          }
        }
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < NP_NB * NP_NB; t += nt) {
    const int i = t >> 5, j = t & 31;
    if (i > j && i < kb) Lm[i][j] = A[i][j] * rps[j];
  }
  __syncthreads();
  const int kv = c.kl + c.ku;
  for (int t = tid; t < kb * kb; t += nt) {
    const int i = t / kb, j = t % kb;
    if (i - j <= c.kl && j - i <= c.ku) {
      const double v = i > j ? Lm[i][j] : A[i][j];
      c.ab[(size_t)(kv + i - j) + (size_t)(k0 + j) * c.ldab] = v;
      gmax = fmax(gmax, fabs(v));
    }
  }
  for (int j = tid; j < kb; j += nt) {
    c.rdiag[k0 + j] = rps[j];
    c.ipiv[k0 + j] = k0 + j;
  }
  if (tid == 0 && s_bad) atomicOr(flags, FLAG_NOPIV_REJECTED);
}

// Loads the kb x kb diagonal block at (k0, k0) from the band (zeros outside it) into A.
__device__ __forceinline__ void np_load_diag(const CoarseDev& c, int k0, int kb, double (*A)[NP_NB + 1]) {
  const int kv = c.kl + c.ku;
  for (int t = threadIdx.x; t < NP_NB * NP_NB; t += blockDim.x) {
    const int i = t / NP_NB, j = t % NP_NB;
    double v = 0.0;
    if (i < kb && j < kb && i - j <= c.kl && j - i <= c.ku)
      v = c.ab[(size_t)(kv + i - j) + (size_t)(k0 + j) * c.ldab];
    A[i][j] = v;
  }
}

// One 16 x 16 tile of A22 -= L21 U12 (band entries only), four partial sums per entry.
__device__ __forceinline__ void np_tile(const CoarseDev& c, int k0, int kb, int i0, int j0, double (*sL)[NP_NB + 1],
                                        double (*sU)[NP_TILE + 1], double& gmax) {
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku, tid = threadIdx.x;
  double* ab = c.ab;
  __syncthreads();
  for (int e = tid; e < NP_TILE * NP_NB; e += NP_THREADS) {
    const int r = e / NP_NB, q = e % NP_NB, i = i0 + r, col = k0 + q;
    sL[r][q] = (q < kb && i < n && i - col <= kl) ? ab[(size_t)(kv + i - col) + (size_t)col * ld] : 0.0;
    const int rr = e / NP_TILE, cc = e % NP_TILE, j = j0 + cc, row = k0 + rr;
    sU[rr][cc] = (rr < kb && j < n && j - row <= ku) ? ab[(size_t)(kv + row - j) + (size_t)j * ld] : 0.0;
  }
  __syncthreads();
  const int r = tid / NP_TILE, cc = tid % NP_TILE, i = i0 + r, j = j0 + cc;
  if (i < n && j < n && i - j <= kl && j - i <= ku) {
    double* a = ab + (size_t)(kv + i - j) + (size_t)j * ld;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
    for (int q = 0; q < NP_NB; q += 4) {
      s0 += sL[r][q] * sU[q][cc];
      s1 += sL[r][q + 1] * sU[q + 1][cc];
      s2 += sL[r][q + 2] * sU[q + 2][cc];
      s3 += sL[r][q + 3] * sU[q + 3][cc];
    }
    const double v = *a - ((s0 + s1) + (s2 + s3));
    *a = v;
    gmax = fmax(gmax, fabs(v));
  }
}

__global__ void __launch_bounds__(NP_THREADS) k_gbtrf_np(CoarseDev c, int* flags, unsigned* bar,
                                                         unsigned long long* stats) {
  __shared__ double A[NP_NB][NP_NB + 1];       // diagonal block (L11 and U11)
  __shared__ double Lm[NP_NB][NP_NB + 1];      // multipliers of the diagonal block being factored
  __shared__ double rd[NP_NB];                 // 1 / U11(j, j)
  __shared__ double sL[NP_TILE][NP_NB + 1];    // tile rows of L21
  __shared__ double sU[NP_NB][NP_TILE + 1];    // tile columns of U12
  const int n = c.n, kl = c.kl, ku = c.ku, ld = c.ldab, kv = kl + ku;
  double* ab = c.ab;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NP_THREADS / 32;
  const int G = gridDim.x, b = blockIdx.x;
  unsigned* dcount = bar + 6;                  // diagonal-block tiles updated so far (monotonic)
  // with enough CTAs the next diagonal block's tiles go to CTAs 1..4, CTA 0 factors it, the other
  // tiles go to the remaining CTAs
  const bool split = G >= 8;
  const int first_other = split ? 5 : (G > 1 ? 1 : 0), n_other = G - first_other;
  unsigned dtarget = 0;
  double gmax = 0.0;
  {
    double m = 0.0;
    for (size_t t = (size_t)b * NP_THREADS + tid; t < (size_t)n * (kl + ku + 1); t += (size_t)G * NP_THREADS) {
      const int j = (int)(t / (kl + ku + 1)), r = (int)(t % (kl + ku + 1));
      const int i = j - ku + r;
      if (i >= 0 && i < n) m = fmax(m, fabs(ab[(size_t)(kv + i - j) + (size_t)j * ld]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) np_max_abs(&stats[0], m);
  }
  if (b == 0) {
    const int kb = min(NP_NB, n);
    np_load_diag(c, 0, kb, A);
    __syncthreads();
    np_factor_diag(c, 0, kb, A, Lm, gmax, flags);
  }
  if (!grid_barrier(bar, flags)) return;
  for (int k0 = 0; k0 < n; k0 += NP_NB) {
    const int kb = min(NP_NB, n - k0), r0 = k0 + kb;
    const int nr = min(kl, n - r0), nc = min(ku, n - r0);
    if (nr <= 0 && nc <= 0) break;
    np_load_diag(c, k0, kb, A);
    for (int j = tid; j < NP_NB; j += NP_THREADS) rd[j] = j < kb ? c.rdiag[k0 + j] : 0.0;
    __syncthreads();
    for (int task = b * nw + warp; task < nr + nc; task += G * nw) {
      if (task < nr) {
        const int i = r0 + task, col = k0 + lane;
        double acc = (lane < kb && i - col <= kl) ? ab[(size_t)(kv + i - col) + (size_t)col * ld] : 0.0;
        double x = 0.0;
        for (int m = 0; m < kb; ++m) {
          const double xm = __shfl_sync(0xffffffffu, acc, m) * rd[m];
          if (lane == m) x = xm;
          if (lane > m) acc -= xm * A[m][lane];
        }
        if (lane < kb && i - col <= kl) {
          ab[(size_t)(kv + i - col) + (size_t)col * ld] = x;
          gmax = fmax(gmax, fabs(x));
        }
      } else {
        const int j = r0 + task - nr, row = k0 + lane;
        double acc = (lane < kb && j - row <= ku) ? ab[(size_t)(kv + row - j) + (size_t)j * ld] : 0.0;
        for (int m = 0; m < kb; ++m) {
          const double ym = __shfl_sync(0xffffffffu, acc, m);
          if (lane > m) acc -= A[lane][m] * ym;
        }
        if (lane < kb && j - row <= ku) {
          ab[(size_t)(kv + row - j) + (size_t)j * ld] = acc;
          gmax = fmax(gmax, fabs(acc));
        }
      }
    }
    if (!grid_barrier(bar, flags)) return;
    const int ntr = (nr + NP_TILE - 1) / NP_TILE, ntc = (nc + NP_TILE - 1) / NP_TILE;
    const int kb2 = min(NP_NB, n - r0);
    const int dt = kb2 > 0 ? (kb2 + NP_TILE - 1) / NP_TILE : 0;
    // diagonal-block tiles: CTAs 1..dt^2 (split) or CTA 0
    if (split ? (b >= 1 && b <= dt * dt) : b == 0) {
      for (int d = split ? b - 1 : 0; d < (split ? b : dt * dt); ++d) {
        const int ti = d / dt, tj = d % dt;
        np_tile(c, k0, kb, r0 + ti * NP_TILE, r0 + tj * NP_TILE, sL, sU, gmax);
      }
      if (split) {
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          atomicAdd(dcount, 1u);
        }
      }
    }
    if (split) dtarget += dt * dt;
    // the other tiles of the band, round robin over the remaining CTAs
    if (b >= first_other || n_other == 0) {
      for (int t = (n_other > 0 ? b - first_other : 0); t < ntr * ntc; t += (n_other > 0 ? n_other : 1)) {
        const int ti = t / ntc, tj = t % ntc;
        if (ti < dt && tj < dt) continue;
        const int i0 = r0 + ti * NP_TILE, j0 = r0 + tj * NP_TILE;
        if (i0 - (j0 + NP_TILE - 1) > kl || j0 - (i0 + NP_TILE - 1) > ku) continue;
        np_tile(c, k0, kb, i0, j0, sL, sU, gmax);
      }
    }
    if (b == 0 && kb2 > 0) {
      if (split && tid == 0) {
        volatile unsigned* dc = dcount;
        long long spins = 0;
        while (*dc < dtarget) {
          if (++spins > BARRIER_SPIN_LIMIT) {
            atomicOr(flags, FLAG_TIMEOUT);
            break;
          }
        }
        __threadfence();
      }
      __syncthreads();
      np_load_diag(c, r0, kb2, A);
      __syncthreads();
      np_factor_diag(c, r0, kb2, A, Lm, gmax, flags);
    }
    if (!grid_barrier(bar, flags)) return;
  }
  for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) np_max_abs(&stats[1], gmax);
  if (!grid_barrier(bar, flags)) return;
  if (b == 0 && tid == 0) {
    const double g0 = __longlong_as_double((long long)stats[0]), g1 = __longlong_as_double((long long)stats[1]);
    if (!(g1 <= NOPIV_MAX_GROWTH * g0)) atomicOr(flags, FLAG_NOPIV_REJECTED);
  }
}


cudaError_t launch_coarse_factor_nopiv(const CoarseDev& c, int* flags, unsigned* scratch, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gbtrf_np, NP_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  // barrier words [0, 2), the two statistics (8-byte aligned at word 2) and the diagonal-tile
  // counter (word 6) start at zero
  e = cudaMemsetAsync(scratch, 0, 8 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  CoarseDev cc = c;
  unsigned* bar = scratch;
  unsigned long long* stats = reinterpret_cast<unsigned long long*>(scratch + 2);
  void* args[] = {(void*)&cc, (void*)&flags, (void*)&bar, (void*)&stats};
  e = cudaLaunchCooperativeKernel((const void*)k_gbtrf_np, dim3(sms), dim3(NP_THREADS), args, 0, st);
  count_launch(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_coarse_assemble(const CoarseDev& c, const double* mom, int E, cudaStream_t st) {
  if (E == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(c.ab, 0, sizeof(double) * (size_t)c.ldab * c.n, st);
  if (e != cudaSuccess) return e;
  k_coarse_assemble<<<(E + 127) / 128, 128, 0, st>>>(c, mom, E);
  count_launch(1);
  return cudaGetLastError();
}

// variant: 16 or 8, the cluster LU with that many CTAs; 1, the single-CTA window; 0, the
// global-memory kernel; -1, the first of these that the device runs for this band.  All variants
// take the same steps in the same order, so they give identical factors.
cudaError_t launch_coarse_factor(const CoarseDev& c, int* flags, cudaStream_t st, int variant) {
  if (c.n == 0) return cudaSuccess;
  if (variant < 0) {
    int v[COARSE_FACTOR_MAX_VARIANTS];
    coarse_factor_variants(c, v);
    variant = v[0];
  }
  if (variant >= 8) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    int NS = 0;
    if (!gbtrf_cluster_config(c, variant, &cfg, attr, &NS)) return cudaErrorInvalidConfiguration;
    cfg.stream = st;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_gbtrf_cluster, c, flags, NS);
    count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  if (variant == 1) {
    const cudaError_t e = raise_smem_limit<k_gbtf2_win>();
    if (e != cudaSuccess) return e;
    k_gbtf2_win<<<1, GBW_THREADS, gbtf2_win_smem(c), st>>>(c, flags);
  } else {
    k_gbtf2<<<1, 512, 0, st>>>(c, flags);
  }
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_rhs(const CoarseDev& c, const double* mom0, int E, cudaStream_t st) {
  if (E == 0) return cudaSuccess;
  k_coarse_rhs<<<(E * c.nq + 127) / 128, 128, 0, st>>>(c, mom0, E);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const CoarseDev& c, const double* mom0, int E, cudaStream_t st) {
  if (c.n == 0) return cudaSuccess;
  if (gbb_usable(c)) return launch_gbb_solve(c, mom0, E, st);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the deepest ring that fits next to the right-hand side: the band data come from HBM and one
  // step is short, so several steps must be in flight
  const int rows = (c.kl + c.ku + 1 + GBS_THREADS - 1) / GBS_THREADS;
  int depth = 0;
  for (int d : {8, 4})
    if (gbtrs_smem(c, d) <= (size_t)optin) {
      depth = d;
      break;
    }
  if (depth > 0 && rows <= 8) {
    const size_t sm = gbtrs_smem(c, depth);
    cudaError_t e = cudaSuccess;
    const int R = rows <= 2 ? 2 : rows <= 4 ? 4 : 8;
#define MRCM_GBTRS(RR, DD)                                                               \
  if (R == RR && depth == DD) {                                                          \
    if ((e = raise_smem_limit<k_gbtrs_smem<RR, DD>>()) == cudaSuccess)                   \
      k_gbtrs_smem<RR, DD><<<1, GBS_THREADS, sm, st>>>(c, mom0, E);                      \
  }
    MRCM_GBTRS(2, 4) MRCM_GBTRS(2, 8)
    MRCM_GBTRS(4, 4) MRCM_GBTRS(4, 8)
    MRCM_GBTRS(8, 4) MRCM_GBTRS(8, 8)
#undef MRCM_GBTRS
    if (e != cudaSuccess) return e;
    count_launch(1);
    return cudaGetLastError();
  }
  const cudaError_t e = launch_coarse_rhs(c, mom0, E, st);
  if (e != cudaSuccess) return e;
  k_gbtrs<<<1, 256, 0, st>>>(c);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace mrcm
