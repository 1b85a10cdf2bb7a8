// Coupling system of MRCM-O (Eq. 13-14) by a multifrontal LU over a nested dissection of the
// subdomain grid, without row interchanges.
//
// Each interface carries 2 nq unknowns and the 2 nq rows homed at them (flux and pressure rows),
// and a row couples the unknowns of the one or two subdomains it joins, so a rectangle of
// subdomains whose interior interfaces are eliminated leaves couplings only among the interfaces of
// its boundary.  The host plan (plan.cpp) cuts the grid recursively; a front eliminates the
// separator of its rectangle (or every interior interface of a leaf rectangle).  With the front
// F = [F11 F12; F21 F22] (pivot unknowns P first, boundary unknowns U after),
//   F11^-1 (Gauss-Jordan without pivoting),  D = F11^-1 F12,  B = F21 F11^-1,
//   S = F22 - F21 D  (added into the parent front),
// and a solve of G x = g runs forward through the levels, v_P = g_P + children's w, w_U = v_U - B v_P,
// then backward, x_P = F11^-1 v_P - D x_U.  Every product has a fixed order, so the solution is
// deterministic.  A zero or non-finite pivot, or |S| above NOPIV_MAX_GROWTH max |G|, sets
// FLAG_NOPIV_REJECTED and the caller falls back to the pivoted band LU of k_coarse.cu.
#include <cooperative_groups.h>

#include "common.cuh"

namespace mrcm {

constexpr int MF_THREADS = 256;
constexpr int MF_GJ_CL = 8;          // CTAs of the cluster that inverts a large pivot block
constexpr int MF_GJ_CLUSTER_NP = 64; // pivot blocks this large (and divisible by MF_GJ_CL) use it

// largest of a non-negative double across the CTA into an 8-byte maximum in global memory (the
// bit patterns of non-negative doubles order like the values; +inf above every finite value)
__device__ __forceinline__ void cta_max_to(double v, unsigned long long* dst) {
  __shared__ double red[MF_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    atomicMax(dst, (unsigned long long)__double_as_longlong(m));
  }
}

__device__ __forceinline__ double mag(double v) { return isfinite(v) ? fabs(v) : __longlong_as_double(0x7ff0000000000000LL); }

// C (M x N) = (acc ? C : 0) + alpha A (M x K) B (K x N), row-major operands with leading
// dimensions, in global or shared memory; one CTA of MF_THREADS, 32 x 32 output tiles with 2 x 2
// outputs per thread, K in chunks of 32 staged in shared memory (sm: 2048 doubles).  Returns the
// largest |C| written (+inf for a non-finite entry).
__device__ double cta_gemm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                           int ldc, double alpha, bool acc, double* sm) {
  double* As = sm;          // As[k * 32 + r] = A[m0 + r][k0 + k]
  double* Bs = sm + 1024;   // Bs[k * 32 + c] = B[k0 + k][n0 + c]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double cmax = 0.0;
  for (int m0 = 0; m0 < M; m0 += 32)
    for (int n0 = 0; n0 < N; n0 += 32) {
      double c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = 0.0;
      for (int k0 = 0; k0 < K; k0 += 32) {
        for (int t = tid; t < 1024; t += MF_THREADS) {
          const int k = t >> 5, r = t & 31;
          As[t] = (m0 + r < M && k0 + k < K) ? A[(size_t)(m0 + r) * lda + k0 + k] : 0.0;
          Bs[t] = (k0 + k < K && n0 + r < N) ? B[(size_t)(k0 + k) * ldb + n0 + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          const double a0 = As[k * 32 + ty], a1 = As[k * 32 + ty + 16];
          const double b0 = Bs[k * 32 + tx], b1 = Bs[k * 32 + tx + 16];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        __syncthreads();
      }
      const double cv[2][2] = {{c00, c01}, {c10, c11}};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
          if (r < M && c < N) {
            double* p = C + (size_t)r * ldc + c;
            const double v = (acc ? *p : 0.0) + alpha * cv[i][j];
            *p = v;
            cmax = fmax(cmax, mag(v));
          }
        }
    }
  return cmax;
}

__device__ __forceinline__ unsigned long long* mf_stats(const MfDev& m) {
  return reinterpret_cast<unsigned long long*>(m.scr + 2);
}

// One CTA per front of a level: assembly (zero, the original entries of the pivot rows and
// columns, the children's Schur complements in child order) and F11^-1 in place.
__global__ void __launch_bounds__(MF_THREADS) k_mf_front(MfDev m, const double* __restrict__ ab, int first,
                                                         int* flags) {
  extern __shared__ __align__(16) double smd[];
  const int fid = m.order[first + blockIdx.x];
  const MfFront fr = m.fr[fid];
  const int np = fr.np, nu = fr.nu, f = np + nu;
  double* __restrict__ F = m.F + fr.fo;
  for (size_t t = threadIdx.x; t < (size_t)f * f; t += MF_THREADS) F[t] = 0.0;
  __syncthreads();
  // assembly in batches of AB entries per thread, every load of a batch issued before its stores
  // (the positions within one batch, and within one child, are distinct)
  constexpr int AB = 8;
  double amax = 0.0;
  for (int t0 = threadIdx.x; t0 < fr.na; t0 += AB * MF_THREADS) {
    int dst[AB];
    double v[AB];
#pragma unroll
    for (int e = 0; e < AB; ++e) {
      const int t = t0 + e * MF_THREADS;
      dst[e] = -1;
      v[e] = 0.0;
      if (t < fr.na) {
        const int2 p = m.asmv[fr.ao + t];
        dst[e] = p.x;
        v[e] = ab[p.y];
      }
    }
#pragma unroll
    for (int e = 0; e < AB; ++e)
      if (dst[e] >= 0) {
        F[dst[e]] = v[e];
        amax = fmax(amax, mag(v[e]));
      }
  }
  __syncthreads();
  for (int c = 0; c < fr.nch; ++c) {
    const MfFront cf = m.fr[c == 0 ? fr.ch[0] : fr.ch[1]];
    const int fc = cf.np + cf.nu, nuc = cf.nu;
    const double* __restrict__ S = m.F + cf.fo + (size_t)cf.np * fc + cf.np;
    const int* mp = m.map + (c == 0 ? fr.mo[0] : fr.mo[1]);
    for (int t0 = threadIdx.x; t0 < nuc * nuc; t0 += AB * MF_THREADS) {
      size_t dst[AB];
      double v[AB], o[AB];
#pragma unroll
      for (int e = 0; e < AB; ++e) {
        const int t = t0 + e * MF_THREADS;
        dst[e] = ~(size_t)0;
        v[e] = o[e] = 0.0;
        if (t < nuc * nuc) {
          const int i = t / nuc, j = t - i * nuc;
          dst[e] = (size_t)mp[i] * f + mp[j];
          v[e] = S[(size_t)i * fc + j];
        }
      }
#pragma unroll
      for (int e = 0; e < AB; ++e)
        if (dst[e] != ~(size_t)0) o[e] = F[dst[e]];
#pragma unroll
      for (int e = 0; e < AB; ++e)
        if (dst[e] != ~(size_t)0) F[dst[e]] = o[e] + v[e];
    }
    __syncthreads();
  }
  cta_max_to(amax, mf_stats(m));
  if (np >= MF_GJ_CLUSTER_NP && np % MF_GJ_CL == 0) return;   // F11^-1 by k_mf_gj_cluster
  // Gauss-Jordan on F11 (np x np) in shared memory: pivot k takes the scaled row r_k = A_k. / a_kk
  // and the column c_k = A_.k, then a_ij -= c_i r_j off row and column k, row k = r_k, column
  // k = -c_k / a_kk, a_kk = 1 / a_kk; after the np pivots A = F11^-1
  double* A = smd;
  double* rk = A + np * np;
  double* ck = rk + np;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < np; i += MF_THREADS / 32)
    for (int j = lane; j < np; j += 32) A[i * np + j] = F[(size_t)i * f + j];
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < np; ++k) {
    double d = A[k * np + k];
    if (!(fabs(d) > 0.0) || !isfinite(d)) {
      bad = true;
      d = 1.0;
    }
    const double r = 1.0 / d;
    for (int j = threadIdx.x; j < np; j += MF_THREADS) {
      rk[j] = A[k * np + j] * r;
      ck[j] = A[j * np + k];
    }
    __syncthreads();
    for (int i = wid; i < np; i += MF_THREADS / 32) {
      const double ci = ck[i];
      for (int j = lane; j < np; j += 32) {
        double v;
        if (i == k) v = j == k ? r : rk[j];
        else if (j == k) v = -ci * r;
        else v = fma(-ci, rk[j], A[i * np + j]);
        A[i * np + j] = v;
      }
    }
    __syncthreads();
  }
  for (int i = wid; i < np; i += MF_THREADS / 32)
    for (int j = lane; j < np; j += 32) F[(size_t)i * f + j] = A[i * np + j];
  if (bad && lane == 0) atomicOr(flags, FLAG_NOPIV_REJECTED);
}

// F11^-1 of a large pivot block by the same Gauss-Jordan steps, over a cluster of MF_GJ_CL CTAs:
// CTA q keeps columns [q cw, (q + 1) cw) of F11 in shared memory (cw = np / MF_GJ_CL); per pivot the
// owner of column k publishes it (double-buffered), one cluster barrier, every CTA copies it through
// distributed shared memory and updates its columns.  Entry by entry the arithmetic is that of the
// one-CTA form.  One cluster per front of the level; fronts too small for it return at once.
__global__ void __launch_bounds__(MF_THREADS, 1) k_mf_gj_cluster(MfDev m, int first, int* flags) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double smd[];
  const int q = (int)cl.block_rank();
  const int fid = m.order[first + blockIdx.x / MF_GJ_CL];
  const MfFront fr = m.fr[fid];
  const int np = fr.np, f = fr.np + fr.nu;
  if (np < MF_GJ_CLUSTER_NP || np % MF_GJ_CL != 0) return;   // uniform over the cluster
  const int cw = np / MF_GJ_CL, c0 = q * cw;
  double* F = m.F + fr.fo;
  double* A = smd;                 // [np][cw] this CTA's columns
  double* pub = A + np * cw;       // [2][np] the pivot column, published by its owner
  double* col = pub + 2 * np;      // [np] the pivot column, copied
  double* rk = col + np;           // [cw] this CTA's part of the scaled pivot row
  const int tid = threadIdx.x;
  for (int t = tid; t < np * cw; t += MF_THREADS) {
    const int i = t / cw, jj = t - i * cw;
    A[t] = F[(size_t)i * f + c0 + jj];
  }
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < np; ++k) {
    const int owner = k / cw, kk = k - owner * cw;
    double* pb = pub + (k & 1) * np;
    if (q == owner)
      for (int i = tid; i < np; i += MF_THREADS) pb[i] = A[i * cw + kk];
    cl.sync();
    const double* rp = cl.map_shared_rank(pb, owner);
    for (int i = tid; i < np; i += MF_THREADS) col[i] = rp[i];
    __syncthreads();
    double d = col[k];
    if (!(fabs(d) > 0.0) || !isfinite(d)) {
      bad = true;
      d = 1.0;
    }
    const double r = 1.0 / d;
    for (int jj = tid; jj < cw; jj += MF_THREADS) rk[jj] = A[k * cw + jj] * r;
    __syncthreads();
    for (int t = tid; t < np * cw; t += MF_THREADS) {
      const int i = t / cw, jj = t - i * cw;
      const int j = c0 + jj;
      double v;
      if (i == k) v = j == k ? r : rk[jj];
      else if (j == k) v = -col[i] * r;
      else v = fma(-col[i], rk[jj], A[t]);
      A[t] = v;
    }
    __syncthreads();
  }
  cl.sync();   // no CTA leaves while another may still read its published column
  for (int t = tid; t < np * cw; t += MF_THREADS) {
    const int i = t / cw, jj = t - i * cw;
    F[(size_t)i * f + c0 + jj] = A[t];
  }
  if (bad && tid == 0) atomicOr(flags, FLAG_NOPIV_REJECTED);
}

// Tile tasks of a level: kind 0, columns c0.. of D = F11^-1 F12 (in place of F12, from a shared
// copy); kind 1, rows r0.. of B = F21 F11^-1; kind 2, the (r0, c0) tile of S = F22 - F21 D.
__global__ void __launch_bounds__(MF_THREADS) k_mf_tiles(MfDev m, int first) {
  extern __shared__ __align__(16) double smd[];
  const int4 tk = m.task[first + blockIdx.x];
  const MfFront fr = m.fr[tk.x];
  const int np = fr.np, nu = fr.nu, f = np + nu;
  double* F = m.F + fr.fo;
  double* Bx = F + (size_t)f * f;
  double* stage = smd + 2048;
  if (tk.y == 0) {
    const int cols = min(MF_TILE, nu - tk.w);
    for (int t = threadIdx.x; t < np * MF_TILE; t += MF_THREADS) {
      const int i = t / MF_TILE, j = t - i * MF_TILE;
      stage[t] = j < cols ? F[(size_t)i * f + np + tk.w + j] : 0.0;
    }
    __syncthreads();
    cta_gemm(np, cols, np, F, f, stage, MF_TILE, F + np + tk.w, f, 1.0, false, smd);
  } else if (tk.y == 1) {
    const int rows = min(MF_TILE, nu - tk.z);
    cta_gemm(rows, np, np, F + (size_t)(np + tk.z) * f, f, F, f, Bx + (size_t)tk.z * np, np, 1.0, false, smd);
  } else {
    const int rows = min(MF_TILE, nu - tk.z), cols = min(MF_TILE, nu - tk.w);
    const double smax = cta_gemm(rows, cols, np, F + (size_t)(np + tk.z) * f, f, F + np + tk.w, f,
                                 F + (size_t)(np + tk.z) * f + np + tk.w, f, -1.0, true, smd);
    cta_max_to(smax, mf_stats(m) + 1);
  }
}

__global__ void k_mf_check(MfDev m, int* flags) {
  const unsigned long long* st = mf_stats(m);
  const double gmax = __longlong_as_double((long long)st[0]), smax = __longlong_as_double((long long)st[1]);
  if (!(smax <= NOPIV_MAX_GROWTH * gmax) || !isfinite(gmax)) atomicOr(flags, FLAG_NOPIV_REJECTED);
}

cudaError_t launch_mf_factor(const MfDev& m, const Plan& P, const double* ab, int* flags, cudaStream_t st) {
  const size_t sm_front = 8 * ((size_t)P.mf_max_np * P.mf_max_np + 2 * (size_t)P.mf_max_np);
  const size_t sm_tiles = 8 * (2048 + (size_t)P.mf_max_np * MF_TILE);
  // the limits go to the device maximum once (raise_smem_limit): request workers launch these kernels
  // from several host threads with different sizes, and a per-launch limit could be lowered by
  // another thread between its set and its launch
  cudaError_t e = raise_smem_limit<k_mf_front>();
  if (e == cudaSuccess) e = raise_smem_limit<k_mf_tiles>();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(m.scr + 2, 0, 16, st);   // the statistics; the solve epoch runs on
  if (e != cudaSuccess) return e;
  for (int L = 0; L + 1 < (int)P.mf_level.size(); ++L) {
    const int nf = P.mf_level[L + 1] - P.mf_level[L];
    if (nf > 0) {
      k_mf_front<<<nf, MF_THREADS, sm_front, st>>>(m, ab, P.mf_level[L], flags);
      count_launch(1);
      bool big = false;   // a pivot block for the cluster form
      for (int i = P.mf_level[L]; i < P.mf_level[L + 1]; ++i) {
        const MfFront& fr = P.mf_front[P.mf_order[i]];
        big = big || (fr.np >= MF_GJ_CLUSTER_NP && fr.np % MF_GJ_CL == 0);
      }
      if (big) {
        const size_t sm_gj = 8 * ((size_t)P.mf_max_np * (P.mf_max_np / MF_GJ_CL) + 3 * (size_t)P.mf_max_np +
                                  P.mf_max_np / MF_GJ_CL);
        cudaError_t e2 = raise_smem_limit<k_mf_gj_cluster>();
        if (e2 != cudaSuccess) return e2;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = MF_GJ_CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(nf * MF_GJ_CL);
        cfg.blockDim = dim3(MF_THREADS);
        cfg.dynamicSmemBytes = sm_gj;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e2 = cudaLaunchKernelEx(&cfg, k_mf_gj_cluster, m, P.mf_level[L], flags);
        if (e2 != cudaSuccess) return e2;
        count_launch(1);
      }
    }
    const int nb = P.mf_task_c[L] - P.mf_task_b[L];
    if (nb > 0) {
      k_mf_tiles<<<nb, MF_THREADS, sm_tiles, st>>>(m, P.mf_task_b[L]);
      count_launch(1);
    }
    const int nc = P.mf_task_b[L + 1] - P.mf_task_c[L];
    if (nc > 0) {
      k_mf_tiles<<<nc, MF_THREADS, sm_tiles, st>>>(m, P.mf_task_c[L]);
      count_launch(1);
    }
  }
  k_mf_check<<<1, 1, 0, st>>>(m, flags);
  count_launch(1);
  return cudaGetLastError();
}

// y_r = sum_k A[r][k] x[k] for r < rows (A row-major with leading dimension lda, in shared or global
// memory): tpr threads per row (a power of two up to 8, as many as the CTA has for the rows), each
// with four partial sums over its columns k = q, q + tpr, ..., then the tpr sums in a fixed shuffle
// order; emit(r, y) by the first thread of the row.  Deterministic.
template <class Emit>
__device__ __forceinline__ void mf_rows(const double* A, int lda, int rows, int cols, const double* x, Emit emit) {
  int tpr = 1;
  while (tpr < 8 && tpr * 2 * rows <= MF_THREADS) tpr *= 2;
  const int q = threadIdx.x % tpr, per = MF_THREADS / tpr;
  for (int r0 = 0; r0 < rows; r0 += per) {
    const int r = r0 + threadIdx.x / tpr;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (r < rows) {
      const double* a = A + (size_t)r * lda;
      int k = q;
      for (; k + 3 * tpr < cols; k += 4 * tpr) {
        s0 = fma(a[k], x[k], s0);
        s1 = fma(a[k + tpr], x[k + tpr], s1);
        s2 = fma(a[k + 2 * tpr], x[k + 2 * tpr], s2);
        s3 = fma(a[k + 3 * tpr], x[k + 3 * tpr], s3);
      }
      for (; k < cols; k += tpr) s0 = fma(a[k], x[k], s0);
    }
    double t = (s0 + s1) + (s2 + s3);
    for (int o = 1; o < tpr; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (r < rows && q == 0) emit(r, t);
  }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Solve, one cooperative launch (one CTA per SM), fronts taken level by level in round robin: a
// front's forward step waits for its children's, its backward step for its parent's (the
// ancestors have then written x_U), through completion flags stamped with the solve's epoch.  The
// epoch lives in device memory: every CTA reads it at the start, the last CTA to finish advances
// it, so repeated launches (also from a captured graph) never see a stale flag as current.  All
// CTAs are resident and each takes its fronts in increasing level (decreasing, backward), so
// every wait ends; the spins are bounded all the same (FLAG_TIMEOUT).  Everything a step reads
// that does not depend on the wait (the front's indices, its right-hand side entries, its B or
// [F11^-1 D] rows, copied asynchronously into shared memory) is requested before the wait, so a
// level costs about one flag hand-over and one read.  A front's rows are dotted by whole warps
// (up to eight threads per row, four partial sums each, combined in a fixed order), so the result
// is deterministic.
__global__ void __launch_bounds__(MF_THREADS) k_mf_solve(MfDev m, double* __restrict__ g, int* flags, int mcap) {
  extern __shared__ __align__(16) double smd[];
  double* v = smd;                                   // [max_f]
  double* M = v + m.max_f;                           // [mcap] rows of B or of [F11^-1 D]
  int* ix = reinterpret_cast<int*>(M + mcap);        // [max_f]
  __shared__ unsigned s_ep;
  __shared__ int s_ok;
  volatile unsigned* vep = m.scr + 8;
  if (threadIdx.x == 0) {
    s_ep = *vep + 1u;
    s_ok = 1;
  }
  __syncthreads();
  const unsigned E = s_ep;
  volatile unsigned* fdone = m.done;
  volatile unsigned* bdone = m.done + m.nfront;
  // thread 0 polls the flag; the CTA proceeds together (false: the wait gave up)
  auto wait_for = [&](volatile unsigned* fl) -> bool {
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (*fl != E) {
        if (++spins > BARRIER_SPIN_LIMIT) {
          atomicOr(flags, FLAG_TIMEOUT);
          s_ok = 0;
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
  };
  auto publish = [&](volatile unsigned* fl) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *fl = E;
  };
  bool ok = true;
  // forward: v_P = g_P + the children's w mapped into P, v_U = their part mapped into U;
  // keep v_P, pass w_U = v_U - B v_P up
  for (int L = 0; L < m.levels && ok; ++L) {
    for (int b = m.lvl[L] + blockIdx.x; b < m.lvl[L + 1] && ok; b += gridDim.x) {
      const int fid = m.order[b];
      const MfFront fr = m.fr[fid];
      const int np = fr.np, nu = fr.nu, f = np + nu;
      const double* Bx = m.F + fr.fo + (size_t)f * f;
      // B staged row by row with an odd stride in doubles (np + 1): the rows a warp reads start in
      // different banks
      const bool staged = nu * (np + 1) <= mcap;
      if (staged)
        for (int r = threadIdx.x >> 5; r < nu; r += MF_THREADS / 32)
          for (int k = threadIdx.x & 31; k < np; k += 32) cp_async8(M + (size_t)r * (np + 1) + k, Bx + (size_t)r * np + k);
      for (int t = threadIdx.x; t < f; t += MF_THREADS) v[t] = t < np ? g[m.idx[fr.io + t]] : 0.0;
      __syncthreads();
      for (int c = 0; c < fr.nch && ok; ++c) {
        const int cid = c == 0 ? fr.ch[0] : fr.ch[1];
        const MfFront cf = m.fr[cid];
        const int* mp = m.map + (c == 0 ? fr.mo[0] : fr.mo[1]);
        const double* wc = m.V + cf.vo + cf.np;
        ok = wait_for(fdone + cid);
        if (!ok) break;
        for (int t = threadIdx.x; t < cf.nu; t += MF_THREADS) v[mp[t]] += __ldcg(wc + t);
        __syncthreads();
      }
      if (!ok) break;
      cp_async_wait_all();
      __syncthreads();
      double* Vf = m.V + fr.vo;
      for (int t = threadIdx.x; t < np; t += MF_THREADS) Vf[t] = v[t];
      mf_rows(staged ? M : Bx, staged ? np + 1 : np, nu, np, v,
              [&](int r, double t) { Vf[np + r] = v[np + r] - t; });
      publish(fdone + fid);
    }
  }
  // backward: x_P = [F11^-1 D] [v_P; -x_U], x_U written by the ancestors
  for (int L = m.levels - 1; L >= 0 && ok; --L) {
    for (int b = m.lvl[L] + blockIdx.x; b < m.lvl[L + 1] && ok; b += gridDim.x) {
      const int fid = m.order[b];
      const MfFront fr = m.fr[fid];
      const int np = fr.np, nu = fr.nu, f = np + nu;
      const double* F = m.F + fr.fo;
      const double* Vf = m.V + fr.vo;
      const bool staged = np * (f + 1) <= mcap;   // [F11^-1 D], rows with stride f + 1
      if (staged)
        for (int r = threadIdx.x >> 5; r < np; r += MF_THREADS / 32)
          for (int k = threadIdx.x & 31; k < f; k += 32) cp_async8(M + (size_t)r * (f + 1) + k, F + (size_t)r * f + k);
      for (int t = threadIdx.x; t < f; t += MF_THREADS) {
        ix[t] = m.idx[fr.io + t];
        if (t < np) v[t] = Vf[t];
      }
      if (fr.par >= 0) {
        ok = wait_for(bdone + fr.par);
        if (!ok) break;
      } else {
        __syncthreads();
      }
      for (int t = np + threadIdx.x; t < f; t += MF_THREADS) v[t] = -__ldcg(g + ix[t]);
      cp_async_wait_all();
      __syncthreads();
      mf_rows(staged ? M : F, staged ? f + 1 : f, np, f, v, [&](int r, double t) { g[ix[r]] = t; });
      publish(bdone + fid);
    }
  }
  // the last CTA to finish advances the epoch (a CTA that gave up still counts itself)
  cp_async_wait_all();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(m.scr + 9, 1u) == gridDim.x - 1) {
      m.scr[9] = 0u;
      __threadfence();
      *vep = E;
    }
  }
}

cudaError_t launch_mf_solve(const MfDev& m, const CoarseDev& c, const double* mom0, int E, int* flags,
                            cudaStream_t st) {
  cudaError_t e = launch_coarse_rhs(c, mom0, E, st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // shared memory: v and the indices of the largest front, and its matrix rows when they fit in
  // about 192 KB (larger fronts read them from global memory)
  int mcap = m.mcap;
  const size_t sm = 12 * (size_t)m.max_f + 8 * (size_t)mcap;
  e = raise_smem_limit<k_mf_solve>();
  if (e != cudaSuccess) return e;
  MfDev mm = m;
  double* g = c.g;
  int* fl = flags;
  void* args[] = {(void*)&mm, (void*)&g, (void*)&fl, (void*)&mcap};
  e = cudaLaunchCooperativeKernel((const void*)k_mf_solve, dim3(sms), dim3(MF_THREADS), args, sm, st);
  count_launch(1);
  return e;
}

}  // namespace mrcm
