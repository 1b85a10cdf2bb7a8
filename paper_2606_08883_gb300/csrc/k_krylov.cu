// Krylov kernels for Algorithm 1 (restarted right-preconditioned GMRES storing Z), FP64.
//
// Inner step j runs as one cooperative kernel (k_arnoldi_ls below).  For vectors too long for one
// co-resident wave the step falls back to separate launches in MGS pass order: w = A z_j fused with
// h_{0,j} = (w, v_0) and ||w||^2, then "w -= h_{i-1,j} v_{i-1}, h_{i,j} = (w, v_i)" for i = 1..j, a
// last pass for h_{j+1,j} = ||w||, and the Givens update in one thread.  Reductions are
// deterministic: fixed grid, per-block partials, summed in block order.
#include <algorithm>

#include "common.cuh"

namespace mrcm {

__global__ void __launch_bounds__(RED_THREADS) k_norm2(const double* __restrict__ x, size_t n, double* partials,
                                                       unsigned* counter, double* out) {
  __shared__ double sm[32];
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[0] += x[i] * x[i];
  double* const outs[1] = {out};
  grid_reduce<1>(v, partials, counter, outs, sm, 1);
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ denom, size_t n, double* __restrict__ y) {
  const double d = *denom;
  const double r = d != 0.0 ? 1.0 / d : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = d != 0.0 ? x[i] * r : 0.0;
}

// w = A z, out0 = (w, v0), out1 = (w, w)
__global__ void __launch_bounds__(RED_THREADS) k_matvec_dot(Geo g, const double* __restrict__ z,
                                                            const double* __restrict__ v0, double* __restrict__ w,
                                                            double* partials, unsigned* counter, double* out0,
                                                            double* out1) {
  __shared__ double sm[32];
  double v[2] = {0.0, 0.0};
  const size_t n = (size_t)g.nx * g.ny;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const double zc = z[c];
    const double zw = i > 0 ? z[c - 1] : 0.0;
    const double ze = i < g.nx - 1 ? z[c + 1] : 0.0;
    const double zs = j > 0 ? z[c - g.nx] : 0.0;
    const double zn = j < g.ny - 1 ? z[c + g.nx] : 0.0;
    const double* Tx = g.Tx + (size_t)j * (g.nx + 1) + i;
    const double* Ty = g.Ty + (size_t)j * g.nx + i;
    const double wx = Tx[1] * (zc - ze) - Tx[0] * (zw - zc);
    const double wy = Ty[g.nx] * (zc - zn) - Ty[0] * (zs - zc);
    const double wc = wx + wy;
    w[c] = wc;
    v[0] += wc * v0[c];
    v[1] += wc * wc;
  }
  double* const outs[2] = {out0, out1};
  grid_reduce<2>(v, partials, counter, outs, sm, 0);
}

// w -= (*hprev) vprev; then hout = (w, vnext), or ||w|| when vnext is null
__global__ void __launch_bounds__(RED_THREADS) k_mgs_pass(const double* __restrict__ vprev,
                                                          const double* __restrict__ hprev,
                                                          const double* __restrict__ vnext, size_t n,
                                                          double* __restrict__ w, double* partials, unsigned* counter,
                                                          double* hout) {
  __shared__ double sm[32];
  const double h = *hprev;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double wi = w[i] - h * vprev[i];
    w[i] = wi;
    v[0] += vnext ? wi * vnext[i] : wi * wi;
  }
  double* const outs[1] = {hout};
  grid_reduce<1>(v, partials, counter, outs, sm, vnext ? 0 : 1);
}

// Givens update of Hessenberg column j (column-major, leading dimension ldh).
// out[0] = |g_{j+1}| (residual estimate), out[1] = h_{j+1,j} before rotation, out[2] = ||A z_j||.
__global__ void k_givens(double* H, double* cs, double* sn, double* gv, int j, int ldh, const double* wnorm2,
                         double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ldh;
  const double hnext = col[j + 1];
  for (int i = 0; i < j; ++i) {
    const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
    const double t1 = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t0;
    col[i + 1] = t1;
  }
  const double a = col[j], b = col[j + 1];
  double c, s, t;
  if (b == 0.0) {
    c = 1.0;
    s = 0.0;
    t = a;
  } else {
    t = hypot(a, b);
    c = a / t;
    s = b / t;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = t;
  col[j + 1] = 0.0;
  gv[j + 1] = -s * gv[j];
  gv[j] = c * gv[j];
  out[0] = fabs(gv[j + 1]);
  out[1] = hnext;
  out[2] = sqrt(*wnorm2);
}

// y = R^-1 g (R = leading k x k of the rotated H) then p += Z y
__global__ void k_update(double* __restrict__ p, const double* __restrict__ Z, size_t n, const double* __restrict__ H,
                         const double* __restrict__ gv, int k, int ldh) {
  extern __shared__ double y[];
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int t = i + 1; t < k; ++t) acc -= H[(size_t)t * ldh + i] * y[t];
      y[i] = acc / H[(size_t)i * ldh + i];
    }
  }
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = p[i];
    for (int t = 0; t < k; ++t) acc += y[t] * Z[(size_t)t * n + i];
    p[i] = acc;
  }
}

// r = b - A p and out = ||r||
__global__ void __launch_bounds__(RED_THREADS) k_residual_norm(Geo g, const double* __restrict__ b,
                                                               const double* __restrict__ p, double* __restrict__ r,
                                                               double* partials, unsigned* counter, double* out) {
  __shared__ double sm[32];
  double v[1] = {0.0};
  const size_t n = (size_t)g.nx * g.ny;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const double pc = p[c];
    const double pw = i > 0 ? p[c - 1] : 0.0;
    const double pe = i < g.nx - 1 ? p[c + 1] : 0.0;
    const double ps = j > 0 ? p[c - g.nx] : 0.0;
    const double pn = j < g.ny - 1 ? p[c + g.nx] : 0.0;
    const double* Tx = g.Tx + (size_t)j * (g.nx + 1) + i;
    const double* Ty = g.Ty + (size_t)j * g.nx + i;
    const double wx = Tx[1] * (pc - pe) - Tx[0] * (pw - pc);
    const double wy = Ty[g.nx] * (pc - pn) - Ty[0] * (ps - pc);
    const double rc = b[c] - (wx + wy);
    r[c] = rc;
    v[0] += rc * rc;
  }
  double* const outs[1] = {out};
  grid_reduce<1>(v, partials, counter, outs, sm, 1);
}

// ============================================================================================
// Cooperative Arnoldi step.  All blocks are co-resident (cooperative launch); grid barriers are
// an arrival counter plus a generation word, polled with a bounded spin that sets FLAG_TIMEOUT and
// returns instead of waiting forever.
// ============================================================================================
// One Arnoldi step (inner step j) in a single cooperative launch, with the modified
// Gram-Schmidt coefficients obtained from one global reduction.  MGS computes
//   h_i = (w - sum_{k<i} h_k v_k, v_i) = a_i - sum_{k<i} (v_k, v_i) h_k,   a_i = (w, v_i),
// i.e. (I + R) h = a with R the strictly lower Gram matrix of the basis.  T = (I + R)^-1 is kept in
// its compact inverse form and grows by one row per step (t_j = -r^T T_{j-1}, r_k = (v_k, v_j)):
// h_i = (T a)_i for i < j is a product instead of a sequential solve, and the last coefficient is
// the MGS recurrence itself, h_j = a_j - sum_k r_k h_k.
//
// Per step: one sweep over the basis that forms a_k and r_k together for every k < j (one read of
// v_k), plus (w, v_j) and ||A z_j||^2; one sweep for w -= V h and ||w||^2; three grid barriers.
// Each block owns one contiguous slice of the vectors.  GB300's FP64 rate (2 DFMA/clk/SM, 64-clock
// latency) bounds both sweeps, so the kernel is laid out to keep that pipe fed:
//  * dot sweep: every warp of the block busy at any j (each basis vector's task split over
//    nw / (j+1) warps), DOT_UNROLL loads in flight per lane, both sums of a warp reduced with one
//    exchange (half the shuffle adds);
//  * update sweep: every thread streams its UPD_EL elements of UPD_UU basis vectors per stage
//    through a UPD_DS-deep cp.async ring in shared memory (each thread reads back only its own
//    copies, so no block barrier per stage) and keeps each element's MGS order i = 0..j;
//  * the rows of T are copied to shared memory while the first totals are formed, so the
//    coefficients h come from on-chip data;
//  * the previous rotations of the Hessenberg column are a first-order linear recurrence
//    (y_{i+1} = -s_i y_i + c_i h_{i+1}) and are applied by a warp-wide scan in the last block,
//    overlapped with its share of the update sweep.
// Cross-block sums are taken in block order (deterministic).
struct LsArgs {
  const double* z;      // z_j
  double* V;            // basis, V_i at V + i n
  int j;
  size_t n;
  double* H;            // Hessenberg, column-major, leading dimension ldh
  int ldh;
  double* cs;
  double* sn;
  double* gv;
  double* out;          // [0] |g_{j+1}|, [1] h_{j+1,j}, [2] ||A z_j||
  double* wbuf;         // w (n)
  double* part;         // (2 ldh + 3) x gridDim partial sums
  double* tot;          // 2 ldh + 3 totals
  double* Tm;           // (I + R)^-1, row-major lower, leading dimension ldh
  unsigned* bar;
  int* flags;
  int stage_T;          // 1: rows of T staged in shared memory (fits), 0: read from global
};

constexpr int ARN_THREADS = 1024;
constexpr int DOT_UNROLL = 4;   // elements of the swept basis vector in flight per lane
constexpr int UPD_EL = 2;       // vector elements per thread in the update sweep
constexpr int UPD_UU = 2;       // basis vectors per ring stage
constexpr int UPD_DS = 3;       // ring stages
constexpr int ROW_TPR = 4;      // threads per row of T in the coefficient product
constexpr int ARN_SMALL = 5 * 264;                               // a | r | h | cs | sn (doubles)
constexpr int ARN_RING = UPD_DS * UPD_UU * UPD_EL * ARN_THREADS;  // doubles
constexpr int ARN_SMEM_MAX = 227 * 1024 - 1024;                   // dynamic bytes (static use kept apart)

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Sum of two values over a warp with one exchange: lanes < 16 end with the total of s0, lanes >= 16
// with the total of s1.
__device__ __forceinline__ double warp_sum2(double s0, double s1, int lane) {
  const bool low = lane < 16;
  double v = low ? s0 : s1;
  const double u = low ? s1 : s0;
  v += __shfl_xor_sync(0xffffffffu, u, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Applies rotations 0..j-1 to column entries h[0..j] and writes the rotated entries 0..j-1 to col;
// returns the rotated entry j (all lanes).  The running entry obeys y_{i+1} = -s_i y_i + c_i h_{i+1}
// (y_0 = h_0) and rotated entry i is c_i y_i + s_i h_{i+1}; lanes take contiguous index ranges,
// compose their affine maps, scan the maps across the warp and then replay their range.
__device__ __forceinline__ double givens_scan(const double* c_, const double* s_, const double* h, double* col, int j,
                                              int lane) {
  const int per = (j + 31) / 32;
  const int lo = lane * per, hi = min(j, lo + per);
  double A = 1.0, B = 0.0;
  for (int i = lo; i < hi; ++i) {
    const double ai = -s_[i], bi = c_[i] * h[i + 1];
    A = ai * A;
    B = ai * B + bi;
  }
  double eA = A, eB = B;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double pA = __shfl_up_sync(0xffffffffu, eA, o), pB = __shfl_up_sync(0xffffffffu, eB, o);
    if (lane >= o) {
      eB = eA * pB + eB;
      eA = eA * pA;
    }
  }
  double xA = __shfl_up_sync(0xffffffffu, eA, 1), xB = __shfl_up_sync(0xffffffffu, eB, 1);
  if (lane == 0) {
    xA = 1.0;
    xB = 0.0;
  }
  double y = xA * h[0] + xB;
  for (int i = lo; i < hi; ++i) {
    const double c = c_[i], s = s_[i], hn = h[i + 1];
    col[i] = c * y + s * hn;
    y = -s * y + c * hn;
  }
  const int owner = j == 0 ? 0 : (j - 1) / per;
  return __shfl_sync(0xffffffffu, j == 0 ? h[0] : y, owner);
}

// w[c] -= sum_{i<=j} h_i V_i[c] (in order i = 0..j) for the NE elements c = base + e ARN_THREADS of
// this thread, streamed through the thread's slots of the ring; adds their squares to nrm and
// leaves the results in keep.
template <int NE>
__device__ __forceinline__ void update_ring(const double* __restrict__ V, size_t n, int j, const double* sh_h,
                                            size_t base, int tid, double* ring, double* w, double& nrm,
                                            double (&keep)[UPD_EL], int nvalid = NE) {
  constexpr int NT = ARN_THREADS;
  double acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = e < nvalid ? w[base + (size_t)e * NT] : 0.0;
  double* tr = ring + tid;
  const int S = (j + UPD_UU) / UPD_UU;
  auto issue = [&](int s) {
    if (s < S) {
#pragma unroll
      for (int u = 0; u < UPD_UU; ++u) {
        const int i = s * UPD_UU + u;
        if (i <= j)
#pragma unroll
          for (int e = 0; e < NE; ++e)
            if (e < nvalid)
              cp_async8(tr + ((size_t)((s % UPD_DS) * UPD_UU + u) * NE + e) * NT, V + (size_t)i * n + base + (size_t)e * NT);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < UPD_DS; ++s) issue(s);
  for (int s = 0; s < S; ++s) {
    cp_async_wait<UPD_DS - 1>();
#pragma unroll
    for (int u = 0; u < UPD_UU; ++u) {
      const int i = s * UPD_UU + u;
      if (i <= j) {
        const double hu = sh_h[i];
#pragma unroll
        for (int e = 0; e < NE; ++e) acc[e] -= hu * tr[((size_t)((s % UPD_DS) * UPD_UU + u) * NE + e) * NT];
      }
    }
    issue(s + UPD_DS);
  }
  cp_async_wait<0>();
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    if (e < nvalid) {
      w[base + (size_t)e * NT] = acc[e];
      nrm += acc[e] * acc[e];
      keep[e] = acc[e];
    }
  }
}

__global__ void __launch_bounds__(ARN_THREADS, 1) k_arnoldi_ls(Geo g, LsArgs a) {
  extern __shared__ double sh[];      // small arrays | ring (update) or staged rows of T
  __shared__ double sm[32];
  __shared__ double s_dot[2 * (ARN_THREADS / 32)];
  __shared__ double s_hn, s_x;
  constexpr int nt = ARN_THREADS, nw = ARN_THREADS / 32;
  const int j = a.j, G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t n = a.n;
  const size_t chunk = (n + G - 1) / G;
  const size_t lo = (size_t)b * chunk < n ? (size_t)b * chunk : n;
  const size_t hi = lo + chunk < n ? lo + chunk : n;
  double* w = a.wbuf;
  const double* vj = a.V + (size_t)j * n;
  double* ring = sh + ARN_SMALL;
  // 1. w = A z_j on the slice (4 elements per thread, all loads before the stores)
  for (size_t base = lo + tid; base < hi; base += 4 * (size_t)nt) {
    double r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const size_t c = base + (size_t)e * nt;
      r[e] = 0.0;
      if (c < hi) {
        const int i = (int)(c % g.nx), jj = (int)(c / g.nx);
        const double* z = a.z;
        const double zc = z[c];
        const double zw = i > 0 ? z[c - 1] : 0.0;
        const double ze = i < g.nx - 1 ? z[c + 1] : 0.0;
        const double zs = jj > 0 ? z[c - g.nx] : 0.0;
        const double zn = jj < g.ny - 1 ? z[c + g.nx] : 0.0;
        const double* Tx = g.Tx + (size_t)jj * (g.nx + 1) + i;
        const double* Ty = g.Ty + (size_t)jj * g.nx + i;
        // the four face fluxes from the differences (no cancellation against a diagonal term), one
        // product and three FMAs
        double f = Tx[1] * (zc - ze);
        f = fma(Tx[0], zc - zw, f);
        f = fma(Ty[g.nx], zc - zn, f);
        r[e] = fma(Ty[0], zc - zs, f);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const size_t c = base + (size_t)e * nt;
      if (c < hi) w[c] = r[e];
    }
  }
  __syncthreads();
  // 2. block partials: task k < j gives a_k = (w, v_k) and r_k = (v_j, v_k) from one read of v_k;
  //    task j gives a_j = (w, v_j) and ||w||^2.  Slots: a_t at t, r_k at j+1+k, ||w||^2 at 2j+1.
  //    Every warp of the block takes part whatever j is: a round of up to nw tasks gives each task
  //    nw / (tasks in the round) warps over consecutive parts of the slice, and the parts' sums are
  //    added in part order (deterministic).
  const int nd = 2 * j + 2;
  for (int u0 = 0; u0 <= j; u0 += nw) {
    const int nr = min(j + 1 - u0, nw);
    const int wpt = nw / nr;
    const size_t sub = (((hi - lo) + wpt - 1) / wpt + 31) & ~(size_t)31;
    if (warp < nr * wpt) {
      const int t = j - (u0 + warp / wpt), q = warp % wpt;
      const size_t plo = lo + (size_t)q * sub < hi ? lo + (size_t)q * sub : hi;
      const size_t phi = plo + sub < hi ? plo + sub : hi;
      double s0 = 0.0, s1 = 0.0;
      size_t c = plo + lane;
      if (t < j) {
        const double* x = a.V + (size_t)t * n;
        constexpr int U = DOT_UNROLL;
        const size_t nfull = (phi - plo) / (32 * U);
        for (size_t k = 0; k < nfull; ++k, c += 32 * U) {
          double xv[U], wv[U], yv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            xv[u] = __ldcg(x + c + 32 * u);
            wv[u] = w[c + 32 * u];
            yv[u] = vj[c + 32 * u];
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            s0 += wv[u] * xv[u];
            s1 += yv[u] * xv[u];
          }
        }
        double xv[U], wv[U], yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = c + 32 * u < phi;
          xv[u] = in ? __ldcg(x + c + 32 * u) : 0.0;
          wv[u] = in ? w[c + 32 * u] : 0.0;
          yv[u] = in ? vj[c + 32 * u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          s0 += wv[u] * xv[u];
          s1 += yv[u] * xv[u];
        }
      } else {
        for (; c < phi; c += 32) {
          const double wc = w[c];
          s0 += wc * vj[c];
          s1 += wc * wc;
        }
      }
      const double v = warp_sum2(s0, s1, lane);
      if (lane == 0) s_dot[2 * warp] = v;
      if (lane == 16) s_dot[2 * warp + 1] = v;
    }
    __syncthreads();
    if (tid < 2 * nr) {
      const int uu = tid >> 1, which = tid & 1;
      const int t = j - (u0 + uu);
      double acc = 0.0;
      for (int q = 0; q < wpt; ++q) acc += s_dot[2 * (uu * wpt + q) + which];
      const int slot = which == 0 ? t : (t < j ? j + 1 + t : 2 * j + 1);
      a.part[(size_t)slot * G + b] = acc;
    }
    __syncthreads();
  }
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) return;
  // 3. copy rows 1..j-1 of T (lower part, row i at offset i(i-1)/2) to shared memory while the
  //    totals are formed, one dot per block (in block order)
  const int ldt = a.ldh;
  double* Ts = ring;
  if (a.stage_T) {
    for (int i = warp + 1; i < j; i += nw)
      for (int k = lane; k < i; k += 32) cp_async8(Ts + i * (i - 1) / 2 + k, a.Tm + (size_t)i * ldt + k);
    cp_async_commit();
  }
  if (warp == 0)
    for (int t = b; t < nd; t += G) {
      double acc = 0.0;
      for (int k = lane; k < G; k += 32) acc += *((volatile double*)&a.part[(size_t)t * G + k]);
      acc = warp_sum(acc);
      if (lane == 0) a.tot[t] = acc;
    }
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) {
    cp_async_wait<0>();
    return;
  }
  // 4. MGS coefficients: h_i = a_i + sum_{k<i} T_ik a_k (i < j, ROW_TPR threads per row), then
  //    h_j = a_j - sum_k r_k h_k; the new row t_jk = -sum_{i=k}^{j-1} r_i T_ik of T is split over
  //    the blocks by column and read from the next step on.
  double* sa = sh;               // a[0..j]
  double* sr = sa + (j + 1);     // r[0..j-1]
  double* shh = sr + j;          // h[0..j]
  double* scs = shh + (j + 1);   // cs[0..j-1] (last block)
  double* ssn = scs + j;         // sn[0..j-1] (last block)
  for (int t = tid; t < nd - 1; t += nt) sa[t] = *((volatile double*)&a.tot[t]);
  const double wn2 = *((volatile double*)&a.tot[nd - 1]);
  if (b == G - 1)
    for (int k = tid; k < j; k += nt) {
      scs[k] = a.cs[k];
      ssn[k] = a.sn[k];
    }
  cp_async_wait<0>();
  __syncthreads();
  for (int rb = warp * (32 / ROW_TPR); rb < j; rb += nw * (32 / ROW_TPR)) {   // rb is warp-uniform
    const int i = rb + lane / ROW_TPR, q = lane % ROW_TPR;
    double acc = 0.0;
    if (i < j) {
      if (a.stage_T) {
        const double* row = Ts + i * (i - 1) / 2;
        for (int k = q; k < i; k += ROW_TPR) acc += row[k] * sa[k];
      } else {
        const double* row = a.Tm + (size_t)i * ldt;
        for (int k = q; k < i; k += ROW_TPR) acc += row[k] * sa[k];
      }
    }
#pragma unroll
    for (int o = ROW_TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (q == 0 && i < j) shh[i] = acc + sa[i];
  }
  for (int k = b + (warp - 1) * G; warp > 0 && k < j; k += (nw - 1) * G) {
    double acc = 0.0;
    for (int i = k + lane; i < j; i += 32) {
      const double tik = i == k ? 1.0 : (a.stage_T ? Ts[i * (i - 1) / 2 + k] : a.Tm[(size_t)i * ldt + k]);
      acc += sr[i] * tik;
    }
    acc = warp_sum(acc);
    if (lane == 0) a.Tm[(size_t)j * ldt + k] = -acc;
  }
  if (b == 0 && tid == 0) a.Tm[(size_t)j * ldt + j] = 1.0;
  __syncthreads();
  if (warp == 0) {
    double acc = 0.0;
    for (int k = lane; k < j; k += 32) acc += sr[k] * shh[k];
    acc = warp_sum(acc);
    if (lane == 0) shh[j] = sa[j] - acc;
  }
  __syncthreads();
  // previous rotations on column j: last block, warp 0, before its share of the update
  if (b == G - 1 && warp == 0) {
    const double x = givens_scan(scs, ssn, shh, a.H + (size_t)j * a.ldh, j, lane);
    if (lane == 0) s_x = x;
  }
  // 5. w -= V h on the slice, ||w||^2 (UPD_EL elements per thread; warp-uniform counts except
  //    in the one warp that holds the slice end)
  double nrm = 0.0;
  double keep[UPD_EL];
#pragma unroll
  for (int e = 0; e < UPD_EL; ++e) keep[e] = 0.0;
  const bool one_group = hi - lo <= (size_t)UPD_EL * nt;
  for (size_t base = lo + tid; base < hi; base += (size_t)UPD_EL * nt) {
    const size_t left = (hi - base + nt - 1) / nt;
    // the warp that holds the slice end runs the wide path on all its lanes (the missing elements
    // masked) instead of both paths one after the other
    const int nv = left >= (size_t)UPD_EL ? UPD_EL : (int)left;
    if (__any_sync(__activemask(), nv == UPD_EL))
      update_ring<UPD_EL>(a.V, n, j, shh, base, tid, ring, w, nrm, keep, nv);
    else
      update_ring<1>(a.V, n, j, shh, base, tid, ring, w, nrm, keep);
  }
  nrm = block_sum(nrm, sm);
  if (tid == 0) a.part[(size_t)nd * G + b] = nrm;
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) return;
  // 6. h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; last rotation of the column (last block)
  if (warp == 0) {
    double acc = 0.0;
    for (int k = lane; k < G; k += 32) acc += *((volatile double*)&a.part[(size_t)nd * G + k]);
    acc = warp_sum(acc);
    if (lane == 0) s_hn = sqrt(acc);
  }
  __syncthreads();
  const double hn = s_hn;
  if (b == G - 1 && tid == 0) {
    double* col = a.H + (size_t)j * a.ldh;
    const double x = s_x;
    double c, s, t;
    if (hn == 0.0) {
      c = 1.0;
      s = 0.0;
      t = x;
    } else {
      t = hypot(x, hn);
      c = x / t;
      s = hn / t;
    }
    a.cs[j] = c;
    a.sn[j] = s;
    col[j] = t;
    col[j + 1] = 0.0;
    const double gj = a.gv[j];
    a.gv[j + 1] = -s * gj;
    a.gv[j] = c * gj;
    a.out[0] = fabs(-s * gj);
    a.out[1] = hn;
    a.out[2] = sqrt(wn2);
    a.out[3] = 0.0;
  }
  const double rh = hn != 0.0 ? 1.0 / hn : 0.0;
  double* vn = a.V + (size_t)(j + 1) * n;
  if (one_group) {
#pragma unroll
    for (int e = 0; e < UPD_EL; ++e) {
      const size_t c = lo + tid + (size_t)e * nt;
      if (c < hi) vn[c] = keep[e] * rh;
    }
  } else {
    for (size_t c = lo + tid; c < hi; c += nt) vn[c] = w[c] * rh;
  }
}

// Returns cudaErrorNotSupported when one co-resident wave cannot cover the grid.
cudaError_t launch_arnoldi(const Geo& g, const double* z, double* V, int j, size_t n, double* H, int ldh, double* cs,
                           double* sn, double* gv, double* out, double* wbuf, double* part, double* tot, double* Tm,
                           unsigned* bar, int* flags, cudaStream_t st) {
  struct Occ {
    int sms = 0, per_sm = 0;
  };
  static const Occ occ = [] {  // thread-safe one-time initialisation (request workers call this)
    Occ o;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    raise_smem_limit<k_arnoldi_ls>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, k_arnoldi_ls, ARN_THREADS, ARN_SMEM_MAX);
    return o;
  }();
  const int sms = occ.sms, per_sm = occ.per_sm;
  int grid = (int)std::min<size_t>((size_t)sms, (n + ARN_THREADS - 1) / ARN_THREADS);
  if (grid < 1) grid = 1;
  if (grid > ARNOLDI_MAX_BLOCKS || per_sm < 1 || ldh > 257) return cudaErrorNotSupported;
  const size_t tri = (size_t)j * (j > 0 ? j - 1 : 0) / 2;
  const int stage_T = 8 * (ARN_SMALL + std::max<size_t>(ARN_RING, tri)) <= (size_t)ARN_SMEM_MAX ? 1 : 0;
  const size_t smem = 8 * (ARN_SMALL + (stage_T ? std::max<size_t>(ARN_RING, tri) : (size_t)ARN_RING));
  LsArgs a{z, V, j, n, H, ldh, cs, sn, gv, out, wbuf, part, tot, Tm, bar, flags, stage_T};
  void* args[] = {(void*)&g, (void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_arnoldi_ls, dim3(grid), dim3(ARN_THREADS), args, smem, st);
  if (e == cudaSuccess) count_launch(1);
  return e;
}

static int red_grid(size_t n) {
  const size_t want = (n + RED_THREADS - 1) / RED_THREADS;
  return (int)(want < (size_t)RED_BLOCKS ? (want > 0 ? want : 1) : RED_BLOCKS);
}

cudaError_t launch_norm2(const double* x, size_t n, double* partials, unsigned* counter, double* out, cudaStream_t st) {
  k_norm2<<<red_grid(n), RED_THREADS, 0, st>>>(x, n, partials, counter, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* x, const double* denom, size_t n, double* y, cudaStream_t st) {
  k_scale<<<red_grid(n), RED_THREADS, 0, st>>>(x, denom, n, y);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_matvec_dot(const Geo& g, const double* z, const double* v0, double* w, double* partials,
                              unsigned* counter, double* out2, cudaStream_t st) {
  k_matvec_dot<<<red_grid((size_t)g.nx * g.ny), RED_THREADS, 0, st>>>(g, z, v0, w, partials, counter, out2,
                                                                      out2 + 1);
  return cudaGetLastError();
}

cudaError_t launch_mgs_pass(const double* vprev, const double* hprev, const double* vnext, size_t n, double* w,
                            double* partials, unsigned* counter, double* hout, int, cudaStream_t st) {
  k_mgs_pass<<<red_grid(n), RED_THREADS, 0, st>>>(vprev, hprev, vnext, n, w, partials, counter, hout);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_givens(double* H, double* cs, double* sn, double* gv, int j, int ldh, double* wnorm2, double* out,
                          cudaStream_t st) {
  k_givens<<<1, 32, 0, st>>>(H, cs, sn, gv, j, ldh, wnorm2, out);
  count_launch(1);
  return cudaGetLastError();
}

// y = R^-1 g (R = leading k x k of the rotated H, column-major) by column-oriented back
// substitution in one CTA: y_i = g_i / R_ii, then g_t -= R_ti y_i for t < i.  Stores -y, the form
// the update sweep below subtracts.
__global__ void __launch_bounds__(256) k_backsub(const double* __restrict__ H, const double* __restrict__ gv, int k,
                                                 int ldh, double* __restrict__ yneg) {
  __shared__ double g[260];
  __shared__ double s_y;
  for (int t = threadIdx.x; t < k; t += blockDim.x) g[t] = gv[t];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      s_y = g[i] / H[(size_t)i * ldh + i];
      yneg[i] = -s_y;
    }
    __syncthreads();
    const double yi = s_y;
    for (int t = threadIdx.x; t < i; t += blockDim.x) g[t] -= H[(size_t)i * ldh + t] * yi;
    __syncthreads();
  }
}

// p += Z y over the k stored preconditioned vectors: the Arnoldi update sweep (cp.async ring,
// each element summed in order t = 0 .. k-1) with h = -y.
__global__ void __launch_bounds__(ARN_THREADS, 1) k_update_p(double* __restrict__ p, const double* __restrict__ Z,
                                                            size_t n, const double* __restrict__ yneg, int k) {
  extern __shared__ double sh[];   // -y | ring
  constexpr int nt = ARN_THREADS;
  for (int t = threadIdx.x; t < k; t += nt) sh[t] = yneg[t];
  __syncthreads();
  double* ring = sh + ARN_SMALL;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const size_t chunk = (n + G - 1) / G;
  const size_t lo = (size_t)b * chunk < n ? (size_t)b * chunk : n;
  const size_t hi = lo + chunk < n ? lo + chunk : n;
  double nrm = 0.0;
  double keep[UPD_EL];
  for (size_t base = lo + tid; base < hi; base += (size_t)UPD_EL * nt) {
    const size_t left = (hi - base + nt - 1) / nt;
    if (left >= (size_t)UPD_EL)
      update_ring<UPD_EL>(Z, n, k - 1, sh, base, tid, ring, p, nrm, keep);
    else
      update_ring<1>(Z, n, k - 1, sh, base, tid, ring, p, nrm, keep);
  }
}

cudaError_t launch_update(double* p, const double* Z, size_t n, const double* H, const double* gv, int k, int ldh,
                          double* ybuf, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  if (k > ARN_SMALL || k > 256) {
    k_update<<<red_grid(n), RED_THREADS, sizeof(double) * k, st>>>(p, Z, n, H, gv, k, ldh);
    count_launch(1);
    return cudaGetLastError();
  }
  k_backsub<<<1, 256, 0, st>>>(H, gv, k, ldh, ybuf);
  count_launch(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = raise_smem_limit<k_update_p>();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = (int)std::min<size_t>((size_t)sms, (n + ARN_THREADS - 1) / ARN_THREADS);
  if (grid < 1) grid = 1;
  k_update_p<<<grid, ARN_THREADS, sizeof(double) * (ARN_SMALL + ARN_RING), st>>>(p, Z, n, ybuf, k);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm(const Geo& g, const double* b, const double* p, double* r, double* partials,
                                 unsigned* counter, double* out, cudaStream_t st) {
  k_residual_norm<<<red_grid((size_t)g.nx * g.ny), RED_THREADS, 0, st>>>(g, b, p, r, partials, counter, out);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace mrcm
