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
constexpr long long BARRIER_SPIN_LIMIT = 1LL << 24;   // ~1-2 s of polling, then give up

// Returns false if the wait gave up (the flag is set; the caller returns).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned my = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    s_ok = 1;
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == my) {
        if (++spins > BARRIER_SPIN_LIMIT) {
          atomicOr(flags, 8);
          s_ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// One Arnoldi step (inner step j) in a single cooperative launch, with the modified
// Gram-Schmidt coefficients obtained from one global reduction.  MGS computes
//   h_i = (w - sum_{k<i} h_k v_k, v_i) = a_i - sum_{k<i} (v_k, v_i) h_k,   a_i = (w, v_i),
// i.e. (I + R) h = a with R the strictly lower Gram matrix of the basis.  T = (I + R)^-1 is kept in
// its compact inverse form and grows by one row per step (t_j = -r^T T_{j-1}, r_k = (v_k, v_j)),
// so h = T a is a product instead of a sequential solve.  Per step: one sweep over the basis for
// the j+1 coefficients a, the j new Gram entries r and ||A z||^2; one sweep for w -= V h and
// ||w||^2; three grid barriers.  Each block owns one contiguous slice of the vectors; dot products
// are computed one warp per dot over the slice (lanes stride the elements), then reduced across
// blocks in block order (deterministic).
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
  double* part;         // (2 ldh + 2) x gridDim partial sums
  double* tot;          // 2 ldh + 2 totals
  double* Tm;           // (I + R)^-1, row-major lower, leading dimension ldh
  unsigned* bar;
  int* flags;
};

__global__ void __launch_bounds__(512) k_arnoldi_ls(Geo g, LsArgs a) {
  extern __shared__ double sh[];      // a[j+1] | r[j] | tj[j] | h[j+1] | misc
  __shared__ double sm[32];
  __shared__ double s_hn;
  const int j = a.j, G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const size_t n = a.n;
  const size_t chunk = (n + G - 1) / G;
  const size_t lo = (size_t)b * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double* w = a.wbuf;
  const double* vj = a.V + (size_t)j * n;
  // 1. w = A z_j on the slice
  for (size_t c = lo + tid; c < hi; c += nt) {
    const int i = (int)(c % g.nx), jj = (int)(c / g.nx);
    const double* z = a.z;
    const double zc = z[c];
    const double zw = i > 0 ? z[c - 1] : 0.0;
    const double ze = i < g.nx - 1 ? z[c + 1] : 0.0;
    const double zs = jj > 0 ? z[c - g.nx] : 0.0;
    const double zn = jj < g.ny - 1 ? z[c + g.nx] : 0.0;
    const double* Tx = g.Tx + (size_t)jj * (g.nx + 1) + i;
    const double* Ty = g.Ty + (size_t)jj * g.nx + i;
    const double wx = Tx[1] * (zc - ze) - Tx[0] * (zw - zc);
    const double wy = Ty[g.nx] * (zc - zn) - Ty[0] * (zs - zc);
    w[c] = wx + wy;
  }
  __syncthreads();
  // 2. block partials of a_t = (w, v_t) (t <= j), r_k = (v_j, v_k) (k < j), ||w||^2 -- one warp per dot
  const int nd = 2 * j + 2;
  for (int t = warp; t < nd; t += nw) {
    double acc = 0.0;
    if (t <= j) {
      const double* vt = a.V + (size_t)t * n;
      for (size_t c = lo + lane; c < hi; c += 32) acc += w[c] * vt[c];
    } else if (t <= 2 * j) {
      const double* vk = a.V + (size_t)(t - j - 1) * n;
      for (size_t c = lo + lane; c < hi; c += 32) acc += vj[c] * vk[c];
    } else {
      for (size_t c = lo + lane; c < hi; c += 32) acc += w[c] * w[c];
    }
    acc = warp_sum(acc);
    if (lane == 0) a.part[(size_t)t * G + b] = acc;
  }
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) return;
  // 3. totals, one dot per block (in block order)
  if (warp == 0)
    for (int t = b; t < nd; t += G) {
      double acc = 0.0;
      for (int k = lane; k < G; k += 32) acc += *((volatile double*)&a.part[(size_t)t * G + k]);
      acc = warp_sum(acc);
      if (lane == 0) a.tot[t] = acc;
    }
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) return;
  // 4. MGS coefficients h = T_j a, with the new row t_j = -r^T T_{j-1}
  double* sa = sh;               // a[0..j]
  double* sr = sa + (j + 1);     // r[0..j-1]
  double* st = sr + j;           // t_j[0..j-1]
  double* shh = st + j;          // h[0..j]
  for (int t = tid; t < nd - 1; t += nt) sh[t] = *((volatile double*)&a.tot[t]);
  const double wn2 = *((volatile double*)&a.tot[nd - 1]);
  __syncthreads();
  const int ldt = a.ldh;
  for (int k = tid; k < j; k += nt) {
    double acc = 0.0;
    for (int i = k; i < j; ++i) acc += sr[i] * a.Tm[(size_t)i * ldt + k];
    st[k] = -acc;
  }
  __syncthreads();
  for (int i = tid; i <= j; i += nt) {
    double acc = 0.0;
    if (i < j) {
      const double* row = a.Tm + (size_t)i * ldt;
      for (int k = 0; k < i; ++k) acc += row[k] * sa[k];
    } else {
      for (int k = 0; k < j; ++k) acc += st[k] * sa[k];
    }
    shh[i] = acc + sa[i];
  }
  __syncthreads();
  if (b == 0) {
    for (int k = tid; k < j; k += nt) a.Tm[(size_t)j * ldt + k] = st[k];
    if (tid == 0) a.Tm[(size_t)j * ldt + j] = 1.0;
  }
  // 5. w -= V h on the slice, ||w||^2
  double nrm = 0.0;
  for (size_t c = lo + tid; c < hi; c += nt) {
    double acc0 = w[c], acc1 = 0.0;
    int i = 0;
    for (; i + 1 <= j; i += 2) {
      acc0 -= shh[i] * a.V[(size_t)i * n + c];
      acc1 -= shh[i + 1] * a.V[(size_t)(i + 1) * n + c];
    }
    if (i <= j) acc0 -= shh[i] * a.V[(size_t)i * n + c];
    const double wc = acc0 + acc1;
    w[c] = wc;
    nrm += wc * wc;
  }
  nrm = block_sum(nrm, sm);
  if (tid == 0) a.part[(size_t)nd * G + b] = nrm;
  __threadfence();
  if (!grid_barrier(a.bar, a.flags)) return;
  // 6. h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; Hessenberg column and Givens update (block 0)
  if (warp == 0) {
    double acc = 0.0;
    for (int k = lane; k < G; k += 32) acc += *((volatile double*)&a.part[(size_t)nd * G + k]);
    acc = warp_sum(acc);
    if (lane == 0) s_hn = sqrt(acc);
  }
  __syncthreads();
  const double hn = s_hn;
  double* vn = a.V + (size_t)(j + 1) * n;
  for (size_t c = lo + tid; c < hi; c += nt) vn[c] = hn != 0.0 ? w[c] / hn : 0.0;
  if (b == 0 && tid == 0) {
    double* col = a.H + (size_t)j * a.ldh;
    for (int i = 0; i <= j; ++i) col[i] = shh[i];
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t0 = a.cs[i] * col[i] + a.sn[i] * col[i + 1];
      const double t1 = -a.sn[i] * col[i] + a.cs[i] * col[i + 1];
      col[i] = t0;
      col[i + 1] = t1;
    }
    const double x = col[j], y = col[j + 1];
    double c, s, t;
    if (y == 0.0) {
      c = 1.0;
      s = 0.0;
      t = x;
    } else {
      t = hypot(x, y);
      c = x / t;
      s = y / t;
    }
    a.cs[j] = c;
    a.sn[j] = s;
    col[j] = t;
    col[j + 1] = 0.0;
    a.gv[j + 1] = -s * a.gv[j];
    a.gv[j] = c * a.gv[j];
    a.out[0] = fabs(a.gv[j + 1]);
    a.out[1] = hn;
    a.out[2] = sqrt(wn2);
    a.out[3] = 0.0;
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
    cudaFuncSetAttribute(k_arnoldi_ls, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 4 * 260);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, k_arnoldi_ls, 512, 8 * 4 * 260);
    return o;
  }();
  const int sms = occ.sms, per_sm = occ.per_sm;
  int grid = (int)std::min<size_t>((size_t)sms, (n + 511) / 512);
  if (grid < 1) grid = 1;
  if (grid > ARNOLDI_MAX_BLOCKS || per_sm < 1 || ldh > 257) return cudaErrorNotSupported;
  LsArgs a{z, V, j, n, H, ldh, cs, sn, gv, out, wbuf, part, tot, Tm, bar, flags};
  void* args[] = {(void*)&g, (void*)&a};
  const size_t smem = sizeof(double) * (4 * (size_t)(j + 1) + 8);
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_arnoldi_ls, dim3(grid), dim3(512), args, smem, st);
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

cudaError_t launch_update(double* p, const double* Z, size_t n, const double* H, const double* gv, int k, int ldh,
                          cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  k_update<<<red_grid(n), RED_THREADS, sizeof(double) * k, st>>>(p, Z, n, H, gv, k, ldh);
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
