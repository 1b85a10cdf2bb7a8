// Krylov kernels for Algorithm 1 (restarted right-preconditioned GMRES storing Z), FP64.
//
// Inner step j: w = A z_j fused with h_{0,j} = (w, v_0) and ||w||^2; modified Gram-Schmidt passes
// i = 1..j fused as "w -= h_{i-1,j} v_{i-1}, then h_{i,j} = (w, v_i)"; a last pass subtracts
// h_{j,j} v_j and returns h_{j+1,j} = ||w||.  The Givens rotation update of the Hessenberg column
// runs in one thread.  Reductions are deterministic: fixed grid, per-block partials, last block
// sums them in block order.
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
// Fused Arnoldi step (cooperative launch, all blocks co-resident).  Each thread keeps R elements of
// w in registers for the whole step, so the modified Gram-Schmidt passes read only v_i from memory;
// between passes a grid barrier publishes the per-block partial sums, which every block then adds
// in the same (block) order, so all blocks hold bit-identical h_{i,j}.
// ============================================================================================
constexpr long long BARRIER_SPIN_LIMIT = 1LL << 24;   // ~1-2 s of polling, then give up

struct ArnoldiArgs {
  const double* z;      // z_j
  double* V;            // basis, V_i at V + i n
  int j;
  size_t n;
  double* H;            // Hessenberg, column-major, leading dimension ldh
  int ldh;
  double* cs;
  double* sn;
  double* gv;
  double* out;          // [0] |g_{j+1}|, [1] h_{j+1,j}, [2] ||A z_j||, [3] 1 if a barrier timed out
  double* partials;     // 2 buffers x 2 values x gridDim
  unsigned* bar;        // [0] arrivals, [1] generation
  int* flags;
};

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

// Sum of v0 (and v1) over the grid; every block receives the same totals.
template <int NV>
__device__ __forceinline__ bool grid_allreduce(double (&v)[NV], double* partials, int pass, unsigned* bar, int* flags,
                                               double* smem32) {
  const int G = gridDim.x;
  double* buf = partials + (size_t)(pass & 1) * 2 * G;
  for (int k = 0; k < NV; ++k) {
    const double t = block_sum(v[k], smem32);
    if (threadIdx.x == 0) buf[k * G + blockIdx.x] = t;
  }
  __threadfence();
  if (!grid_barrier(bar, flags)) return false;
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) acc += *((volatile double*)&buf[k * G + b]);
    v[k] = block_sum(acc, smem32);
  }
  return true;
}

template <int R>
__global__ void __launch_bounds__(512) k_arnoldi(Geo g, ArnoldiArgs a) {
  __shared__ double sm[32];
  const size_t n = a.n;
  const size_t base = (size_t)blockIdx.x * R * blockDim.x + threadIdx.x;
  const int j = a.j;
  double w[R];
  double red2[2] = {0.0, 0.0};
  // w = A z_j ; (w, v_0) ; (w, w)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const size_t c = base + (size_t)r * blockDim.x;
    w[r] = 0.0;
    if (c < n) {
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
      w[r] = wx + wy;
      red2[0] += w[r] * a.V[c];
      red2[1] += w[r] * w[r];
    }
  }
  int pass = 0;
  if (!grid_allreduce<2>(red2, a.partials, pass++, a.bar, a.flags, sm)) return;
  double hprev = red2[0];
  const double wn2 = red2[1];
  double* col = a.H + (size_t)j * a.ldh;
  if (blockIdx.x == 0 && threadIdx.x == 0) col[0] = hprev;
  // modified Gram-Schmidt passes i = 1..j
  for (int i = 1; i <= j; ++i) {
    const double* vp = a.V + (size_t)(i - 1) * n;
    const double* vi = a.V + (size_t)i * n;
    double red1[1] = {0.0};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t c = base + (size_t)r * blockDim.x;
      if (c < n) {
        w[r] -= hprev * vp[c];
        red1[0] += w[r] * vi[c];
      }
    }
    if (!grid_allreduce<1>(red1, a.partials, pass++, a.bar, a.flags, sm)) return;
    hprev = red1[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) col[i] = hprev;
  }
  // last pass: w -= h_{j,j} v_j, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
  {
    const double* vp = a.V + (size_t)j * n;
    double red1[1] = {0.0};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t c = base + (size_t)r * blockDim.x;
      if (c < n) {
        w[r] -= hprev * vp[c];
        red1[0] += w[r] * w[r];
      }
    }
    if (!grid_allreduce<1>(red1, a.partials, pass++, a.bar, a.flags, sm)) return;
    const double hn = sqrt(red1[0]);
    double* vn = a.V + (size_t)(j + 1) * n;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const size_t c = base + (size_t)r * blockDim.x;
      if (c < n) vn[c] = hn != 0.0 ? w[r] / hn : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      col[j + 1] = hn;
      // Givens update of column j
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
}

template <int R>
static cudaError_t arnoldi_launch(const Geo& g, const ArnoldiArgs& a, int grid, cudaStream_t st) {
  void* args[] = {(void*)&g, (void*)&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_arnoldi<R>, dim3(grid), dim3(512), args, 0, st);
  if (e == cudaSuccess) count_launch(1);
  return e;
}

template <int R>
static int arnoldi_max_blocks() {
  static int cached = -1;
  if (cached < 0) {
    int dev = 0, per_sm = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<R>, 512, 0);
    cached = per_sm * sms;
  }
  return cached;
}

// Returns cudaErrorNotSupported when the vector is too long for one co-resident wave.
cudaError_t launch_arnoldi(const Geo& g, const double* z, double* V, int j, size_t n, double* H, int ldh, double* cs,
                           double* sn, double* gv, double* out, double* partials, unsigned* bar, int* flags,
                           cudaStream_t st) {
  ArnoldiArgs a{z, V, j, n, H, ldh, cs, sn, gv, out, partials, bar, flags};
  const size_t per = 512;
  // about one block per SM: a grid barrier costs roughly in proportion to the arriving blocks,
  // while one block per SM still streams each basis vector at full bandwidth
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
#define MRCM_TRY_R(R_)                                                              \
  {                                                                                 \
    const int mb = arnoldi_max_blocks<R_>();                                        \
    const size_t need = (n + per * R_ - 1) / (per * R_);                            \
    if ((need <= (size_t)sms || R_ == 16) && need <= (size_t)mb &&                  \
        need <= (size_t)ARNOLDI_MAX_BLOCKS)                                         \
      return arnoldi_launch<R_>(g, a, (int)need, st);                               \
  }
  MRCM_TRY_R(1)
  MRCM_TRY_R(2)
  MRCM_TRY_R(4)
  MRCM_TRY_R(8)
  MRCM_TRY_R(16)
#undef MRCM_TRY_R
  return cudaErrorNotSupported;
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
