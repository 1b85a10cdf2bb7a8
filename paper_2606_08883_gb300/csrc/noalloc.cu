// mrcm_residual_norm_noalloc: the true-residual norm ||b - A p||_2 of the GMRES stopping test,
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where device allocation is not allowed or not possible -- in a
// real-time loop that must not touch the allocator, or in a host process that only receives device
// pointers from another component and owns no allocator of its own.  mrcm_gmres_solve computes the same quantity with reduction scratch carved
// from the handle's workspace; this entry point keeps its scratch in a fixed device array that is
// part of the library image instead, so a call allocates nothing.
//
// The scratch array below lives on every GPU that loads the library until the process exits.  Host
// code must not pass the array's name to a kernel (on the host it is only a stand-in); the device
// address is looked up once per device with cudaGetSymbolAddress.
#include <cstdint>
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t NOALLOC_MAX_CELLS = 1u << 20;                 // residual vector capacity
constexpr size_t NOALLOC_PARTIALS = mrcm::RED_BLOCKS;           // one partial sum per block
constexpr size_t NOALLOC_DOUBLES = NOALLOC_MAX_CELLS + NOALLOC_PARTIALS + 32;   // + ticket counter

// residual r = b - A p (cells), then per-block partial sums, then the completion ticket
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {nullptr};

// Same arithmetic, grid and reduction order as the residual-norm kernel of the GMRES path, so the
// two agree bit for bit.
__global__ void __launch_bounds__(mrcm::RED_THREADS) k_residual_norm_static(mrcm::Geo g, const double* __restrict__ b,
                                                                            const double* __restrict__ p,
                                                                            double* scratch, double* out) {
  __shared__ double sm[32];
  double* r = scratch;
  double* partials = scratch + NOALLOC_MAX_CELLS;
  unsigned* counter = reinterpret_cast<unsigned*>(partials + NOALLOC_PARTIALS);
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
  mrcm::grid_reduce<1>(v, partials, counter, outs, sm, 1);
}

}  // namespace

extern "C" mrcm_status mrcm_residual_norm_noalloc(mrcm_handle h, const double* b, const double* p, double* norm_out,
                                                  void* stream) {
  if (!h || !b || !p || !norm_out) return MRCM_ERR_INVALID_ARG;
  if (!h->factored) {
    h->err = "mrcm_factor_local has not completed";
    return MRCM_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)h->n[0] * h->n[1] * h->n[2];
  if (n > NOALLOC_MAX_CELLS) {
    h->err = "mrcm_residual_norm_noalloc supports at most " + std::to_string(NOALLOC_MAX_CELLS) +
             " cells; this grid has " + std::to_string(n);
    return MRCM_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    h->err = std::string("mrcm_residual_norm_noalloc: no usable current device: ") + cudaGetErrorString(e);
    return MRCM_ERR_CUDA;
  }
  if (dev != h->device) {
    // the scratch copy is picked by the current device, the transmissibilities come from the
    // handle's workspace: both must be on the same GPU
    h->err = "mrcm_residual_norm_noalloc: the current device (" + std::to_string(dev) +
             ") is not the one the handle was set up on (" + std::to_string(h->device) + ")";
    return MRCM_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // one-time set-up per device, with that device current
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_addr[dev]), g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        h->err = std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e);
        return MRCM_ERR_CUDA;
      }
    }
    scratch = g_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the completion ticket must start at zero (the array keeps the previous call's contents)
  e = cudaMemsetAsync(scratch + NOALLOC_MAX_CELLS + NOALLOC_PARTIALS, 0, 32 * sizeof(double), st);
  if (e != cudaSuccess) {
    h->err = std::string("mrcm_residual_norm_noalloc: ") + cudaGetErrorString(e);
    return MRCM_ERR_CUDA;
  }
  mrcm::Geo g;
  const mrcm::Plan& P = h->plan;
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
  g.K = reinterpret_cast<const double*>(h->ws + h->lay.K);
  g.Ky = reinterpret_cast<const double*>(h->ws + h->lay.Ky);
  g.Tx = reinterpret_cast<const double*>(h->ws + h->lay.Tx);
  g.Ty = reinterpret_cast<const double*>(h->ws + h->lay.Ty);
  const size_t want = (n + mrcm::RED_THREADS - 1) / mrcm::RED_THREADS;
  const int grid = (int)(want < (size_t)mrcm::RED_BLOCKS ? (want > 0 ? want : 1) : mrcm::RED_BLOCKS);
  k_residual_norm_static<<<grid, mrcm::RED_THREADS, 0, st>>>(g, b, p, scratch, norm_out);
  mrcm::count_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("mrcm_residual_norm_noalloc: ") + cudaGetErrorString(e);
    return MRCM_ERR_CUDA;
  }
  return MRCM_OK;
}
