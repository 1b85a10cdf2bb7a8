// Device helpers shared by the libmrcm kernels.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace mrcm {

// Raises kernel K's dynamic shared-memory limit to the device maximum, once per kernel and
// process (thread-safe).  Launches then pass their own size: the limit only gates launches and
// does not change occupancy, and a limit that never moves cannot be lowered by another thread
// between its own set and launch (request workers launch the same kernels with different sizes).
template <auto K>
cudaError_t raise_smem_limit() {
  static const cudaError_t err = [] {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, K);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
  }();
  return err;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a block (blockDim.x multiple of 32, <= 1024).  Every thread receives the total.
// Deterministic: fixed order for a fixed block size.
__device__ __forceinline__ double block_sum(double v, double* smem32) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem32[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = lane < nw ? smem32[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// Grid-wide deterministic reduction of NV values per thread.  Each block writes its partial sums
// to partials[v * gridDim.x + blockIdx.x]; the last block to finish (atomic ticket) adds the
// partials in block order and writes *outs[v] (the square root for entries with the sqrt bit set
// in sqrt_mask); the ticket counter is reset for the next launch.
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], double* partials, unsigned* counter,
                                            double* const (&outs)[NV], double* smem32, int sqrt_mask = 0) {
  __shared__ bool last;
  for (int k = 0; k < NV; ++k) {
    double t = block_sum(v[k], smem32);
    if (threadIdx.x == 0) partials[k * gridDim.x + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ticket = atomicAdd(counter, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += *((volatile double*)&partials[k * gridDim.x + b]);
    double t = block_sum(acc, smem32);
    if (threadIdx.x == 0) *outs[k] = ((sqrt_mask >> k) & 1) ? sqrt(t) : t;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Two-point-flux pieces (Sec. 3): half transmissibility tau = 2 K |f| / h_a.
__device__ __forceinline__ double half_trans(double k, double area, double ha) { return 2.0 * k * area / ha; }

// Robin face coefficient t_R = (1/tau_in + beta/|f|)^-1, beta = alpha H / K_H (Eq. 5-6).
__device__ __forceinline__ double robin_tr(double k_in, double k_out, double area, double ha, double Hs,
                                           double alpha, double* beta_out, double* tau_out) {
  const double tau = half_trans(k_in, area, ha);
  const double kh = 2.0 * k_in * k_out / (k_in + k_out);
  const double beta = alpha * Hs / kh;
  if (beta_out) *beta_out = beta;
  if (tau_out) *tau_out = tau;
  return 1.0 / (1.0 / tau + beta / area);
}

// Grid-wide barrier for cooperative launches (every block co-resident).  bar[0] counts arrivals
// (zero between barriers), bar[1] is the generation.  A block that polls more than
// BARRIER_SPIN_LIMIT times sets FLAG_TIMEOUT in *flags and returns false instead of waiting on.
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
          atomicOr(flags, FLAG_TIMEOUT);
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

}  // namespace mrcm
