// Launch-shape autotuning for kernels whose variants compute identical results and differ only in
// how they stage data (the local solves' line-block ring depth, the coupling factorisation's
// cluster size).  The first launch of a shape in the process times every variant on the caller's
// own data and stream and keeps the fastest; a process-wide table, guarded by a mutex, serves later
// launches of that shape, from any thread.
#include <array>
#include <map>
#include <mutex>

#include <cuda_runtime_api.h>

#include "internal.h"

namespace mrcm {
namespace {

using Key = std::pair<int, std::array<int, 6>>;

struct Slot {
  bool pending = true;  // being timed by one thread; the others keep the built-in choice meanwhile
  int choice = -1, ncand = 0;
  float best_us = 0.0f;
};

std::mutex g_mu;
std::map<Key, Slot> g_table;
bool g_enabled = true;

}  // namespace

void autotune_mode(int mode) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (mode == 2) {
    for (auto it = g_table.begin(); it != g_table.end();) it = it->second.pending ? std::next(it) : g_table.erase(it);
  }
  g_enabled = mode != 0;
}

std::vector<double> autotune_table() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<double> out;
  for (const auto& kv : g_table) {
    if (kv.second.pending) continue;
    out.push_back(kv.first.first);
    for (int v : kv.first.second) out.push_back(v);
    out.push_back(kv.second.choice);
    out.push_back(kv.second.ncand);
    out.push_back(kv.second.best_us);
  }
  return out;
}

int autotune(int kind, const int key[6], int ncand, cudaStream_t st, const std::function<cudaError_t(int)>& run,
             cudaError_t* err) {
  *err = cudaSuccess;
  if (ncand < 2) return -1;
  Key k{kind, {key[0], key[1], key[2], key[3], key[4], key[5]}};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_enabled) return -1;
    auto it = g_table.find(k);
    if (it != g_table.end()) return it->second.pending ? -1 : it->second.choice;
    g_table.emplace(k, Slot{});
  }
  // a stream under capture cannot be timed: leave the shape untuned
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.erase(k);
    return -1;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best = -1;
  float best_ms = 0.0f;
  for (int c = 0; c < ncand && e == cudaSuccess; ++c) {
    float cand_ms = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // one warm launch, then the best of two
      if (rep > 0) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = run(c);
      if (rep == 0 || e != cudaSuccess) continue;
      if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (rep == 1 || ms < cand_ms) cand_ms = ms;
    }
    if (e == cudaSuccess && (best < 0 || cand_ms < best_ms)) {
      best = c;
      best_ms = cand_ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_mu);
  if (e != cudaSuccess || best < 0) {
    g_table.erase(k);
    *err = e;
    return -1;
  }
  Slot& s = g_table[k];
  s.pending = false;
  s.choice = best;
  s.ncand = ncand;
  s.best_us = 1e3f * best_ms;
  return best;
}

}  // namespace mrcm
