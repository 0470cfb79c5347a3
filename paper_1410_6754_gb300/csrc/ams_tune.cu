// Autotuner: picks levels, groups per level and overpartitioning for a size class.
//
// For (key type, pairs, ceil(log2 n)) it times a small set of candidate plans on n
// synthetic uniform keys (SplitMix64, generated on the device) in the given
// context's scratch, and keeps the fastest in a process-wide table.  Candidates:
// 1, 2 or 3 distribution levels; groups per level r = the power of two nearest to
// (n / t)^(1/levels) for target leaf sizes t = C/2 and C/4 (C the base-case
// capacity), within the limits of b * r (b = 1 for one level, 4 otherwise).
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "ams.h"

namespace {

__global__ void k_fill(void* keys, uint64_t* vals, uint64_t n, int ksize, uint64_t seed) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if (ksize == 8) {
      ((uint64_t*)keys)[i] = z;
    } else {
      ((uint32_t*)keys)[i] = (uint32_t)(z >> 32);
    }
    if (vals) vals[i] = i;
  }
}

struct Cand {
  int levels;
  uint32_t r[8];
  uint32_t b;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int>, ams_tuned> g_table;

uint32_t pow2_near(double x, uint32_t lo, uint32_t hi) {
  const double l = std::round(std::log2(std::max(x, 1.0)));
  double v = std::pow(2.0, l);
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return (uint32_t)v;
}

}  // namespace

extern "C" {

AMS_API ams_status ams_tune(void* ctx, uint64_t n, ams_key_type kt, int pairs, void* stream, ams_tuned* out) {
  if (!out || n == 0 || n >= (1ull << 32)) return AMS_ERR_INVALID;
  if (kt != AMS_U32 && kt != AMS_U64 && kt != AMS_F32) return AMS_ERR_INVALID;
  int lg = 0;
  while ((1ull << lg) < n) ++lg;
  const auto key = std::make_tuple((int)kt, pairs ? 1 : 0, lg);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) {
      *out = it->second;
      return AMS_OK;
    }
  }
  const uint32_t C = ams_default_basecase_cap(kt, pairs);
  std::vector<Cand> cands;
  if (n <= C) {
    Cand c{1, {2}, 1};  // no distribution level is launched for n <= C
    cands.push_back(c);
  } else {
    for (int L = 1; L <= 3; ++L) {
      const uint32_t b = L == 1 ? 1 : 4;
      for (uint32_t t : {C / 2, C / 4}) {
        const double fan = std::pow((double)n / t, 1.0 / L);
        Cand c{L, {}, b};
        const uint32_t r = pow2_near(fan, 2, 2048 / b);
        for (int l = 0; l < L; ++l) c.r[l] = r;
        bool dup = false;
        for (const Cand& o : cands) dup |= o.levels == c.levels && o.r[0] == c.r[0] && o.b == c.b;
        if (!dup) cands.push_back(c);
      }
    }
  }
  const size_t w = kt == AMS_U64 ? 8 : 4;
  void *keys = nullptr, *tmp = nullptr;
  uint64_t *vals = nullptr, *vtmp = nullptr;
  const cudaStream_t s = (cudaStream_t)stream;
  ams_status st = AMS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&keys, n * w) != cudaSuccess || cudaMalloc(&tmp, n * w) != cudaSuccess ||
      (pairs && (cudaMalloc(&vals, n * 8) != cudaSuccess || cudaMalloc(&vtmp, n * 8) != cudaSuccess))) {
    st = AMS_ERR_OOM;
  } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = AMS_ERR_CUDA;
  }
  ams_tuned best{};
  best.ms = -1.f;
  if (st == AMS_OK) {
    k_fill<<<1024, 256, 0, s>>>(keys, vals, n, (int)w, 0x5EEDull + (uint64_t)lg);
    if (cudaGetLastError() != cudaSuccess) st = AMS_ERR_CUDA;
  }
  for (const Cand& c : cands) {
    if (st != AMS_OK) break;
    ams_request rq{};
    rq.keys_in = keys;
    rq.keys_out = tmp;
    rq.vals_in = vals;
    rq.vals_out = pairs ? vtmp : nullptr;
    rq.nseg = 1;
    rq.n = n;
    rq.kt = kt;
    rq.levels = c.levels;
    rq.buckets_per_level = c.r;
    rq.opt.overpartition_b = c.b;
    float ms = 1e30f;
    for (int rep = 0; rep < 4 && st == AMS_OK; ++rep) {  // first one warms up
      cudaEventRecord(e0, s);
      st = ams_sort_request(ctx, &rq, s);
      cudaEventRecord(e1, s);
      if (st == AMS_OK && (st = ams_context_sync(ctx)) == AMS_OK) {
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
          st = AMS_ERR_CUDA;
        } else if (rep > 0) {
          ms = std::min(ms, t);
        }
      }
    }
    if (st == AMS_OK && (best.ms < 0.f || ms < best.ms)) {
      best.levels = c.levels;
      for (int l = 0; l < 8; ++l) best.buckets_per_level[l] = l < c.levels ? c.r[l] : 0;
      best.overpartition_b = c.b;
      best.ms = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (keys) cudaFree(keys);
  if (tmp) cudaFree(tmp);
  if (vals) cudaFree(vals);
  if (vtmp) cudaFree(vtmp);
  if (st != AMS_OK) return st;
  best.candidates = (uint32_t)cands.size();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[key] = best;
  }
  *out = best;
  return AMS_OK;
}

}  // extern "C"
